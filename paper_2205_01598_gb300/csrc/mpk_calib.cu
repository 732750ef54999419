// Arithmetic-rate probe: the denominator of an ALU roofline.  The method's
// per-entry work is one fused multiply-add per stored entry and power
// (Sec. 3.1: 2 flops per nonzero), so the rate that bounds an ALU-bound
// form is the device's sustained FMA rate in that precision, measured here
// rather than taken from a data sheet.
#include "mpk_internal.cuh"

namespace mpk {
namespace {

constexpr int kProbeChains = 8;      // independent FMA chains per thread
constexpr int kProbeUnroll = 4;      // iterations per loop trip
constexpr int kProbeThreads = 256;

// Each thread runs kProbeChains independent chains v <- v * a + b for
// iters iterations (a just below 1 keeps them bounded).  The sum of the
// chains is compared with a value it never takes, so the chains stay live
// without any store in the loop.
template <typename T>
__global__ void __launch_bounds__(kProbeThreads) k_fma_chains(int64_t iters, T a, T b, T *sink) {
    T v[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; c++) v[c] = (T)(threadIdx.x + 1 + c) * (T)1e-3;
    for (int64_t i = 0; i < iters; i += kProbeUnroll) {
#pragma unroll
        for (int u = 0; u < kProbeUnroll; u++)
#pragma unroll
            for (int c = 0; c < kProbeChains; c++) v[c] = fma(v[c], a, b);
    }
    T s = (T)0;
#pragma unroll
    for (int c = 0; c < kProbeChains; c++) s += v[c];
    if (s == (T)-1) sink[0] = s;
}

}  // namespace
}  // namespace mpk

using namespace mpk;

extern "C" int mpk_probe_fma(int32_t prec, int32_t blocks_per_sm, int64_t iters, void *sink, void *stream,
                             double *flops) {
    if (!sink || !flops || (prec != MPK_F64 && prec != MPK_F32) || blocks_per_sm < 1 || blocks_per_sm > 32 ||
        iters < kProbeUnroll || iters % kProbeUnroll)
        return MPK_ERR_INVALID;
    int dev = 0, sms = 0;
    MPK_CUDA(cudaGetDevice(&dev));
    MPK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int grid = sms * blocks_per_sm;
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == MPK_F64)
        k_fma_chains<double><<<grid, kProbeThreads, 0, st>>>(iters, 0.9999999, 1e-7, (double *)sink);
    else
        k_fma_chains<float><<<grid, kProbeThreads, 0, st>>>(iters, 0.9999f, 1e-4f, (float *)sink);
    MPK_CUDA(cudaGetLastError());
    *flops = 2.0 * (double)grid * kProbeThreads * kProbeChains * (double)iters;
    return MPK_OK;
}
