// Execution kernels of the level-blocked MPK: the persistent (level group,
// power) wavefront (Fig. 5 over level groups, with the point-to-point
// conditions of Sec. 4.3 refined to work items), the baseline of back-to-back
// SpMVs (Fig. 1) and the Chebyshev sweep (Sec. 7, Eq. 7-9).
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>

#include "mpk_internal.cuh"

namespace mpk {

namespace {

template <typename MT, typename VT>
__device__ __forceinline__ VT to_vt(MT v) { return (VT)v; }
template <typename MT>
__device__ __forceinline__ double as_double(MT v) { return (double)v; }
template <>
__device__ __forceinline__ double as_double<__nv_bfloat16>(__nv_bfloat16 v) { return (double)__bfloat162float(v); }
template <>
__device__ __forceinline__ float to_vt<__nv_bfloat16, float>(__nv_bfloat16 v) { return __bfloat162float(v); }

// y_out[r] = sum_j A[r, j] * y_in[j] for the (up to) 32 rows of SELL chunk c,
// one row per lane (Fig. 1, restricted to the chunk's row range).  W columns
// of the row-major block vectors are done per pass; EXACT means nrhs == W.
// Padding entries (column -1) sit at the end of each row and are skipped.
template <typename VT, typename MT, int W, bool EXACT, bool DIAG>
__device__ __forceinline__ void chunk_rows(const ExecArgs &a, int32_t c, int lane, const VT *yin, VT *yout) {
    const int32_t row0 = __ldg(a.chunk_row + c);
    const int32_t nrows = __ldg(a.chunk_row + c + 1) - row0;
    if (lane >= nrows) return;
    const int64_t off = __ldg(a.chunk_off + c);
    const int32_t w = (int32_t)((__ldg(a.chunk_off + c + 1) - off) / kChunk);
    const int32_t r = row0 + lane;
    const int nrhs = EXACT ? W : a.nrhs;
    const int32_t *cp = a.pcol + off + lane;
    const MT *vp = (const MT *)a.pval + off + lane;
    for (int cb = 0; cb < nrhs; cb += W) {
        VT acc[W];
#pragma unroll
        for (int i = 0; i < W; i++) acc[i] = VT(0);
#pragma unroll 4
        for (int32_t j = 0; j < w; j++) {
            const int32_t col = __ldg(cp + (int64_t)j * kChunk);
            const VT v = to_vt<MT, VT>(__ldg(vp + (int64_t)j * kChunk));
            if (col >= 0) {
                const VT *src = yin + (int64_t)col * nrhs + cb;
#pragma unroll
                for (int i = 0; i < W; i++)
                    if (EXACT || cb + i < nrhs) acc[i] = fma(v, src[i], acc[i]);
            }
        }
        if (DIAG) {
            const VT d = (VT)__ldg(a.diag + r);
            const VT *src = yin + (int64_t)r * nrhs + cb;
#pragma unroll
            for (int i = 0; i < W; i++)
                if (EXACT || cb + i < nrhs) acc[i] = fma(d, src[i], acc[i]);
        }
        VT *dst = yout + (int64_t)r * nrhs + cb;
#pragma unroll
        for (int i = 0; i < W; i++)
            if (EXACT || cb + i < nrhs) dst[i] = acc[i];
    }
}

// Warp 0 of a CTA waits until power k-1 is complete on every tile in
// [dep_lo[t], dep_hi[t]] (the tiles holding the columns of tile t: the
// conditions (A)-(C) of Sec. 4.3 at tile granularity).  Bounded: after
// timeout_ns it records MPK_ERR_TIMEOUT with the node, raises the abort word
// and returns false; it also returns false once another CTA has aborted.
__device__ bool wait_deps(const ExecArgs &a, int32_t k, int32_t t, uint32_t epoch, int lane) {
    const uint32_t *f = a.flags + (int64_t)(k - 1) * a.n_tiles;
    const int32_t lo = __ldg(a.dep_lo + t), hi = __ldg(a.dep_hi + t);
    uint64_t t0 = 0;
    unsigned ns = 32;
    for (int it = 0;; it++) {
        bool ok = true;
        for (int32_t i = lo + lane; i <= hi; i += 32) ok &= (ld_relaxed_u32(f + i) == epoch);
        if (__all_sync(0xffffffffu, ok)) break;
        int stop = 0;
        if (lane == 0) {
            if (it == 0) t0 = global_ns();
            if (ld_relaxed_s32(a.ctl + CTL_ABORT)) {
                stop = 1;
            } else if (it > 0 && global_ns() - t0 > a.timeout_ns) {
                if (atomicCAS(a.ctl + CTL_ERR, 0, (int)MPK_ERR_TIMEOUT) == 0) {
                    atomicExch(a.ctl + CTL_ERR_K, k);
                    atomicExch(a.ctl + CTL_ERR_T, t);
                }
                atomicExch(a.ctl + CTL_ABORT, 1);
                stop = 1;
            }
        }
        if (__shfl_sync(0xffffffffu, stop, 0)) return false;
        __nanosleep(ns);
        if (ns < 512) ns <<= 1;
    }
    fence_acq_rel_gpu();
    return true;
}

// The last CTA to leave resets the dispatch words and publishes the epoch.
__device__ __forceinline__ void wave_teardown(const ExecArgs &a, uint32_t epoch) {
    if (threadIdx.x == 0) {
        __threadfence();
        int done = atomicAdd(a.ctl + CTL_FINISHED, 1);
        if (done == (int)gridDim.x - 1) {
            atomicExch(a.ctl + CTL_NEXT, 0);
            atomicExch(a.ctl + CTL_FINISHED, 0);
            atomicExch(a.ctl + CTL_ABORT, 0);
            atomicExch(a.ctl + CTL_EPOCH, (int)epoch);
            __threadfence();
        }
    }
}

// Body of one work item (tile t, power k) of the plain MPK.
template <typename VT, typename MT, int W, bool EXACT, bool DIAG>
struct MpkNode {
    __device__ __forceinline__ static void run(const ExecArgs &a, int32_t t, int32_t k, int warp, int nwarps, int lane) {
        const VT *yin = k == 1 ? (const VT *)a.x : (const VT *)a.Y + (int64_t)(k - 2) * a.blk;
        VT *yout = (VT *)a.Y + (int64_t)(k - 1) * a.blk;
        const int32_t c1 = __ldg(a.tile_chunk + t + 1);
        for (int32_t c = __ldg(a.tile_chunk + t) + warp; c < c1; c += nwarps)
            chunk_rows<VT, MT, W, EXACT, DIAG>(a, c, lane, yin, yout);
    }
};

// Persistent wavefront: CTAs take work items in the order of the Lp diagram
// over level groups (diagonals ascending, powers ascending inside a
// diagonal, tiles ascending inside a group).  Items are handed out in order
// by one counter, so every item's dependencies were taken earlier by running
// CTAs and the launch cannot deadlock even when not all CTAs are resident.
template <typename Node, typename Extra>
__device__ __forceinline__ void wave_loop(const ExecArgs &a, const Extra &extra) {
    __shared__ int s_item[2];
    __shared__ int s_ok;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const uint32_t epoch = (uint32_t)ld_relaxed_s32(a.ctl + CTL_EPOCH) + 1u;
    if (threadIdx.x == 0) s_item[0] = atomicAdd(a.ctl + CTL_NEXT, 1);
    __syncthreads();
    int cur = s_item[0], buf = 1;
    while (cur < a.n_items) {
        if (threadIdx.x == 0) s_item[buf] = ld_relaxed_s32(a.ctl + CTL_ABORT) ? INT_MAX : atomicAdd(a.ctl + CTL_NEXT, 1);
        const int32_t wk = __ldg(a.work + cur);
        const int32_t t = wk >> 8, k = wk & 255;
        if (k <= a.p) {
            if (warp == 0) {
                bool ok = k == 1 ? true : wait_deps(a, k, t, epoch, lane);
                if (lane == 0) s_ok = ok;
            }
            __syncthreads();
            if (s_ok) {
                Node::run(a, t, k, warp, nwarps, lane, extra);
                __syncthreads();
                if (threadIdx.x == 0 && !(t == a.drop_tile && k == a.drop_k)) {
                    fence_acq_rel_gpu();
                    st_release_u32(a.flags + (int64_t)k * a.n_tiles + t, epoch);
                }
            }
        }
        __syncthreads();
        cur = s_item[buf];
        buf ^= 1;
    }
    wave_teardown(a, epoch);
}

template <typename VT, typename MT, int W, bool EXACT, bool DIAG>
struct MpkNodeX {
    __device__ __forceinline__ static void run(const ExecArgs &a, int32_t t, int32_t k, int warp, int nwarps, int lane,
                                               const int &) {
        MpkNode<VT, MT, W, EXACT, DIAG>::run(a, t, k, warp, nwarps, lane);
    }
};

template <typename VT, typename MT, int W, bool EXACT, bool DIAG>
__global__ void __launch_bounds__(kWaveThreads) k_wave(ExecArgs a) {
    wave_loop<MpkNodeX<VT, MT, W, EXACT, DIAG>, int>(a, 0);
}

// Baseline: one SpMV over all chunks (warp per chunk, grid-stride).
template <typename VT, typename MT, int W, bool EXACT, bool DIAG>
__global__ void __launch_bounds__(kWaveThreads) k_spmv(ExecArgs a, const VT *yin, VT *yout) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t c = gw; c < a.n_chunks; c += nw) chunk_rows<VT, MT, W, EXACT, DIAG>(a, (int32_t)c, lane, yin, yout);
}

// ---------------------------------------------------------------- Chebyshev
// Node of sweep powers: global power k = k0 + j.  With Ahat = (A - c)/r:
//   v_1 = Ahat v_0,  v_k = 2 Ahat v_{k-1} - v_{k-2},  acc += coef_k v_k,
// vectors complex (two columns re, im) in a ring of three blocks; A v is
// summed in the storage precision, the scaling, the recurrence update and
// the coefficient sum are done in FP64.
template <typename VT, typename MT, bool DIAG>
struct ChebNode {
    __device__ __forceinline__ static void run(const ExecArgs &a, int32_t t, int32_t j, int warp, int nwarps, int lane,
                                               const ChebArgs &ca) {
        const int32_t k = ca.k0 + j;
        VT *ring = (VT *)ca.ring;
        const VT *yin = ring + (int64_t)((k - 1) % 3) * a.blk;
        const VT *yprev = ring + (int64_t)((k + 1) % 3) * a.blk;   // (k-2) mod 3
        VT *yout = ring + (int64_t)(k % 3) * a.blk;
        const double cre = ca.coef[2 * k], cim = ca.coef[2 * k + 1];
        const int32_t c1 = __ldg(a.tile_chunk + t + 1);
        for (int32_t c = __ldg(a.tile_chunk + t) + warp; c < c1; c += nwarps) {
            const int32_t row0 = __ldg(a.chunk_row + c);
            const int32_t nrows = __ldg(a.chunk_row + c + 1) - row0;
            if (lane >= nrows) continue;
            const int64_t off = __ldg(a.chunk_off + c);
            const int32_t w = (int32_t)((__ldg(a.chunk_off + c + 1) - off) / kChunk);
            const int32_t r = row0 + lane;
            const int32_t *cp = a.pcol + off + lane;
            const MT *vp = (const MT *)a.pval + off + lane;
            VT s0 = VT(0), s1 = VT(0);
#pragma unroll 4
            for (int32_t q = 0; q < w; q++) {
                const int32_t col = __ldg(cp + (int64_t)q * kChunk);
                const VT v = to_vt<MT, VT>(__ldg(vp + (int64_t)q * kChunk));
                if (col >= 0) {
                    s0 = fma(v, yin[2 * (int64_t)col], s0);
                    s1 = fma(v, yin[2 * (int64_t)col + 1], s1);
                }
            }
            const double u0 = (double)yin[2 * (int64_t)r], u1 = (double)yin[2 * (int64_t)r + 1];
            double a0, a1;
            if (DIAG) {   // the diagonal term enters in FP64 together with the shift
                const double d = (double)__ldg(a.diag + r);
                a0 = ca.alpha * ((double)s0 + d * u0) + ca.beta * u0;
                a1 = ca.alpha * ((double)s1 + d * u1) + ca.beta * u1;
            } else {
                a0 = ca.alpha * (double)s0 + ca.beta * u0;
                a1 = ca.alpha * (double)s1 + ca.beta * u1;
            }
            double n0 = a0, n1 = a1;
            if (k > 1) {
                n0 = 2.0 * a0 - (double)yprev[2 * (int64_t)r];
                n1 = 2.0 * a1 - (double)yprev[2 * (int64_t)r + 1];
            }
            yout[2 * (int64_t)r] = (VT)n0;
            yout[2 * (int64_t)r + 1] = (VT)n1;
            double *acc = ca.acc + 2 * (int64_t)r;
            acc[0] += cre * n0 - cim * n1;
            acc[1] += cre * n1 + cim * n0;
        }
    }
};

template <typename VT, typename MT, bool DIAG>
__global__ void __launch_bounds__(kWaveThreads) k_cheb_wave(ChebArgs ca) {
    wave_loop<ChebNode<VT, MT, DIAG>, ChebArgs>(ca.e, ca);
}

// acc = coef_0 * v_0 (complex), v_0 = ring block 0
template <typename VT>
__global__ void k_cheb_init(int32_t n, const VT *v0, const double *coef, double *acc) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const double x0 = (double)v0[2 * r], x1 = (double)v0[2 * r + 1];
    acc[2 * r] = coef[0] * x0 - coef[1] * x1;
    acc[2 * r + 1] = coef[0] * x1 + coef[1] * x0;
}

// Gershgorin row bounds -> per-block min/max (lo in [2b], hi in [2b+1])
template <typename MT>
__global__ void k_gersh(ExecArgs a, double *out) {
    __shared__ double slo[8], shi[8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double lo = INFINITY, hi = -INFINITY;
    for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < a.n_chunks;
         c += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int32_t row0 = a.chunk_row[c], nrows = a.chunk_row[c + 1] - row0;
        if (lane < nrows) {
            const int64_t off = a.chunk_off[c];
            const int32_t wd = (int32_t)((a.chunk_off[c + 1] - off) / kChunk);
            const int32_t r = row0 + lane;
            double d = a.diag ? (double)a.diag[r] : 0.0, s = 0.0;
            for (int32_t j = 0; j < wd; j++) {
                int32_t col = a.pcol[off + (int64_t)j * kChunk + lane];
                double v = as_double<MT>(((const MT *)a.pval)[off + (int64_t)j * kChunk + lane]);
                if (col == r) d += v;
                else if (col >= 0) s += fabs(v);
            }
            lo = fmin(lo, d - s);
            hi = fmax(hi, d + s);
        }
    }
    for (int o = 16; o; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (lane == 0) { slo[w] = lo; shi[w] = hi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < (int)(blockDim.x >> 5); i++) { lo = fmin(lo, slo[i]); hi = fmax(hi, shi[i]); }
        out[2 * blockIdx.x] = fmin(lo, slo[0]);
        out[2 * blockIdx.x + 1] = fmax(hi, shi[0]);
    }
}

// dst[r] = src[perm[r]] (to_level) or dst[perm[r]] = src[r], in 4-byte words
__global__ void k_permute(int32_t n, int32_t words, int32_t count, const int32_t *perm, const uint32_t *src,
                          uint32_t *dst, int to_level) {
    const int64_t per = (int64_t)n * words;
    const int64_t total = per * count;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = g / per, rem = g % per;
        const int32_t r = (int32_t)(rem / words), w = (int32_t)(rem % words);
        const int64_t o = (int64_t)perm[r] * words + w;
        if (to_level) dst[b * per + rem] = src[b * per + o];
        else dst[b * per + o] = src[b * per + rem];
    }
}

// ---------------------------------------------------------------- dispatch
template <typename VT, typename MT, bool DIAG>
const void *wave_ptr(int nrhs) {
    switch (nrhs) {
    case 1: return (const void *)k_wave<VT, MT, 1, true, DIAG>;
    case 2: return (const void *)k_wave<VT, MT, 2, true, DIAG>;
    case 4: return (const void *)k_wave<VT, MT, 4, true, DIAG>;
    case 8: return (const void *)k_wave<VT, MT, 8, true, DIAG>;
    default: return (const void *)k_wave<VT, MT, 8, false, DIAG>;
    }
}
template <typename VT, typename MT, bool DIAG>
const void *spmv_ptr(int nrhs) {
    switch (nrhs) {
    case 1: return (const void *)k_spmv<VT, MT, 1, true, DIAG>;
    case 2: return (const void *)k_spmv<VT, MT, 2, true, DIAG>;
    case 4: return (const void *)k_spmv<VT, MT, 4, true, DIAG>;
    case 8: return (const void *)k_spmv<VT, MT, 8, true, DIAG>;
    default: return (const void *)k_spmv<VT, MT, 8, false, DIAG>;
    }
}

const void *pick_wave(const Plan *pl) {
    if (pl->prec == MPK_F64) return wave_ptr<double, double, false>(pl->nrhs);
    if (!pl->has_diag) return wave_ptr<float, float, false>(pl->nrhs);
    if (pl->val_bytes == 2) return wave_ptr<float, __nv_bfloat16, true>(pl->nrhs);
    return wave_ptr<float, float, true>(pl->nrhs);
}
const void *pick_spmv(const Plan *pl) {
    if (pl->prec == MPK_F64) return spmv_ptr<double, double, false>(pl->nrhs);
    if (!pl->has_diag) return spmv_ptr<float, float, false>(pl->nrhs);
    if (pl->val_bytes == 2) return spmv_ptr<float, __nv_bfloat16, true>(pl->nrhs);
    return spmv_ptr<float, float, true>(pl->nrhs);
}
const void *pick_cheb(const Plan *pl) {
    if (pl->prec == MPK_F64) return (const void *)k_cheb_wave<double, double, false>;
    if (!pl->has_diag) return (const void *)k_cheb_wave<float, float, false>;
    if (pl->val_bytes == 2) return (const void *)k_cheb_wave<float, __nv_bfloat16, true>;
    return (const void *)k_cheb_wave<float, float, true>;
}

}  // namespace

int wave_occupancy(const Plan *pl, int *ctas_per_sm) {
    int occ = 0;
    MPK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pick_wave(pl), kWaveThreads, 0));
    int occ2 = 0;
    if (pl->nrhs == 2) {
        MPK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2, pick_cheb(pl), kWaveThreads, 0));
        occ = std::min(occ, occ2);
    }
    *ctas_per_sm = std::max(1, occ);
    return MPK_OK;
}

ExecArgs exec_args(const Plan *pl, const void *x, void *Y) {
    ExecArgs a;
    a.chunk_row = pl->d_chunk_row;
    a.chunk_off = pl->d_chunk_off;
    a.tile_chunk = pl->d_tile_chunk;
    a.dep_lo = pl->d_dep_lo;
    a.dep_hi = pl->d_dep_hi;
    a.work = pl->d_work;
    a.pcol = pl->d_pcol;
    a.pval = pl->d_pval;
    a.diag = pl->d_diag;
    a.flags = pl->d_flags;
    a.ctl = pl->d_ctl;
    a.n_tiles = pl->n_tiles;
    a.n_items = pl->n_tiles * pl->p;
    a.n_chunks = pl->n_chunks;
    a.nrhs = pl->nrhs;
    a.p = pl->p;
    a.blk = (int64_t)pl->n * pl->nrhs;
    a.x = x;
    a.Y = Y;
    a.timeout_ns = (uint64_t)(pl->timeout_s * 1e9);
    a.drop_tile = -1;
    a.drop_k = -1;
    return a;
}

// Epochs are 32-bit: before they could wrap onto stale flag values, clear all.
static int epoch_guard(Plan *pl, cudaStream_t st) {
    if (pl->launches >= 0xFFFFFF00ull) {
        MPK_CUDA(cudaMemsetAsync(pl->d_flags, 0, sizeof(uint32_t) * (size_t)(pl->p + 1) * pl->n_tiles, st));
        MPK_CUDA(cudaMemsetAsync(pl->d_ctl, 0, sizeof(int32_t) * CTL_WORDS, st));
        pl->launches = 0;
    }
    pl->launches++;
    return MPK_OK;
}

int launch_wavefront(Plan *pl, const void *x, void *Y, cudaStream_t st) {
    int rc = epoch_guard(pl, st);
    if (rc) return rc;
    ExecArgs a = exec_args(pl, x, Y);
    a.drop_tile = pl->drop_tile;
    a.drop_k = pl->drop_k;
    pl->drop_tile = pl->drop_k = -1;
    void *args[] = {(void *)&a};
    MPK_CUDA(cudaLaunchKernel(pick_wave(pl), dim3(pl->grid_ctas), dim3(kWaveThreads), args, 0, st));
    return MPK_OK;
}

int launch_baseline(Plan *pl, const void *x, void *Y, cudaStream_t st) {
    ExecArgs a = exec_args(pl, x, Y);
    const void *fn = pick_spmv(pl);
    int occ = 0;
    MPK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kWaveThreads, 0));
    int64_t warps_needed = pl->n_chunks;
    int64_t grid = std::min<int64_t>((int64_t)pl->num_sms * std::max(1, occ), (warps_needed + 7) / 8);
    grid = std::max<int64_t>(1, grid);
    const size_t eb = (size_t)elem_bytes_of(pl);
    for (int k = 1; k <= pl->p; k++) {
        const void *yin = k == 1 ? x : (const char *)Y + (size_t)(k - 2) * a.blk * eb;
        void *yout = (char *)Y + (size_t)(k - 1) * a.blk * eb;
        void *args[] = {(void *)&a, (void *)&yin, (void *)&yout};
        MPK_CUDA(cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(kWaveThreads), args, 0, st));
    }
    return MPK_OK;
}

int read_device_error(Plan *pl, cudaStream_t st) {
    int32_t w[CTL_WORDS];
    MPK_CUDA(cudaMemcpyAsync(w, pl->d_ctl, sizeof(w), cudaMemcpyDeviceToHost, st));
    MPK_CUDA(cudaStreamSynchronize(st));
    if (w[CTL_ERR] != 0) {
        MPK_CUDA(cudaMemsetAsync(pl->d_ctl + CTL_ERR, 0, 3 * sizeof(int32_t), st));
        MPK_CUDA(cudaStreamSynchronize(st));
        return w[CTL_ERR];
    }
    return MPK_OK;
}

int ensure_io(Plan *pl, size_t bytes) {
    if (pl->io_bytes >= bytes) return MPK_OK;
    if (pl->d_io) {
        cudaStreamSynchronize(pl->stream);
        cudaFree(pl->d_io);
        pl->d_io = nullptr;
        pl->io_bytes = 0;
    }
    char *p = nullptr;
    int rc = dev_alloc<char>(nullptr, &p, bytes);
    if (rc) return rc;
    pl->d_io = p;
    pl->io_bytes = bytes;
    return MPK_OK;
}

int permute_vectors(Plan *pl, const void *src, void *dst, int32_t count, int32_t elem_bytes, int32_t to_level,
                    cudaStream_t st) {
    const int32_t words = pl->nrhs * elem_bytes / 4;
    const int64_t total = (int64_t)pl->n * words * count;
    if (total == 0) return MPK_OK;
    unsigned grid = (unsigned)std::min<int64_t>((total + 255) / 256, (int64_t)pl->num_sms * 16);
    k_permute<<<grid, 256, 0, st>>>(pl->n, words, count, pl->d_perm, (const uint32_t *)src, (uint32_t *)dst,
                                    to_level);
    MPK_CUDA(cudaGetLastError());
    return MPK_OK;
}

}  // namespace mpk

using namespace mpk;

namespace {

// Runs `body(x_level, Y_level)` in level order; gathers / scatters through
// the plan-owned buffer when the caller's vectors are in original order.
template <typename F>
int with_level_io(Plan *pl, const void *x, void *Y, int32_t nout, uint32_t flags, F body) {
    cudaStream_t st = pl->stream;
    if (flags & MPK_IO_PERMUTED) return body(x, Y);
    const size_t blk = (size_t)pl->n * pl->nrhs * elem_bytes_of(pl);
    int rc = ensure_io(pl, blk * (size_t)(nout + 1));
    if (rc) return rc;
    char *xb = (char *)pl->d_io, *yb = xb + blk;
    if ((rc = permute_vectors(pl, x, xb, 1, elem_bytes_of(pl), 1, st))) return rc;
    if ((rc = body(xb, yb))) return rc;
    return permute_vectors(pl, yb, Y, nout, elem_bytes_of(pl), 0, st);
}

}  // namespace

extern "C" {

int mpk_run(mpk_plan_t plan, const void *x, void *Y, uint32_t flags) {
    if (!plan || !x || !Y) return MPK_ERR_INVALID;
    Plan *pl = &plan->pl;
    int rc = with_level_io(pl, x, Y, pl->p, flags, [&](const void *xl, void *yl) {
        return launch_wavefront(pl, xl, yl, pl->stream);
    });
    if (rc) return rc;
    MPK_CUDA(cudaGetLastError());
    if (flags & MPK_ASYNC) return MPK_OK;
    return read_device_error(pl, pl->stream);
}

int mpk_baseline_run(mpk_plan_t plan, const void *x, void *Y, uint32_t flags) {
    if (!plan || !x || !Y) return MPK_ERR_INVALID;
    Plan *pl = &plan->pl;
    int rc = with_level_io(pl, x, Y, pl->p, flags, [&](const void *xl, void *yl) {
        return launch_baseline(pl, xl, yl, pl->stream);
    });
    if (rc) return rc;
    MPK_CUDA(cudaGetLastError());
    if (flags & MPK_ASYNC) return MPK_OK;
    MPK_CUDA(cudaStreamSynchronize(pl->stream));
    return MPK_OK;
}

int mpk_permute_vectors(mpk_plan_t plan, const void *src, void *dst, int32_t count, int32_t elem_bytes,
                        int32_t to_level) {
    if (!plan || !src || !dst || count < 0 || (elem_bytes != 4 && elem_bytes != 8)) return MPK_ERR_INVALID;
    Plan *pl = &plan->pl;
    int rc = permute_vectors(pl, src, dst, count, elem_bytes, to_level ? 1 : 0, pl->stream);
    if (rc) return rc;
    MPK_CUDA(cudaStreamSynchronize(pl->stream));
    return MPK_OK;
}

int mpk_gershgorin(mpk_plan_t plan, double *lo, double *hi) {
    if (!plan || !lo || !hi) return MPK_ERR_INVALID;
    Plan *pl = &plan->pl;
    cudaStream_t st = pl->stream;
    ExecArgs a = exec_args(pl, nullptr, nullptr);
    const int grid = std::max(1, std::min(pl->num_sms * 4, (pl->n_chunks + 7) / 8));
    double *d = nullptr;
    int rc = dev_alloc<double>(nullptr, &d, (size_t)2 * grid);
    if (rc) return rc;
    if (pl->val_bytes == 8) k_gersh<double><<<grid, 256, 0, st>>>(a, d);
    else if (pl->val_bytes == 4) k_gersh<float><<<grid, 256, 0, st>>>(a, d);
    else k_gersh<__nv_bfloat16><<<grid, 256, 0, st>>>(a, d);
    std::vector<double> h((size_t)2 * grid);
    cudaError_t e = cudaMemcpyAsync(h.data(), d, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_status(e, "gershgorin", __LINE__);
    double l = INFINITY, u = -INFINITY;
    for (int b = 0; b < grid; b++) {
        l = std::min(l, h[2 * b]);
        u = std::max(u, h[2 * b + 1]);
    }
    *lo = l;
    *hi = u;
    return MPK_OK;
}

int mpk_cheb(mpk_plan_t plan, const double *coef, int32_t M, double c, double r, const void *x, double *y,
             uint32_t flags) {
    if (!plan || !coef || !x || !y || M < 1 || !(r != 0.0)) return MPK_ERR_INVALID;
    Plan *pl = &plan->pl;
    if (pl->nrhs != 2) return MPK_ERR_INVALID;
    cudaStream_t st = pl->stream;
    const int eb = elem_bytes_of(pl);
    const size_t blk = (size_t)pl->n * 2;
    // device storage: 3-block ring (storage precision), FP64 accumulator, coefficients
    const size_t ring_b = 3 * blk * eb, acc_b = (flags & MPK_IO_PERMUTED) ? 0 : blk * sizeof(double);
    const size_t coef_b = sizeof(double) * 2 * ((size_t)M + 1);
    const size_t need = ring_b + acc_b + coef_b + 256;
    if (pl->cheb_bytes < need) {
        if (pl->d_cheb) {
            cudaStreamSynchronize(st);
            cudaFree(pl->d_cheb);
            pl->d_cheb = nullptr;
            pl->cheb_bytes = 0;
        }
        char *p = nullptr;
        int rc = dev_alloc<char>(nullptr, &p, need);
        if (rc) return rc;
        pl->d_cheb = p;
        pl->cheb_bytes = need;
    }
    char *base = (char *)pl->d_cheb;
    void *ring = base;
    double *acc = (flags & MPK_IO_PERMUTED) ? y : (double *)(base + ring_b);
    double *dcoef = (double *)(base + ring_b + acc_b);
    MPK_CUDA(cudaMemcpyAsync(dcoef, coef, coef_b, cudaMemcpyHostToDevice, st));
    int rc;
    if (flags & MPK_IO_PERMUTED) {
        MPK_CUDA(cudaMemcpyAsync(ring, x, blk * eb, cudaMemcpyDeviceToDevice, st));
    } else if ((rc = permute_vectors(pl, x, ring, 1, eb, 1, st))) {
        return rc;
    }
    const unsigned nb = (unsigned)((pl->n + 255) / 256);
    if (eb == 8) k_cheb_init<double><<<nb, 256, 0, st>>>(pl->n, (const double *)ring, dcoef, acc);
    else k_cheb_init<float><<<nb, 256, 0, st>>>(pl->n, (const float *)ring, dcoef, acc);
    MPK_CUDA(cudaGetLastError());
    ChebArgs ca;
    ca.ring = ring;
    ca.acc = acc;
    ca.coef = dcoef;
    ca.alpha = 1.0 / r;
    ca.beta = -c / r;
    for (int32_t k0 = 0; k0 < M; k0 += pl->p) {
        const int32_t pw = std::min(pl->p, M - k0);
        if ((rc = epoch_guard(pl, st))) return rc;
        ca.e = exec_args(pl, nullptr, nullptr);
        ca.e.p = pw;   // items of powers above pw are skipped
        ca.k0 = k0;
        void *args[] = {(void *)&ca};
        MPK_CUDA(cudaLaunchKernel(pick_cheb(pl), dim3(pl->grid_ctas), dim3(kWaveThreads), args, 0, st));
    }
    if (!(flags & MPK_IO_PERMUTED)) {
        // acc (level order, n x 2 doubles) -> y (original order)
        if ((rc = permute_vectors(pl, acc, y, 1, 8, 0, st))) return rc;
    }
    MPK_CUDA(cudaGetLastError());
    if (flags & MPK_ASYNC) return MPK_OK;
    return read_device_error(pl, st);
}

int mpk_plan_last_error(mpk_plan_t plan, int32_t *code, int32_t *power, int32_t *tile) {
    if (!plan) return MPK_ERR_INVALID;
    Plan *pl = &plan->pl;
    int32_t w[CTL_WORDS];
    MPK_CUDA(cudaMemcpyAsync(w, pl->d_ctl, sizeof(w), cudaMemcpyDeviceToHost, pl->stream));
    MPK_CUDA(cudaStreamSynchronize(pl->stream));
    if (code) *code = w[CTL_ERR];
    if (power) *power = w[CTL_ERR_K];
    if (tile) *tile = w[CTL_ERR_T];
    return MPK_OK;
}

int mpk_plan_debug_drop_flag(mpk_plan_t plan, int32_t tile, int32_t power) {
    if (!plan) return MPK_ERR_INVALID;
    Plan *pl = &plan->pl;
    if (tile < 0) {
        pl->drop_tile = pl->drop_k = -1;
        return MPK_OK;
    }
    if (tile >= pl->n_tiles || power < 1 || power > pl->p) return MPK_ERR_INVALID;
    pl->drop_tile = tile;
    pl->drop_k = power;
    return MPK_OK;
}

int mpk_cheb_coeffs_schroedinger(int32_t M, double c, double r, double dt, double *coef) {
    if (M < 0 || !coef) return MPK_ERR_INVALID;
    // exp(-i c dt) * (2 - delta_k0) * (-i)^k * J_k(r dt)   (Jacobi-Anger expansion)
    const double pr = cos(c * dt), pi = -sin(c * dt);
    for (int32_t k = 0; k <= M; k++) {
        const double a = (k == 0 ? 1.0 : 2.0) * jn(k, r * dt);
        static const double ire[4] = {1.0, 0.0, -1.0, 0.0}, iim[4] = {0.0, -1.0, 0.0, 1.0};
        const double tr = a * ire[k & 3], ti = a * iim[k & 3];
        coef[2 * k] = pr * tr - pi * ti;
        coef[2 * k + 1] = pr * ti + pi * tr;
    }
    return MPK_OK;
}

}  // extern "C"
