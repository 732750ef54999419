// Internal declarations of the GB300 level-blocked MPK library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <new>
#include <vector>

#include "mpk.h"

namespace mpk {

constexpr int kChunk = 32;         // rows per SELL chunk = one warp, one row per lane
constexpr int kMaxP = 255;         // powers are packed in 8 bits of a work item
constexpr int kMaxNrhs = 64;
#ifndef MPK_COMPUTE_WARPS
#define MPK_COMPUTE_WARPS 8
#endif
constexpr int kComputeWarps = MPK_COMPUTE_WARPS;         // warps that compute work items
constexpr int kFp64Warps = 16;                           // compute warps of the FP64 MPK wavefront
#ifndef MPK_F32_WARPS
#define MPK_F32_WARPS MPK_COMPUTE_WARPS
#endif
constexpr int kFp32Warps = MPK_F32_WARPS;                // compute warps of the FP32 / BF16 MPK wavefront
constexpr int kWaveThreads = (kComputeWarps + 1) * 32;   // plus one scheduler warp
constexpr int kSpmvThreads = 256;                        // baseline SpMV CTA
#ifndef MPK_RES_WARPS
#define MPK_RES_WARPS 16
#endif
constexpr int kResWarps = MPK_RES_WARPS;                 // compute warps of a resident-schedule CTA
constexpr int kResThreads = (kResWarps + 1) * 32;
constexpr int kMaxStages = 3;                            // shared-memory stages of the staged work-list form
// A dependency range wider than a flag probe is checked by counters of
// finished tiles per block of kFlagBlock tiles (each finished item adds one),
// and flag by flag only at its ragged ends.
constexpr int kFlagBlock = 128;
// Widest dependency range (in flags, from its start rounded down to 4) that
// one 16-byte-per-lane probe of a warp covers; wider ranges use the counters.
constexpr int kProbeFlags = 256;

// Control words of a plan (device int32 array).
enum Ctl : int {
    CTL_UNUSED = 0,
    CTL_FINISHED = 1,   // CTAs that left the dispatch loop in this launch
    CTL_EPOCH = 2,      // epoch of the last completed launch (flags hold epochs)
    CTL_ABORT = 3,      // set when a wait expired: every CTA stops taking work
    CTL_ERR = 4,        // mpk_status of the first device-side error (0 = none)
    CTL_ERR_K = 5,      // power of the node whose wait expired
    CTL_ERR_T = 6,      // tile of the node whose wait expired
    CTL_WORDS = 8
};

struct Plan {
    // sizes and options
    int32_t n = 0, p = 0, nrhs = 1, prec = MPK_F64;
    int64_t nnz = 0;
    int32_t n_levels = 0, n_groups = 0, n_tiles = 0, n_chunks = 0;
    int32_t tile_rows = 0, max_level_rows = 0;
    int32_t grid_ctas = 0, ctas_per_sm = 0;
    int32_t val_bytes = 8;
    int32_t has_diag = 0;           // diagonal stored apart (BF16 values)
    double cache_bytes = 0, safety_f = 0.5, timeout_s = 2.0, lag = -1.0, slope = 1.0;
    cudaStream_t stream = nullptr;
    int device = 0, num_sms = 0;
    int64_t packed_entries = 0, device_bytes = 0;
    double plan_ms = 0;
    static constexpr int kFeatures = 25;   // matrix features for the learned planner
    float features[kFeatures] = {};
    uint64_t launches = 0;
    int32_t drop_tile = -1, drop_k = -1;   // one-shot test hook (mpk_plan_debug_drop_flag)
    uint32_t tune = 0;              // MPK_TUNE_* bits
    int32_t staged = 0;             // matrix slices staged in shared memory by bulk copies
    int32_t n_stages = 0;           // stages of the staged form (2 or 3: copies issued that many items ahead, less one)
    int32_t sorted = 0;             // rows of each tile packed in order of decreasing length
    int32_t resident = 0;           // resident schedule (a CTA keeps a tile's slice for all powers)
    int32_t wave_warps = kComputeWarps;   // compute warps of the MPK wavefront kernel
    int32_t cheb_grid = 0;          // CTAs of the Chebyshev wavefront launch
    int32_t dep_span = 0;           // max over tiles of dep_hi[t] - t
    int32_t stage_recs = 0;         // chunk records one resident stage holds
    int32_t max_row_len = 0;        // longest row of P A P^T
    int32_t *d_row_map = nullptr;   // packed position -> row (only when sorted)
    int64_t stage_entries = 0;      // capacity of one stage in packed entries
    size_t smem_bytes = 0;          // dynamic shared memory per wavefront CTA
    // host copies kept to build the issue order of shorter sweeps
    std::vector<int32_t> h_tile_row, h_group_tile, h_dep_lo, h_dep_hi;
    int32_t *d_work_rem = nullptr;  // issue order for rem_p powers (Chebyshev remainder sweep)
    int32_t rem_p = 0;

    std::vector<int32_t> h_level_ptr, h_group_ptr;   // finest levels (after recursion) and their groups
    std::vector<int32_t> h_group_stage;              // recursion stage that made each group (Sec. 4.4)
    int32_t rec_stages = 0;                          // stages of recursion that refined something
    int32_t sweep = 0;                               // powers per sweep of the issue order (q of mpk_opts.sweep)
    double phase_ms[8] = {};                         // wall time of planning by phase (mpk_plan_stats.phase_ms)

    // device arrays (plan-owned)
    int32_t *d_perm = nullptr, *d_iperm = nullptr, *d_level = nullptr;
    int32_t *d_level_ptr = nullptr, *d_group_ptr = nullptr;
    int32_t *d_chunk_row = nullptr;    // n_chunks+1: first row of each chunk (sentinel n)
    int64_t *d_chunk_off = nullptr;    // n_chunks+1: first packed entry of each chunk
    int4 *d_chunk_rec = nullptr;       // n_chunks: {first row, rows, first entry / 32, width}
    int32_t *d_tile_chunk = nullptr;   // n_tiles+1: first chunk of each tile
    int64_t *d_tile_off = nullptr;     // n_tiles+1: first packed entry of each tile
    int32_t *d_dep_lo = nullptr, *d_dep_hi = nullptr;  // n_tiles: tiles read at power k-1
    int32_t *d_work = nullptr;         // p*n_tiles items, (tile << 8) | power
    int32_t *d_pcol = nullptr;         // packed column indices, -1 = padding
    void *d_pval = nullptr;            // packed values (double / float / bf16)
    float *d_diag = nullptr;           // diagonal (only with has_diag)
    double *d_gersh = nullptr;         // Gershgorin row bounds scratch (lazily)
    uint32_t *d_flags = nullptr;       // (p+1) rows of fstride completion epochs
    uint32_t *d_bcnt = nullptr;        // (p+1) rows of bstride per-block completion counts (zero between launches)
    int32_t wide_deps = 0;             // some tile's dependency range is wider than a probe (counters in use)
    int32_t bstride = 0;               // blocks of kFlagBlock tiles
    int32_t fstride = 0;               // flag row length: n_tiles rounded up to 4, plus 4
    int32_t *d_ctl = nullptr;          // CTL_WORDS control words
    void *d_io = nullptr;              // permuted copies for unpermuted I/O (lazily)
    size_t io_bytes = 0;
    cudaStream_t copy_stream = nullptr;   // device-to-host copies of mpk_run_host (lazily)
    cudaEvent_t io_ev[4] = {};            // staging buffers unpermuted [0..1] / copied out [2..3]
    void *d_cheb = nullptr;            // Chebyshev vector ring (lazily)
    size_t cheb_bytes = 0;
    float2 *d_shadow = nullptr;        // double-float copies of the current and previous power (MPK_F64_DF)
    void *d_kry = nullptr;             // Krylov solver work space (lazily)
    size_t kry_bytes = 0;
    uint64_t df_xlim_bits = 0;         // largest |x| (FP64 bit pattern) the double-float range allows
};

// Parameters of the wavefront / baseline kernels.
struct ExecArgs {
    const int32_t *chunk_row;
    const int64_t *chunk_off;
    const int32_t *tile_chunk;
    const int32_t *dep_lo, *dep_hi;
    const int32_t *work;
    const int32_t *pcol;
    const void *pval;
    const float *diag;
    uint32_t *flags;
    int32_t *ctl;
    int32_t n_tiles, n_items, n_chunks, nrhs, p;
    int32_t fstride;        // flags of power k start at flags + k * fstride
    int64_t blk;            // elements of one vector block (n * nrhs)
    const void *x;          // y_0
    void *Y;                // p blocks
    uint64_t timeout_ns;
    int32_t drop_tile, drop_k;   // completion not published (test hook), -1 = none
    const int64_t *tile_off;     // first packed entry of each tile
    int64_t stage_entries;       // entries one shared-memory stage holds
    uint32_t tune;               // MPK_TUNE_* bits
    const int32_t *row_map;      // chunk position -> row (rows sorted by length in a tile); null = identity
    const int4 *chunk_rec;       // per chunk {first row, rows, first entry / 32, width}
    int32_t stage_recs;          // chunk records one resident stage holds
    int32_t n_stages;            // stages of the staged work-list form
    float2 *shadow;              // MPK_F64_DF: 2 blocks of n double-float pairs, power k in block k mod 2
    uint32_t *bcnt;              // finished tiles per block of kFlagBlock tiles, power k at bcnt + k * bstride;
                                 // null when every dependency range fits a probe (no counting)
    int32_t bstride;
};

// Chebyshev sweep parameters (one wavefront launch computes powers k0+1 .. k0+pw).
// Plans with FP32 vectors keep the coefficient sum and the spectral scaling
// in double-float (a value is the unevaluated sum hi + lo of two FP32
// numbers); FP64 plans keep them in FP64.
struct ChebArgs {
    ExecArgs e;
    void *ring;             // 3 vector blocks (n x G) cycling v_{k-2}, v_{k-1}, v_k
    void *acc;              // n x G coefficient sum: FP64 (FP64 plans) or
                            // double-float pairs (hi, lo) per column (FP32 plans)
    const double *coef;     // FP64 coefficients, G per k (interleaved complex for G = 2)
    const float4 *coef_df;  // double-float coefficients per k: (re hi, re lo, im hi, im lo)
    double alpha, beta;     // Ahat v = alpha*(A v) + beta*v with alpha = 1/r, beta = -c/r
    float alpha_hi, alpha_lo, beta_hi, beta_lo, c_hi, c_lo;   // the same as double-float pairs
    int32_t k0;             // powers already computed before this sweep (all time steps)
    int32_t pw;             // powers of this sweep
    int32_t M;              // powers (degree) of one time step
    int32_t total;          // powers of the whole propagation (time steps x M)
    int32_t step0, kin0;    // time step and power within it (1..M) of the sweep's first power
};

// Launch-wide arguments of a batched wavefront (several plans, one launch).
constexpr int kMaxBatch = 1024;
struct BatchArgs {
    ExecArgs g;                  // merged issue order, batch control words, limits
    const ExecArgs *table;       // per plan
    const int32_t *wplan;        // plan of each work item
    int32_t *const *plan_ctl;    // control words of each plan
    int32_t count;
};

// ---------------------------------------------------------------- host helpers
int cuda_status(cudaError_t e, const char *what, int line);
#define MPK_CUDA(call)                                                   \
    do {                                                                 \
        cudaError_t _e = (call);                                         \
        if (_e != cudaSuccess) return ::mpk::cuda_status(_e, #call, __LINE__); \
    } while (0)

template <typename T>
int dev_alloc(Plan *pl, T **ptr, size_t count) {
    *ptr = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void **)ptr, count * sizeof(T));
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        *ptr = nullptr;
        return e == cudaErrorMemoryAllocation ? MPK_ERR_OOM : MPK_ERR_CUDA;
    }
    if (pl) pl->device_bytes += (int64_t)(count * sizeof(T));
    return MPK_OK;
}

// Exclusive scans used by the planner (device, on `st`); tmp is sized by the helper.
int exclusive_scan_i32(const int32_t *in, int32_t *out, int64_t n, cudaStream_t st, int32_t *total);
int exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t st, int64_t *total);

// Execution entry points used across translation units.
int launch_wavefront(Plan *pl, const void *x, void *Y, cudaStream_t st);
int launch_baseline(Plan *pl, const void *x, void *Y, cudaStream_t st);
int launch_spmv1(Plan *pl, const void *x, void *y, cudaStream_t st);
int launch_cheb_sweep(Plan *pl, const ChebArgs &a, int32_t powers, cudaStream_t st);
int read_device_error(Plan *pl, cudaStream_t st);
int permute_vectors(Plan *pl, const void *src, void *dst, int32_t count, int32_t elem_bytes,
                    int32_t to_level, cudaStream_t st);
ExecArgs exec_args(const Plan *pl, const void *x, void *Y);
int ensure_io(Plan *pl, size_t bytes);
// Issue order of the (tile, power) items for powers 1..p_sweep (mpk_plan.cu).
double order_items(const Plan *pl, int32_t p_sweep, double lag, std::vector<int32_t> &work);
// Tile positions v(t) in level-group units and the slope of that order (lag
// resolved in place when negative).
double order_slope(const Plan *pl, int32_t p, double &lag, std::vector<double> &v);
// The plan's issue order (d_work), copied to the host (synchronises the plan's stream).
int work_to_host(const Plan *pl, std::vector<int32_t> &work);
int wave_occupancy(const Plan *pl, int *wave_ctas, int *cheb_ctas);
const void *batch_kernel(int prec);
int launch_coop(const void *fn, int grid, size_t smem, void **args, cudaStream_t st, int threads = kWaveThreads);

inline bool is_f64_vec(int prec) { return prec == MPK_F64 || prec == MPK_F64_DF; }
inline int elem_bytes_of(const Plan *pl) { return is_f64_vec(pl->prec) ? 8 : 4; }
inline int wave_threads(const Plan *pl) { return pl->resident ? kResThreads : (pl->wave_warps + 1) * 32; }
inline int cheb_threads(const Plan *pl) {
    if (pl->resident) return kResThreads;
    return pl->prec == MPK_F64 && pl->nrhs == 1 ? (kFp64Warps + 1) * 32 : kWaveThreads;   // see k_cheb_wave
}

}  // namespace mpk

struct mpk_plan_s {
    mpk::Plan pl;
};

// ---------------------------------------------------------------- device helpers
namespace mpk {

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int32_t ld_relaxed_s32(const int32_t *p) {
    int32_t v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(uint32_t *p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void fence_acq_rel_gpu() {
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
}

}  // namespace mpk
