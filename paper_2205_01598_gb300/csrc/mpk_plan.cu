// Plan construction of the level-blocked MPK: levels (Eq. 3), renumbering
// (Sec. 4.1), level groups (Eq. 5), packed SELL-32 matrix and the
// dependency ranges of the (level group, power) wavefront (Fig. 5, Sec. 4.3).
#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstring>
#include <mutex>

#include "mpk_internal.cuh"

namespace mpk {


int cuda_status(cudaError_t e, const char *what, int line) {
    (void)cudaGetLastError();
    if (getenv("MPK_DEBUG")) fprintf(stderr, "mpk: %s failed at line %d: %s\n", what, line, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? MPK_ERR_OOM : MPK_ERR_CUDA;
}

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

// ---------------------------------------------------------------- scans
template <typename T>
__device__ T block_exclusive_scan(T v, T *warp_sums, T *total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[w] = x;
    __syncthreads();
    if (w == 0) {
        T s = lane < nw ? warp_sums[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) warp_sums[lane] = s;
    }
    __syncthreads();
    T before = (w > 0 ? warp_sums[w - 1] : T(0)) + x - v;
    if (total) *total = warp_sums[nw - 1];
    __syncthreads();
    return before;
}

template <typename T>
__global__ void k_scan_reduce(const T *in, int64_t n, T *sums) {
    __shared__ T ws[32];
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    T s = 0;
    for (int i = 0; i < kScanItems; i++)
        if (base + i < n) s += in[base + i];
    T tot;
    block_exclusive_scan<T>(s, ws, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

template <typename T>
__global__ void k_scan_sums(T *sums, int64_t nb, T *grand) {   // one block, in place
    __shared__ T ws[32];
    T carry = 0;
    for (int64_t b0 = 0; b0 < nb; b0 += blockDim.x) {
        int64_t i = b0 + threadIdx.x;
        T v = i < nb ? sums[i] : T(0);
        T tot;
        T ex = block_exclusive_scan<T>(v, ws, &tot);
        if (i < nb) sums[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) *grand = carry;
}

template <typename T>
__global__ void k_scan_apply(const T *in, T *out, int64_t n, const T *sums) {
    __shared__ T ws[32];
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    T vals[kScanItems];
    T s = 0;
    for (int i = 0; i < kScanItems; i++) {
        vals[i] = base + i < n ? in[base + i] : T(0);
        s += vals[i];
    }
    T run = block_exclusive_scan<T>(s, ws, nullptr) + sums[blockIdx.x];
    for (int i = 0; i < kScanItems; i++) {
        if (base + i < n) out[base + i] = run;
        run += vals[i];
    }
}

template <typename T>
int exclusive_scan(const T *in, T *out, int64_t n, cudaStream_t st, T *total) {
    int64_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb < 1) nb = 1;
    T *sums = nullptr;
    MPK_CUDA(cudaMallocAsync((void **)&sums, sizeof(T) * (size_t)(nb + 1), st));
    k_scan_reduce<T><<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, sums);
    k_scan_sums<T><<<1, 1024, 0, st>>>(sums, nb, sums + nb);
    k_scan_apply<T><<<(unsigned)nb, kScanThreads, 0, st>>>(in, out, n, sums);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && total) e = cudaMemcpyAsync(total, sums + nb, sizeof(T), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && total) e = cudaStreamSynchronize(st);
    cudaFreeAsync(sums, st);
    if (e != cudaSuccess) return cuda_status(e, "scan", __LINE__);
    return MPK_OK;
}

// ---------------------------------------------------------------- validation
__global__ void k_validate(int32_t n, int64_t nnz, const int32_t *rp, const int32_t *col, int32_t *bad) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r > n) return;
    if (r == 0 && rp[0] != 0) atomicOr(bad, 1);
    if (r == n) {
        if ((int64_t)rp[n] != nnz) atomicOr(bad, 2);
        return;
    }
    int32_t a = rp[r], b = rp[r + 1];
    if (b < a || a < 0 || (int64_t)b > nnz) {
        atomicOr(bad, 4);
        return;
    }
    for (int32_t e = a; e < b; e++) {
        int32_t c = col[e];
        if (c < 0 || c >= n) {
            atomicOr(bad, 8);
            return;
        }
    }
}

// ---------------------------------------------------------------- transpose pattern
__global__ void k_count_cols(int64_t nnz, const int32_t *col, int32_t *cnt) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[col[e]], 1);
}
__global__ void k_fill_transpose(int32_t n, const int32_t *rp, const int32_t *col, int32_t *fill, int32_t *tcol) {
    int32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    for (int32_t e = rp[r]; e < rp[r + 1]; e++) tcol[atomicAdd(&fill[col[e]], 1)] = r;
}

// ---------------------------------------------------------------- BFS (Eq. 3)
struct BfsCtl {
    unsigned bar_count;    // arrivals at grid barriers (never reset within a launch)
    unsigned unused;
    int cnt[3];            // frontier sizes by grid-barrier round mod 3 (see k_bfs)
    int found[3];          // restart search results, rotating by search round mod 3
    int nlevels;
    int err;
    int narrow_L[3];       // after a turn of one-CTA levels: first level not yet expanded,
    int narrow_start[3];   // and the queue offset of its frontier (by round mod 3)
};

constexpr int kBfsThreads = 1024;   // one CTA per SM
constexpr int kBfsBatch = 8;        // neighbours a lane loads before it tests them
// Levels whose frontier fits one CTA (one vertex per thread) are expanded by
// CTA 0 alone, level after level with __syncthreads between them, while the
// other CTAs wait at the next grid barrier; a turn ends after kBfsNarrowRun
// levels, so that the waits of the others stay short.
constexpr int kBfsNarrowRun = 512;

// Grid-wide barrier of a cooperative launch with a bounded wait.  The
// arrival counter only grows: the b-th barrier of the launch is complete when
// it reaches b * gridDim.x, so an arrival is one atomic add and nothing has to
// be reset or released by the last CTA.  `b` counts the barriers every CTA
// has called (all CTAs call them in the same sequence).
__device__ bool grid_sync(BfsCtl *c, uint32_t &b, uint64_t timeout_ns) {
    __shared__ int s_ok;
    __syncthreads();
    b++;
    if (threadIdx.x == 0) {
        int ok = 1;
        const uint32_t target = b * gridDim.x;
        fence_acq_rel_gpu();   // this CTA's writes before the arrival
        const uint32_t arrived = atomicAdd(&c->bar_count, 1u) + 1u;
        if ((int32_t)(arrived - target) < 0) {
            const uint64_t t0 = global_ns();
            while ((int32_t)(ld_relaxed_u32(&c->bar_count) - target) < 0) {
                if (ld_relaxed_s32(&c->err)) { ok = 0; break; }
                if (global_ns() - t0 > timeout_ns) { atomicCAS(&c->err, 0, (int)MPK_ERR_TIMEOUT); ok = 0; break; }
                __nanosleep(32);
            }
        }
        fence_acq_rel_gpu();   // the other CTAs' writes before this CTA's next reads
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Expands the frontier queue[start, end) of level L: warps warp0,
// warp0 + nwarps, ... take 32 frontier vertices each; a lane loads up to
// kBfsBatch neighbours, then tests them, then claims the unvisited ones with
// a compare-and-swap (so the loads of a batch overlap), and the warp appends
// its claims to the queue after end with one atomic add.
__device__ __forceinline__ void bfs_expand(int64_t start, int64_t end, int64_t warp0, int64_t nwarps, int lane,
                                           const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                                           const int32_t *__restrict__ trp, const int32_t *__restrict__ tcol,
                                           int32_t L, int32_t *level, int32_t *queue, int *next_cnt) {
    for (int64_t base = start + warp0 * 32; base < end; base += nwarps * 32) {
        const int64_t i = base + lane;
        const bool valid = i < end;
        int32_t a0 = 0, da = 0, t0 = 0, dt = 0;
        if (valid) {
            const int32_t u = queue[i];
            a0 = __ldg(rp + u);
            da = __ldg(rp + u + 1) - a0;
            if (trp) {
                t0 = __ldg(trp + u);
                dt = __ldg(trp + u + 1) - t0;
            }
        }
        const int32_t deg = da + dt;
        const int32_t maxdeg = (int32_t)__reduce_max_sync(0xffffffffu, (unsigned)deg);
        for (int32_t j0 = 0; j0 < maxdeg; j0 += kBfsBatch) {
            int32_t v[kBfsBatch];
#pragma unroll
            for (int b = 0; b < kBfsBatch; b++) {
                const int32_t j = j0 + b;
                v[b] = j < deg ? (j < da ? __ldg(col + a0 + j) : __ldg(tcol + t0 + (j - da))) : -1;
            }
            unsigned disc = 0;
#pragma unroll
            for (int b = 0; b < kBfsBatch; b++)
                if (v[b] >= 0 && ld_relaxed_s32(&level[v[b]]) < 0) disc |= 1u << b;
#pragma unroll
            for (int b = 0; b < kBfsBatch; b++)
                if (((disc >> b) & 1u) && atomicCAS(&level[v[b]], -1, L + 1) != -1) disc &= ~(1u << b);
            const int mine = __popc(disc);
            int incl = mine;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const int total = __shfl_sync(0xffffffffu, incl, 31);
            if (total == 0) continue;
            int at = 0;
            if (lane == 31) at = atomicAdd(next_cnt, total);
            at = __shfl_sync(0xffffffffu, at, 31);
            int64_t pos = end + at + (incl - mine);
#pragma unroll
            for (int b = 0; b < kBfsBatch; b++)
                if ((disc >> b) & 1u) queue[pos++] = v[b];
        }
    }
}

// Level-synchronous top-down BFS over the pattern (and its transpose when
// trp != null).  Levels are hop distances from the root; when a level comes
// out empty while vertices remain, the lowest-numbered unvisited vertex
// starts the next level.  level[] must be -1 on entry.  The levels do not
// depend on the order in which a level's vertices are queued or claimed.
//
// Rounds are the stretches between grid barriers (R counts the barriers
// passed).  The frontier size every CTA reads after barrier R is cnt[R % 3];
// during round R only cnt[(R+1) % 3] (the next size) and cnt[(R+2) % 3]
// (cleared for round R+1) are written, so no CTA can overwrite a size
// another CTA has yet to read.  A narrow frontier (at most one vertex per
// thread of a CTA) is expanded by CTA 0 alone for up to kBfsNarrowRun levels
// in one round, counting in shared memory; it hands the state on through the
// round's slots.
__global__ void __launch_bounds__(kBfsThreads) k_bfs(int32_t n, const int32_t *rp, const int32_t *col,
                                                     const int32_t *trp, const int32_t *tcol, int32_t root,
                                                     int32_t *level, int32_t *queue, BfsCtl *c, uint64_t timeout_ns) {
    __shared__ int s_cnt[3];
    const int lane = threadIdx.x & 31;
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gsize = (int64_t)gridDim.x * blockDim.x;
    const int64_t gwarp = gtid >> 5, nwarps = gsize >> 5;
    if (gtid == 0) {
        level[root] = 0;
        queue[0] = root;
        c->cnt[1] = 1;   // read after the first barrier (round 1)
        c->cnt[2] = 0;
        c->found[0] = c->found[1] = c->found[2] = INT_MAX;
    }
    uint32_t nbar = 0;
    if (!grid_sync(c, nbar, timeout_ns)) return;
    uint32_t R = 1;
    int32_t L = 0;
    int64_t start = 0, cursor = 0;
    int round = 0;
    for (;;) {
        int32_t size = ld_relaxed_s32(&c->cnt[R % 3]);
        if (size == 0) {   // component finished: restart at the lowest unvisited vertex
            int32_t f = INT_MAX;
            for (;;) {
                const int slot = round % 3;
                if (gtid == 0) c->found[(round + 1) % 3] = INT_MAX;
                int64_t idx = cursor + gtid;
                if (idx < n && ld_relaxed_s32(&level[idx]) < 0) atomicMin(&c->found[slot], (int)idx);
                if (!grid_sync(c, nbar, timeout_ns)) return;
                R++;
                f = ld_relaxed_s32(&c->found[slot]);
                round++;
                if (f != INT_MAX) break;
                cursor += gsize;
                if (cursor >= n) break;
            }
            if (f == INT_MAX) break;
            cursor = f + 1;
            if (gtid == 0) {
                level[f] = L;
                queue[start] = f;
                atomicExch(&c->cnt[(R + 1) % 3], 1);
                atomicExch(&c->cnt[(R + 2) % 3], 0);
            }
            if (!grid_sync(c, nbar, timeout_ns)) return;
            R++;
            size = 1;
        }
        if (size <= kBfsThreads) {
            // narrow levels: CTA 0 alone, __syncthreads between levels
            if (blockIdx.x == 0) {
                if (threadIdx.x == 0) s_cnt[0] = s_cnt[1] = 0;
                __syncthreads();
                int32_t l = L, sz = size;
                int64_t s0 = start;
                for (int run = 0; run < kBfsNarrowRun; run++) {
                    // level l counts into s_cnt[run % 3]; s_cnt[(run + 1) % 3] is
                    // cleared for the next level (its last reads were before the
                    // previous __syncthreads)
                    if (threadIdx.x == 0) s_cnt[(run + 1) % 3] = 0;
                    const int64_t e = s0 + sz;
                    bfs_expand(s0, e, threadIdx.x >> 5, blockDim.x >> 5, lane, rp, col, trp, tcol, l, level, queue,
                               &s_cnt[run % 3]);
                    __syncthreads();
                    s0 = e;
                    l++;
                    sz = *(volatile int *)&s_cnt[run % 3];
                    if (sz == 0 || sz > kBfsThreads) break;
                }
                if (threadIdx.x == 0) {
                    c->narrow_L[(R + 1) % 3] = l;
                    c->narrow_start[(R + 1) % 3] = (int)s0;
                    atomicExch(&c->cnt[(R + 1) % 3], sz);
                    atomicExch(&c->cnt[(R + 2) % 3], 0);
                }
            }
            if (!grid_sync(c, nbar, timeout_ns)) return;
            R++;
            L = ld_relaxed_s32(&c->narrow_L[R % 3]);
            start = ld_relaxed_s32(&c->narrow_start[R % 3]);
            continue;
        }
        if (gtid == 0) atomicExch(&c->cnt[(R + 2) % 3], 0);
        bfs_expand(start, start + size, gwarp, nwarps, lane, rp, col, trp, tcol, L, level, queue,
                   &c->cnt[(R + 1) % 3]);
        if (!grid_sync(c, nbar, timeout_ns)) return;
        R++;
        start += size;
        L++;
    }
    if (gtid == 0) c->nlevels = L;
}

// Cooperative launch of k_bfs: one CTA per SM.
int launch_bfs(int32_t n, const int32_t *rp, const int32_t *col, const int32_t *trp, const int32_t *tcol, int32_t root,
               int32_t *level, int32_t *queue, BfsCtl *c, uint64_t timeout_ns, int num_sms, cudaStream_t st) {
    int occ = 0;
    MPK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_bfs, kBfsThreads, 0));
    if (occ < 1) return MPK_ERR_CUDA;
    void *args[] = {(void *)&n, (void *)&rp, (void *)&col, (void *)&trp, (void *)&tcol, (void *)&root,
                    (void *)&level, (void *)&queue, (void *)&c, (void *)&timeout_ns};
    MPK_CUDA(cudaLaunchCooperativeKernel((void *)k_bfs, dim3(num_sms), dim3(kBfsThreads), args, 0, st));
    return MPK_OK;
}

// ---------------------------------------------------------------- issue order on the GPU
// The order of order_items for a plan without recursion, one thread per
// item: item (t, k) of sweep s (powers k0..k1) goes to position s*q*T plus,
// over the sweep's powers k', the number of items (t', k') that sort before
// it by (key, k, t), key(t, k) = v(t) + sigma * (k - k0).  Keys of one power
// do not decrease with t, so each count is a binary search (for k' = k it is
// t itself); the keys are rounded as the host rounds them (no contraction).
__global__ void k_issue_order(int32_t T, int32_t p, int32_t q, double sigma, const double *__restrict__ v,
                              int32_t *work) {
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (int64_t)T * p) return;
    const int32_t k = (int32_t)(id / T) + 1, t = (int32_t)(id % T);
    const int32_t s = (k - 1) / q, k0 = s * q + 1, k1 = min(p, k0 + q - 1);
    const double key = __dadd_rn(__ldg(v + t), __dmul_rn(sigma, (double)(k - k0)));
    int64_t pos = (int64_t)s * q * T;
    for (int32_t kk = k0; kk <= k1; kk++) {
        if (kk == k) {
            pos += t;
            continue;
        }
        const double sh = __dmul_rn(sigma, (double)(kk - k0));
        int32_t lo = 0, hi = T;   // first t' that sorts after (t, k)
        while (lo < hi) {
            const int32_t mid = (lo + hi) >> 1;
            const double km = __dadd_rn(__ldg(v + mid), sh);
            if (kk < k ? km <= key : km < key) lo = mid + 1;
            else hi = mid;
        }
        pos += lo;
    }
    work[pos] = (t << 8) | k;
}

// ---------------------------------------------------------------- stable radix sort by level
constexpr int kRsThreads = 256, kRsRounds = 16, kRsTile = kRsThreads * kRsRounds;

__global__ void k_rs_hist(const int32_t *keys, int32_t n, int shift, int32_t *hist, int32_t nb) {
    __shared__ int h[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kRsTile;
    for (int i = threadIdx.x; i < kRsTile; i += blockDim.x)
        if (base + i < n) atomicAdd(&h[((uint32_t)keys[base + i] >> shift) & 255u], 1);
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += blockDim.x) hist[(int64_t)d * nb + blockIdx.x] = h[d];
}

// Stable scatter: items keep their input order inside each digit bucket.
__global__ void __launch_bounds__(kRsThreads) k_rs_scatter(const int32_t *kin, const int32_t *vin, int32_t *kout,
                                                           int32_t *vout, int32_t n, int shift,
                                                           const int32_t *hscan, int32_t nb) {
    __shared__ int wc[kRsThreads / 32][257];
    __shared__ int base[256];
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    for (int d = tid; d < 256; d += blockDim.x) base[d] = hscan[(int64_t)d * nb + blockIdx.x];
    for (int r = 0; r < kRsRounds; r++) {
        for (int i = tid; i < (kRsThreads / 32) * 257; i += blockDim.x) (&wc[0][0])[i] = 0;
        __syncthreads();
        int64_t i = (int64_t)blockIdx.x * kRsTile + r * kRsThreads + tid;
        bool valid = i < n;
        int32_t key = valid ? kin[i] : 0;
        int d = valid ? (int)(((uint32_t)key >> shift) & 255u) : 256;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int rank = __popc(peers & ((1u << lane) - 1u));
        if (rank == 0) wc[w][d] = __popc(peers);
        __syncthreads();
        if (tid < 256) {
            int run = base[tid];
            for (int ww = 0; ww < kRsThreads / 32; ww++) {
                int t = wc[ww][tid];
                wc[ww][tid] = run;
                run += t;
            }
            base[tid] = run;
        }
        __syncthreads();
        if (valid) {
            int pos = wc[w][d] + rank;
            kout[pos] = key;
            vout[pos] = vin ? vin[i] : (int32_t)i;
        }
        __syncthreads();
    }
}

__global__ void k_inverse_perm(int32_t n, const int32_t *perm, int32_t *iperm) {
    int32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) iperm[perm[r]] = r;
}

__global__ void k_level_ptr(int32_t n, const int32_t *sorted_level, int32_t *level_ptr, int32_t nlevels) {
    int32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    if (r == 0) {
        level_ptr[0] = 0;
        level_ptr[nlevels] = n;
    } else if (sorted_level[r] != sorted_level[r - 1]) {
        level_ptr[sorted_level[r]] = r;   // levels are consecutive integers
    }
}

// ---------------------------------------------------------------- permuted CRS
__global__ void k_perm_len(int32_t n, const int32_t *rp, const int32_t *perm, int32_t *len) {
    int32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) len[r] = rp[perm[r] + 1] - rp[perm[r]];
}

// Row r of P A P^T = old row perm[r], columns renumbered through iperm and
// put in ascending order (stable).  kPermGroup lanes share a row, so its
// entries are read and written as contiguous runs: a row of at most
// kPermGroup * kPermSlots entries is held in registers and every entry's
// place is its rank among the row's entries (shuffles within the group);
// longer rows fall back to an insertion sort by the group's first lane.
constexpr int kPermGroup = 8, kPermSlots = 8;
__global__ void k_perm_fill(int32_t n, const int32_t *rp, const int32_t *col, const double *val,
                            const int32_t *perm, const int32_t *iperm, const int32_t *prow,
                            int32_t *pcol, double *pval) {
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t r = gid / kPermGroup;
    const int sub = (int)(gid % kPermGroup), lane = threadIdx.x & 31;
    const unsigned gmask = ((1u << kPermGroup) - 1u) << (lane & ~(kPermGroup - 1));
    if (r >= n) return;   // whole groups (kPermGroup divides 32 and the block size)
    const int32_t o = __ldg(perm + r), a = __ldg(rp + o), len = __ldg(rp + o + 1) - a, base = __ldg(prow + r);
    if (len <= kPermGroup * kPermSlots) {
        int32_t c[kPermSlots];
#pragma unroll
        for (int k = 0; k < kPermSlots; k++) {
            const int32_t j = sub + k * kPermGroup;
            c[k] = j < len ? __ldg(iperm + __ldg(col + a + j)) : INT_MAX;
        }
        int32_t rank[kPermSlots] = {};
        const int32_t used = (len + kPermGroup - 1) / kPermGroup;   // slots in use (uniform in the group)
#pragma unroll
        for (int k2 = 0; k2 < kPermSlots; k2++) {
            if (k2 >= used) break;   // uniform in the group
            for (int q = 0; q < kPermGroup; q++) {
                const int32_t cq = __shfl_sync(gmask, c[k2], q, kPermGroup);
                const int32_t jq = q + k2 * kPermGroup;
#pragma unroll
                for (int k = 0; k < kPermSlots; k++) {
                    const int32_t j = sub + k * kPermGroup;
                    rank[k] += (cq < c[k]) || (cq == c[k] && jq < j);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < kPermSlots; k++) {
            const int32_t j = sub + k * kPermGroup;
            if (j < len) {
                pcol[base + rank[k]] = c[k];
                pval[base + rank[k]] = __ldg(val + a + j);
            }
        }
        return;
    }
    if (sub != 0) return;
    for (int32_t j = 0; j < len; j++) {
        int32_t cc = iperm[col[a + j]];
        double v = val[a + j];
        int32_t k = base + j;
        while (k > base && pcol[k - 1] > cc) {
            pcol[k] = pcol[k - 1];
            pval[k] = pval[k - 1];
            k--;
        }
        pcol[k] = cc;
        pval[k] = v;
    }
}

// Row statistics of P A P^T for the planner's features: sum and sum of
// squares of row lengths, the longest row, and the sum / maximum of the
// distance |column - row| (bandwidth of the level-ordered matrix).
__global__ void k_row_stats(int32_t n, const int32_t *prow, const int32_t *pcol, unsigned long long *acc) {
    __shared__ unsigned long long s[5];
    if (threadIdx.x < 5) s[threadIdx.x] = 0;
    __syncthreads();
    unsigned long long len_sum = 0, len_sq = 0, len_max = 0, dist_sum = 0, dist_max = 0;
    for (int32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        const unsigned long long len = (unsigned long long)(prow[r + 1] - prow[r]);
        len_sum += len;
        len_sq += len * len;
        len_max = len > len_max ? len : len_max;
        for (int32_t e = prow[r]; e < prow[r + 1]; e++) {
            const unsigned long long d = (unsigned long long)abs(pcol[e] - r);
            dist_sum += d;
            dist_max = d > dist_max ? d : dist_max;
        }
    }
    atomicAdd(&s[0], len_sum);
    atomicAdd(&s[1], len_sq);
    atomicMax(&s[2], len_max);
    atomicAdd(&s[3], dist_sum);
    atomicMax(&s[4], dist_max);
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicAdd(&acc[0], s[0]);
        atomicAdd(&acc[1], s[1]);
        atomicMax(&acc[2], s[2]);
        atomicAdd(&acc[3], s[3]);
        atomicMax(&acc[4], s[4]);
    }
}

__global__ void k_level_nnz(int32_t nlevels, const int32_t *level_ptr, const int32_t *prow, int64_t *lnnz) {
    int32_t l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l < nlevels) lnnz[l] = (int64_t)prow[level_ptr[l + 1]] - prow[level_ptr[l]];
}

// 1 if every off-diagonal value is exactly a bfloat16
__global__ void k_bf16_exact(int32_t n, const int32_t *prow, const int32_t *pcol, const double *pval, int32_t *not_exact) {
    int32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    for (int32_t e = prow[r]; e < prow[r + 1]; e++) {
        if (pcol[e] == r) continue;
        double v = pval[e];
        float f = (float)v;
        __nv_bfloat16 b = __float2bfloat16_rn(f);
        if ((double)__bfloat162float(b) != v) { atomicOr(not_exact, 1); return; }
    }
}

// Double-float plans: flags[0] = 1 if some value is not exactly an FP32
// number, flags[1] = 1 if some nonzero |value| lies outside [2^-60, 2^60];
// *rowsum_bits = the largest row sum of |a_ij| (the bit pattern of a
// non-negative double orders like the double, so an integer maximum works).
__global__ void k_df_values(int32_t n, const int32_t *prow, const double *pval, int32_t *flags,
                            unsigned long long *rowsum_bits) {
    const int32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    double sum = 0.0;
    int32_t inexact = 0, out = 0;
    for (int32_t e = prow[r]; e < prow[r + 1]; e++) {
        const double v = pval[e], av = fabs(v);
        sum += av;
        inexact |= (double)(float)v != v;
        out |= v != 0.0 && !(av >= 0x1p-60 && av <= 0x1p60);
    }
    if (inexact) atomicOr(flags, 1);
    if (out) atomicOr(flags + 1, 1);
    atomicMax(rowsum_bits, (unsigned long long)__double_as_longlong(sum));
}

// ---------------------------------------------------------------- packing
// Entries of row r that go into the SELL arrays (all of them, or all but the
// diagonal when the diagonal is stored apart).
__device__ __forceinline__ int32_t packed_len(int32_t r, const int32_t *prow, const int32_t *pcol, int split_diag) {
    int32_t len = prow[r + 1] - prow[r];
    if (split_diag)
        for (int32_t e = prow[r]; e < prow[r + 1]; e++) len -= (pcol[e] == r);
    return len;
}

__global__ void k_row_len(int32_t n, const int32_t *prow, const int32_t *pcol, int split_diag, int32_t *len) {
    int32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) len[r] = packed_len(r, prow, pcol, split_diag);
}

// SELL-C-sigma with sigma = the tile: the rows of each tile are put in
// order of decreasing packed length (ties: ascending row) so that a chunk
// holds rows of similar length; row_map[position] = row.  One CTA per tile.
__global__ void k_sort_tile_rows(int32_t n_tiles, const int32_t *tile_row, const int32_t *len, int32_t *row_map) {
    extern __shared__ int32_t s_len[];
    const int32_t t = blockIdx.x;
    if (t >= n_tiles) return;
    const int32_t r0 = tile_row[t], nr = tile_row[t + 1] - r0;
    for (int32_t i = threadIdx.x; i < nr; i += blockDim.x) s_len[i] = len[r0 + i];
    __syncthreads();
    for (int32_t i = threadIdx.x; i < nr; i += blockDim.x) {
        const int32_t li = s_len[i];
        int32_t rank = 0;
        for (int32_t q = 0; q < nr; q++) rank += (s_len[q] > li) || (s_len[q] == li && q < i);
        row_map[r0 + rank] = r0 + i;
    }
}

__global__ void k_chunk_width(int32_t n_chunks, const int32_t *chunk_row, const int32_t *len, const int32_t *row_map,
                              int64_t *cw) {
    int32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_chunks) return;
    int32_t w = 0;
    for (int32_t q = chunk_row[c]; q < chunk_row[c + 1]; q++) w = max(w, len[row_map ? row_map[q] : q]);
    cw[c] = (int64_t)w * kChunk;
}

template <typename MT>
__device__ __forceinline__ MT cvt_val(double v);
template <> __device__ __forceinline__ double cvt_val<double>(double v) { return v; }
template <> __device__ __forceinline__ float cvt_val<float>(double v) { return (float)v; }
template <> __device__ __forceinline__ __nv_bfloat16 cvt_val<__nv_bfloat16>(double v) {
    return __float2bfloat16_rn((float)v);
}
// double-float pair: hi = v rounded to FP32, lo = the rest rounded to FP32
template <> __device__ __forceinline__ float2 cvt_val<float2>(double v) {
    const float hi = (float)v;
    return make_float2(hi, (float)(v - (double)hi));
}

// Column-major SELL-32: entry j of lane l of chunk c sits at off[c] + 32*j + l.
template <typename MT>
__global__ void k_pack(int32_t n_chunks, const int32_t *chunk_row, const int64_t *chunk_off, const int32_t *row_map,
                       const int32_t *prow, const int32_t *pcol, const double *pval, int split_diag, int32_t *scol,
                       MT *sval, float *diag) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int32_t c = (int32_t)(g / kChunk);
    int lane = (int)(g % kChunk);
    if (c >= n_chunks) return;
    int64_t off = chunk_off[c] + lane;
    int32_t w = (int32_t)((chunk_off[c + 1] - chunk_off[c]) / kChunk);
    const int32_t pos = chunk_row[c] + lane;
    int32_t j = 0;
    if (pos < chunk_row[c + 1]) {
        const int32_t r = row_map ? row_map[pos] : pos;
        double d = 0.0;
        for (int32_t e = prow[r]; e < prow[r + 1]; e++) {
            if (split_diag && pcol[e] == r) { d += pval[e]; continue; }
            scol[off + (int64_t)j * kChunk] = pcol[e];
            sval[off + (int64_t)j * kChunk] = cvt_val<MT>(pval[e]);
            j++;
        }
        if (split_diag) diag[r] = (float)d;
    }
    for (; j < w; j++) {
        scol[off + (int64_t)j * kChunk] = -1;
        sval[off + (int64_t)j * kChunk] = cvt_val<MT>(0.0);
    }
}

// ---------------------------------------------------------------- dependency ranges
__global__ void k_tile_of_row(int32_t n_tiles, const int32_t *tile_row, int32_t *tor) {
    int32_t t = blockIdx.x;
    if (t >= n_tiles) return;
    for (int32_t r = tile_row[t] + threadIdx.x; r < tile_row[t + 1]; r += blockDim.x) tor[r] = t;
}

// Tile t at power k reads y_{k-1} on the columns of its rows; the tiles that
// hold those rows form a contiguous range (Eq. 4: columns of a level lie in
// the neighbouring levels).  For a non-symmetric pattern the range is closed
// under transposition so that "t reads u" implies "u reads t".
__global__ void k_deps(int32_t n, const int32_t *prow, const int32_t *pcol, const int32_t *tor, int symmetric,
                       int32_t *lo, int32_t *hi) {
    const int32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = r < n;
    int32_t t = valid ? tor[r] : -1, mn = t, mx = t;
    if (valid) {
        for (int32_t e = prow[r]; e < prow[r + 1]; e++) {
            int32_t u = tor[pcol[e]];
            mn = min(mn, u);
            mx = max(mx, u);
            if (!symmetric) {
                atomicMin(&lo[u], t);
                atomicMax(&hi[u], t);
            }
        }
    }
    // the rows of a warp lie in one or two tiles: one atomic pair per tile
    const unsigned same = __match_any_sync(0xffffffffu, t);
    mn = __reduce_min_sync(same, mn);   // rows past n form their own group (t = -1)
    mx = __reduce_max_sync(same, mx);
    if (valid && (threadIdx.x & 31) == __ffs(same) - 1) {
        atomicMin(&lo[t], mn);
        atomicMax(&hi[t], mx);
    }
}

__global__ void k_widen(int32_t n, const int32_t *a, int64_t *b) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = a[i];
}

__global__ void k_tile_off(int32_t n_tiles, const int32_t *tile_chunk, const int64_t *chunk_off, int64_t *tile_off) {
    int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t <= n_tiles) tile_off[t] = chunk_off[tile_chunk[t]];
}

// Chunk records {first row, rows, first packed entry / 32, width}: the four
// facts a warp needs about a chunk, in one 16-byte load.
__global__ void k_chunk_rec(int32_t n_chunks, const int32_t *chunk_row, const int64_t *chunk_off, int4 *rec) {
    int32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_chunks) return;
    const int32_t r0 = chunk_row[c];
    const int64_t o0 = chunk_off[c];
    rec[c] = make_int4(r0, chunk_row[c + 1] - r0, (int32_t)(o0 / kChunk), (int32_t)((chunk_off[c + 1] - o0) / kChunk));
}

__global__ void k_fill_i32(int32_t *p, int64_t n, int32_t v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = v;
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

// Temporary device buffers of the planner, freed on scope exit.
// ---------------------------------------------------------------- recursion (Sec. 4.4)
// The rows being refined are the runs of bulky level groups: run i covers
// rows run_a[i] .. and the compacted indices run_base[i] .. run_base[i+1]-1.
// comp_row[j] = the row of compacted index j; run_of[r] = run of row r (-1 if
// none, preset), comp_of[r] = compacted index of row r.
__global__ void k_runs_index(int32_t nruns, const int32_t *run_a, const int32_t *run_base, int32_t m,
                             int32_t *comp_row, int32_t *run_of, int32_t *comp_of) {
    const int32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    int32_t lo = 0, hi = nruns - 1;   // the run with run_base[i] <= j < run_base[i+1]
    while (lo < hi) {
        const int32_t mid = (lo + hi + 1) >> 1;
        if (run_base[mid] <= j) lo = mid;
        else hi = mid - 1;
    }
    const int32_t r = run_a[lo] + (j - run_base[lo]);
    comp_row[j] = r;
    run_of[r] = lo;
    comp_of[r] = j;
}

// The subgraph each run induces: compacted vertex j keeps the columns of its
// row that lie in the same run, as compacted indices (the stored order).
__global__ void k_sub_len(int32_t m, const int32_t *comp_row, const int32_t *prow, const int32_t *pcol,
                          const int32_t *run_of, int32_t *len) {
    const int32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    const int32_t r = comp_row[j], ri = run_of[r];
    int32_t c = 0;
    for (int32_t e = prow[r]; e < prow[r + 1]; e++) c += run_of[pcol[e]] == ri;
    len[j] = c;
}
__global__ void k_sub_fill(int32_t m, const int32_t *comp_row, const int32_t *prow, const int32_t *pcol,
                           const int32_t *run_of, const int32_t *comp_of, const int32_t *srow, int32_t *scol) {
    const int32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    const int32_t r = comp_row[j], ri = run_of[r];
    int32_t o = srow[j];
    for (int32_t e = prow[r]; e < prow[r + 1]; e++)
        if (run_of[pcol[e]] == ri) scol[o++] = comp_of[pcol[e]];
}

// Renumbering of the runs by sub-level: ord[j] = the compacted vertex at
// position j of the stable sort by sub-level (runs stay in their blocks,
// their sub-levels being numbered run after run), so the row of compacted
// index j receives the vertex of row comp_row[ord[j]].
__global__ void k_apply_sub_order(int32_t m, const int32_t *ord, const int32_t *comp_row, const int32_t *perm_in,
                                  int32_t *perm_out) {
    const int32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < m) perm_out[comp_row[j]] = perm_in[comp_row[ord[j]]];
}

// Temporary device memory of one planning call: buffers are carved out of
// slabs (256-byte aligned) and released together when planning returns, so
// planning makes a few allocations instead of one per buffer.  The first slab
// is sized by `hint`; a request that does not fit gets a slab of its own size.
struct Scratch {
    std::vector<void *> slabs;
    char *cur = nullptr;
    size_t left = 0, hint = 0;
    ~Scratch() {
        for (void *p : slabs) cudaFree(p);
    }
    template <typename T>
    int alloc(T **p, size_t count) {
        const size_t bytes = (std::max<size_t>(count, 1) * sizeof(T) + 255) & ~(size_t)255;
        if (bytes > left) {
            const size_t size = std::max(bytes, hint);
            hint = 0;
            char *q = nullptr;
            const int rc = dev_alloc<char>(nullptr, &q, size);
            if (rc != MPK_OK) {
                *p = nullptr;
                return rc;
            }
            slabs.push_back(q);
            cur = q;
            left = size;
        }
        *p = (T *)cur;
        cur += bytes;
        left -= bytes;
        return MPK_OK;
    }
};

#define MPK_TRY(x)                 \
    do {                           \
        int _rc = (x);             \
        if (_rc != MPK_OK) return _rc; \
    } while (0)

void free_plan(Plan *pl) {
    void *ps[] = {pl->d_perm, pl->d_iperm, pl->d_level, pl->d_level_ptr, pl->d_group_ptr, pl->d_chunk_row,
                  pl->d_chunk_off, pl->d_tile_chunk, pl->d_dep_lo, pl->d_dep_hi, pl->d_work, pl->d_pcol,
                  pl->d_pval, pl->d_diag, pl->d_gersh, pl->d_flags, pl->d_bcnt, pl->d_ctl, pl->d_io, pl->d_cheb,
                  pl->d_tile_off, pl->d_work_rem, pl->d_row_map, pl->d_chunk_rec, pl->d_shadow, pl->d_kry};
    for (void *p : ps)
        if (p) cudaFree(p);
    for (cudaEvent_t e : pl->io_ev)
        if (e) cudaEventDestroy(e);
    if (pl->copy_stream) cudaStreamDestroy(pl->copy_stream);
}

// Stable LSD radix sort (8-bit digits) of the n keys in kA (values in
// [0, maxkey]); on return kA holds the sorted keys and vA the input position
// of each (ties keep their input order).  kB, vB and hist (256 counters per
// tile of kRsTile keys) are scratch.
static int radix_sort_keys(int32_t n, int32_t maxkey, int32_t *&kA, int32_t *&kB, int32_t *&vA, int32_t *&vB,
                           int32_t *hist, cudaStream_t st) {
    const int32_t nb = (int32_t)((n + kRsTile - 1) / kRsTile);
    int passes = 0;
    for (uint32_t m = (uint32_t)maxkey; m; m >>= 8) passes++;
    if (passes == 0) passes = 1;
    bool first = true;
    for (int ps = 0; ps < passes; ps++) {
        k_rs_hist<<<nb, kRsThreads, 0, st>>>(kA, n, 8 * ps, hist, nb);
        MPK_TRY(exclusive_scan<int32_t>(hist, hist, (int64_t)256 * nb, st, nullptr));
        k_rs_scatter<<<nb, kRsThreads, 0, st>>>(kA, first ? nullptr : vA, kB, vB, n, 8 * ps, hist, nb);
        first = false;
        std::swap(kA, kB);
        std::swap(vA, vB);
    }
    return MPK_OK;
}

// P A P^T with sorted rows for the permutation pl->d_perm (and its inverse).
static int permute_matrix(Plan *pl, const mpk_csr *A, int32_t *prow, int32_t *plen, int32_t *pcol, double *pval,
                          cudaStream_t st) {
    const int32_t n = pl->n;
    k_inverse_perm<<<blocks_for(n, 256), 256, 0, st>>>(n, pl->d_perm, pl->d_iperm);
    MPK_CUDA(cudaMemsetAsync(plen + n, 0, sizeof(int32_t), st));
    k_perm_len<<<blocks_for(n, 256), 256, 0, st>>>(n, A->rowptr, pl->d_perm, plen);
    MPK_TRY(exclusive_scan<int32_t>(plen, prow, (int64_t)n + 1, st, nullptr));
    k_perm_fill<<<blocks_for((int64_t)n * kPermGroup, 256), 256, 0, st>>>(n, A->rowptr, A->col, A->val, pl->d_perm,
                                                                          pl->d_iperm, prow,
                                                    pcol, pval);
    MPK_CUDA(cudaGetLastError());
    return MPK_OK;
}

// Sec. 4.4: up to s_max stages, every maximal run of consecutive bulky level
// groups (a single level with (p+1) * weight >= f * C) is refined by the
// levels of the subgraph it induces: one cooperative BFS over the union of
// the runs' subgraphs (its components come run after run in the current
// numbering, so the restart rule roots each run at its first vertex, as a
// separate search per run would), a stable sort of the runs' rows by
// sub-level, and Eq. 5 groups of the sub-levels.  Updates the permutation,
// P A P^T (prow, plen, pcol, pval), the finest levels pl->h_level_ptr with
// their stored entries lnnz, the groups pl->h_group_ptr and their stages.
static int refine_levels(Plan *pl, const mpk_csr *A, int32_t p, int32_t s_max, double bpe, double budget,
                         int32_t *prow, int32_t *plen, int32_t *pcol, double *pval, std::vector<int64_t> &lnnz,
                         int32_t *kA, int32_t *kB, int32_t *vA, int32_t *vB, int32_t *hist, Scratch &S,
                         cudaStream_t st, uint64_t timeout_ns) {
    const int32_t n = pl->n;
    std::vector<int32_t> &lp = pl->h_level_ptr, &gp = pl->h_group_ptr;
    pl->h_group_stage.assign(gp.size() - 1, 0);
    int32_t *run_of, *comp_of, *comp_row, *slen, *srow, *scol, *slev, *queue, *perm2, *d_meta, *d_lp;
    BfsCtl *bc;
    MPK_TRY(S.alloc(&run_of, (size_t)n));
    MPK_TRY(S.alloc(&comp_of, (size_t)n));
    MPK_TRY(S.alloc(&comp_row, (size_t)n));
    MPK_TRY(S.alloc(&slen, (size_t)n + 1));
    MPK_TRY(S.alloc(&srow, (size_t)n + 1));
    MPK_TRY(S.alloc(&scol, (size_t)std::max<int64_t>(1, A->nnz)));
    MPK_TRY(S.alloc(&slev, (size_t)n));
    MPK_TRY(S.alloc(&queue, (size_t)n));
    MPK_TRY(S.alloc(&perm2, (size_t)n));
    MPK_TRY(S.alloc(&d_meta, 2 * (size_t)n + 2));
    MPK_TRY(S.alloc(&d_lp, (size_t)n + 1));
    MPK_TRY(S.alloc(&bc, 1));
    for (int32_t s = 0; s < s_max; s++) {
        const int32_t G = (int32_t)gp.size() - 1;
        auto bulky = [&](int32_t g) {
            return gp[g + 1] - gp[g] == 1 && (double)(p + 1) * (double)lnnz[gp[g]] * bpe >= budget;
        };
        std::vector<int32_t> rg0, rg1, run_a, run_base(1, 0);
        for (int32_t g = 0; g < G;) {
            if (!bulky(g)) { g++; continue; }
            int32_t g1 = g;
            while (g1 < G && bulky(g1)) g1++;
            rg0.push_back(g);
            rg1.push_back(g1);
            run_a.push_back(lp[gp[g]]);
            run_base.push_back(run_base.back() + (lp[gp[g1]] - lp[gp[g]]));
            g = g1;
        }
        const int32_t nruns = (int32_t)rg0.size();
        if (nruns == 0) break;
        const int32_t m = run_base.back();
        // the union of the runs' induced subgraphs, compacted
        MPK_CUDA(cudaMemcpyAsync(d_meta, run_a.data(), sizeof(int32_t) * nruns, cudaMemcpyHostToDevice, st));
        MPK_CUDA(cudaMemcpyAsync(d_meta + nruns, run_base.data(), sizeof(int32_t) * (nruns + 1), cudaMemcpyHostToDevice,
                                 st));
        MPK_CUDA(cudaMemsetAsync(run_of, 0xff, sizeof(int32_t) * (size_t)n, st));
        k_runs_index<<<blocks_for(m, 256), 256, 0, st>>>(nruns, d_meta, d_meta + nruns, m, comp_row, run_of, comp_of);
        k_sub_len<<<blocks_for(m, 256), 256, 0, st>>>(m, comp_row, prow, pcol, run_of, slen);
        MPK_CUDA(cudaMemsetAsync(slen + m, 0, sizeof(int32_t), st));
        MPK_TRY(exclusive_scan<int32_t>(slen, srow, (int64_t)m + 1, st, nullptr));
        k_sub_fill<<<blocks_for(m, 256), 256, 0, st>>>(m, comp_row, prow, pcol, run_of, comp_of, srow, scol);
        // Eq. 3 on it, rooted at compacted vertex 0 (the first run's first row)
        MPK_CUDA(cudaMemsetAsync(slev, 0xff, sizeof(int32_t) * (size_t)m, st));
        MPK_CUDA(cudaMemsetAsync(bc, 0, sizeof(BfsCtl), st));
        MPK_TRY(launch_bfs(m, srow, scol, nullptr, nullptr, 0, slev, queue, bc, timeout_ns, pl->num_sms, st));
        BfsCtl h_bc;
        MPK_CUDA(cudaMemcpyAsync(&h_bc, bc, sizeof(BfsCtl), cudaMemcpyDeviceToHost, st));
        MPK_CUDA(cudaStreamSynchronize(st));
        if (h_bc.err) return h_bc.err;
        const int32_t Ls = h_bc.nlevels;
        if (Ls < 1 || Ls > m) return MPK_ERR_CUDA;
        // stable sort of the compacted vertices by sub-level; new permutation
        MPK_CUDA(cudaMemcpyAsync(kA, slev, sizeof(int32_t) * (size_t)m, cudaMemcpyDeviceToDevice, st));
        MPK_TRY(radix_sort_keys(m, Ls - 1, kA, kB, vA, vB, hist, st));
        k_level_ptr<<<blocks_for(m, 256), 256, 0, st>>>(m, kA, d_lp, Ls);
        MPK_CUDA(cudaMemcpyAsync(perm2, pl->d_perm, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, st));
        k_apply_sub_order<<<blocks_for(m, 256), 256, 0, st>>>(m, vA, comp_row, pl->d_perm, perm2);
        MPK_CUDA(cudaMemcpyAsync(pl->d_perm, perm2, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, st));
        MPK_TRY(permute_matrix(pl, A, prow, plen, pcol, pval, st));
        std::vector<int32_t> slp((size_t)Ls + 1);
        MPK_CUDA(cudaMemcpyAsync(slp.data(), d_lp, sizeof(int32_t) * ((size_t)Ls + 1), cudaMemcpyDeviceToHost, st));
        MPK_CUDA(cudaStreamSynchronize(st));
        // the new finest levels: the runs' levels replaced by their sub-levels
        // (run i owns the sub-levels starting in [run_base[i], run_base[i+1]))
        std::vector<int32_t> nlp, ngp, ngs, run_l0(nruns), run_l1(nruns);
        int32_t q = 0, sl = 0;
        for (int32_t g = 0; g < G;) {
            if (q < nruns && g == rg0[q]) {
                run_l0[q] = (int32_t)nlp.size();
                for (; sl < Ls && slp[sl] < run_base[q + 1]; sl++) nlp.push_back(run_a[q] + (slp[sl] - run_base[q]));
                run_l1[q] = (int32_t)nlp.size();
                ngp.push_back(-1 - q);   // placeholder: the run's groups come after its weights are known
                ngs.push_back(s + 1);
                g = rg1[q++];
                continue;
            }
            ngp.push_back((int32_t)nlp.size());
            ngs.push_back(pl->h_group_stage[g]);
            for (int32_t l = gp[g]; l < gp[g + 1]; l++) nlp.push_back(lp[l]);
            g++;
        }
        const int32_t L2 = (int32_t)nlp.size();
        nlp.push_back(n);
        // stored entries of the new levels
        int64_t *d_ln;
        MPK_TRY(S.alloc(&d_ln, (size_t)L2));
        MPK_CUDA(cudaMemcpyAsync(d_lp, nlp.data(), sizeof(int32_t) * ((size_t)L2 + 1), cudaMemcpyHostToDevice, st));
        k_level_nnz<<<blocks_for(L2, 256), 256, 0, st>>>(L2, d_lp, prow, d_ln);
        std::vector<int64_t> nln((size_t)L2);
        MPK_CUDA(cudaMemcpyAsync(nln.data(), d_ln, sizeof(int64_t) * (size_t)L2, cudaMemcpyDeviceToHost, st));
        MPK_CUDA(cudaStreamSynchronize(st));
        // Eq. 5 groups of each run's sub-levels, in place of its placeholder
        std::vector<int32_t> fgp, fgs;
        for (size_t k = 0; k < ngp.size(); k++) {
            if (ngp[k] >= 0) {
                fgp.push_back(ngp[k]);
                fgs.push_back(ngs[k]);
                continue;
            }
            const int32_t r = -1 - ngp[k];
            for (int32_t s0 = run_l0[r]; s0 < run_l1[r];) {
                double acc = (double)nln[s0] * bpe;
                int32_t e = s0 + 1;
                while (e < run_l1[r] && (double)(p + 1) * (acc + (double)nln[e] * bpe) < budget) {
                    acc += (double)nln[e] * bpe;
                    e++;
                }
                fgp.push_back(s0);
                fgs.push_back(s + 1);
                s0 = e;
            }
        }
        fgp.push_back(L2);
        lp = std::move(nlp);
        lnnz = std::move(nln);
        gp = std::move(fgp);
        pl->h_group_stage = std::move(fgs);
        pl->rec_stages = s + 1;
    }
    return MPK_OK;
}

int build_plan(Plan *pl, const mpk_csr *A, int32_t p, const mpk_opts *o) {
    const auto t_start = std::chrono::steady_clock::now();
    cudaStream_t st = (cudaStream_t)o->stream;
    pl->stream = st;
    pl->n = A->n;
    pl->nnz = A->nnz;
    pl->p = p;
    const int32_t q = o->sweep > 0 ? std::min(o->sweep, p) : p;   // p_m of Eq. 5
    pl->sweep = q;
    pl->nrhs = o->nrhs;
    pl->prec = o->prec;
    pl->safety_f = o->safety_f;
    pl->timeout_s = o->timeout_s > 0 ? o->timeout_s : 2.0;
    const uint64_t timeout_ns = (uint64_t)(pl->timeout_s * 1e9);
    auto t_mark = t_start;
    auto mark = [&](int phase) {
        const auto now = std::chrono::steady_clock::now();
        pl->phase_ms[phase] += std::chrono::duration<double, std::milli>(now - t_mark).count();
        t_mark = now;
    };
    MPK_CUDA(cudaGetDevice(&pl->device));
    struct {
        int multiProcessorCount, l2CacheSize, sharedMemPerBlockOptin, sharedMemPerMultiprocessor;
    } prop;   // the four attributes planning needs (a full property query costs milliseconds)
    MPK_CUDA(cudaDeviceGetAttribute(&prop.multiProcessorCount, cudaDevAttrMultiProcessorCount, pl->device));
    MPK_CUDA(cudaDeviceGetAttribute(&prop.l2CacheSize, cudaDevAttrL2CacheSize, pl->device));
    MPK_CUDA(cudaDeviceGetAttribute(&prop.sharedMemPerBlockOptin, cudaDevAttrMaxSharedMemoryPerBlockOptin, pl->device));
    MPK_CUDA(cudaDeviceGetAttribute(&prop.sharedMemPerMultiprocessor, cudaDevAttrMaxSharedMemoryPerMultiprocessor,
                                    pl->device));
    pl->num_sms = prop.multiProcessorCount;
    pl->cache_bytes = o->cache_bytes > 0 ? o->cache_bytes : (double)prop.l2CacheSize;
    const int32_t n = A->n;
    const int64_t nnz = A->nnz;
    Scratch S;
    // what the buffers below take for n rows and nnz entries (transposed
    // pattern included when symmetry is not promised)
    S.hint = (size_t)(64 + (A->assume_symmetric ? 0 : 12)) * (size_t)A->n +
             (size_t)(12 + (A->assume_symmetric ? 0 : 4)) * (size_t)A->nnz + ((size_t)1 << 20);

    // 1. validation of the CRS arrays on the device
    int32_t *d_bad;
    MPK_TRY(S.alloc(&d_bad, 4));
    MPK_CUDA(cudaMemsetAsync(d_bad, 0, 4 * sizeof(int32_t), st));
    k_validate<<<blocks_for((int64_t)n + 1, 256), 256, 0, st>>>(n, nnz, A->rowptr, A->col, d_bad);
    int32_t h_bad = 0;
    MPK_CUDA(cudaMemcpyAsync(&h_bad, d_bad, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    MPK_CUDA(cudaStreamSynchronize(st));
    if (h_bad) return MPK_ERR_INVALID;
    mark(0);

    // 2. transposed pattern when symmetry is not promised
    int32_t *d_trp = nullptr, *d_tcol = nullptr;
    if (!A->assume_symmetric) {
        int32_t *cnt;
        MPK_TRY(S.alloc(&cnt, (size_t)n + 1));
        MPK_TRY(S.alloc(&d_trp, (size_t)n + 1));
        MPK_TRY(S.alloc(&d_tcol, (size_t)nnz));
        MPK_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * ((size_t)n + 1), st));
        k_count_cols<<<std::min<unsigned>(blocks_for(nnz, 256), 4096), 256, 0, st>>>(nnz, A->col, cnt);
        MPK_TRY(exclusive_scan<int32_t>(cnt, d_trp, (int64_t)n + 1, st, nullptr));
        MPK_CUDA(cudaMemcpyAsync(cnt, d_trp, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, st));
        k_fill_transpose<<<blocks_for(n, 256), 256, 0, st>>>(n, A->rowptr, A->col, cnt, d_tcol);
    }

    // 3. BFS levels (Eq. 3), one cooperative launch
    int32_t *d_queue;
    BfsCtl *d_bc;
    MPK_TRY(dev_alloc(pl, &pl->d_level, (size_t)n));
    MPK_TRY(S.alloc(&d_queue, (size_t)n));
    MPK_TRY(S.alloc(&d_bc, 1));
    MPK_CUDA(cudaMemsetAsync(pl->d_level, 0xff, sizeof(int32_t) * (size_t)n, st));
    MPK_CUDA(cudaMemsetAsync(d_bc, 0, sizeof(BfsCtl), st));
    MPK_TRY(launch_bfs(n, A->rowptr, A->col, d_trp, d_tcol, (o->root >= 0 && o->root < n) ? o->root : 0, pl->d_level,
                       d_queue, d_bc, timeout_ns, pl->num_sms, st));
    BfsCtl h_bc;
    MPK_CUDA(cudaMemcpyAsync(&h_bc, d_bc, sizeof(BfsCtl), cudaMemcpyDeviceToHost, st));
    MPK_CUDA(cudaStreamSynchronize(st));
    if (h_bc.err) return h_bc.err;
    const int32_t L = h_bc.nlevels;
    if (L < 1 || L > n) return MPK_ERR_CUDA;
    pl->n_levels = L;
    mark(1);

    // 4. stable renumbering by (level, original index): LSD radix sort on levels
    int32_t *kA, *kB, *vA, *vB, *hist;
    const int32_t nb = (int32_t)((n + kRsTile - 1) / kRsTile);
    MPK_TRY(S.alloc(&kA, (size_t)n));
    MPK_TRY(S.alloc(&kB, (size_t)n));
    MPK_TRY(S.alloc(&vA, (size_t)n));
    MPK_TRY(S.alloc(&vB, (size_t)n));
    MPK_TRY(S.alloc(&hist, (size_t)256 * nb));
    MPK_CUDA(cudaMemcpyAsync(kA, pl->d_level, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, st));
    MPK_TRY(radix_sort_keys(n, L - 1, kA, kB, vA, vB, hist, st));
    MPK_TRY(dev_alloc(pl, &pl->d_perm, (size_t)n));
    MPK_TRY(dev_alloc(pl, &pl->d_iperm, (size_t)n));
    MPK_TRY(dev_alloc(pl, &pl->d_level_ptr, (size_t)L + 1));
    MPK_CUDA(cudaMemcpyAsync(pl->d_perm, vA, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, st));
    k_inverse_perm<<<blocks_for(n, 256), 256, 0, st>>>(n, pl->d_perm, pl->d_iperm);
    k_level_ptr<<<blocks_for(n, 256), 256, 0, st>>>(n, kA, pl->d_level_ptr, L);

    // 5. symmetric permutation P A P^T with sorted rows
    int32_t *prow, *plen, *pcol;
    double *pval;
    MPK_TRY(S.alloc(&prow, (size_t)n + 1));
    MPK_TRY(S.alloc(&plen, (size_t)n + 1));
    MPK_TRY(S.alloc(&pcol, (size_t)nnz));
    MPK_TRY(S.alloc(&pval, (size_t)nnz));
    MPK_CUDA(cudaMemsetAsync(plen + n, 0, sizeof(int32_t), st));
    k_perm_len<<<blocks_for(n, 256), 256, 0, st>>>(n, A->rowptr, pl->d_perm, plen);
    MPK_TRY(exclusive_scan<int32_t>(plen, prow, (int64_t)n + 1, st, nullptr));
    k_perm_fill<<<blocks_for((int64_t)n * kPermGroup, 256), 256, 0, st>>>(n, A->rowptr, A->col, A->val, pl->d_perm,
                                                                          pl->d_iperm, prow,
                                                    pcol, pval);

    // features of the matrix for the learned planner (host array of the plan)
    {
        unsigned long long *d_acc;
        MPK_TRY(S.alloc(&d_acc, 5));
        MPK_CUDA(cudaMemsetAsync(d_acc, 0, 5 * sizeof(unsigned long long), st));
        k_row_stats<<<std::min<unsigned>(blocks_for(n, 256), (unsigned)pl->num_sms * 8), 256, 0, st>>>(n, prow, pcol,
                                                                                                      d_acc);
        unsigned long long h[5];
        MPK_CUDA(cudaMemcpyAsync(h, d_acc, sizeof(h), cudaMemcpyDeviceToHost, st));
        MPK_CUDA(cudaStreamSynchronize(st));
        const double N = (double)n, mean = (double)h[0] / N;
        const double var = std::max(0.0, (double)h[1] / N - mean * mean);
        float *f = pl->features;
        f[0] = (float)std::log10(N);
        f[1] = (float)mean;
        f[2] = (float)std::sqrt(var);
        f[3] = (float)std::log10(1.0 + (double)h[2]);
        pl->max_row_len = (int32_t)h[2];
        f[4] = (float)((double)h[3] / std::max(1.0, (double)h[0]) / N);   // mean |col-row| / N
        f[5] = (float)((double)h[4] / N);                                  // max |col-row| / N
    }
    mark(2);

    // 6. level sizes to the host
    int64_t *d_lnnz;
    MPK_TRY(S.alloc(&d_lnnz, (size_t)L));
    k_level_nnz<<<blocks_for(L, 256), 256, 0, st>>>(L, pl->d_level_ptr, prow, d_lnnz);
    std::vector<int64_t> lnnz((size_t)L);
    pl->h_level_ptr.resize((size_t)L + 1);
    MPK_CUDA(cudaMemcpyAsync(lnnz.data(), d_lnnz, sizeof(int64_t) * (size_t)L, cudaMemcpyDeviceToHost, st));
    MPK_CUDA(cudaMemcpyAsync(pl->h_level_ptr.data(), pl->d_level_ptr, sizeof(int32_t) * ((size_t)L + 1),
                             cudaMemcpyDeviceToHost, st));

    // precision: bytes per stored entry (value + 32-bit column index)
    int split_diag = 0;
    if (pl->prec == MPK_F64) {
        pl->val_bytes = 8;
    } else if (pl->prec == MPK_F64_DF) {
        // FP32 values when every value is exactly one, else (hi, lo) pairs;
        // the run-time range guard: max|x| * ||A||_inf^p < 2^100
        int32_t *d_fl;
        unsigned long long *d_rs;
        MPK_TRY(S.alloc(&d_fl, 2));
        MPK_TRY(S.alloc(&d_rs, 1));
        MPK_CUDA(cudaMemsetAsync(d_fl, 0, 2 * sizeof(int32_t), st));
        MPK_CUDA(cudaMemsetAsync(d_rs, 0, sizeof(unsigned long long), st));
        if (nnz > 0) k_df_values<<<blocks_for(n, 256), 256, 0, st>>>(n, prow, pval, d_fl, d_rs);
        int32_t h_fl[2] = {0, 0};
        unsigned long long h_rs = 0;
        MPK_CUDA(cudaMemcpyAsync(h_fl, d_fl, sizeof(h_fl), cudaMemcpyDeviceToHost, st));
        MPK_CUDA(cudaMemcpyAsync(&h_rs, d_rs, sizeof(h_rs), cudaMemcpyDeviceToHost, st));
        MPK_CUDA(cudaStreamSynchronize(st));
        if (h_fl[1]) return MPK_ERR_UNSUPPORTED;
        pl->val_bytes = h_fl[0] ? 8 : 4;
        double norm;
        memcpy(&norm, &h_rs, sizeof(norm));
        const double lim = 100.0 - (double)p * std::log2(std::max(norm, 1.0));
        if (lim < -60.0) return MPK_ERR_UNSUPPORTED;   // no input could stay in range
        const double xlim = std::ldexp(1.0, (int)std::floor(lim));
        memcpy(&pl->df_xlim_bits, &xlim, sizeof(xlim));
    } else if (pl->prec == MPK_F32) {
        pl->val_bytes = 4;
    } else {
        int32_t *d_ne;
        MPK_TRY(S.alloc(&d_ne, 1));
        MPK_CUDA(cudaMemsetAsync(d_ne, 0, sizeof(int32_t), st));
        k_bf16_exact<<<blocks_for(n, 256), 256, 0, st>>>(n, prow, pcol, pval, d_ne);
        int32_t h_ne = 0;
        MPK_CUDA(cudaMemcpyAsync(&h_ne, d_ne, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        MPK_CUDA(cudaStreamSynchronize(st));
        split_diag = 1;
        pl->val_bytes = h_ne ? 4 : 2;
    }
    pl->has_diag = split_diag;
    MPK_CUDA(cudaStreamSynchronize(st));
    for (int32_t l = 0; l < L; l++)
        pl->max_level_rows = std::max(pl->max_level_rows, pl->h_level_ptr[l + 1] - pl->h_level_ptr[l]);
    {   // level features: count, largest level, and the share of rows in each
        // sixteenth of the level range (shape of the level-size profile)
        float *f = pl->features;
        f[6] = (float)std::log10((double)L);
        f[7] = (float)((double)pl->max_level_rows / n);
        f[8] = (float)((double)n / L / std::max(1, pl->max_level_rows));   // mean / largest level size
        for (int b = 0; b < 16; b++) {
            const int32_t l0 = (int32_t)((int64_t)L * b / 16), l1 = (int32_t)((int64_t)L * (b + 1) / 16);
            f[9 + b] = (float)((double)(pl->h_level_ptr[l1] - pl->h_level_ptr[l0]) / n);
        }
    }
    mark(3);

    // 7. level groups (Eq. 5): add levels while (q+1) * weight(T) < f * C,
    //    q the powers of one sweep
    {
        const double budget = pl->safety_f * pl->cache_bytes;
        const double bpe = (double)(pl->val_bytes + 4);
        std::vector<int32_t> gp;
        int32_t s0 = 0;
        while (s0 < L) {
            double acc = (double)lnnz[s0] * bpe;
            int32_t e = s0 + 1;
            while (e < L && (double)(q + 1) * (acc + (double)lnnz[e] * bpe) < budget) {
                acc += (double)lnnz[e] * bpe;
                e++;
            }
            gp.push_back(s0);
            s0 = e;
        }
        gp.push_back(L);
        pl->h_group_ptr = gp;
        pl->n_groups = (int32_t)gp.size() - 1;
    }

    // 7b. recursion (Sec. 4.4): bulky groups refined by the levels of the
    //     subgraphs they induce; the finest levels replace the levels
    pl->h_group_stage.assign((size_t)pl->n_groups, 0);
    if (o->recursion > 0) {
        const double budget = pl->safety_f * pl->cache_bytes;
        const double bpe = (double)(pl->val_bytes + 4);
        MPK_TRY(refine_levels(pl, A, q, o->recursion, bpe, budget, prow, plen, pcol, pval, lnnz, kA, kB, vA, vB, hist,
                              S, st, timeout_ns));
        if (pl->rec_stages > 0) {
            pl->n_levels = (int32_t)pl->h_level_ptr.size() - 1;
            pl->n_groups = (int32_t)pl->h_group_ptr.size() - 1;
            cudaFree(pl->d_level_ptr);
            pl->d_level_ptr = nullptr;
            MPK_TRY(dev_alloc(pl, &pl->d_level_ptr, pl->h_level_ptr.size()));
            MPK_CUDA(cudaMemcpyAsync(pl->d_level_ptr, pl->h_level_ptr.data(), sizeof(int32_t) * pl->h_level_ptr.size(),
                                     cudaMemcpyHostToDevice, st));
        }
    }

    mark(4);

    // 8. tiles (work items) inside groups, chunks of 32 rows inside tiles
    // Work items of 512 rows by default: small enough that the rows in flight
    // (CTAs x tile rows) stay a small part of the level-group window, large
    // enough to amortise the per-item synchronisation; tiny matrices get
    // smaller tiles so that every SM has work.
    //    Resident schedule: a tile must fit one of the two shared-memory
    //    stages of its CTA; rows are at most max_row_len entries wide, so
    //    tile_rows * max_row_len entries (plus a record per chunk) bound it.
    const bool want_res =
        (o->tune & MPK_TUNE_RESIDENT) && (o->nrhs == 1 || o->nrhs == 2) && o->prec != MPK_F64_DF && q == p;
    const int res_per_sm = std::max(1, std::min(2, o->ctas_per_sm > 0 ? o->ctas_per_sm : 1));
    size_t res_stage = 0;
    if (want_res) {
        const size_t per_cta = std::min<size_t>((size_t)prop.sharedMemPerBlockOptin,
                                                (size_t)prop.sharedMemPerMultiprocessor / res_per_sm) -
                               2048;   // static shared memory and the per-CTA reservation
        res_stage = (per_cta / 2) / 128 * 128;
    }
    int32_t tr = o->tile_rows;
    if (tr <= 0 && want_res) {
        const double per_row = (double)std::max(1, pl->max_row_len) * (double)(4 + pl->val_bytes) + 16.0 / kChunk;
        const int64_t rows = (int64_t)((double)(res_stage - 256) / per_row);
        tr = (int32_t)std::min<int64_t>(8192, (rows / kChunk) * kChunk);
        if (tr < kChunk) tr = 0;   // rows too wide for a stage: work-list schedule
    }
    if (tr <= 0) {
        int64_t target = (int64_t)n / ((int64_t)pl->num_sms * 4);
        tr = (int32_t)std::min<int64_t>(512, std::max<int64_t>(kChunk, (target / kChunk) * kChunk));
    }
    tr = std::max(kChunk, (tr / kChunk) * kChunk);
    pl->tile_rows = tr;
    std::vector<int32_t> tile_row, tile_chunk, chunk_row, group_tile;
    for (int32_t g = 0; g < pl->n_groups; g++) {
        group_tile.push_back((int32_t)tile_row.size());
        int32_t r0 = pl->h_level_ptr[pl->h_group_ptr[g]], r1 = pl->h_level_ptr[pl->h_group_ptr[g + 1]];
        for (int32_t a = r0; a < r1; a += tr) {
            int32_t b = std::min(r1, a + tr);
            tile_row.push_back(a);
            tile_chunk.push_back((int32_t)chunk_row.size());
            for (int32_t c = a; c < b; c += kChunk) chunk_row.push_back(c);
        }
    }
    group_tile.push_back((int32_t)tile_row.size());
    tile_row.push_back(n);
    tile_chunk.push_back((int32_t)chunk_row.size());
    chunk_row.push_back(n);
    pl->n_tiles = (int32_t)tile_row.size() - 1;
    pl->n_chunks = (int32_t)chunk_row.size() - 1;
    if ((int64_t)pl->n_tiles >= (1LL << 23)) return MPK_ERR_UNSUPPORTED;

    int32_t *d_tile_row;
    MPK_TRY(S.alloc(&d_tile_row, tile_row.size()));
    MPK_TRY(dev_alloc(pl, &pl->d_tile_chunk, tile_chunk.size()));
    MPK_TRY(dev_alloc(pl, &pl->d_chunk_row, chunk_row.size()));
    MPK_TRY(dev_alloc(pl, &pl->d_chunk_off, chunk_row.size()));
    MPK_TRY(dev_alloc(pl, &pl->d_group_ptr, pl->h_group_ptr.size()));
    MPK_CUDA(cudaMemcpyAsync(d_tile_row, tile_row.data(), tile_row.size() * 4, cudaMemcpyHostToDevice, st));
    MPK_CUDA(cudaMemcpyAsync(pl->d_tile_chunk, tile_chunk.data(), tile_chunk.size() * 4, cudaMemcpyHostToDevice, st));
    MPK_CUDA(cudaMemcpyAsync(pl->d_chunk_row, chunk_row.data(), chunk_row.size() * 4, cudaMemcpyHostToDevice, st));
    MPK_CUDA(cudaMemcpyAsync(pl->d_group_ptr, pl->h_group_ptr.data(), pl->h_group_ptr.size() * 4,
                             cudaMemcpyHostToDevice, st));

    // 9. packed SELL-32 matrix; rows of a tile sorted by length when that
    //    removes more than a tenth of the padding (SELL-C-sigma, sigma = tile)
    int64_t *cw;
    int32_t *rlen;
    MPK_TRY(S.alloc(&cw, (size_t)pl->n_chunks + 1));
    MPK_TRY(S.alloc(&rlen, (size_t)n));
    MPK_CUDA(cudaMemsetAsync(cw + pl->n_chunks, 0, sizeof(int64_t), st));
    k_row_len<<<blocks_for(n, 256), 256, 0, st>>>(n, prow, pcol, split_diag, rlen);
    k_chunk_width<<<blocks_for(pl->n_chunks, 256), 256, 0, st>>>(pl->n_chunks, pl->d_chunk_row, rlen, nullptr, cw);
    int64_t total = 0;
    MPK_TRY(exclusive_scan<int64_t>(cw, pl->d_chunk_off, (int64_t)pl->n_chunks + 1, st, &total));
    {
        int64_t stored = 0;
        int64_t *d_len64;
        MPK_TRY(S.alloc(&d_len64, (size_t)n + 1));
        k_widen<<<blocks_for(n, 256), 256, 0, st>>>(n, rlen, d_len64);
        MPK_CUDA(cudaMemsetAsync(d_len64 + n, 0, sizeof(int64_t), st));
        MPK_TRY(exclusive_scan<int64_t>(d_len64, d_len64, (int64_t)n + 1, st, &stored));
        if (!(o->tune & MPK_TUNE_NO_SORT) && tr <= 8192 && (double)total > 1.1 * (double)stored) {
            MPK_TRY(dev_alloc(pl, &pl->d_row_map, (size_t)n));
            const size_t sm = sizeof(int32_t) * (size_t)tr;
            k_sort_tile_rows<<<pl->n_tiles, 256, sm, st>>>(pl->n_tiles, d_tile_row, rlen, pl->d_row_map);
            k_chunk_width<<<blocks_for(pl->n_chunks, 256), 256, 0, st>>>(pl->n_chunks, pl->d_chunk_row, rlen,
                                                                        pl->d_row_map, cw);
            MPK_TRY(exclusive_scan<int64_t>(cw, pl->d_chunk_off, (int64_t)pl->n_chunks + 1, st, &total));
            pl->sorted = 1;
        }
    }
    pl->packed_entries = total;
    if (total / kChunk >= (int64_t)INT32_MAX) return MPK_ERR_UNSUPPORTED;   // chunk records hold offset / 32
    MPK_TRY(dev_alloc(pl, &pl->d_chunk_rec, (size_t)pl->n_chunks));
    k_chunk_rec<<<blocks_for(pl->n_chunks, 256), 256, 0, st>>>(pl->n_chunks, pl->d_chunk_row, pl->d_chunk_off,
                                                              pl->d_chunk_rec);
    MPK_TRY(dev_alloc(pl, &pl->d_pcol, (size_t)total));
    if (split_diag) MPK_TRY(dev_alloc(pl, &pl->d_diag, (size_t)n));
    if (pl->prec == MPK_F64_DF) MPK_TRY(dev_alloc(pl, &pl->d_shadow, 2 * (size_t)n));
    {
        const unsigned nbk = blocks_for((int64_t)pl->n_chunks * kChunk, 256);
        if (pl->prec == MPK_F64_DF && pl->val_bytes == 8) {
            float2 *v;
            MPK_TRY(dev_alloc(pl, &v, (size_t)total));
            pl->d_pval = v;
            k_pack<float2><<<nbk, 256, 0, st>>>(pl->n_chunks, pl->d_chunk_row, pl->d_chunk_off, pl->d_row_map, prow,
                                                pcol, pval, split_diag, pl->d_pcol, v, pl->d_diag);
        } else if (pl->val_bytes == 8) {
            double *v;
            MPK_TRY(dev_alloc(pl, &v, (size_t)total));
            pl->d_pval = v;
            k_pack<double><<<nbk, 256, 0, st>>>(pl->n_chunks, pl->d_chunk_row, pl->d_chunk_off, pl->d_row_map, prow,
                                                pcol, pval, split_diag, pl->d_pcol, v, pl->d_diag);
        } else if (pl->val_bytes == 4) {
            float *v;
            MPK_TRY(dev_alloc(pl, &v, (size_t)total));
            pl->d_pval = v;
            k_pack<float><<<nbk, 256, 0, st>>>(pl->n_chunks, pl->d_chunk_row, pl->d_chunk_off, pl->d_row_map, prow,
                                               pcol, pval, split_diag, pl->d_pcol, v, pl->d_diag);
        } else {
            __nv_bfloat16 *v;
            MPK_TRY(dev_alloc(pl, &v, (size_t)total));
            pl->d_pval = v;
            k_pack<__nv_bfloat16><<<nbk, 256, 0, st>>>(pl->n_chunks, pl->d_chunk_row, pl->d_chunk_off, pl->d_row_map,
                                                       prow, pcol, pval, split_diag, pl->d_pcol, v, pl->d_diag);
        }
    }

    // 10. dependency ranges of every tile
    int32_t *tor;
    MPK_TRY(S.alloc(&tor, (size_t)n));
    MPK_TRY(dev_alloc(pl, &pl->d_dep_lo, (size_t)pl->n_tiles));
    MPK_TRY(dev_alloc(pl, &pl->d_dep_hi, (size_t)pl->n_tiles));
    k_tile_of_row<<<pl->n_tiles, 256, 0, st>>>(pl->n_tiles, d_tile_row, tor);
    k_fill_i32<<<256, 256, 0, st>>>(pl->d_dep_lo, pl->n_tiles, INT_MAX);
    k_fill_i32<<<256, 256, 0, st>>>(pl->d_dep_hi, pl->n_tiles, -1);
    k_deps<<<blocks_for(n, 256), 256, 0, st>>>(n, prow, pcol, tor, A->assume_symmetric ? 1 : 0, pl->d_dep_lo,
                                               pl->d_dep_hi);

    // tile offsets into the packed arrays, and the shared-memory stage size
    {
        MPK_TRY(dev_alloc(pl, &pl->d_tile_off, (size_t)pl->n_tiles + 1));
        k_tile_off<<<blocks_for(pl->n_tiles + 1, 256), 256, 0, st>>>(pl->n_tiles, pl->d_tile_chunk, pl->d_chunk_off,
                                                                    pl->d_tile_off);
        std::vector<int64_t> toff((size_t)pl->n_tiles + 1);
        MPK_CUDA(cudaMemcpyAsync(toff.data(), pl->d_tile_off, sizeof(int64_t) * toff.size(), cudaMemcpyDeviceToHost, st));
        MPK_CUDA(cudaStreamSynchronize(st));
        int64_t mx = 0;
        int32_t mc = 0;
        for (int32_t t = 0; t < pl->n_tiles; t++) {
            mx = std::max(mx, toff[t + 1] - toff[t]);
            mc = std::max(mc, tile_chunk[t + 1] - tile_chunk[t]);
        }
        mark(5);
        pl->stage_entries = ((mx + kChunk - 1) / kChunk) * kChunk;
        pl->stage_recs = ((mc + 7) / 8) * 8;
        pl->tune = o->tune;
        const size_t res_need =
            (((size_t)pl->stage_recs * 16 + (size_t)pl->stage_entries * (4 + pl->val_bytes) + 127) / 128) * 128;
        if (want_res && res_need <= res_stage) {
            pl->resident = 1;
            pl->staged = 0;
            pl->smem_bytes = 2 * res_need;
        } else {
            // staged work-list form (block widths 1 and 2): three stages, so
            // that each copy is issued two items ahead, when the wanted CTAs
            // per SM (ctas_per_sm, default 2) still fit; else two
            const size_t optin = (size_t)prop.sharedMemPerBlockOptin, per_sm = (size_t)prop.sharedMemPerMultiprocessor;
            const size_t want = (size_t)(o->ctas_per_sm > 0 ? o->ctas_per_sm : 2);
            int nst = 0;
            if ((o->tune & MPK_TUNE_STAGE) && o->nrhs <= 2 && o->prec != MPK_F64_DF) {
                if (3 * res_need + 1024 <= optin && want * (3 * res_need + 1024) <= per_sm) nst = 3;
                else if (2 * res_need + 1024 <= optin) nst = 2;
            }
            pl->staged = nst > 0;
            pl->n_stages = nst;
            pl->smem_bytes = (size_t)nst * res_need;
        }
        pl->wave_warps = pl->resident ? kComputeWarps : (is_f64_vec(pl->prec) ? kFp64Warps : kFp32Warps);
    }

    // 11. grid size, then the work list: a skewed diagonal order of the Lp
    //     diagram over level groups (see order_items)
    pl->h_dep_lo.resize((size_t)pl->n_tiles);
    MPK_CUDA(cudaMemcpyAsync(pl->h_dep_lo.data(), pl->d_dep_lo, sizeof(int32_t) * pl->h_dep_lo.size(),
                             cudaMemcpyDeviceToHost, st));
    pl->h_dep_hi.resize((size_t)pl->n_tiles);
    MPK_CUDA(cudaMemcpyAsync(pl->h_dep_hi.data(), pl->d_dep_hi, sizeof(int32_t) * pl->h_dep_hi.size(),
                             cudaMemcpyDeviceToHost, st));
    MPK_CUDA(cudaStreamSynchronize(st));
    for (int32_t t = 0; t < pl->n_tiles; t++) {
        pl->dep_span = std::max(pl->dep_span, pl->h_dep_hi[t] - t);
        if (pl->h_dep_hi[t] - (pl->h_dep_lo[t] & ~3) >= kProbeFlags) pl->wide_deps = 1;
    }
    if (pl->resident) {
        // resident schedule: res_per_sm CTAs per SM, each owning whole tiles;
        // the wait chains cannot close when G > (p-1) * span (or every tile
        // has its own CTA)
        int occ_w = 0, occ_c = 0;
        MPK_TRY(wave_occupancy(pl, &occ_w, &occ_c));
        const int64_t G = std::min<int64_t>((int64_t)pl->num_sms * res_per_sm, pl->n_tiles);
        const bool acyclic = G >= pl->n_tiles || G > (int64_t)(p - 1) * pl->dep_span;
        if (std::min(occ_w, occ_c) >= res_per_sm && acyclic) {
            pl->ctas_per_sm = res_per_sm;
            pl->grid_ctas = pl->cheb_grid = (int32_t)G;
        } else {
            pl->resident = 0;
            pl->smem_bytes = 0;
            pl->wave_warps = is_f64_vec(pl->prec) ? kFp64Warps : kFp32Warps;
        }
    }
    if (!pl->resident) {
        int occ_w = 0, occ_c = 0;
        MPK_TRY(wave_occupancy(pl, &occ_w, &occ_c));
        const int64_t items = (int64_t)pl->n_tiles * p;
        auto grid_of = [&](int occ) {
            const int per_sm = std::max(1, o->ctas_per_sm > 0 ? std::min(o->ctas_per_sm, occ) : occ);
            return (int32_t)std::max<int64_t>(1, std::min<int64_t>((int64_t)pl->num_sms * per_sm, items));
        };
        pl->ctas_per_sm = std::max(1, o->ctas_per_sm > 0 ? std::min(o->ctas_per_sm, occ_w) : occ_w);
        pl->grid_ctas = grid_of(occ_w);
        pl->cheb_grid = occ_c < (1 << 30) ? grid_of(occ_c) : pl->grid_ctas;
    }
    {
        pl->h_tile_row = tile_row;
        pl->h_group_tile = group_tile;
        pl->lag = o->lag;
        const size_t items = (size_t)pl->n_tiles * p;
        MPK_TRY(dev_alloc(pl, &pl->d_work, items));
        if (pl->rec_stages == 0) {
            // without recursion the order is a merge of shifted copies of one
            // sorted list: placed on the GPU (k_issue_order)
            double lag = o->lag;
            std::vector<double> v;
            pl->slope = order_slope(pl, p, lag, v);
            double *d_v;
            MPK_TRY(S.alloc(&d_v, v.size()));
            MPK_CUDA(cudaMemcpyAsync(d_v, v.data(), sizeof(double) * v.size(), cudaMemcpyHostToDevice, st));
            const int32_t q = pl->sweep > 0 ? std::min(pl->sweep, p) : p;
            k_issue_order<<<blocks_for((int64_t)items, 256), 256, 0, st>>>(pl->n_tiles, p, q, pl->slope, d_v,
                                                                          pl->d_work);
            MPK_CUDA(cudaGetLastError());
        } else {
            std::vector<int32_t> work;
            pl->slope = order_items(pl, p, o->lag, work);
            MPK_CUDA(cudaMemcpyAsync(pl->d_work, work.data(), work.size() * 4, cudaMemcpyHostToDevice, st));
        }
        MPK_CUDA(cudaStreamSynchronize(st));
    }
    mark(6);
    pl->fstride = ((pl->n_tiles + 3) / 4) * 4 + 4;
    MPK_TRY(dev_alloc(pl, &pl->d_flags, (size_t)(p + 1) * pl->fstride));
    pl->bstride = (pl->n_tiles + kFlagBlock - 1) / kFlagBlock;
    MPK_TRY(dev_alloc(pl, &pl->d_bcnt, (size_t)(p + 1) * pl->bstride));
    MPK_CUDA(cudaMemsetAsync(pl->d_bcnt, 0, sizeof(uint32_t) * (size_t)(p + 1) * pl->bstride, st));
    MPK_TRY(dev_alloc(pl, &pl->d_ctl, CTL_WORDS));
    MPK_CUDA(cudaMemsetAsync(pl->d_flags, 0, sizeof(uint32_t) * (size_t)(p + 1) * pl->fstride, st));
    MPK_CUDA(cudaMemsetAsync(pl->d_ctl, 0, sizeof(int32_t) * CTL_WORDS, st));

    MPK_CUDA(cudaStreamSynchronize(st));
    MPK_CUDA(cudaGetLastError());
    return MPK_OK;
}

// ---------------------------------------------------------------- allocation-free levels
// Scratch of mpk_levels_noalloc: words [0, kStaticCtlWords) hold the control
// block of the BFS kernel and the validation flag, the rest the frontier
// queue.  It lives in the library's own device memory (reserved when the
// module is loaded on a device and kept until the process exits).
constexpr int32_t kStaticLevelsMaxN = 1 << 20;
constexpr int32_t kStaticCtlWords = 64;
constexpr int32_t kStaticBadWord = 32;
static_assert(sizeof(BfsCtl) <= kStaticBadWord * sizeof(int32_t), "control block must fit");

}  // namespace

static __device__ __align__(256) int32_t g_levels_scratch[kStaticCtlWords + kStaticLevelsMaxN];

namespace {

// Device address of the static scratch in the current device's context.  It
// is looked up on every call (cudaGetSymbolAddress is cheap): a cached
// address would go stale once the primary context is torn down and created
// again (cudaDeviceReset), and the kernels would then write through an
// address the new context does not own.
int static_levels_scratch(int32_t **out) {
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_levels_scratch);
    if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress(g_levels_scratch)", __LINE__);
    *out = (int32_t *)ptr;
    return MPK_OK;
}

}  // namespace

// Issue order of the (tile, power) work items.  The Lp diagram of Fig. 5 is
// traversed along diagonals: node (i, k) of level group i and power k sits on
// diagonal i + k, and the paper visits a diagonal with k ascending, so node
// (i, k) directly follows the node (i+1, k-1) it depends on (condition (C) of
// Sec. 4.3).  A GPU runs hundreds of items at once, and that order would put
// p dependent steps on every diagonal's critical path.  Items here are ordered
// by the key v(t) + sigma * (k - 1), with v(t) the position of tile t in units
// of level groups (group index plus the fraction of the group's rows before
// the tile): the diagonals of the Lp diagram get slope sigma and the tiles of
// the p nodes on a diagonal are interleaved.  sigma is the least slope that
// puts every dependency (the tiles up to dep_hi[t] at power k-1) strictly
// before its item, plus a lag that covers the items in flight, and at least 1
// (the paper's slope, i.e. p+1 level groups between the first and last power
// front, the working set Eq. 5 budgets for).  Ties go to the lower power, so
// dependencies always come first and in-order hand-out cannot deadlock.
// With sweeps of q < p powers (Sec. 5.1 splits a power into sweeps) the
// powers of sweep s = (k-1) / q come after every item of sweep s-1, each
// sweep traversed as above with k - 1 replaced by its power within the sweep.
// Tile positions v(t) in level-group units and the slope sigma of the
// issue order below (its lag resolved), for p powers in sweeps of q.
double order_slope(const Plan *pl, int32_t p, double &lag, std::vector<double> &v) {
    const std::vector<int32_t> &tile_row = pl->h_tile_row, &group_tile = pl->h_group_tile, &hi = pl->h_dep_hi;
    const int32_t T = pl->n_tiles, G = pl->n_groups;
    const int32_t q = pl->sweep > 0 ? std::min(pl->sweep, p) : p;
    v.assign((size_t)T, 0.0);
    for (int32_t g = 0; g < G; g++) {
        const double r0 = tile_row[group_tile[g]], r1 = tile_row[group_tile[g + 1]];
        for (int32_t t = group_tile[g]; t < group_tile[g + 1]; t++) v[t] = g + (tile_row[t] - r0) / (r1 - r0);
    }
    double need = 0.0;
    for (int32_t t = 0; t < T; t++) need = std::max(need, v[hi[t]] - v[t]);
    if (lag < 0) {   // in-flight items measured in level groups per power front
        const double tiles_per_group = (double)T / G;
        // the order is shared by the MPK and the Chebyshev launches: size the
        // lag for the smaller of their grids
        const int32_t grid = pl->cheb_grid > 0 ? std::min(pl->grid_ctas, pl->cheb_grid) : pl->grid_ctas;
        lag = 1.5 * (double)grid / ((double)q * tiles_per_group);
    }
    return std::max(1.0, need + lag);
}

double order_items(const Plan *pl, int32_t p, double lag, std::vector<int32_t> &work) {
    const std::vector<int32_t> &hi = pl->h_dep_hi;
    const int32_t T = pl->n_tiles;
    const int32_t q = pl->sweep > 0 ? std::min(pl->sweep, p) : p;
    std::vector<double> v;
    const double sigma = order_slope(pl, p, lag, v);
    struct Item { int32_t s; double key; int32_t k, t; };
    std::vector<Item> items;
    items.reserve((size_t)T * p);
    double slope = sigma;
    if (pl->rec_stages == 0) {
        // v(t) increases with t, so each power's items are already in key
        // order: a merge of the q lists of each sweep (a heap over powers)
        // gives the order of a full sort by (key, k, t) in O(T p log q).
        work.clear();
        work.reserve((size_t)T * p);
        struct Head { double key; int32_t k, t; };
        auto later = [](const Head &a, const Head &b) {
            if (a.key != b.key) return a.key > b.key;
            if (a.k != b.k) return a.k > b.k;
            return a.t > b.t;
        };
        std::vector<Head> heap;
        for (int32_t k0 = 1; k0 <= p; k0 += q) {
            const int32_t k1 = std::min(p, k0 + q - 1);
            heap.clear();
            if (T > 0)
                for (int32_t k = k0; k <= k1; k++) heap.push_back({v[0] + sigma * (k - k0), k, 0});
            std::make_heap(heap.begin(), heap.end(), later);
            while (!heap.empty()) {
                std::pop_heap(heap.begin(), heap.end(), later);
                Head &h = heap.back();
                work.push_back((h.t << 8) | h.k);
                if (++h.t < T) {
                    h.key = v[h.t] + sigma * (h.k - k0);
                    std::push_heap(heap.begin(), heap.end(), later);
                } else {
                    heap.pop_back();
                }
            }
        }
        return slope;
    } else {
        // After recursion a tile next to a refined subgraph may read rows
        // spread over all its sub-levels: one slope for every tile would
        // have to cover the widest such span.  Instead each item is placed
        // by its own latest dependency,
        //   key(t, 1) = v(t),
        //   key(t, k) = max(key(t, k-1) + 1, max over the tiles t' in
        //               [dep_lo[t], dep_hi[t]] of key(t', k-1) + lag),
        // so items near the boundary of a refined region are delayed as far
        // as their dependencies need and no further (the "diamond" of
        // Sec. 4.4); every dependency still comes strictly earlier.  The
        // range maxima come from a sparse table per power.  The first power
        // of every sweep starts again from v(t).
        const std::vector<int32_t> &lo = pl->h_dep_lo;
        const double dl = std::max(lag, 0.5);
        std::vector<double> key(v), nk((size_t)T);
        int32_t levels = 1;
        while ((1 << levels) < T) levels++;
        std::vector<std::vector<double>> tab((size_t)levels + 1, std::vector<double>((size_t)T));
        std::vector<int32_t> lg((size_t)T + 1, 0);
        for (int32_t i = 2; i <= T; i++) lg[i] = lg[i / 2] + 1;
        for (int32_t t = 0; t < T; t++) items.push_back({0, key[t], 1, t});
        double slope_sum = 0.0;
        for (int32_t k = 2; k <= p; k++) {
            if ((k - 1) % q == 0) {
                key = v;
            } else {
                tab[0] = key;
                for (int32_t j = 1; j <= levels; j++)
                    for (int32_t t = 0; t + (1 << j) <= T; t++)
                        tab[j][t] = std::max(tab[j - 1][t], tab[j - 1][t + (1 << (j - 1))]);
                for (int32_t t = 0; t < T; t++) {
                    double m = key[t] + 1.0;
                    const int32_t a = lo[t], b = hi[t];
                    if (a <= b) {
                        const int32_t j = lg[b - a + 1];
                        m = std::max(m, std::max(tab[j][a], tab[j][b - (1 << j) + 1]) + dl);
                    }
                    nk[t] = m;
                }
                key.swap(nk);
            }
            if (k == q)
                for (int32_t t = 0; t < T; t++) slope_sum += (key[t] - v[t]) / (q - 1);
            for (int32_t t = 0; t < T; t++) items.push_back({(k - 1) / q, key[t], k, t});
        }
        slope = T > 0 && q > 1 ? slope_sum / T : 1.0;
    }
    std::sort(items.begin(), items.end(), [](const Item &a, const Item &b) {
        if (a.s != b.s) return a.s < b.s;
        if (a.key != b.key) return a.key < b.key;
        if (a.k != b.k) return a.k < b.k;
        return a.t < b.t;
    });
    work.resize(items.size());
    for (size_t i = 0; i < items.size(); i++) work[i] = (items[i].t << 8) | items[i].k;
    return slope;
}

int work_to_host(const Plan *pl, std::vector<int32_t> &work) {
    work.resize((size_t)pl->n_tiles * pl->p);
    MPK_CUDA(cudaMemcpyAsync(work.data(), pl->d_work, sizeof(int32_t) * work.size(), cudaMemcpyDeviceToHost,
                             pl->stream));
    MPK_CUDA(cudaStreamSynchronize(pl->stream));
    return MPK_OK;
}

int exclusive_scan_i32(const int32_t *in, int32_t *out, int64_t n, cudaStream_t st, int32_t *total) {
    return exclusive_scan<int32_t>(in, out, n, st, total);
}
int exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t st, int64_t *total) {
    return exclusive_scan<int64_t>(in, out, n, st, total);
}

}  // namespace mpk

using namespace mpk;

extern "C" {

int mpk_opts_default(mpk_opts *o) {
    if (!o) return MPK_ERR_INVALID;
    memset(o, 0, sizeof(*o));
    o->root = 0;
    o->cache_bytes = 0.0;
    o->safety_f = 0.5;
    o->prec = MPK_F64;
    o->nrhs = 1;
    o->tile_rows = 0;
    o->ctas_per_sm = 0;
    o->timeout_s = 2.0;
    o->stream = nullptr;
    o->lag = -1.0;
    o->tune = 0;
    o->recursion = 0;
    o->sweep = 0;
    return MPK_OK;
}

int mpk_plan(const mpk_csr *A, int32_t p, const mpk_opts *o, mpk_plan_t *out) {
    if (!out) return MPK_ERR_INVALID;
    *out = nullptr;
    if (!A || !o || !A->rowptr) return MPK_ERR_INVALID;
    if (A->nnz > 0 && (!A->col || !A->val)) return MPK_ERR_INVALID;   // unused when there are no entries
    if (A->n < 1 || A->nnz < 0 || A->nnz >= (int64_t)INT32_MAX) return MPK_ERR_INVALID;
    if (p < 1 || p > kMaxP) return MPK_ERR_INVALID;
    if (o->nrhs < 1 || o->nrhs > kMaxNrhs) return MPK_ERR_INVALID;
    if (o->prec < MPK_F64 || o->prec > MPK_F64_DF) return MPK_ERR_INVALID;
    if (o->prec == MPK_F64_DF && o->nrhs != 1) return MPK_ERR_UNSUPPORTED;
    if (!(o->safety_f > 0.0) || o->cache_bytes < 0.0 || o->tile_rows < 0 || o->ctas_per_sm < 0) return MPK_ERR_INVALID;
    if (o->recursion < 0 || o->recursion > 16) return MPK_ERR_INVALID;
    if (o->sweep < 0 || o->sweep > kMaxP) return MPK_ERR_INVALID;
    mpk_plan_s *h = new (std::nothrow) mpk_plan_s();
    if (!h) return MPK_ERR_OOM;
    const auto t0 = std::chrono::steady_clock::now();
    int rc = build_plan(&h->pl, A, p, o);   // its temporary device memory is released on return
    if (rc != MPK_OK) {
        cudaStreamSynchronize((cudaStream_t)o->stream);
        free_plan(&h->pl);
        delete h;
        return rc;
    }
    Plan &pl = h->pl;
    pl.plan_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    double rest = pl.plan_ms;
    for (int i = 0; i < 7; i++) rest -= pl.phase_ms[i];
    pl.phase_ms[7] = std::max(0.0, rest);
    *out = h;
    return MPK_OK;
}

int mpk_plan_destroy(mpk_plan_t plan) {
    if (!plan) return MPK_OK;
    cudaStreamSynchronize(plan->pl.stream);
    free_plan(&plan->pl);
    delete plan;
    return MPK_OK;
}

int mpk_plan_info(mpk_plan_t plan, mpk_plan_stats *s) {
    if (!plan || !s) return MPK_ERR_INVALID;
    const Plan &pl = plan->pl;
    memset(s, 0, sizeof(*s));
    s->n = pl.n;
    s->p = pl.p;
    s->nrhs = pl.nrhs;
    s->prec = pl.prec;
    s->nnz = pl.nnz;
    s->n_levels = pl.n_levels;
    s->n_groups = pl.n_groups;
    s->n_tiles = pl.n_tiles;
    s->max_level_rows = pl.max_level_rows;
    s->tile_rows = pl.tile_rows;
    s->grid_ctas = pl.grid_ctas;
    s->val_bytes = pl.val_bytes;
    s->packed_entries = pl.packed_entries;
    s->matrix_bytes = pl.packed_entries * (int64_t)(pl.val_bytes + 4) + (pl.has_diag ? (int64_t)pl.n * 4 : 0);
    s->device_bytes = pl.device_bytes + (int64_t)pl.io_bytes + (int64_t)pl.cheb_bytes;
    s->plan_ms = pl.plan_ms;
    s->cache_bytes = pl.cache_bytes;
    s->slope = pl.slope;
    s->staged = pl.staged;
    s->sorted = pl.sorted;
    s->resident = pl.resident;
    s->dep_span = pl.dep_span;
    s->rec_stages = pl.rec_stages;
    s->sweep = pl.sweep;
    for (int i = 0; i < 8; i++) s->phase_ms[i] = pl.phase_ms[i];
    s->smem_bytes = (int32_t)pl.smem_bytes;
    return MPK_OK;
}

int mpk_plan_features(mpk_plan_t plan, float *out, int32_t count) {
    if (!plan || !out || count < 1) return MPK_ERR_INVALID;
    for (int32_t i = 0; i < count; i++) out[i] = i < Plan::kFeatures ? plan->pl.features[i] : 0.0f;
    return Plan::kFeatures;
}

int mpk_plan_perm(mpk_plan_t plan, int32_t *perm, int32_t *level_ptr, int32_t *group_ptr, int32_t *level) {
    if (!plan) return MPK_ERR_INVALID;
    Plan &pl = plan->pl;
    cudaStream_t st = pl.stream;
    if (perm) MPK_CUDA(cudaMemcpyAsync(perm, pl.d_perm, sizeof(int32_t) * pl.n, cudaMemcpyDeviceToDevice, st));
    if (level_ptr)
        MPK_CUDA(cudaMemcpyAsync(level_ptr, pl.d_level_ptr, sizeof(int32_t) * (pl.n_levels + 1),
                                 cudaMemcpyDeviceToDevice, st));
    if (group_ptr)
        MPK_CUDA(cudaMemcpyAsync(group_ptr, pl.d_group_ptr, sizeof(int32_t) * (pl.n_groups + 1),
                                 cudaMemcpyDeviceToDevice, st));
    if (level) MPK_CUDA(cudaMemcpyAsync(level, pl.d_level, sizeof(int32_t) * pl.n, cudaMemcpyDeviceToDevice, st));
    MPK_CUDA(cudaStreamSynchronize(st));
    return MPK_OK;
}

const char *mpk_strerror(int status) {
    switch (status) {
    case MPK_OK: return "ok";
    case MPK_ERR_INVALID: return "invalid argument or malformed matrix";
    case MPK_ERR_CUDA: return "CUDA runtime error";
    case MPK_ERR_OOM: return "out of memory";
    case MPK_ERR_TIMEOUT: return "device-side dependency wait timed out";
    case MPK_ERR_UNSUPPORTED: return "unsupported request";
    default: return "unknown status";
    }
}

int mpk_levels_noalloc(int32_t n, int64_t nnz, const int32_t *rowptr, const int32_t *col, int32_t root,
                       int32_t *level, int32_t *n_levels, void *stream, double timeout_s) {
    if (!rowptr || (nnz > 0 && !col) || !level || !n_levels || n < 1 || nnz < 0 || nnz >= (int64_t)INT32_MAX)
        return MPK_ERR_INVALID;
    if (root < 0 || root >= n) return MPK_ERR_INVALID;
    if (n > kStaticLevelsMaxN) return MPK_ERR_UNSUPPORTED;   // beyond the static scratch
    cudaStream_t st = (cudaStream_t)stream;
    int32_t *scratch = nullptr;
    int rc = static_levels_scratch(&scratch);
    if (rc) return rc;
    BfsCtl *ctl = (BfsCtl *)scratch;
    int32_t *bad = scratch + kStaticBadWord;
    int32_t *queue = scratch + kStaticCtlWords;
    // the array keeps the previous call's contents: clear what must start at zero
    MPK_CUDA(cudaMemsetAsync(scratch, 0, sizeof(int32_t) * kStaticCtlWords, st));
    MPK_CUDA(cudaMemsetAsync(level, 0xff, sizeof(int32_t) * (size_t)n, st));
    k_validate<<<blocks_for((int64_t)n + 1, 256), 256, 0, st>>>(n, nnz, rowptr, col, bad);
    MPK_CUDA(cudaGetLastError());
    int32_t h_bad = 0;
    MPK_CUDA(cudaMemcpyAsync(&h_bad, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    MPK_CUDA(cudaStreamSynchronize(st));
    if (h_bad) return MPK_ERR_INVALID;
    int dev = 0, sms = 0;
    MPK_CUDA(cudaGetDevice(&dev));
    MPK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const uint64_t tns = (uint64_t)((timeout_s > 0 ? timeout_s : 2.0) * 1e9);
    rc = launch_bfs(n, rowptr, col, nullptr, nullptr, root, level, queue, ctl, tns, sms, st);
    if (rc) return rc;
    BfsCtl h_bc;
    MPK_CUDA(cudaMemcpyAsync(&h_bc, ctl, sizeof(BfsCtl), cudaMemcpyDeviceToHost, st));
    MPK_CUDA(cudaStreamSynchronize(st));
    if (h_bc.err) return h_bc.err;
    if (h_bc.nlevels < 1 || h_bc.nlevels > n) return MPK_ERR_CUDA;
    *n_levels = h_bc.nlevels;
    return MPK_OK;
}

}  // extern "C"
