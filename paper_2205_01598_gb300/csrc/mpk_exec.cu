// Execution kernels of the level-blocked MPK: the persistent (level group,
// power) wavefront (Fig. 5 over level groups, with the point-to-point
// conditions of Sec. 4.3 refined to work items), the baseline of back-to-back
// SpMVs (Fig. 1) and the Chebyshev sweep (Sec. 7, Eq. 7-9).
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>

#include <type_traits>

#include "mpk_internal.cuh"

// Compile-time tuning of the wavefront kernels: entries of a row fetched per
// batch for one vector column, and the minimum resident CTAs per SM that the
// register allocation must allow (0 = no bound).
#ifndef MPK_BATCH
#define MPK_BATCH 8
#endif
#ifndef MPK_WAVE_MIN_BLOCKS
#define MPK_WAVE_MIN_BLOCKS 0
#endif

namespace mpk {

namespace {

template <typename MT, typename VT>
__device__ __forceinline__ VT to_vt(MT v) { return (VT)v; }
template <>
__device__ __forceinline__ float to_vt<__nv_bfloat16, float>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <typename MT>
__device__ __forceinline__ double as_double(MT v) { return (double)v; }
template <>
__device__ __forceinline__ double as_double<__nv_bfloat16>(__nv_bfloat16 v) { return (double)__bfloat162float(v); }
template <>
__device__ __forceinline__ double as_double<float2>(float2 v) { return (double)v.x + (double)v.y; }

// ---------------------------------------------------------------- TMA / mbarrier helpers
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *m, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(m)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t *m, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(m)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *m, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(m)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the completion of phase `parity` of an mbarrier.
__device__ __forceinline__ bool mbar_wait(uint64_t *m, uint32_t parity, uint64_t timeout_ns) {
    if (mbar_try_wait(m, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(m, parity))
        if (global_ns() - t0 > timeout_ns) return false;
    return true;
}
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ uint64_t l2_policy_evict_last() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ uint64_t l2_policy_evict_normal() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
// Bulk (non-tensor) TMA copy global -> shared, completing on an mbarrier.
// dst, src and bytes must be multiples of 16 bytes.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *m, uint64_t pol) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(m)), "l"(pol)
        : "memory");
}

// L2 prefetch of a contiguous range (16-byte aligned address, size a multiple of 16).
__device__ __forceinline__ void bulk_prefetch_l2(const void *p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Where a work item reads its slice of the packed matrix: global memory, or
// the shared-memory stage that a bulk copy filled (entries base..).
template <typename MT, bool STAGED>
struct MatView {
    const int32_t *col;
    const MT *val;
    int64_t base;
    __device__ __forceinline__ int32_t c(int64_t i) const { return STAGED ? col[i - base] : __ldg(col + i); }
    __device__ __forceinline__ MT v(int64_t i) const { return STAGED ? val[i - base] : __ldg(val + i); }
};

// y_out[r] = sum_j A[r, j] * y_in[j] for the (up to) 32 rows of SELL chunk c,
// one row per lane (Fig. 1, restricted to the chunk's row range).  W columns
// of the row-major block vectors are done per pass; EXACT means nrhs == W.
// Padding entries (column -1) sit at the end of each row and are skipped.
template <typename VT, typename MT, int W, bool EXACT, bool DIAG, bool STAGED, int GB = 32>
__device__ __forceinline__ void chunk_rows(const ExecArgs &a, const MatView<MT, STAGED> &mv, int32_t c, int lane,
                                           const VT *yin, VT *yout) {
    const int32_t row0 = __ldg(a.chunk_row + c);
    const int32_t nrows = __ldg(a.chunk_row + c + 1) - row0;
    if (lane >= nrows) return;
    const int64_t off = __ldg(a.chunk_off + c);
    const int32_t w = (int32_t)((__ldg(a.chunk_off + c + 1) - off) / kChunk);
    const int32_t r = a.row_map ? __ldg(a.row_map + row0 + lane) : row0 + lane;
    const int nrhs = EXACT ? W : a.nrhs;
    const int64_t e0 = off + lane;
    // B entries of the row are fetched together (indices and values first,
    // then the B gathers) so that each lane keeps many loads in flight.  When
    // the block width allows, a row of the block vector is gathered with
    // 16-byte loads (VEC values each) and B is set so that about GB FP32
    // values' worth of gathers are in flight per lane (fewer in kernels that
    // must keep registers low for occupancy).
    constexpr int VEC = 16 / (int)sizeof(VT);
    constexpr bool CAN_VEC = W % VEC == 0 && GB > 0;   // GB = 0: scalar gathers only
    constexpr int BW = GB * 4 / (W * (int)sizeof(VT));
    constexpr int BV = BW < 2 ? 2 : (BW > 8 ? 8 : BW);
    constexpr int B = CAN_VEC ? BV : (W <= 2 ? MPK_BATCH : (W <= 4 ? 4 : 2));
    // vectors only when every VEC group lies inside a row of the block vector
    const bool vec = CAN_VEC && (EXACT || nrhs % VEC == 0);
    using V = typename std::conditional<sizeof(VT) == 4, float4, double2>::type;
    for (int cb = 0; cb < nrhs; cb += W) {
        VT acc[W];
#pragma unroll
        for (int i = 0; i < W; i++) acc[i] = VT(0);
        for (int32_t j0 = 0; j0 < w; j0 += B) {
            int32_t cols[B];
            VT vals[B];
#pragma unroll
            for (int u = 0; u < B; u++) {
                const bool in = j0 + u < w;
                cols[u] = in ? mv.c(e0 + (int64_t)(j0 + u) * kChunk) : -1;
                vals[u] = in ? to_vt<MT, VT>(mv.v(e0 + (int64_t)(j0 + u) * kChunk)) : VT(0);
            }
            if (CAN_VEC && vec) {
                VT g[B][W];
#pragma unroll
                for (int u = 0; u < B; u++)
#pragma unroll
                    for (int q = 0; q < W / VEC; q++) {
                        V t;
                        if (cols[u] >= 0 && (EXACT || cb + q * VEC < nrhs))
                            t = *reinterpret_cast<const V *>(yin + (int64_t)cols[u] * nrhs + cb + q * VEC);
                        else
                            memset(&t, 0, sizeof(t));
                        memcpy(&g[u][q * VEC], &t, sizeof(t));
                    }
#pragma unroll
                for (int u = 0; u < B; u++)
                    if (cols[u] >= 0)
#pragma unroll
                        for (int i = 0; i < W; i++)
                            if (EXACT || cb + i < nrhs) acc[i] = fma(vals[u], g[u][i], acc[i]);
            } else {
#pragma unroll
                for (int u = 0; u < B; u++) {
                    if (cols[u] >= 0) {
                        const VT *src = yin + (int64_t)cols[u] * nrhs + cb;
#pragma unroll
                        for (int i = 0; i < W; i++)
                            if (EXACT || cb + i < nrhs) acc[i] = fma(vals[u], src[i], acc[i]);
                    }
                }
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

__device__ __forceinline__ uint4 ld_relaxed_v4(const uint32_t *p) {
    uint4 v;
    asm volatile("ld.relaxed.gpu.global.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p)
                 : "memory");
    return v;
}

// Dependency check of a work item (tile t, power k), run by warp 0: power
// k-1 must be complete on every tile in [dep_lo[t], dep_hi[t]] (the tiles
// holding the columns of tile t; conditions (A)-(C) of Sec. 4.3 at tile
// granularity).  The flags of the next item are loaded (16-byte relaxed loads,
// 4 flags each) before the current item is computed, so that in steady state
// the check costs no round trip.  Flag rows are padded so that a 16-byte load
// that starts at a multiple of 4 inside [lo, hi] stays in bounds.
constexpr int kProbeVec = 2;   // 2 x 32 lanes x 4 flags = 256 flags per probe
static_assert(kProbeVec * 128 == kProbeFlags, "probe width");

struct FlagProbe {
    uint4 v[kProbeVec];
    int32_t lo, hi, base;

    __device__ __forceinline__ void issue(const ExecArgs &a, int32_t t, int32_t k, int lane) {
        issue_range(a, __ldg(a.dep_lo + t), __ldg(a.dep_hi + t), k, lane);
    }
    // with the dependency range [lo_, hi_] of the item's tile already loaded
    __device__ __forceinline__ void issue_range(const ExecArgs &a, int32_t lo_, int32_t hi_, int32_t k, int lane) {
        lo = lo_;
        hi = hi_;
        base = lo & ~3;
        const uint32_t *f = a.flags + (int64_t)(k - 1) * a.fstride;
#pragma unroll
        for (int q = 0; q < kProbeVec; q++) {
            const int32_t i = base + (q * 32 + lane) * 4;
            v[q] = i <= hi ? ld_relaxed_v4(f + i) : make_uint4(0, 0, 0, 0);
        }
    }
    __device__ __forceinline__ bool fits() const { return hi - base < kProbeVec * 128; }
    // `skip`: a tile whose flag need not be read (the caller's own tile at
    // the previous power, finished by the same CTA), -1 for none.
    __device__ __forceinline__ bool ready(uint32_t epoch, int lane, int32_t skip = -1) const {
        bool good = true;
#pragma unroll
        for (int q = 0; q < kProbeVec; q++) {
            const int32_t i = base + (q * 32 + lane) * 4;
            const uint32_t w[4] = {v[q].x, v[q].y, v[q].z, v[q].w};
#pragma unroll
            for (int s = 0; s < 4; s++)
                if (i + s >= lo && i + s <= hi && i + s != skip) good &= (w[s] == epoch);
        }
        return __all_sync(0xffffffffu, good);
    }
};

// Check of a range wider than one probe (huge levels, small tiles): blocks
// of kFlagBlock tiles that lie inside [lo, hi] by their counters of finished
// tiles (a full count means every flag of the block holds this launch's
// epoch: counters are zeroed at the end of every launch), the ragged ends and
// the block holding `skip` flag by flag.
template <bool COUNT = true>
__device__ bool ready_wide(const ExecArgs &a, int32_t t, int32_t k, uint32_t epoch, int lane, int32_t skip = -1) {
    const uint32_t *f = a.flags + (int64_t)(k - 1) * a.fstride;
    const int32_t lo = __ldg(a.dep_lo + t), hi = __ldg(a.dep_hi + t);
    const int32_t b0 = (lo + kFlagBlock - 1) / kFlagBlock, b1 = (hi + 1) / kFlagBlock;   // full blocks [b0, b1)
    bool ok = true;
    if (!COUNT || b0 >= b1 || !a.bcnt) {
        for (int32_t i = lo + lane; i <= hi; i += 32) ok &= (i == skip || ld_relaxed_u32(f + i) == epoch);
    } else {
        const int32_t sb = skip >= 0 ? skip / kFlagBlock : -1;
        for (int32_t i = lo + lane; i < b0 * kFlagBlock; i += 32) ok &= (i == skip || ld_relaxed_u32(f + i) == epoch);
        for (int32_t i = b1 * kFlagBlock + lane; i <= hi; i += 32) ok &= (i == skip || ld_relaxed_u32(f + i) == epoch);
        const uint32_t *cnt = a.bcnt + (int64_t)(k - 1) * a.bstride;
        for (int32_t b = b0 + lane; b < b1; b += 32)
            if (b != sb) ok &= (ld_relaxed_u32(cnt + b) == (uint32_t)kFlagBlock);
        if (sb >= b0 && sb < b1)
            for (int32_t i = sb * kFlagBlock + lane; i < (sb + 1) * kFlagBlock; i += 32)
                ok &= (i == skip || ld_relaxed_u32(f + i) == epoch);
    }
    return __all_sync(0xffffffffu, ok);
}

// Completion of item (t, k): its epoch flag, then, in plans with ranges wider
// than a probe, one more finished tile in its block (both with release
// semantics: the item's outputs are visible to whoever observes either).
__device__ __forceinline__ void publish_item(const ExecArgs &a, int32_t t, int32_t k, uint32_t epoch) {
    st_release_u32(a.flags + (int64_t)k * a.fstride + t, epoch);
    if (a.bcnt)
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(a.bcnt + (int64_t)k * a.bstride + t / kFlagBlock)
                     : "memory");
}

// Zeroes the block counters of a plan (one warp), for the next launch.
__device__ __forceinline__ void clear_block_counts(const ExecArgs &a, int lane) {
    if (!a.bcnt) return;
    const int64_t total = (int64_t)(a.p + 1) * a.bstride;
    for (int64_t i = lane; i < total; i += 32) a.bcnt[i] = 0u;
}

__device__ void record_timeout(const ExecArgs &a, int32_t k, int32_t t) {
    if (atomicCAS(a.ctl + CTL_ERR, 0, (int)MPK_ERR_TIMEOUT) == 0) {
        atomicExch(a.ctl + CTL_ERR_K, k);
        atomicExch(a.ctl + CTL_ERR_T, t);
    }
    atomicExch(a.ctl + CTL_ABORT, 1);
}

// Polls until the item's dependencies are complete.  Bounded: after
// timeout_ns it records MPK_ERR_TIMEOUT with the node, raises the abort word
// and returns false; it also returns false once another CTA has aborted.
template <bool COUNT = true>
__device__ bool wait_deps(const ExecArgs &a, FlagProbe &pr, int32_t t, int32_t k, uint32_t epoch, int lane,
                          int32_t skip = -1) {
    const bool wide = !pr.fits();
    if (wide ? ready_wide<COUNT>(a, t, k, epoch, lane, skip) : pr.ready(epoch, lane, skip)) {
        fence_acq_rel_gpu();
        return true;
    }
    const uint64_t t0 = global_ns();
    unsigned ns = 32;
    for (;;) {
        int stop = 0;
        if (lane == 0) {
            if (ld_relaxed_s32(a.ctl + CTL_ABORT)) {
                stop = 1;
            } else if (global_ns() - t0 > a.timeout_ns) {
                record_timeout(a, k, t);
                stop = 1;
            }
        }
        if (__shfl_sync(0xffffffffu, stop, 0)) return false;
        __nanosleep(ns);
        if (ns < 256) ns <<= 1;
        if (wide) {
            if (ready_wide<COUNT>(a, t, k, epoch, lane, skip)) break;
        } else {
            pr.issue(a, t, k, lane);
            if (pr.ready(epoch, lane, skip)) break;
        }
    }
    fence_acq_rel_gpu();
    return true;
}

// Bytes of one shared-memory stage: the chunk records of a tile, then its
// column indices, then its values, each part 128-byte aligned.
template <typename MT>
__device__ __forceinline__ size_t stage_bytes_of(const ExecArgs &a) {
    return (((size_t)a.stage_recs * 16 + (size_t)a.stage_entries * (4 + sizeof(MT)) + 127) / 128) * 128;
}

// Bulk copy of tile t's packed slice -- chunk records, column indices,
// values -- into a shared-memory stage (layout of stage_bytes_of), completing
// on mbar.  Every part starts on a 128-byte boundary in global and shared
// memory and is a multiple of 16 bytes long (chunks hold 32 entries).
template <typename MT>
__device__ __forceinline__ void stage_slice(const ExecArgs &a, int32_t t, unsigned char *stage, uint64_t *mbar,
                                            int32_t *s_nch, int64_t *s_ebase, uint64_t pol) {
    const int32_t c0 = __ldg(a.tile_chunk + t), c1 = __ldg(a.tile_chunk + t + 1);
    const int64_t o0 = __ldg(a.tile_off + t), o1 = __ldg(a.tile_off + t + 1);
    const uint32_t rb = (uint32_t)(c1 - c0) * 16u, cb = (uint32_t)(o1 - o0) * 4u,
                   vb = (uint32_t)(o1 - o0) * (uint32_t)sizeof(MT);
    *s_nch = c1 - c0;
    *s_ebase = o0;
    fence_proxy_async_smem();
    mbar_expect_tx(mbar, rb + cb + vb);
    unsigned char *cols = stage + (size_t)a.stage_recs * 16;
    if (rb) bulk_g2s(stage, a.chunk_rec + c0, rb, mbar, pol);
    if (cb) bulk_g2s(cols, a.pcol + o0, cb, mbar, pol);
    if (vb) bulk_g2s(cols + (size_t)a.stage_entries * 4, (const MT *)a.pval + o0, vb, mbar, pol);
}

// The slice of work item wk (tile, power): evict-first in L2 at its last
// power (no later reuse), evict-normal (or evict-last when asked) before.
template <typename MT>
__device__ __forceinline__ void stage_item(const ExecArgs &a, int32_t wk, unsigned char *stage, uint64_t *mbar,
                                           int32_t *s_nch, int64_t *s_ebase) {
    const int32_t k = wk & 255;
    const uint64_t pol = k >= a.p ? l2_policy_evict_first()
                                  : ((a.tune & MPK_TUNE_EVICT_LAST) ? l2_policy_evict_last() : l2_policy_evict_normal());
    stage_slice<MT>(a, wk >> 8, stage, mbar, s_nch, s_ebase, pol);
}

// ---------------------------------------------------------------- register-held slices
// A compute warp handles chunks c0 + warp + i*ncw of a work item's tile.  The
// first kPC of them -- chunk record, row, and the first kPE entries of the
// lane's row -- are loaded into registers one work item ahead.  Those loads
// read only the matrix, never a vector, so they are issued before the item's
// dependencies are known to be complete; once the item is released only the
// gathers of the input vector remain on its critical path.
#ifndef MPK_PIPE_CHUNKS
#define MPK_PIPE_CHUNKS 2
#endif
#ifndef MPK_PIPE_ENTRIES
#define MPK_PIPE_ENTRIES 8
#endif
constexpr int kPC = MPK_PIPE_CHUNKS;    // chunks of a warp held in registers
constexpr int kPE = MPK_PIPE_ENTRIES;   // entries of a row held in registers

template <typename MT, int PC>
struct Slice {
    int4 rec[PC];            // {first row, rows, first entry / 32, width}; rows 0 = no chunk
    int32_t row[PC];         // output row of this lane, -1 = none
    int32_t col[PC][kPE];    // -1 = past the row's end
    MT val[PC][kPE];
    int32_t c0, c1;          // chunk range of the item's tile
};

template <int PC>
__device__ __forceinline__ void slice_recs(const ExecArgs &a, int32_t c0, int32_t c1, int warp, int ncw,
                                           int4 (&rec)[PC]) {
#pragma unroll
    for (int i = 0; i < PC; i++) {
        const int32_t c = c0 + warp + i * ncw;
        rec[i] = c < c1 ? __ldg(a.chunk_rec + c) : make_int4(0, 0, 0, 0);
    }
}

template <typename MT, int PC>
__device__ __forceinline__ void slice_entries(const ExecArgs &a, Slice<MT, PC> &s, int lane) {
#pragma unroll
    for (int i = 0; i < PC; i++) {
        const int4 r = s.rec[i];
        const bool on = lane < r.y;
        s.row[i] = on ? (a.row_map ? __ldg(a.row_map + r.x + lane) : r.x + lane) : -1;
        const int64_t e0 = (int64_t)r.z * kChunk + lane;
#pragma unroll
        for (int u = 0; u < kPE; u++) {
            const bool in = on && u < r.w;
            s.col[i][u] = in ? __ldg(a.pcol + e0 + (int64_t)u * kChunk) : -1;
            s.val[i][u] = in ? __ldg((const MT *)a.pval + e0 + (int64_t)u * kChunk) : MT{};
        }
    }
}

// acc[i][q] = sum over the entries of the lane's row in held chunk i of
// value * yin[col * G + q], in entry order (the order of chunk_rows, so both
// paths round alike).  All gathers of the held entries are issued first.
template <typename VT, typename MT, int G, int PC>
__device__ __forceinline__ void slice_sum(const ExecArgs &a, const Slice<MT, PC> &s, const VT *yin, int lane,
                                          VT (&acc)[PC][G]) {
    VT g[PC][kPE][G];
#pragma unroll
    for (int i = 0; i < PC; i++)
#pragma unroll
        for (int u = 0; u < kPE; u++)
#pragma unroll
            for (int q = 0; q < G; q++) g[i][u][q] = s.col[i][u] >= 0 ? yin[(int64_t)s.col[i][u] * G + q] : VT(0);
#pragma unroll
    for (int i = 0; i < PC; i++)
#pragma unroll
        for (int q = 0; q < G; q++) acc[i][q] = VT(0);
#pragma unroll
    for (int i = 0; i < PC; i++)
#pragma unroll
        for (int u = 0; u < kPE; u++)
            if (s.col[i][u] >= 0) {
                const VT v = to_vt<MT, VT>(s.val[i][u]);
#pragma unroll
                for (int q = 0; q < G; q++) acc[i][q] = fma(v, g[i][u][q], acc[i][q]);
            }
    // entries past the held ones (rows wider than kPE)
#pragma unroll
    for (int i = 0; i < PC; i++) {
        const int32_t w = s.rec[i].w;
        if (s.row[i] < 0 || w <= kPE) continue;
        const int64_t e0 = (int64_t)s.rec[i].z * kChunk + lane;
        constexpr int B = 8;
        for (int32_t j0 = kPE; j0 < w; j0 += B) {
            int32_t cols[B];
            VT vals[B];
#pragma unroll
            for (int u = 0; u < B; u++) {
                const bool in = j0 + u < w;
                cols[u] = in ? __ldg(a.pcol + e0 + (int64_t)(j0 + u) * kChunk) : -1;
                vals[u] = in ? to_vt<MT, VT>(__ldg((const MT *)a.pval + e0 + (int64_t)(j0 + u) * kChunk)) : VT(0);
            }
#pragma unroll
            for (int u = 0; u < B; u++)
                if (cols[u] >= 0)
#pragma unroll
                    for (int q = 0; q < G; q++) acc[i][q] = fma(vals[u], yin[(int64_t)cols[u] * G + q], acc[i][q]);
        }
    }
}

// Rows of a tile whose chunk records, indices and values sit in a
// shared-memory stage (resident schedule): kRC chunks of a warp per pass, the
// gathers of all their entries (kGb per row per pass) in flight together,
// entries summed in stored order with padding skipped (as chunk_rows does, so
// both round alike).  out(row, acc) writes a row.
constexpr int kRC = 2;   // chunks of a warp handled together
constexpr int kGb = 8;   // entries of a row per pass

template <typename VT, typename MT, int G, typename Out>
__device__ __forceinline__ void resident_rows(const ExecArgs &a, const int4 *srec, const int32_t *scol,
                                              const MT *sval, int64_t ebase, int32_t nch, int warp, int ncw, int lane,
                                              const VT *yin, const Out &out) {
    for (int32_t cb = warp; cb < nch; cb += kRC * ncw) {
        int32_t row[kRC], w[kRC], e0[kRC];
        int32_t wmax = 0;
#pragma unroll
        for (int i = 0; i < kRC; i++) {
            const int32_t c = cb + i * ncw;
            row[i] = -1;
            w[i] = 0;
            e0[i] = 0;
            if (c < nch) {
                const int4 r = srec[c];
                if (lane < r.y) {
                    row[i] = a.row_map ? __ldg(a.row_map + r.x + lane) : r.x + lane;
                    w[i] = r.w;
                    e0[i] = (int32_t)((int64_t)r.z * kChunk - ebase) + lane;
                }
            }
            wmax = max(wmax, w[i]);
        }
        VT acc[kRC][G];
#pragma unroll
        for (int i = 0; i < kRC; i++)
#pragma unroll
            for (int q = 0; q < G; q++) acc[i][q] = VT(0);
        for (int32_t j0 = 0; j0 < wmax; j0 += kGb) {
            int32_t cols[kRC][kGb];
            VT g[kRC][kGb][G];
#pragma unroll
            for (int i = 0; i < kRC; i++)
#pragma unroll
                for (int u = 0; u < kGb; u++) {
                    cols[i][u] = j0 + u < w[i] ? scol[e0[i] + (j0 + u) * kChunk] : -1;
#pragma unroll
                    for (int q = 0; q < G; q++)
                        g[i][u][q] = cols[i][u] >= 0 ? yin[(int64_t)cols[i][u] * G + q] : VT(0);
                }
#pragma unroll
            for (int i = 0; i < kRC; i++)
#pragma unroll
                for (int u = 0; u < kGb; u++)
                    if (cols[i][u] >= 0) {
                        const VT v = to_vt<MT, VT>(sval[e0[i] + (j0 + u) * kChunk]);
#pragma unroll
                        for (int q = 0; q < G; q++) acc[i][q] = fma(v, g[i][u][q], acc[i][q]);
                    }
        }
#pragma unroll
        for (int i = 0; i < kRC; i++)
            if (row[i] >= 0) out(row[i], acc[i]);
    }
}

// Body of one work item (tile t, power k) of the plain MPK.
template <typename VT, typename MT, int W, bool EXACT, bool DIAG, int GB = 32>
struct MpkNode {
    // prefetch power-1 slices into L2 ahead of time (measured on 160^3: the
    // FP64 MPK 2 % faster; the FP32 MPK and the FP64 heat propagation slower)
    static constexpr bool kL2First = sizeof(MT) == 8;
    static constexpr bool kPipe = W == 1 && EXACT;   // single vectors run from register-held slices

    template <typename Extra, int PC>
    __device__ __forceinline__ static void pipe_run(const ExecArgs &a, const Slice<MT, PC> &s, int32_t t, int32_t k,
                                                    int warp, int nwarps, int lane, const Extra &) {
        const VT *yin = k == 1 ? (const VT *)a.x : (const VT *)a.Y + (int64_t)(k - 2) * a.blk;
        VT *yout = (VT *)a.Y + (int64_t)(k - 1) * a.blk;
        VT acc[PC][1];
        slice_sum<VT, MT, 1, PC>(a, s, yin, lane, acc);
        if (DIAG) {   // the diagonal terms' loads before any store (see row_out of ChebNode)
            VT dv[PC], xv[PC];
#pragma unroll
            for (int i = 0; i < PC; i++) {
                const int32_t r = s.row[i];
                dv[i] = r >= 0 ? (VT)__ldg(a.diag + r) : VT(0);
                xv[i] = r >= 0 ? yin[r] : VT(0);
            }
#pragma unroll
            for (int i = 0; i < PC; i++) acc[i][0] = fma(dv[i], xv[i], acc[i][0]);
        }
#pragma unroll
        for (int i = 0; i < PC; i++)
            if (s.row[i] >= 0) yout[s.row[i]] = acc[i][0];
        const MatView<MT, false> mv{a.pcol, (const MT *)a.pval, 0};
        for (int32_t c = s.c0 + warp + PC * nwarps; c < s.c1; c += nwarps)
            chunk_rows<VT, MT, 1, true, DIAG, false>(a, mv, c, lane, yin, yout);
    }

    // resident schedule (block vectors of width W = nrhs in {1, 2})
    template <typename Extra>
    __device__ __forceinline__ static void res_run(const ExecArgs &a, const int4 *srec, const int32_t *scol,
                                                   const MT *sval, int64_t ebase, int32_t nch, int32_t k, int warp,
                                                   int nwarps, int lane, const Extra &) {
        const VT *yin = k == 1 ? (const VT *)a.x : (const VT *)a.Y + (int64_t)(k - 2) * a.blk;
        VT *yout = (VT *)a.Y + (int64_t)(k - 1) * a.blk;
        resident_rows<VT, MT, W>(a, srec, scol, sval, ebase, nch, warp, nwarps, lane, yin,
                                 [&](int32_t r, const VT (&acc)[W]) {
#pragma unroll
                                     for (int q = 0; q < W; q++) {
                                         VT v = acc[q];
                                         if (DIAG) v = fma((VT)__ldg(a.diag + r), yin[(int64_t)r * W + q], v);
                                         yout[(int64_t)r * W + q] = v;
                                     }
                                 });
    }

    template <bool STAGED>
    __device__ __forceinline__ static void run(const ExecArgs &a, const MatView<MT, STAGED> &mv, int32_t t, int32_t k,
                                               int warp, int nwarps, int lane, const int &) {
        const VT *yin = k == 1 ? (const VT *)a.x : (const VT *)a.Y + (int64_t)(k - 2) * a.blk;
        VT *yout = (VT *)a.Y + (int64_t)(k - 1) * a.blk;
        const int32_t c1 = __ldg(a.tile_chunk + t + 1);
        for (int32_t c = __ldg(a.tile_chunk + t) + warp; c < c1; c += nwarps)
            chunk_rows<VT, MT, W, EXACT, DIAG, STAGED, GB>(a, mv, c, lane, yin, yout);
    }
};

__device__ __forceinline__ void named_sync(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}
__device__ __forceinline__ void named_arrive(int id, int nthreads) {
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}
constexpr int kBarReady = 1;   // scheduler -> compute warps: the next item may start
constexpr int kBarDone = 2;    // compute warps -> scheduler: the current item is finished

// Where the arguments and the epoch of a work item come from: one plan, or
// one of the plans of a batch (per-item plan index, per-plan epoch).
struct OnePlan {
    const ExecArgs &a;
    uint32_t epoch;
    __device__ __forceinline__ int32_t plan_of(int32_t) const { return 0; }
    __device__ __forceinline__ const ExecArgs &args(int32_t) const { return a; }
    __device__ __forceinline__ uint32_t epoch_of(int32_t) const { return epoch; }
    __device__ __forceinline__ void publish_epochs() const { atomicExch(a.ctl + CTL_EPOCH, (int)epoch); }
    __device__ __forceinline__ void clear_counts(int lane) const { clear_block_counts(a, lane); }
};
struct ManyPlans {
    const ExecArgs *table;      // per plan (device memory)
    const int32_t *wplan;       // plan of each work item
    const uint32_t *epochs;     // per plan (shared memory)
    int32_t *const *plan_ctl;   // control words of each plan (their epochs advance)
    int32_t count;
    __device__ __forceinline__ int32_t plan_of(int32_t j) const { return __ldg(wplan + j); }
    __device__ __forceinline__ const ExecArgs &args(int32_t m) const { return table[m]; }
    __device__ __forceinline__ uint32_t epoch_of(int32_t m) const { return epochs[m]; }
    __device__ __forceinline__ void publish_epochs() const {
        for (int32_t m = 0; m < count; m++) atomicExch(plan_ctl[m] + CTL_EPOCH, (int)epochs[m]);
    }
    __device__ __forceinline__ void clear_counts(int lane) const {
        for (int32_t m = 0; m < count; m++) clear_block_counts(table[m], lane);
    }
};

// Persistent, warp-specialised wavefront.  Work items are dealt round-robin
// in the issue order (item j goes to CTA j mod gridDim.x; each CTA runs its
// items in order).  Every dependency of an item comes earlier in that order,
// the launch is cooperative (all CTAs resident), and a CTA publishes a
// finished item before it blocks on the dependencies of its next one, so the
// lowest unfinished item can always run: the launch cannot deadlock.
//
// The last warp of the CTA schedules: it checks the dependencies of the next
// item (flags loaded ahead of time), performs the acquire fence, has the
// item's matrix slice copied into a shared-memory stage (bulk copy, staged
// form), starts the compute warps, and publishes the previous item with a
// release store.  Its fences overlap the compute warps' work instead of
// stalling them.  `g` holds the launch-wide fields (issue order, control
// words, limits); `src` the per-item plan arguments.
//
// With one plan and no stage, the compute warps hold the next item's matrix
// slice in registers (Slice): they know which item comes next because the
// dealing is static -- the scheduler hands them items blockIdx.x,
// blockIdx.x + gridDim.x, ... in that order, or -1 to stop.
// COUNT: the completion counters may be in use (see ready_wide); without
// it the plan's ranges all fit a probe and an item publishes its flag alone.
template <typename Node, typename MT, bool STAGED, typename Src, typename Extra, int PC = kPC, bool COUNT = true>
__device__ __forceinline__ void wave_loop(const ExecArgs &g, const Src &src, const Extra &extra) {
    extern __shared__ __align__(128) unsigned char dsmem[];
    __shared__ int s_item, s_stage, s_plan;
    __shared__ __align__(8) uint64_t mbar[kMaxStages];
    __shared__ int32_t s_nch[kMaxStages];
    __shared__ int64_t s_ebase[kMaxStages];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ncw = (int)(blockDim.x >> 5) - 1;
    const int nthr = (int)blockDim.x;
    // staged form: the i-th item of this CTA uses stage i mod nst, whose
    // mbarrier completes its (i / nst)-th phase when the copy has landed
    const int nst = STAGED ? g.n_stages : 1;
    const size_t stage_bytes = STAGED ? stage_bytes_of<MT>(g) : 0;
    if (STAGED && threadIdx.x == 0) {
        for (int q = 0; q < nst; q++) mbar_init(&mbar[q], 1);
        fence_mbar_init();
    }
    __syncthreads();

    if (warp == ncw) {
        // ------------------------------------------------------------ scheduler warp
        const int G = (int)gridDim.x;
        int32_t issued = 0, consumed = 0;   // bulk copies issued / items finished (staged form)
        auto issue = [&](int32_t jj) {      // the next copy goes to stage issued mod nst
            if (STAGED) {
                const int st = issued % nst;
                if (lane == 0)
                    stage_item<MT>(src.args(src.plan_of(jj)), __ldg(g.work + jj), dsmem + st * stage_bytes, &mbar[st],
                                   &s_nch[st], &s_ebase[st]);
                issued++;
            }
        };
        FlagProbe pr;
        int32_t j = blockIdx.x;
        bool ok = j < g.n_items;
        int32_t m = 0;
        if (ok) {
            for (int q = 0; q < nst; q++)
                if (j + q * G < g.n_items) issue(j + q * G);
            const int32_t wk = __ldg(g.work + j);
            m = src.plan_of(j);
            if ((wk & 255) > 1) {
                const ExecArgs &aj = src.args(m);
                pr.issue(aj, wk >> 8, wk & 255, lane);
                ok = wait_deps<COUNT>(aj, pr, wk >> 8, wk & 255, src.epoch_of(m), lane);
            }
        }
        if (lane == 0) {
            s_item = ok ? __ldg(g.work + j) : -1;
            s_plan = m;
            s_stage = 0;
        }
        __syncwarp();
        named_arrive(kBarReady, nthr);
        // What the dependency check of an item needs besides its flags is
        // loaded ahead: the work word and plan of item j + G one item ahead,
        // the dependency range of its tile two items ahead (so that the
        // check of an item waits for the flag loads alone).
        auto work_of = [&](int32_t jj) { return jj < g.n_items ? __ldg(g.work + jj) : 0; };
        auto plan_at = [&](int32_t jj) { return jj < g.n_items ? src.plan_of(jj) : 0; };
        int32_t wA = work_of(j + G), mA = plan_at(j + G);           // item j + G
        int32_t wB = work_of(j + 2 * G), mB = plan_at(j + 2 * G);   // item j + 2G
        int32_t loA = 0, hiA = -1;                                  // deps of item j + G
        if (j + G < g.n_items) {
            loA = __ldg(src.args(mA).dep_lo + (wA >> 8));
            hiA = __ldg(src.args(mA).dep_hi + (wA >> 8));
        }
        // Nodes with kL2First (the FP64 MPK): the slice of a power-1 item is
        // the one read from HBM (later powers find it in L2); its bulk
        // prefetch into L2 is issued four items ahead, after two steps of
        // loads (work word, then slice range) spread over the items before.
        constexpr bool kL2Ahead = Node::kL2First && !STAGED;
        int32_t pfw = -1, pfmw = 0;   // item j + 5G: work word (-1 none) and plan
        int64_t pfo0 = 0, pfo1 = 0;   // item j + 4G: packed entries, when a power-1 item
        int32_t pfm = 0;
        int32_t i = 0;
        while (ok) {
            const int32_t wk = __ldg(g.work + j);
            const int32_t jn = j + G;
            if constexpr (kL2Ahead) {
                if (pfo1 > pfo0 && lane == 0) {
                    const ExecArgs &ap = src.args(pfm);
                    bulk_prefetch_l2(ap.pcol + pfo0, (uint32_t)((pfo1 - pfo0) * 4));
                    bulk_prefetch_l2((const MT *)ap.pval + pfo0, (uint32_t)((pfo1 - pfo0) * (int64_t)sizeof(MT)));
                }
                pfo0 = pfo1 = 0;
                if (pfw >= 0 && (pfw & 255) == 1) {
                    const ExecArgs &ap = src.args(pfmw);
                    pfo0 = __ldg(ap.tile_off + (pfw >> 8));
                    pfo1 = __ldg(ap.tile_off + (pfw >> 8) + 1);
                    pfm = pfmw;
                }
                const int32_t jq = j + 6 * G;
                pfw = jq < g.n_items ? __ldg(g.work + jq) : -1;
                pfmw = jq < g.n_items ? src.plan_of(jq) : 0;
            }
            int32_t wn = 0, mn = 0;
            bool ready = true;
            if (jn < g.n_items) {
                wn = wA;
                mn = mA;
                const int32_t lon = loA, hin = hiA;
                // loads for the next items (used one and two items from now)
                if (jn + G < g.n_items) {
                    loA = __ldg(src.args(mB).dep_lo + (wB >> 8));
                    hiA = __ldg(src.args(mB).dep_hi + (wB >> 8));
                }
                wA = wB;
                mA = mB;
                wB = work_of(jn + 2 * G);
                mB = plan_at(jn + 2 * G);
                if ((wn & 255) > 1) {
                    const ExecArgs &an = src.args(mn);
                    pr.issue_range(an, lon, hin, wn & 255, lane);
                    ready = pr.fits() ? pr.ready(src.epoch_of(mn), lane)
                                      : ready_wide<COUNT>(an, wn >> 8, wn & 255, src.epoch_of(mn), lane);
                    if (ready) fence_acq_rel_gpu();
                }
            }
            named_sync(kBarDone, nthr);   // compute warps finished item j
            if (STAGED) consumed++;
            bool published = false;
            auto publish = [&]() {
                if constexpr (COUNT) {   // a repeat store of the flag is harmless, a repeat count is not
                    if (published) return;
                    published = true;
                }
                const ExecArgs &aj = src.args(m);
                const int32_t t = wk >> 8, k = wk & 255;
                if (lane == 0 && !(t == aj.drop_tile && k == aj.drop_k)) {
                    if constexpr (COUNT)
                        publish_item(aj, t, k, src.epoch_of(m));
                    else
                        st_release_u32(aj.flags + (int64_t)k * aj.fstride + t, src.epoch_of(m));
                }
            };
            if (jn >= g.n_items) {
                publish();
                if (lane == 0) s_item = -1;
                __syncwarp();
                named_arrive(kBarReady, nthr);
                break;
            }
            if (!ready) {   // publish first, then block on the next item's dependencies
                publish();
                ready = wait_deps<COUNT>(src.args(mn), pr, wn >> 8, wn & 255, src.epoch_of(mn), lane);
            }
            if (ready && j + nst * G < g.n_items) issue(j + nst * G);   // the stage of item j is free
            if (lane == 0) {
                s_item = ready ? wn : -1;
                s_plan = mn;
                s_stage = (i + 1) % nst;
            }
            __syncwarp();
            named_arrive(kBarReady, nthr);
            if (!ready) break;
            publish();   // off the compute warps' critical path (unless published above)
            j = jn;
            m = mn;
            i++;
        }
        // never leave with a bulk copy in flight (abort path): copy q went to
        // stage q mod nst and completes that mbarrier's (q / nst)-th phase
        for (int32_t q = consumed; STAGED && q < issued; q++)
            if (!mbar_wait(&mbar[q % nst], (uint32_t)((q / nst) & 1), g.timeout_ns) && lane == 0)
                record_timeout(g, 0, -1);
        __syncwarp();
        int done = 0;
        if (lane == 0) {
            __threadfence();
            done = atomicAdd(g.ctl + CTL_FINISHED, 1);
        }
        done = __shfl_sync(0xffffffffu, done, 0);
        if (done == (int)gridDim.x - 1) {   // last CTA: clear the block counts, publish the epoch(s), reset
            if constexpr (COUNT) {
                fence_acq_rel_gpu();
                src.clear_counts(lane);
                __syncwarp();
            }
            if (lane == 0) {
                atomicExch(g.ctl + CTL_FINISHED, 0);
                atomicExch(g.ctl + CTL_ABORT, 0);
                src.publish_epochs();
                __threadfence();
            }
        }
    } else if constexpr (!STAGED && Node::kPipe && std::is_same<Src, OnePlan>::value) {
        // ------------------------------------------------------------ compute warps, register-held slices
        const ExecArgs &a = src.args(0);
        const int64_t G = gridDim.x;
        int64_t j = blockIdx.x;
        auto range = [&](int64_t jj, int32_t &c0, int32_t &c1) {
            c0 = c1 = 0;
            if (jj < g.n_items) {
                const int32_t t = __ldg(g.work + jj) >> 8;
                c0 = __ldg(a.tile_chunk + t);
                c1 = __ldg(a.tile_chunk + t + 1);
            }
        };
        Slice<MT, PC> s;
        range(j, s.c0, s.c1);
        slice_recs(a, s.c0, s.c1, warp, ncw, s.rec);
        slice_entries(a, s, lane);
        int32_t n0, n1;   // chunk range of item j + G
        range(j + G, n0, n1);
        for (;;) {
            named_sync(kBarReady, nthr);
            const int32_t wk = *(volatile int *)&s_item;
            if (wk < 0) break;
            int4 rn[PC];   // records of item j + G, and the chunk range of item j + 2G
            slice_recs(a, n0, n1, warp, ncw, rn);
            int32_t m0, m1;
            range(j + 2 * G, m0, m1);
            Node::template pipe_run<Extra, PC>(a, s, wk >> 8, wk & 255, warp, ncw, lane, extra);
            s.c0 = n0;
            s.c1 = n1;
#pragma unroll
            for (int i = 0; i < PC; i++) s.rec[i] = rn[i];
            slice_entries(a, s, lane);   // item j + G, used after its release
            n0 = m0;
            n1 = m1;
            j += G;
            named_arrive(kBarDone, nthr);
        }
    } else if constexpr (STAGED) {
        // ------------------------------------------------------------ compute warps, staged slices
        // The item's chunk records, indices and values are in its stage, so
        // the first global access of an item is the gather of its inputs.
        const size_t rec_bytes = (size_t)g.stage_recs * 16;
        for (int32_t i = 0;; i++) {
            named_sync(kBarReady, nthr);
            const int32_t wk = *(volatile int *)&s_item;
            const int st = *(volatile int *)&s_stage;
            const int32_t m = *(volatile int *)&s_plan;
            if (wk < 0) break;
            const ExecArgs &a = src.args(m);
            if (!mbar_wait(&mbar[st], (uint32_t)((i / nst) & 1), g.timeout_ns)) {
                if (lane == 0) record_timeout(g, wk & 255, wk >> 8);
                named_arrive(kBarDone, nthr);
                continue;
            }
            const unsigned char *sb = dsmem + st * stage_bytes;
            Node::res_run(a, (const int4 *)sb, (const int32_t *)(sb + rec_bytes),
                          (const MT *)(sb + rec_bytes + (size_t)g.stage_entries * 4), s_ebase[st], s_nch[st],
                          wk & 255, warp, ncw, lane, extra);
            named_arrive(kBarDone, nthr);
        }
    } else {
        // ------------------------------------------------------------ compute warps
        for (;;) {
            named_sync(kBarReady, nthr);
            const int32_t wk = *(volatile int *)&s_item;
            const int32_t m = *(volatile int *)&s_plan;
            if (wk < 0) break;
            const int32_t t = wk >> 8, k = wk & 255;
            const ExecArgs &a = src.args(m);
            const MatView<MT, false> mv{a.pcol, (const MT *)a.pval, 0};
            Node::template run<false>(a, mv, t, k, warp, ncw, lane, extra);
            named_arrive(kBarDone, nthr);
        }
    }
}

// ---------------------------------------------------------------- resident schedule
// CTA b owns tiles b, b + G, b + 2G, ... (G = gridDim.x) and runs powers
// 1..P of a tile before its next tile.  The tile's packed slice (chunk
// records, column indices, values) is bulk-copied into a shared-memory stage
// at its first power and read from there for all P powers: the matrix leaves
// HBM once per sweep, the level-group blocking of Sec. 4 with shared memory
// as the cache.  Two stages alternate, so the copy of a CTA's next tile runs
// while it works on the current one.  The warp split, the flag protocol
// (epoch-tagged completion flags, acquire before and release after an item,
// publish before blocking) and the bounded waits are those of wave_loop.
//
// Cycle freedom: item (t, k) waits for items of power k-1 in tiles up to
// t + span (span = max dep_hi[t] - t) and for item (t, k-1); the first power
// of tile t waits for the CTA's previous tile t - G.  Along a chain of waits
// the power falls at every dependency step, so a chain advances at most
// (p-1)*span tiles before it has to step back G tiles: with G > (p-1)*span
// (checked when the plan is built) no chain closes.
template <typename MT>
__device__ __forceinline__ void stage_tile(const ExecArgs &a, int32_t t, unsigned char *stage, uint64_t *mbar,
                                           int32_t *s_nch, int64_t *s_ebase) {
    stage_slice<MT>(a, t, stage, mbar, s_nch, s_ebase, l2_policy_evict_first());   // read once per sweep
}

template <typename Node, typename MT, typename Extra>
__device__ __forceinline__ void resident_loop(const ExecArgs &a, uint32_t epoch, const Extra &extra) {
    extern __shared__ __align__(128) unsigned char dsmem[];
    __shared__ int s_item, s_stage;
    __shared__ int32_t s_nch[2];
    __shared__ int64_t s_ebase[2];
    __shared__ __align__(8) uint64_t mbar[2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ncw = (int)(blockDim.x >> 5) - 1;
    const int nthr = (int)blockDim.x;
    const size_t rec_bytes = (size_t)a.stage_recs * 16;
    const size_t stage_bytes = stage_bytes_of<MT>(a);
    const int32_t P = a.p;
    const int32_t G = (int32_t)gridDim.x;
    if (threadIdx.x == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();

    if (warp == ncw) {
        // ------------------------------------------------------------ scheduler warp
        int32_t issued[2] = {0, 0}, consumed[2] = {0, 0};
        auto issue = [&](int32_t q) {   // tile q of this CTA into stage q & 1
            const int64_t t = (int64_t)blockIdx.x + (int64_t)q * G;
            if (t < a.n_tiles) {
                if (lane == 0)
                    stage_tile<MT>(a, (int32_t)t, dsmem + (q & 1) * stage_bytes, &mbar[q & 1], &s_nch[q & 1],
                                   &s_ebase[q & 1]);
                issued[q & 1]++;
            }
        };
        issue(0);
        issue(1);
        FlagProbe pr;
        int32_t q = 0, k = 1, t = blockIdx.x;
        bool ok = t < a.n_tiles;
        if (lane == 0) {
            s_item = ok ? ((t << 8) | 1) : -1;
            s_stage = 0;
        }
        __syncwarp();
        named_arrive(kBarReady, nthr);
        while (ok) {
            int32_t qn = q, kn = k + 1;
            if (kn > P) {
                qn = q + 1;
                kn = 1;
            }
            const int64_t tn64 = (int64_t)blockIdx.x + (int64_t)qn * G;
            const bool more = tn64 < a.n_tiles;
            const int32_t tn = more ? (int32_t)tn64 : 0;
            const int32_t self = qn == q ? t : -1;   // (t, k) is this CTA's own, finished before (t, k+1)
            bool ready = true;
            if (more && kn > 1) {
                pr.issue(a, tn, kn, lane);
                ready = pr.fits() ? pr.ready(epoch, lane, self) : ready_wide(a, tn, kn, epoch, lane, self);
                if (ready) fence_acq_rel_gpu();
            }
            named_sync(kBarDone, nthr);   // compute warps finished (t, k)
            if (k == P) consumed[q & 1]++;
            bool published = false;
            auto publish = [&]() {
                if (published) return;
                published = true;
                if (lane == 0 && !(t == a.drop_tile && k == a.drop_k)) publish_item(a, t, k, epoch);
            };
            if (!more) {
                publish();
                if (lane == 0) s_item = -1;
                __syncwarp();
                named_arrive(kBarReady, nthr);
                break;
            }
            if (!ready) {   // publish first, then block on the next item's dependencies
                publish();
                ready = wait_deps(a, pr, tn, kn, epoch, lane, self);
            }
            if (ready && k == P) issue(q + 2);   // the stage of tile q is free
            if (lane == 0) {
                s_item = ready ? ((tn << 8) | kn) : -1;
                s_stage = qn & 1;
            }
            __syncwarp();
            named_arrive(kBarReady, nthr);
            if (!ready) break;
            publish();   // off the compute warps' critical path (unless published above)
            q = qn;
            k = kn;
            t = tn;
        }
        // never leave with a bulk copy in flight (abort path)
        for (int st = 0; st < 2; st++)
            while (consumed[st] < issued[st]) {
                if (!mbar_wait(&mbar[st], (uint32_t)(consumed[st] & 1), a.timeout_ns) && lane == 0)
                    record_timeout(a, 0, -1);
                consumed[st]++;
            }
        __syncwarp();
        int done = 0;
        if (lane == 0) {
            __threadfence();
            done = atomicAdd(a.ctl + CTL_FINISHED, 1);
        }
        done = __shfl_sync(0xffffffffu, done, 0);
        if (done == (int)gridDim.x - 1) {   // last CTA: clear the block counts, publish the epoch, reset
            fence_acq_rel_gpu();
            clear_block_counts(a, lane);
            __syncwarp();
            if (lane == 0) {
                atomicExch(a.ctl + CTL_FINISHED, 0);
                atomicExch(a.ctl + CTL_ABORT, 0);
                atomicExch(a.ctl + CTL_EPOCH, (int)epoch);
                __threadfence();
            }
        }
    } else {
        // ------------------------------------------------------------ compute warps
        uint32_t ph[2] = {0u, 0u};
        for (;;) {
            named_sync(kBarReady, nthr);
            const int32_t wk = *(volatile int *)&s_item;
            const int st = *(volatile int *)&s_stage;
            if (wk < 0) break;
            const int32_t t = wk >> 8, k = wk & 255;
            if (k == 1) {   // first power of the tile: its slice must have landed
                const bool landed = mbar_wait(&mbar[st], ph[st], a.timeout_ns);
                ph[st] ^= 1u;
                if (!landed) {
                    if (lane == 0) record_timeout(a, k, t);
                    named_arrive(kBarDone, nthr);
                    continue;
                }
            }
            const unsigned char *sb = dsmem + st * stage_bytes;
            Node::res_run(a, (const int4 *)sb, (const int32_t *)(sb + rec_bytes),
                          (const MT *)(sb + rec_bytes + (size_t)a.stage_entries * 4), s_ebase[st], s_nch[st], k,
                          warp, ncw, lane, extra);
            named_arrive(kBarDone, nthr);
        }
    }
}

template <typename VT, typename MT, int W, bool DIAG>
__global__ void __launch_bounds__(kResThreads) k_res_wave(ExecArgs a) {
    const uint32_t epoch = (uint32_t)ld_relaxed_s32(a.ctl + CTL_EPOCH) + 1u;
    resident_loop<MpkNode<VT, MT, W, true, DIAG>, MT>(a, epoch, 0);
}

#if MPK_WAVE_MIN_BLOCKS > 0
#define MPK_WAVE_BOUNDS(threads) __launch_bounds__(threads, MPK_WAVE_MIN_BLOCKS)
#else
#define MPK_WAVE_BOUNDS(threads) __launch_bounds__(threads)
#endif
// NW compute warps per CTA; with 16 of them a warp holds one chunk of a
// 512-row item (more warps, fewer registers each: the FP64 form, whose
// FP64 pipe wants more independent rows in flight), with 8 it holds two.
template <typename VT, typename MT, int W, bool EXACT, bool DIAG, bool STAGED, int NW, bool COUNT>
__global__ void MPK_WAVE_BOUNDS((NW + 1) * 32) k_wave(ExecArgs a) {
    const OnePlan src{a, (uint32_t)ld_relaxed_s32(a.ctl + CTL_EPOCH) + 1u};
    wave_loop<MpkNode<VT, MT, W, EXACT, DIAG>, MT, STAGED, OnePlan, int, (NW >= 16 ? 1 : kPC), COUNT>(a, src, 0);
}

// Baseline: one SpMV over all chunks (warp per chunk, grid-stride).
template <typename VT, typename MT, int W, bool EXACT, bool DIAG>
__global__ void __launch_bounds__(kSpmvThreads) k_spmv(ExecArgs a, const VT *yin, VT *yout) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const MatView<MT, false> mv{a.pcol, (const MT *)a.pval, 0};
    for (int64_t c = gw; c < a.n_chunks; c += nw)
        chunk_rows<VT, MT, W, EXACT, DIAG, false>(a, mv, (int32_t)c, lane, yin, yout);
}

// ---------------------------------------------------------------- double-float arithmetic
// A double-float value is the unevaluated sum hi + lo of two FP32 numbers.
// Sums are split exactly by Knuth's branch-free TwoSum, products by the FMA
// form of Dekker's product (p = a b, e = fma(a, b, -p) is the exact
// rounding error); FP32's 24-bit significand gives pairs of about 48
// significant bits.  GB300 runs FP32 at about 60 times its FP64 rate, so
// the parts of the Chebyshev node that need more than FP32 run in pairs.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
    p = a * b;
    e = fmaf(a, b, -p);
}
// acc = (hi, lo) += (ch + cl) * v: the exact product ch*v, the small cl*v,
// and a TwoSum whose error goes to lo (one step of the compensated dot
// product of Ogita, Rump and Oishi, Dot2).  Terms are added one at a time in
// a fixed order, so the result does not depend on where acc is kept between
// terms.
__device__ __forceinline__ void dot2_add(float &hi, float &lo, float ch, float cl, float v) {
    float p, r, s, q;
    two_prod(ch, v, p, r);
    r = fmaf(cl, v, r);
    two_sum(hi, p, s, q);
    hi = s;
    lo += q + r;
}

// ---------------------------------------------------------------- Chebyshev
// Node of a sweep.  The propagation runs T time steps of M powers each; the
// node of global power g (k0 < g <= k0 + pw) is power k = g - step*M of time
// step `step`.  With Ahat = (A - c)/r:
//   v_1 = Ahat v_0,  v_k = 2 Ahat v_{k-1} - v_{k-2},  acc = sum_k coef_k v_k,
// and v_0 of the next time step is the finished acc.  G columns: G = 2
// complex (re, im; the Schroedinger propagator, complex coefficients), G = 1
// real (the heat propagator, real coefficients).  A v is summed in the
// storage precision.  FP64 plans do the rest in FP64.  FP32 plans do the
// spectral scaling in double-float (the diagonal shift d - c exactly, then
// 1/r), round once to FP32 at the recurrence, and keep acc in double-float.
//
// Vectors live in a ring of three blocks.  Time step s holds v_0 .. v_M at
// the virtual positions s*(M+1) + k, block = position mod 3.  The node of
// power M writes the next step's v_0 (its row of the finished acc, in the
// storage precision) at position s*(M+1) + M + 1, the block of v_{M-2},
// whose last readers -- the neighbours' power M-1 and this node -- are done;
// the next step's v_1 lands on v_{M-1}'s block, whose readers are the
// power-M nodes it waits for.  So sweeps may run across time steps, and one
// launch may hold several steps.
//
// acc (one array, only ever read by its own row) starts as coef_0 v_0 (a
// kernel before the first sweep; for the later time steps the node of the
// previous step's last power, right after it hands v_0 on).  It is read and
// written every third power of a sweep, at the sweep's last power and at
// power M: the node of power k holds v_{k-2} and v_{k-1} (its own row of the
// two input vectors) and v_k, so it adds the terms not yet added, in
// ascending k.  The terms and their order do not
// depend on how the powers are split into sweeps, so every split gives the
// same bits.
// MULTI: the step-aware node (several time steps, v_0 handed on at a step's
// last power); single-step propagations use the lean node (MULTI = false),
// whose power k is simply k0 + j.
template <typename VT, typename MT, bool DIAG, int G, bool MULTI>
struct ChebNode {
    static constexpr bool kL2First = false;
    static_assert(G == 1 || G == 2, "real or complex vectors");
    static constexpr bool kPipe = true;
    static constexpr bool kF64 = sizeof(VT) == 8;

    struct Vecs {
        const VT *yin, *yprev;
        VT *yout;
        VT *ynext;       // the next time step's v_0 (at the step's last power), else null
        int32_t k;       // power within the time step, 1..M
        int32_t nterm;   // coefficient terms this node adds (0: none, else 1..3 ending at k)
    };
    __device__ __forceinline__ static Vecs vecs(const ExecArgs &a, const ChebArgs &ca, int32_t j) {
        VT *ring = (VT *)ca.ring;
        if constexpr (!MULTI) {   // one time step: power k0 + j, flushes every third power of the sweep
            const int32_t k = ca.k0 + j;
            const int32_t flush = (j % 3 == 0 || j == ca.pw) ? j - 3 * ((j - 1) / 3) : 0;
            return Vecs{ring + (int64_t)((k - 1) % 3) * a.blk, ring + (int64_t)((k + 1) % 3) * a.blk,
                        ring + (int64_t)(k % 3) * a.blk, nullptr, k, flush};
        }
        // power k of time step `step` (32-bit arithmetic, no division by M:
        // the host gives the sweep's first step and power)
        int32_t step = ca.step0, k = ca.kin0 + j - 1;
        while (k > ca.M) {
            k -= ca.M;
            step++;
        }
        const int32_t pos = step * (ca.M + 1) + k;   // virtual position of v_k
        // flush points: every third power of the sweep, its last power and
        // the last power of a time step; the terms not yet added start after
        // the latest of the sweep's start, the last flush at a multiple of 3
        // inside the sweep and the start of this time step
        const int32_t last = max(ca.k0 + 3 * ((j - 1) / 3), step * ca.M);
        const int32_t lo = last + 1 - step * ca.M;
        const bool flush = j % 3 == 0 || k == ca.M || j == ca.pw;
        auto blk = [&](int32_t q) { return ring + (int64_t)(q % 3) * a.blk; };
        return Vecs{blk(pos - 1), blk(pos + 1),   // (pos - 2) mod 3
                    blk(pos), (k == ca.M && ca.k0 + j < ca.total) ? blk(pos + 1) : nullptr, k, flush ? k - lo + 1 : 0};
    }

    // Row r of the node, given s = the row's sum of value * v_{k-1} over its
    // stored entries (without the diagonal when it is stored apart).  Every
    // load comes before the first store: the ring blocks may alias as far as
    // the compiler knows, and a load behind a store waits for it.
    __device__ __forceinline__ static void row_out(const ExecArgs &a, const ChebArgs &ca, const Vecs &v, int32_t r,
                                                   const VT (&s)[G]) {
        VT u[G], pv[G], nv[G];
#pragma unroll
        for (int q = 0; q < G; q++) {
            u[q] = v.yin[G * (int64_t)r + q];
            pv[q] = v.k > 1 ? v.yprev[G * (int64_t)r + q] : VT(0);
        }
        if constexpr (kF64) {
            double *acc = (double *)ca.acc + G * (int64_t)r;
            double ac[G];
            if (v.nterm) {
#pragma unroll
                for (int q = 0; q < G; q++) ac[q] = acc[q];
            }
#pragma unroll
            for (int q = 0; q < G; q++) {
                const double ah = ca.alpha * (double)s[q] + ca.beta * (double)u[q];
                nv[q] = v.k > 1 ? 2.0 * ah - (double)pv[q] : ah;
            }
#pragma unroll
            for (int q = 0; q < G; q++) v.yout[G * (int64_t)r + q] = nv[q];
            if (v.nterm) {
                auto add = [&](const VT (&t)[G], int32_t kt) {
                    if constexpr (G == 2) {
                        const double cre = ca.coef[2 * kt], cim = ca.coef[2 * kt + 1];
                        ac[0] = fma(cre, (double)t[0], fma(-cim, (double)t[1], ac[0]));
                        ac[1] = fma(cre, (double)t[1], fma(cim, (double)t[0], ac[1]));
                    } else {
                        ac[0] = fma(ca.coef[kt], (double)t[0], ac[0]);
                    }
                };
                if (v.nterm >= 3) add(pv, v.k - 2);
                if (v.nterm >= 2) add(u, v.k - 1);
                add(nv, v.k);
                if (MULTI && v.ynext) {   // hand v_0 to the next step and restart acc as coef_0 v_0
                    VT v0[G];
#pragma unroll
                    for (int q = 0; q < G; q++) {
                        v0[q] = (VT)ac[q];
                        v.ynext[G * (int64_t)r + q] = v0[q];
                        ac[q] = 0.0;
                    }
                    add(v0, 0);
                }
#pragma unroll
                for (int q = 0; q < G; q++) acc[q] = ac[q];
            }
        } else {
            float *acc = (float *)ca.acc + 2 * G * (int64_t)r;   // (hi, lo) per column
            float ac[2 * G];
            if (v.nterm) {
                if constexpr (G == 2) {
                    const float4 t = *reinterpret_cast<const float4 *>(acc);
                    ac[0] = t.x, ac[1] = t.y, ac[2] = t.z, ac[3] = t.w;
                } else {
                    const float2 t = *reinterpret_cast<const float2 *>(acc);
                    ac[0] = t.x, ac[1] = t.y;
                }
            }
            float dh = 0.f, dl = 0.f;
            if (DIAG) {   // d - c, exactly up to the rounding of c's low part
                two_sum((float)__ldg(a.diag + r), -ca.c_hi, dh, dl);
                dl -= ca.c_lo;
            }
#pragma unroll
            for (int q = 0; q < G; q++) {
                float h, l;
                if (DIAG) {   // Ahat v = (s + (d - c) u) / r
                    float p, pe, wh, wl;
                    two_prod(dh, (float)u[q], p, pe);
                    pe = fmaf(dl, (float)u[q], pe);
                    two_sum((float)s[q], p, wh, wl);
                    wl += pe;
                    two_prod(ca.alpha_hi, wh, h, l);
                    l = fmaf(ca.alpha_hi, wl, fmaf(ca.alpha_lo, wh, l));
                } else {      // Ahat v = s / r - (c / r) u
                    float h1, l1, h2, l2;
                    two_prod(ca.alpha_hi, (float)s[q], h1, l1);
                    l1 = fmaf(ca.alpha_lo, (float)s[q], l1);
                    two_prod(ca.beta_hi, (float)u[q], h2, l2);
                    l2 = fmaf(ca.beta_lo, (float)u[q], l2);
                    two_sum(h1, h2, h, l);
                    l += l1 + l2;
                }
                nv[q] = v.k > 1 ? fmaf(2.f, h, -(float)pv[q]) + 2.f * l : h + l;
            }
#pragma unroll
            for (int q = 0; q < G; q++) v.yout[G * (int64_t)r + q] = nv[q];
            if (v.nterm) {
                auto add = [&](const VT (&t)[G], int32_t kt) {
                    const float4 c = __ldg(ca.coef_df + kt);
                    if constexpr (G == 2) {   // (c_re + i c_im)(t_re + i t_im)
                        dot2_add(ac[0], ac[1], c.x, c.y, (float)t[0]);
                        dot2_add(ac[0], ac[1], -c.z, -c.w, (float)t[1]);
                        dot2_add(ac[2], ac[3], c.x, c.y, (float)t[1]);
                        dot2_add(ac[2], ac[3], c.z, c.w, (float)t[0]);
                    } else {
                        dot2_add(ac[0], ac[1], c.x, c.y, (float)t[0]);
                    }
                };
                if (v.nterm >= 3) add(pv, v.k - 2);
                if (v.nterm >= 2) add(u, v.k - 1);
                add(nv, v.k);
                if (MULTI && v.ynext) {   // hand v_0 (hi + lo rounded once to FP32) on, restart acc as coef_0 v_0
                    VT v0[G];
#pragma unroll
                    for (int q = 0; q < G; q++) {
                        v0[q] = ac[2 * q] + ac[2 * q + 1];
                        v.ynext[G * (int64_t)r + q] = v0[q];
                        ac[2 * q] = ac[2 * q + 1] = 0.f;
                    }
                    add(v0, 0);
                }
                if constexpr (G == 2)
                    *reinterpret_cast<float4 *>(acc) = make_float4(ac[0], ac[1], ac[2], ac[3]);
                else
                    *reinterpret_cast<float2 *>(acc) = make_float2(ac[0], ac[1]);
            }
        }
    }

    template <bool STAGED>
    __device__ __forceinline__ static void chunk(const ExecArgs &a, const MatView<MT, STAGED> &mv, int32_t c, int lane,
                                                 const ChebArgs &ca, const Vecs &v) {
        const int32_t row0 = __ldg(a.chunk_row + c);
        const int32_t nrows = __ldg(a.chunk_row + c + 1) - row0;
        if (lane >= nrows) return;
        const int64_t off = __ldg(a.chunk_off + c);
        const int32_t w = (int32_t)((__ldg(a.chunk_off + c + 1) - off) / kChunk);
        const int32_t r = a.row_map ? __ldg(a.row_map + row0 + lane) : row0 + lane;
        const int64_t e0 = off + lane;
        VT sum[G];
#pragma unroll
        for (int q = 0; q < G; q++) sum[q] = VT(0);
        constexpr int B = 8;
        for (int32_t q0 = 0; q0 < w; q0 += B) {
            int32_t cols[B];
            VT vals[B];
#pragma unroll
            for (int u = 0; u < B; u++) {
                const bool in = q0 + u < w;
                cols[u] = in ? mv.c(e0 + (int64_t)(q0 + u) * kChunk) : -1;
                vals[u] = in ? to_vt<MT, VT>(mv.v(e0 + (int64_t)(q0 + u) * kChunk)) : VT(0);
            }
#pragma unroll
            for (int u = 0; u < B; u++)
                if (cols[u] >= 0)
#pragma unroll
                    for (int q = 0; q < G; q++) sum[q] = fma(vals[u], v.yin[G * (int64_t)cols[u] + q], sum[q]);
        }
        row_out(a, ca, v, r, sum);
    }

    template <bool STAGED>
    __device__ __forceinline__ static void run(const ExecArgs &a, const MatView<MT, STAGED> &mv, int32_t t, int32_t j,
                                               int warp, int nwarps, int lane, const ChebArgs &ca) {
        const Vecs v = vecs(a, ca, j);
        const int32_t c1 = __ldg(a.tile_chunk + t + 1);
        for (int32_t c = __ldg(a.tile_chunk + t) + warp; c < c1; c += nwarps) chunk<STAGED>(a, mv, c, lane, ca, v);
    }

    __device__ __forceinline__ static void res_run(const ExecArgs &a, const int4 *srec, const int32_t *scol,
                                                   const MT *sval, int64_t ebase, int32_t nch, int32_t j, int warp,
                                                   int nwarps, int lane, const ChebArgs &ca) {
        const Vecs v = vecs(a, ca, j);
        resident_rows<VT, MT, G>(a, srec, scol, sval, ebase, nch, warp, nwarps, lane, v.yin,
                                 [&](int32_t r, const VT (&acc)[G]) { row_out(a, ca, v, r, acc); });
    }

    template <typename Extra, int PC>
    __device__ __forceinline__ static void pipe_run(const ExecArgs &a, const Slice<MT, PC> &s, int32_t t, int32_t j,
                                                    int warp, int nwarps, int lane, const Extra &ca) {
        const Vecs v = vecs(a, ca, j);
        VT acc[PC][G];
        slice_sum<VT, MT, G, PC>(a, s, v.yin, lane, acc);
#pragma unroll
        for (int i = 0; i < PC; i++)
            if (s.row[i] >= 0) row_out(a, ca, v, s.row[i], acc[i]);
        const MatView<MT, false> mv{a.pcol, (const MT *)a.pval, 0};
        for (int32_t c = s.c0 + warp + PC * nwarps; c < s.c1; c += nwarps) chunk<false>(a, mv, c, lane, ca, v);
    }
};

template <typename VT, typename MT, bool DIAG, bool STAGED, int G, bool MULTI>
__global__ void __launch_bounds__(kWaveThreads) k_cheb_wave(ChebArgs ca) {
    const OnePlan src{ca.e, (uint32_t)ld_relaxed_s32(ca.e.ctl + CTL_EPOCH) + 1u};
    wave_loop<ChebNode<VT, MT, DIAG, G, MULTI>, MT, STAGED>(ca.e, src, ca);
}
// The real FP64 propagation: 16 compute warps holding one chunk each at two
// CTAs per SM, as the FP64 MPK (more rows in flight for the FP64 pipe).  (A
// minimum of blocks in the bounds of the 8-warp kernel above changes its
// register allocation: the Anderson propagation went from 72 to 96 registers
// and 9.4 to 22.5 ms.)
template <bool STAGED, bool MULTI>
__global__ void __launch_bounds__((kFp64Warps + 1) * 32, 2) k_cheb_wave_f64r(ChebArgs ca) {
    const OnePlan src{ca.e, (uint32_t)ld_relaxed_s32(ca.e.ctl + CTL_EPOCH) + 1u};
    wave_loop<ChebNode<double, double, false, 1, MULTI>, double, STAGED, OnePlan, ChebArgs, 1>(ca.e, src, ca);
}

// Two CTAs per SM must fit (the resident schedule's grid may use them).
template <typename VT, typename MT, bool DIAG, int G>
__global__ void __launch_bounds__(kResThreads, 2) k_res_cheb(ChebArgs ca) {
    const uint32_t epoch = (uint32_t)ld_relaxed_s32(ca.e.ctl + CTL_EPOCH) + 1u;
    resident_loop<ChebNode<VT, MT, DIAG, G, true>, MT>(ca.e, epoch, ca);
}

// ---------------------------------------------------------------- double-float MPK (MPK_F64_DF)
// FP64 input and outputs with the arithmetic on the FP32 pipe in
// double-float pairs.  x is split once into pairs (shadow block 0); power k
// gathers its inputs from shadow block (k-1) mod 2 and writes y_k to Y (FP64)
// and to shadow block k mod 2.  Overwriting block k mod 2 (power k-2) is
// safe: a tile's power k waits for power k-1 on every tile that reads the
// tile's rows (the dependency ranges are closed under that symmetry), and
// those were the last readers of its rows of power k-2.

// FP64 -> double-float pair.  For |v| in [2^-74, 2^101) by integer
// operations: hi = the leading 24 significant bits (truncated), lo = the
// remaining 29 bits, rounded to FP32 by the integer-to-float conversion and
// scaled by an exact power of two (hi + lo = v within 2^-47 |v|).  Other
// values (zero included) through the conversion instructions.
__device__ __forceinline__ float2 f64_to_df(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const uint32_t H = (uint32_t)(b >> 32), L = (uint32_t)b;
    const uint32_t e = (H >> 20) & 0x7FFu;
    if (e < 949u || e > 1123u) {
        const float hi = (float)v;
        return make_float2(hi, (float)(v - (double)hi));
    }
    const uint32_t hb = (H & 0x80000000u) | (((H & 0x7FFFFFFFu) - (896u << 20)) << 3) | (L >> 29);
    float lo = __uint2float_rn(L & 0x1FFFFFFFu) * __uint_as_float((e - 948u) << 23);   // * 2^(e - 1075)
    if (H & 0x80000000u) lo = -lo;
    return make_float2(__uint_as_float(hb), lo);
}

// FP32 -> FP64: zero and normal numbers by integer operations (the exponent
// rebiased, the significand widened; exact), subnormal, infinite and NaN
// inputs through the conversion instruction.
__device__ __forceinline__ double f32_to_f64(float f) {
    const uint32_t u = __float_as_uint(f);
    const uint32_t e = (u >> 23) & 0xFFu;
    if ((u & 0x7FFFFFFFu) == 0u) return __hiloint2double((int)(u & 0x80000000u), 0);
    if (e == 0u || e == 255u) return (double)f;
    return __hiloint2double((int)((u & 0x80000000u) | (((u & 0x7FFFFFFFu) >> 3) + (896u << 20))), (int)(u << 29));
}

// (s, c) += a * x, x = xh + xl: the product a * xh split exactly by FMA, the
// small cross terms added to its error, its high part added to s by TwoSum,
// and every error summed in c (one step of the compensated dot product Dot2
// of Ogita, Rump and Oishi).  Values are FP32 (exact) or pairs (hi, lo).
__device__ __forceinline__ void df_term(float &s, float &c, float a, float2 x) {
    float p, e, t, q;
    two_prod(a, x.x, p, e);
    e = fmaf(a, x.y, e);
    two_sum(s, p, t, q);
    s = t;
    c += q + e;
}
__device__ __forceinline__ void df_term(float &s, float &c, float2 a, float2 x) {
    float p, e, t, q;
    two_prod(a.x, x.x, p, e);
    e = fmaf(a.x, x.y, fmaf(a.y, x.x, e));
    two_sum(s, p, t, q);
    s = t;
    c += q + e;
}

template <typename MT>
struct DfNode {
    static constexpr bool kL2First = true;   // power-1 slices prefetched into L2, as in the FP64 MPK
    static constexpr bool kPipe = true;

    __device__ __forceinline__ static const float2 *in_of(const ExecArgs &a, int32_t k) {
        return a.shadow + (int64_t)((k - 1) & 1) * a.blk;
    }
    // row r of power k from its compensated sum (s, c): the normalised pair
    // to the shadow, hi + lo rounded once to FP64 into Y
    __device__ __forceinline__ static void row_out(const ExecArgs &a, int32_t k, int32_t r, float s, float c) {
        float h, l;
        two_sum(s, c, h, l);
        a.shadow[(int64_t)(k & 1) * a.blk + r] = make_float2(h, l);
        double y = f32_to_f64(h);
        if (l != 0.f) y += f32_to_f64(l);
        ((double *)a.Y)[(int64_t)(k - 1) * a.blk + r] = y;
    }
    // entries j0.. of the lane's row (stored order, padding skipped)
    __device__ __forceinline__ static void entries(const ExecArgs &a, int64_t e0, int32_t j0, int32_t w,
                                                   const float2 *xin, float &s, float &c) {
        constexpr int B = 8;
        for (; j0 < w; j0 += B) {
            int32_t cols[B];
            MT vals[B];
            float2 g[B];
#pragma unroll
            for (int u = 0; u < B; u++) {
                const bool in = j0 + u < w;
                cols[u] = in ? __ldg(a.pcol + e0 + (int64_t)(j0 + u) * kChunk) : -1;
                vals[u] = in ? __ldg((const MT *)a.pval + e0 + (int64_t)(j0 + u) * kChunk) : MT{};
            }
#pragma unroll
            for (int u = 0; u < B; u++) g[u] = cols[u] >= 0 ? xin[cols[u]] : make_float2(0.f, 0.f);
#pragma unroll
            for (int u = 0; u < B; u++)
                if (cols[u] >= 0) df_term(s, c, vals[u], g[u]);
        }
    }
    __device__ __forceinline__ static void chunk(const ExecArgs &a, int32_t c, int lane, int32_t k) {
        const int32_t row0 = __ldg(a.chunk_row + c);
        const int32_t nrows = __ldg(a.chunk_row + c + 1) - row0;
        if (lane >= nrows) return;
        const int64_t off = __ldg(a.chunk_off + c);
        const int32_t w = (int32_t)((__ldg(a.chunk_off + c + 1) - off) / kChunk);
        const int32_t r = a.row_map ? __ldg(a.row_map + row0 + lane) : row0 + lane;
        float s = 0.f, cc = 0.f;
        entries(a, off + lane, 0, w, in_of(a, k), s, cc);
        row_out(a, k, r, s, cc);
    }
    template <typename Extra, int PC>
    __device__ __forceinline__ static void pipe_run(const ExecArgs &a, const Slice<MT, PC> &sl, int32_t t, int32_t k,
                                                    int warp, int nwarps, int lane, const Extra &) {
        const float2 *xin = in_of(a, k);
        float2 g[PC][kPE];
#pragma unroll
        for (int i = 0; i < PC; i++)
#pragma unroll
            for (int u = 0; u < kPE; u++) g[i][u] = sl.col[i][u] >= 0 ? xin[sl.col[i][u]] : make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 0; i < PC; i++) {
            if (sl.row[i] < 0) continue;
            float s = 0.f, cc = 0.f;
#pragma unroll
            for (int u = 0; u < kPE; u++)
                if (sl.col[i][u] >= 0) df_term(s, cc, sl.val[i][u], g[i][u]);
            if (sl.rec[i].w > kPE) entries(a, (int64_t)sl.rec[i].z * kChunk + lane, kPE, sl.rec[i].w, xin, s, cc);
            row_out(a, k, sl.row[i], s, cc);
        }
        for (int32_t c = sl.c0 + warp + PC * nwarps; c < sl.c1; c += nwarps) chunk(a, c, lane, k);
    }
    template <bool STAGED>
    __device__ __forceinline__ static void run(const ExecArgs &a, const MatView<MT, STAGED> &, int32_t t, int32_t k,
                                               int warp, int nwarps, int lane, const int &) {
        const int32_t c1 = __ldg(a.tile_chunk + t + 1);
        for (int32_t c = __ldg(a.tile_chunk + t) + warp; c < c1; c += nwarps) chunk(a, c, lane, k);
    }
    // the resident and staged forms do not run double-float plans
    __device__ __forceinline__ static void res_run(const ExecArgs &, const int4 *, const int32_t *, const MT *, int64_t,
                                                   int32_t, int32_t, int, int, int, const int &) {}
};

template <typename MT>
__global__ void MPK_WAVE_BOUNDS((kFp64Warps + 1) * 32) k_wave_df(ExecArgs a) {
    const OnePlan src{a, (uint32_t)ld_relaxed_s32(a.ctl + CTL_EPOCH) + 1u};
    wave_loop<DfNode<MT>, MT, false, OnePlan, int, 1>(a, src, 0);
}

// Baseline power k of a double-float plan: one SpMV with the same row arithmetic.
template <typename MT>
__global__ void __launch_bounds__(kSpmvThreads) k_spmv_df(ExecArgs a, int32_t k) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t c = gw; c < a.n_chunks; c += nw) DfNode<MT>::chunk(a, (int32_t)c, lane, k);
}

// x (FP64, level order) -> double-float pairs in shadow block 0.  An |x_i|
// above the plan's range limit (or a NaN) sets MPK_ERR_UNSUPPORTED in the
// plan's error word.
__global__ void k_df_split(int32_t n, const double *__restrict__ x, float2 *__restrict__ out, uint64_t lim_bits,
                           int32_t *ctl) {
    bool bad = false;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const double v = x[r];
        bad |= ((unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull) > lim_bits;
        out[r] = f64_to_df(v);
    }
    if (bad) atomicCAS(ctl + CTL_ERR, 0, (int)MPK_ERR_UNSUPPORTED);
}

// ---------------------------------------------------------------- batched MPK
// Plans of a batch may differ in block width and number of powers; the node
// dispatches on the plan's nrhs.
// Gather budget of the batch's row kernel: 16-byte gathers of 16 values in
// FP32; scalar gathers in FP64 (fits the batch kernel's register budget).
template <typename VT>
constexpr int kBatchGatherBudget = sizeof(VT) == 4 ? 16 : 0;

template <typename VT, typename MT>
struct BatchNode {
    static constexpr bool kL2First = false;
    static constexpr bool kPipe = false;
    template <typename Extra, int PC>
    __device__ __forceinline__ static void pipe_run(const ExecArgs &, const Slice<MT, PC> &, int32_t, int32_t, int, int,
                                                    int, const Extra &) {}

    template <bool STAGED>
    __device__ __forceinline__ static void run(const ExecArgs &a, const MatView<MT, STAGED> &mv, int32_t t, int32_t k,
                                               int warp, int nwarps, int lane, const int &x) {
        constexpr int GB = kBatchGatherBudget<VT>;
        switch (a.nrhs) {
        case 1: MpkNode<VT, MT, 1, true, false, GB>::template run<STAGED>(a, mv, t, k, warp, nwarps, lane, x); break;
        case 2: MpkNode<VT, MT, 2, true, false, GB>::template run<STAGED>(a, mv, t, k, warp, nwarps, lane, x); break;
        case 4: MpkNode<VT, MT, 4, true, false, GB>::template run<STAGED>(a, mv, t, k, warp, nwarps, lane, x); break;
        case 8: MpkNode<VT, MT, 8, true, false, GB>::template run<STAGED>(a, mv, t, k, warp, nwarps, lane, x); break;
        default: MpkNode<VT, MT, 8, false, false, GB>::template run<STAGED>(a, mv, t, k, warp, nwarps, lane, x); break;
        }
    }
};

#ifndef MPK_BATCH_MIN_BLOCKS
#define MPK_BATCH_MIN_BLOCKS 4
#endif
// Four CTAs per SM: the batch's items are short and latency-bound, so
// resident warps matter more than the gathers in flight per lane.
template <typename VT, typename MT>
__global__ void __launch_bounds__(kWaveThreads, MPK_BATCH_MIN_BLOCKS) k_batch_wave(BatchArgs b) {
    __shared__ uint32_t s_epochs[kMaxBatch];
    for (int32_t m = threadIdx.x; m < b.count; m += blockDim.x)
        s_epochs[m] = (uint32_t)ld_relaxed_s32(b.plan_ctl[m] + CTL_EPOCH) + 1u;
    __syncthreads();
    const ManyPlans src{b.table, b.wplan, s_epochs, b.plan_ctl, b.count};
    wave_loop<BatchNode<VT, MT>, MT, false>(b.g, src, 0);
}

// acc = coef_0 * v_0 (complex for G = 2, real for G = 1), v_0 = ring block 0,
// before the first sweep: FP64 for FP64 plans, double-float pairs (the
// node's arithmetic, from zero) for FP32 plans.
template <int G>
__global__ void k_cheb_init_f64(int32_t n, const double *v0, const double *coef, double *acc) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    if (G == 2) {
        const double x0 = v0[2 * r], x1 = v0[2 * r + 1];
        acc[2 * r] = fma(coef[0], x0, fma(-coef[1], x1, 0.0));
        acc[2 * r + 1] = fma(coef[0], x1, fma(coef[1], x0, 0.0));
    } else {
        acc[r] = fma(coef[0], v0[r], 0.0);
    }
}
template <int G>
__global__ void k_cheb_init_df(int32_t n, const float *v0, const float4 *coef_df, float *acc) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const float4 c = coef_df[0];
    if (G == 2) {
        const float x0 = v0[2 * r], x1 = v0[2 * r + 1];
        float a[4] = {0.f, 0.f, 0.f, 0.f};
        dot2_add(a[0], a[1], c.x, c.y, x0);
        dot2_add(a[0], a[1], -c.z, -c.w, x1);
        dot2_add(a[2], a[3], c.x, c.y, x1);
        dot2_add(a[2], a[3], c.z, c.w, x0);
        reinterpret_cast<float4 *>(acc)[r] = make_float4(a[0], a[1], a[2], a[3]);
    } else {
        float a[2] = {0.f, 0.f};
        dot2_add(a[0], a[1], c.x, c.y, v0[r]);
        reinterpret_cast<float2 *>(acc)[r] = make_float2(a[0], a[1]);
    }
}

// y[r] = hi + lo in FP64 for each column of row idx[r] (idx = NULL: row r)
// of a double-float sum.  With idx = NULL, y may be the sum itself (each row's
// 8G bytes are read, then written, by the same thread).
template <int G>
__global__ void k_cheb_df_to_f64(int32_t n, const float *acc, const int32_t *__restrict__ idx, double *y) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t from = idx ? (int64_t)__ldg(idx + r) : r;
        if (G == 2) {
            const float4 t = reinterpret_cast<const float4 *>(acc)[from];
            const double2 o = make_double2((double)t.x + (double)t.y, (double)t.z + (double)t.w);
            reinterpret_cast<double2 *>(y)[r] = o;
        } else {
            const float2 t = reinterpret_cast<const float2 *>(acc)[from];
            y[r] = (double)t.x + (double)t.y;
        }
    }
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
            const int32_t r = a.row_map ? a.row_map[row0 + lane] : row0 + lane;
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

// dst[r] = src[idx[r]] for the n rows of block blockIdx.y (rows of wpr
// words of type W: 4, 8 or 16 bytes).  Both directions of the level
// permutation are gathers (idx = perm into level order, iperm out of it):
// the stores are coalesced, and the scattered loads of one block (one
// vector) find its lines in L2, where consecutive blocks follow.
template <typename W>
__global__ void k_permute(int32_t n, int32_t wpr, const int32_t *__restrict__ idx, const W *__restrict__ src,
                          W *__restrict__ dst) {
    const int64_t base = (int64_t)blockIdx.y * n * wpr;
    for (int32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        const int64_t from = base + (int64_t)__ldg(idx + r) * wpr, to = base + (int64_t)r * wpr;
        for (int32_t w = 0; w < wpr; w++) dst[to + w] = src[from + w];
    }
}

// ---------------------------------------------------------------- dispatch
template <typename VT, typename MT, bool DIAG, bool STAGED, int NW, bool COUNT>
const void *wave_ptr_c(int nrhs) {
    switch (nrhs) {
    case 1: return (const void *)k_wave<VT, MT, 1, true, DIAG, STAGED, NW, COUNT>;
    case 2: return (const void *)k_wave<VT, MT, 2, true, DIAG, STAGED, NW, COUNT>;
    case 4: return (const void *)k_wave<VT, MT, 4, true, DIAG, STAGED, NW, COUNT>;
    case 8: return (const void *)k_wave<VT, MT, 8, true, DIAG, STAGED, NW, COUNT>;
    default: return (const void *)k_wave<VT, MT, 8, false, DIAG, STAGED, NW, COUNT>;
    }
}
// plans whose dependency ranges all fit a probe run the variant without counters
template <typename VT, typename MT, bool DIAG, bool STAGED, int NW = kComputeWarps>
const void *wave_ptr(const Plan *pl) {
    return pl->wide_deps ? wave_ptr_c<VT, MT, DIAG, STAGED, NW, true>(pl->nrhs)
                         : wave_ptr_c<VT, MT, DIAG, STAGED, NW, false>(pl->nrhs);
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

template <typename VT, typename MT, bool DIAG, int NW>
const void *staged_wave_ptr(int nrhs) {   // the staged form runs block widths 1 and 2
    return nrhs == 1 ? (const void *)k_wave<VT, MT, 1, true, DIAG, true, NW, true>
                     : (const void *)k_wave<VT, MT, 2, true, DIAG, true, NW, true>;
}
template <bool STAGED>
const void *pick_wave_t(const Plan *pl) {
    if constexpr (STAGED) {
        if (pl->prec == MPK_F64) return staged_wave_ptr<double, double, false, kFp64Warps>(pl->nrhs);
        if (!pl->has_diag) return staged_wave_ptr<float, float, false, kFp32Warps>(pl->nrhs);
        if (pl->val_bytes == 2) return staged_wave_ptr<float, __nv_bfloat16, true, kFp32Warps>(pl->nrhs);
        return staged_wave_ptr<float, float, true, kFp32Warps>(pl->nrhs);
    } else {
        if (pl->prec == MPK_F64) return wave_ptr<double, double, false, false, kFp64Warps>(pl);
        if (!pl->has_diag) return wave_ptr<float, float, false, false, kFp32Warps>(pl);
        if (pl->val_bytes == 2) return wave_ptr<float, __nv_bfloat16, true, false, kFp32Warps>(pl);
        return wave_ptr<float, float, true, false, kFp32Warps>(pl);
    }
}
template <bool STAGED, int G>
const void *pick_cheb_g(const Plan *pl, bool multi) {
    if (multi) {
        if (pl->prec == MPK_F64)
            return G == 1 ? (const void *)k_cheb_wave_f64r<STAGED, true>
                          : (const void *)k_cheb_wave<double, double, false, STAGED, G, true>;
        if (!pl->has_diag) return (const void *)k_cheb_wave<float, float, false, STAGED, G, true>;
        if (pl->val_bytes == 2) return (const void *)k_cheb_wave<float, __nv_bfloat16, true, STAGED, G, true>;
        return (const void *)k_cheb_wave<float, float, true, STAGED, G, true>;
    }
    if (pl->prec == MPK_F64)
        return G == 1 ? (const void *)k_cheb_wave_f64r<STAGED, false>
                      : (const void *)k_cheb_wave<double, double, false, STAGED, G, false>;
    if (!pl->has_diag) return (const void *)k_cheb_wave<float, float, false, STAGED, G, false>;
    if (pl->val_bytes == 2) return (const void *)k_cheb_wave<float, __nv_bfloat16, true, STAGED, G, false>;
    return (const void *)k_cheb_wave<float, float, true, STAGED, G, false>;
}
template <bool STAGED>
const void *pick_cheb_t(const Plan *pl, bool multi) {
    return pl->nrhs == 1 ? pick_cheb_g<STAGED, 1>(pl, multi) : pick_cheb_g<STAGED, 2>(pl, multi);
}
template <int W>
const void *pick_res_w(const Plan *pl) {
    if (pl->prec == MPK_F64) return (const void *)k_res_wave<double, double, W, false>;
    if (!pl->has_diag) return (const void *)k_res_wave<float, float, W, false>;
    if (pl->val_bytes == 2) return (const void *)k_res_wave<float, __nv_bfloat16, W, true>;
    return (const void *)k_res_wave<float, float, W, true>;
}
template <int G>
const void *pick_res_cheb_g(const Plan *pl) {
    if (pl->prec == MPK_F64) return (const void *)k_res_cheb<double, double, false, G>;
    if (!pl->has_diag) return (const void *)k_res_cheb<float, float, false, G>;
    if (pl->val_bytes == 2) return (const void *)k_res_cheb<float, __nv_bfloat16, true, G>;
    return (const void *)k_res_cheb<float, float, true, G>;
}
const void *pick_res_cheb(const Plan *pl) { return pl->nrhs == 1 ? pick_res_cheb_g<1>(pl) : pick_res_cheb_g<2>(pl); }
const void *pick_wave(const Plan *pl) {
    if (pl->prec == MPK_F64_DF)
        return pl->val_bytes == 4 ? (const void *)k_wave_df<float> : (const void *)k_wave_df<float2>;
    if (pl->resident) return pl->nrhs == 1 ? pick_res_w<1>(pl) : pick_res_w<2>(pl);
    return pl->staged ? pick_wave_t<true>(pl) : pick_wave_t<false>(pl);
}

}  // namespace

const void *batch_kernel(int prec) {
    return prec == MPK_F64 ? (const void *)k_batch_wave<double, double> : (const void *)k_batch_wave<float, float>;
}

namespace {

const void *pick_cheb(const Plan *pl, bool multi = true) {
    if (pl->resident) return pick_res_cheb(pl);
    return pl->staged ? pick_cheb_t<true>(pl, multi) : pick_cheb_t<false>(pl, multi);
}
const void *pick_spmv(const Plan *pl) {
    if (pl->prec == MPK_F64) return spmv_ptr<double, double, false>(pl->nrhs);
    if (!pl->has_diag) return spmv_ptr<float, float, false>(pl->nrhs);
    if (pl->val_bytes == 2) return spmv_ptr<float, __nv_bfloat16, true>(pl->nrhs);
    return spmv_ptr<float, float, true>(pl->nrhs);
}

}  // namespace

// Resident CTAs per SM of the plan's MPK wavefront kernel and of its
// Chebyshev kernel (with the plan's dynamic shared memory; 1 << 30 when the
// plan has no Chebyshev kernel); also raises the kernels' limit of dynamic
// shared memory to what the plan needs.
int wave_occupancy(const Plan *pl, int *wave_ctas, int *cheb_ctas) {
    // the MPK kernel, then the Chebyshev kernels (single- and multi-step)
    const bool cheb = pl->nrhs <= 2 && pl->prec != MPK_F64_DF;
    const void *fns[3] = {pick_wave(pl), cheb ? pick_cheb(pl, false) : nullptr, cheb ? pick_cheb(pl, true) : nullptr};
    const int threads[3] = {wave_threads(pl), cheb_threads(pl), cheb_threads(pl)};
    int occ[3] = {1 << 30, 1 << 30, 1 << 30};
    for (int i = 0; i < 3; i++) {
        if (!fns[i]) continue;
        MPK_CUDA(cudaFuncSetAttribute(fns[i], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl->smem_bytes));
        MPK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[i], fns[i], threads[i], pl->smem_bytes));
    }
    *wave_ctas = occ[0];
    *cheb_ctas = std::min(occ[1], occ[2]);
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
    a.fstride = pl->fstride;
    a.bcnt = pl->wide_deps ? pl->d_bcnt : nullptr;
    a.bstride = pl->bstride;
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
    a.tile_off = pl->d_tile_off;
    a.row_map = pl->d_row_map;
    a.chunk_rec = pl->d_chunk_rec;
    a.stage_recs = pl->stage_recs;
    a.stage_entries = pl->stage_entries;
    a.tune = pl->tune;
    a.n_stages = pl->n_stages;
    a.shadow = pl->d_shadow;
    return a;
}

// Cooperative launch (all CTAs co-resident), expressed with cudaLaunchKernelEx
// so that it can also be captured in a CUDA graph.
int launch_coop(const void *fn, int grid, size_t smem, void **args, cudaStream_t st, int threads) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    MPK_CUDA(cudaLaunchKernelExC(&cfg, fn, args));
    return MPK_OK;
}

// Epochs are 32-bit: before they could wrap onto stale flag values, clear all.
static int epoch_guard(Plan *pl, cudaStream_t st) {
    if (pl->launches >= 0xFFFFFF00ull) {
        MPK_CUDA(cudaMemsetAsync(pl->d_flags, 0, sizeof(uint32_t) * (size_t)(pl->p + 1) * pl->fstride, st));
        MPK_CUDA(cudaMemsetAsync(pl->d_ctl, 0, sizeof(int32_t) * CTL_WORDS, st));
        pl->launches = 0;
    }
    pl->launches++;
    return MPK_OK;
}

// Double-float plans: x split into pairs (shadow block 0), with the range guard.
static int df_split(Plan *pl, const void *x, cudaStream_t st) {
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(((int64_t)pl->n + 255) / 256, (int64_t)pl->num_sms * 8));
    k_df_split<<<g, 256, 0, st>>>(pl->n, (const double *)x, pl->d_shadow, pl->df_xlim_bits, pl->d_ctl);
    MPK_CUDA(cudaGetLastError());
    return MPK_OK;
}

int launch_wavefront(Plan *pl, const void *x, void *Y, cudaStream_t st) {
    int rc = epoch_guard(pl, st);
    if (rc) return rc;
    if (pl->prec == MPK_F64_DF && (rc = df_split(pl, x, st))) return rc;
    ExecArgs a = exec_args(pl, x, Y);
    a.drop_tile = pl->drop_tile;
    a.drop_k = pl->drop_k;
    pl->drop_tile = pl->drop_k = -1;
    void *args[] = {(void *)&a};
    return launch_coop(pick_wave(pl), pl->grid_ctas, pl->smem_bytes, args, st, wave_threads(pl));
}

int launch_baseline(Plan *pl, const void *x, void *Y, cudaStream_t st) {
    ExecArgs a = exec_args(pl, x, Y);
    if (pl->prec == MPK_F64_DF) {
        int rc = df_split(pl, x, st);
        if (rc) return rc;
        const void *fn = pl->val_bytes == 4 ? (const void *)k_spmv_df<float> : (const void *)k_spmv_df<float2>;
        int occ = 0;
        MPK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kSpmvThreads, 0));
        const int wpb = kSpmvThreads / 32;
        const int64_t grid = std::max<int64_t>(
            1, std::min<int64_t>((int64_t)pl->num_sms * std::max(1, occ), ((int64_t)pl->n_chunks + wpb - 1) / wpb));
        for (int32_t k = 1; k <= pl->p; k++) {
            void *args[] = {(void *)&a, (void *)&k};
            MPK_CUDA(cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(kSpmvThreads), args, 0, st));
        }
        return MPK_OK;
    }
    const void *fn = pick_spmv(pl);
    int occ = 0;
    MPK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kSpmvThreads, 0));
    int64_t warps_needed = pl->n_chunks;
    const int wpb = kSpmvThreads / 32;
    int64_t grid = std::min<int64_t>((int64_t)pl->num_sms * std::max(1, occ), (warps_needed + wpb - 1) / wpb);
    grid = std::max<int64_t>(1, grid);
    const size_t eb = (size_t)elem_bytes_of(pl);
    for (int k = 1; k <= pl->p; k++) {
        const void *yin = k == 1 ? x : (const char *)Y + (size_t)(k - 2) * a.blk * eb;
        void *yout = (char *)Y + (size_t)(k - 1) * a.blk * eb;
        void *args[] = {(void *)&a, (void *)&yin, (void *)&yout};
        MPK_CUDA(cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(kSpmvThreads), args, 0, st));
    }
    return MPK_OK;
}

// One SpMV of the plan's packed matrix, y = A x (x, y: n x nrhs in level
// order, the plan's element type): the row kernel of the baseline.
int launch_spmv1(Plan *pl, const void *x, void *y, cudaStream_t st) {
    if (pl->prec == MPK_F64_DF) return MPK_ERR_UNSUPPORTED;
    ExecArgs a = exec_args(pl, x, y);
    const void *fn = pick_spmv(pl);
    int occ = 0;
    MPK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kSpmvThreads, 0));
    const int wpb = kSpmvThreads / 32;
    const int64_t grid = std::max<int64_t>(
        1, std::min<int64_t>((int64_t)pl->num_sms * std::max(1, occ), ((int64_t)pl->n_chunks + wpb - 1) / wpb));
    void *args[] = {(void *)&a, (void *)&x, (void *)&y};
    MPK_CUDA(cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(kSpmvThreads), args, 0, st));
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
    const int32_t row_bytes = pl->nrhs * elem_bytes;
    if ((uintptr_t)src % 4 || (uintptr_t)dst % 4) return MPK_ERR_INVALID;   // elements are 4 or 8 bytes
    if ((int64_t)pl->n * count == 0) return MPK_OK;
    const int32_t *idx = to_level ? pl->d_perm : pl->d_iperm;
    // widest word that divides the row and both base addresses
    const uintptr_t align = (uintptr_t)src | (uintptr_t)dst | (uintptr_t)row_bytes;
    const size_t blk_bytes = (size_t)pl->n * row_bytes;
    for (int32_t b0 = 0; b0 < count; b0 += 65535) {   // grid rows: one per vector block
        const char *s = (const char *)src + blk_bytes * (size_t)b0;
        char *d = (char *)dst + blk_bytes * (size_t)b0;
        const dim3 grid((unsigned)std::min<int64_t>((pl->n + 255) / 256, (int64_t)pl->num_sms * 8),
                        (unsigned)std::min(count - b0, 65535));
        if (align % 16 == 0)
            k_permute<uint4><<<grid, 256, 0, st>>>(pl->n, row_bytes / 16, idx, (const uint4 *)s, (uint4 *)d);
        else if (align % 8 == 0)
            k_permute<uint2><<<grid, 256, 0, st>>>(pl->n, row_bytes / 8, idx, (const uint2 *)s, (uint2 *)d);
        else
            k_permute<uint32_t><<<grid, 256, 0, st>>>(pl->n, row_bytes / 4, idx, (const uint32_t *)s, (uint32_t *)d);
        MPK_CUDA(cudaGetLastError());
    }
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

int mpk_run_host(mpk_plan_t plan, const void *x_host, void *Y_host, uint32_t flags) {
    if (!plan || !x_host || !Y_host) return MPK_ERR_INVALID;
    Plan *pl = &plan->pl;
    cudaStream_t st = pl->stream;
    const int eb = elem_bytes_of(pl);
    const size_t blk = (size_t)pl->n * pl->nrhs * eb;
    const bool level_io = flags & MPK_IO_PERMUTED;
    int rc = ensure_io(pl, blk * (size_t)(pl->p + 3));
    if (rc) return rc;
    if (!pl->copy_stream) MPK_CUDA(cudaStreamCreateWithFlags(&pl->copy_stream, cudaStreamNonBlocking));
    for (cudaEvent_t &e : pl->io_ev)
        if (!e) MPK_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    char *xb = (char *)pl->d_io, *yb = xb + blk, *stage = yb + blk * (size_t)pl->p;
    // input: host -> device, into level order
    MPK_CUDA(cudaMemcpyAsync(level_io ? xb : stage, x_host, blk, cudaMemcpyHostToDevice, st));
    if (!level_io && (rc = permute_vectors(pl, stage, xb, 1, eb, 1, st))) return rc;
    if ((rc = launch_wavefront(pl, xb, yb, st))) return rc;
    // outputs: each power into the caller's numbering (two staging blocks,
    // alternating), then device -> host on the copy stream
    for (int32_t k = 0; k < pl->p; k++) {
        const char *src = yb + blk * (size_t)k;
        if (!level_io) {
            char *sb = stage + blk * (size_t)(k & 1);
            if (k >= 2) MPK_CUDA(cudaStreamWaitEvent(st, pl->io_ev[2 + (k & 1)], 0));   // copy of power k-2 done
            if ((rc = permute_vectors(pl, src, sb, 1, eb, 0, st))) return rc;
            src = sb;
        }
        MPK_CUDA(cudaEventRecord(pl->io_ev[k & 1], st));
        MPK_CUDA(cudaStreamWaitEvent(pl->copy_stream, pl->io_ev[k & 1], 0));
        MPK_CUDA(cudaMemcpyAsync((char *)Y_host + blk * (size_t)k, src, blk, cudaMemcpyDeviceToHost,
                                 pl->copy_stream));
        MPK_CUDA(cudaEventRecord(pl->io_ev[2 + (k & 1)], pl->copy_stream));
    }
    // the plan's stream covers the copies too
    MPK_CUDA(cudaStreamWaitEvent(st, pl->io_ev[2 + ((pl->p - 1) & 1)], 0));
    if (flags & MPK_ASYNC) return MPK_OK;
    return read_device_error(pl, st);
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
    return read_device_error(pl, pl->stream);   // the double-float range guard reports here
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
    if (pl->prec == MPK_F64_DF && pl->val_bytes == 8) k_gersh<float2><<<grid, 256, 0, st>>>(a, d);
    else if (pl->val_bytes == 8) k_gersh<double><<<grid, 256, 0, st>>>(a, d);
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

// Splits x into FP32 hi + lo with hi = x rounded to FP32 (exact pairs for
// the double-float node).
static inline void split_f64(double x, float &hi, float &lo) {
    hi = (float)x;
    lo = (float)(x - (double)hi);
}

// Chebyshev propagation with G vector columns (2: complex state and
// coefficients, 1: real); the plan's block width must be G.
static int cheb_run(mpk_plan_t plan, const double *coef, int32_t M, double c, double r, const void *x, double *y,
                    uint32_t flags, int G, int32_t T) {
    if (!plan || !coef || !x || !y || M < 1 || T < 1 || !(r != 0.0) || (int64_t)M * T > INT32_MAX / 2)
        return MPK_ERR_INVALID;
    Plan *pl = &plan->pl;
    if (pl->nrhs != G) return MPK_ERR_INVALID;
    if (pl->prec == MPK_F64_DF) return MPK_ERR_UNSUPPORTED;
    cudaStream_t st = pl->stream;
    const int eb = elem_bytes_of(pl);
    const bool df = eb == 4;   // FP32 vectors: double-float scaling and coefficient sum
    const size_t blk = (size_t)pl->n * G;
    std::vector<float4> cdf;
    ChebArgs ca;
    ca.alpha = 1.0 / r;
    ca.beta = -c / r;
    if (df) {
        // the pairs must stay inside FP32's range
        const double lim = 1e30;
        if (!(std::fabs(ca.alpha) <= lim && std::fabs(ca.beta) <= lim && std::fabs(c) <= lim)) return MPK_ERR_UNSUPPORTED;
        cdf.resize((size_t)M + 1);
        for (int32_t k = 0; k <= M; k++) {
            const double re = coef[(size_t)G * k], im = G == 2 ? coef[(size_t)G * k + 1] : 0.0;
            if (!(std::fabs(re) <= lim && std::fabs(im) <= lim)) return MPK_ERR_UNSUPPORTED;
            split_f64(re, cdf[k].x, cdf[k].y);
            split_f64(im, cdf[k].z, cdf[k].w);
        }
        split_f64(ca.alpha, ca.alpha_hi, ca.alpha_lo);
        split_f64(ca.beta, ca.beta_hi, ca.beta_lo);
        split_f64(c, ca.c_hi, ca.c_lo);
    }
    // device storage: 3-block ring (storage precision), the coefficient sum
    // (FP64, or double-float pairs of the same size) unless it lives in y,
    // and the coefficients (FP64 and double-float tables)
    const size_t ring_b = 3 * blk * eb, acc_b = (flags & MPK_IO_PERMUTED) ? 0 : blk * sizeof(double);
    const size_t coef_b = sizeof(double) * G * ((size_t)M + 1), coefdf_b = sizeof(float4) * ((size_t)M + 1);
    const size_t need = ring_b + acc_b + coef_b + coefdf_b + 256;
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
    void *acc = (flags & MPK_IO_PERMUTED) ? (void *)y : (void *)(base + ring_b);
    double *dcoef = (double *)(base + ring_b + acc_b);
    float4 *dcoef_df = (float4 *)(((uintptr_t)(base + ring_b + acc_b + coef_b) + 15) & ~(uintptr_t)15);
    MPK_CUDA(cudaMemcpyAsync(dcoef, coef, coef_b, cudaMemcpyHostToDevice, st));
    if (df) MPK_CUDA(cudaMemcpyAsync(dcoef_df, cdf.data(), coefdf_b, cudaMemcpyHostToDevice, st));
    int rc;
    if (flags & MPK_IO_PERMUTED) {
        MPK_CUDA(cudaMemcpyAsync(ring, x, blk * eb, cudaMemcpyDeviceToDevice, st));
    } else if ((rc = permute_vectors(pl, x, ring, 1, eb, 1, st))) {
        return rc;
    }
    const unsigned nb = (unsigned)((pl->n + 255) / 256);
    if (G == 2) {
        if (!df) k_cheb_init_f64<2><<<nb, 256, 0, st>>>(pl->n, (const double *)ring, dcoef, (double *)acc);
        else k_cheb_init_df<2><<<nb, 256, 0, st>>>(pl->n, (const float *)ring, dcoef_df, (float *)acc);
    } else {
        if (!df) k_cheb_init_f64<1><<<nb, 256, 0, st>>>(pl->n, (const double *)ring, dcoef, (double *)acc);
        else k_cheb_init_df<1><<<nb, 256, 0, st>>>(pl->n, (const float *)ring, dcoef_df, (float *)acc);
    }
    MPK_CUDA(cudaGetLastError());
    ca.ring = ring;
    ca.acc = acc;
    ca.coef = dcoef;
    ca.coef_df = dcoef_df;
    ca.M = M;
    ca.total = M * T;
    // sweeps of p powers over all T*M powers: a sweep may run across time
    // steps (the node of a step's last power hands v_0 to the next step)
    const int32_t sweep = (flags & MPK_SWEEP_ONE) ? 1 : pl->p;
    for (int32_t k0 = 0; k0 < ca.total; k0 += sweep) {
        const int32_t pw = std::min(sweep, ca.total - k0);
        if ((rc = epoch_guard(pl, st))) return rc;
        ca.e = exec_args(pl, nullptr, nullptr);
        if (pw < pl->p) {   // a shorter last sweep has its own issue order
            if (pl->rem_p != pw) {
                std::vector<int32_t> work;
                order_items(pl, pw, pl->lag, work);
                if (pl->d_work_rem) {
                    cudaStreamSynchronize(st);
                    cudaFree(pl->d_work_rem);
                    pl->d_work_rem = nullptr;
                }
                if ((rc = dev_alloc<int32_t>(nullptr, &pl->d_work_rem, work.size()))) return rc;
                MPK_CUDA(cudaMemcpyAsync(pl->d_work_rem, work.data(), work.size() * 4, cudaMemcpyHostToDevice, st));
                MPK_CUDA(cudaStreamSynchronize(st));
                pl->rem_p = pw;
            }
            ca.e.work = pl->d_work_rem;
            ca.e.n_items = pl->n_tiles * pw;
            ca.e.p = pw;
        }
        ca.k0 = k0;
        ca.pw = pw;
        ca.step0 = k0 / M;
        ca.kin0 = k0 % M + 1;
        void *args[] = {(void *)&ca};
        if ((rc = launch_coop(pick_cheb(pl, T > 1), pl->cheb_grid, pl->smem_bytes, args, st, cheb_threads(pl))))
            return rc;
    }
    if (df) {
        // double-float sum -> FP64 y (in place in level order, else gathered
        // into the caller's numbering)
        const int32_t *idx = (flags & MPK_IO_PERMUTED) ? nullptr : pl->d_iperm;
        const unsigned g = (unsigned)std::min<int64_t>(((int64_t)pl->n + 255) / 256, (int64_t)pl->num_sms * 8);
        if (G == 2) k_cheb_df_to_f64<2><<<g, 256, 0, st>>>(pl->n, (const float *)acc, idx, y);
        else k_cheb_df_to_f64<1><<<g, 256, 0, st>>>(pl->n, (const float *)acc, idx, y);
    } else if (!(flags & MPK_IO_PERMUTED)) {
        // acc (level order, n x G doubles) -> y (original order)
        if ((rc = permute_vectors(pl, acc, y, 1, 8, 0, st))) return rc;
    }
    MPK_CUDA(cudaGetLastError());
    if (flags & MPK_ASYNC) return MPK_OK;
    return read_device_error(pl, st);
}

int mpk_cheb(mpk_plan_t plan, const double *coef, int32_t M, double c, double r, const void *x, double *y,
             uint32_t flags) {
    return cheb_run(plan, coef, M, c, r, x, y, flags, 2, 1);
}

int mpk_cheb_real(mpk_plan_t plan, const double *coef, int32_t M, double c, double r, const void *x, double *y,
                  uint32_t flags) {
    return cheb_run(plan, coef, M, c, r, x, y, flags, 1, 1);
}

int mpk_cheb_steps(mpk_plan_t plan, const double *coef, int32_t M, double c, double r, int32_t nsteps, const void *x,
                   double *y, uint32_t flags) {
    if (!plan) return MPK_ERR_INVALID;
    const int32_t G = plan->pl.nrhs;
    if (G != 1 && G != 2) return MPK_ERR_INVALID;
    return cheb_run(plan, coef, M, c, r, x, y, flags, G, nsteps);
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

int mpk_cheb_coeffs_heat(int32_t M, double c, double r, double tau, double *coef) {
    if (M < 0 || !coef || !(r > 0.0) || !(tau >= 0.0)) return MPK_ERR_INVALID;
    // exp(-tau c) (2 - delta_k0) (-1)^k I_k(tau r).  The scaled values
    // I_k(z) e^{-z} come from Miller's backward recurrence
    // I_{k-1} = I_{k+1} + (2k/z) I_k, started far above the wanted orders with
    // arbitrary small values and normalised by e^z = I_0 + 2 sum_{k>=1} I_k.
    const double z = tau * r;
    std::vector<double> ik((size_t)M + 1, 0.0);
    if (z == 0.0) {
        ik[0] = 1.0;
    } else {
        const int32_t top = std::max<int32_t>(M, (int32_t)std::ceil(10.0 * std::sqrt(z) + z / 4.0)) + 48;
        double hi = 0.0, cur = 1e-300, sum = 0.0;   // I_{k+1}, I_k (unnormalised)
        for (int32_t k = top; k >= 1; k--) {
            const double lo = hi + (2.0 * k / z) * cur;   // I_{k-1}
            hi = cur;
            cur = lo;
            sum += 2.0 * hi;                            // 2 I_k
            if (k - 1 <= M) ik[(size_t)(k - 1)] = cur;
            if (cur > 1e250) {                           // rescale to stay in range
                for (int32_t q = k - 1; q <= M; q++) ik[(size_t)q] *= 1e-250;
                hi *= 1e-250;
                cur *= 1e-250;
                sum *= 1e-250;
            }
        }
        sum += cur;   // + I_0
        for (int32_t q = 0; q <= M; q++) ik[(size_t)q] /= sum;
    }
    const double scale = std::exp(-tau * (c - r));
    for (int32_t k = 0; k <= M; k++) coef[k] = (k == 0 ? 1.0 : 2.0) * ((k & 1) ? -1.0 : 1.0) * scale * ik[(size_t)k];
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
