// Krylov solvers that consume the matrix-power kernel (Sec. 1: s-step Krylov
// methods build their Krylov basis of s powers with one MPK).  Conjugate
// gradients (Hestenes and Stiefel) as the comparator, and s-step CG with the
// monomial basis: one level-blocked MPK of the block [p r] per s steps, its
// Gram matrix, s steps of CG on coordinate vectors, one fused update.  All
// vectors live in the plan's level order on the device; FP64 throughout.
#include <algorithm>
#include <cmath>
#include <vector>

#include "mpk_internal.cuh"

namespace mpk {
namespace {

constexpr int kRedThreads = 256;
constexpr int kMaxS = 16;                    // basis of 2s+1 <= 33 columns
constexpr int kMaxCols = 2 * kMaxS + 1;
constexpr int kGramRows = 64;                // rows of V per shared-memory tile

int red_blocks(const Plan *pl) { return pl->num_sms * 4; }

// partial[blockIdx.x] = sum over the block's rows of a[i] * b[i] (a fixed
// order per block; the blocks' sums are added by k_sum_partials in order, so
// the result does not change from run to run)
__global__ void __launch_bounds__(kRedThreads) k_dot_partial(int64_t n, const double *a, const double *b,
                                                             double *partial) {
    __shared__ double sw[kRedThreads / 32];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s = fma(a[i], b[i], s);
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kRedThreads / 32; w++) t += sw[w];
        partial[blockIdx.x] = t;
    }
}

// out[q] = sum_b partial[b * count + q], b ascending (one thread per q)
__global__ void k_sum_partials(const double *partial, int32_t nblk, int32_t count, double *out) {
    const int32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= count) return;
    double t = 0.0;
    for (int32_t b = 0; b < nblk; b++) t += partial[(int64_t)b * count + q];
    out[q] = t;
}

// ------------------------------------------------------------------ CG
// Scalars on the device: sc[0] = r.r, sc[1] = p.q, sc[2] = the new r.r.
// r = b - q, p = r
__global__ void k_cg_start(int64_t n, const double *b, const double *q, double *r, double *p) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = b[i] - q[i];
        r[i] = v;
        p[i] = v;
    }
}
// alpha = sc[0] / sc[1] (0 once the residual is exactly zero); x += alpha p; r -= alpha q
__global__ void k_cg_step(int64_t n, const double *sc, double *x, double *r, const double *p, const double *q) {
    const double alpha = sc[1] != 0.0 ? sc[0] / sc[1] : 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        x[i] = fma(alpha, p[i], x[i]);
        r[i] = fma(-alpha, q[i], r[i]);
    }
}
// beta = sc[2] / sc[0] (0 once the residual is exactly zero); p = r + beta p.
// The new r.r moves to sc[0] in a launch of its own (k_cg_roll), after every
// thread of this one has read the old value.
__global__ void k_cg_dir(int64_t n, const double *sc, const double *r, double *p) {
    const double beta = sc[0] != 0.0 ? sc[2] / sc[0] : 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = fma(beta, p[i], r[i]);
}
__global__ void k_cg_roll(double *sc) { sc[0] = sc[2]; }

// ------------------------------------------------------------------ s-step CG
// Column c of the basis V at row i (m = 2s+1 columns): the p block
// p, Ap/rho, .., A^s p/rho^s, then the r block r, Ar/rho, .., A^(s-1) r/rho^(s-1);
// X = [p r] (n x 2), Y = the MPK of X (s blocks of n x 2).
struct Basis {
    const double *X, *Y;
    int64_t n;
    int32_t s;
    double scale[kMaxS + 1];   // rho^-k
    __device__ __forceinline__ double at(int64_t i, int32_t c) const {
        const int32_t col = c <= s ? 0 : 1;
        const int32_t k = c <= s ? c : c - s - 1;
        return k == 0 ? X[2 * i + col] : Y[(int64_t)(k - 1) * 2 * n + 2 * i + col] * scale[k];
    }
};

// Per-block partial Gram matrix (upper triangle, npairs = m(m+1)/2 entries in
// row-major pair order) over the block's tiles of kGramRows rows.
__global__ void __launch_bounds__(kRedThreads) k_gram_partial(Basis V, int32_t m, double *partial) {
    __shared__ double tile[kGramRows][kMaxCols];
    const int32_t npairs = m * (m + 1) / 2;
    constexpr int kPer = (kMaxCols * (kMaxCols + 1) / 2 + kRedThreads - 1) / kRedThreads;
    double acc[kPer];
    int32_t pa[kPer], pb[kPer];
#pragma unroll
    for (int q = 0; q < kPer; q++) {
        acc[q] = 0.0;
        int32_t idx = threadIdx.x + q * kRedThreads, a = 0;
        while (idx >= m - a && a < m) { idx -= m - a; a++; }   // pair number -> (a, a + idx)
        pa[q] = a;
        pb[q] = a + idx;
    }
    const int64_t ntiles = (V.n + kGramRows - 1) / kGramRows;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t r0 = t * kGramRows;
        __syncthreads();
        for (int32_t e = threadIdx.x; e < kGramRows * m; e += blockDim.x) {
            const int32_t ri = e / m, c = e % m;
            tile[ri][c] = r0 + ri < V.n ? V.at(r0 + ri, c) : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kPer; q++) {
            if (threadIdx.x + q * kRedThreads >= npairs) continue;
            double s = acc[q];
            for (int ri = 0; ri < kGramRows; ri++) s = fma(tile[ri][pa[q]], tile[ri][pb[q]], s);
            acc[q] = s;
        }
    }
#pragma unroll
    for (int q = 0; q < kPer; q++)
        if (threadIdx.x + q * kRedThreads < npairs) partial[(int64_t)blockIdx.x * npairs + threadIdx.x + q * kRedThreads] = acc[q];
}

struct Coords {
    double x[kMaxCols], r[kMaxCols], p[kMaxCols];
};

// x += V x', then X = [V p', V r'] in place (row i is read, then written, by
// one thread)
__global__ void k_sstep_update(Basis V, int32_t m, Coords c, double *x, double *X) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < V.n; i += (int64_t)gridDim.x * blockDim.x) {
        double dx = 0.0, np = 0.0, nr = 0.0;
        for (int32_t a = 0; a < m; a++) {
            const double v = V.at(i, a);
            dx = fma(c.x[a], v, dx);
            np = fma(c.p[a], v, np);
            nr = fma(c.r[a], v, nr);
        }
        x[i] += dx;
        X[2 * i] = np;
        X[2 * i + 1] = nr;
    }
}

// X = [x, 0] for the initial residual; X[.,1] = r after it
__global__ void k_interleave_x(int64_t n, const double *x, double *X) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        X[2 * i] = x[i];
        X[2 * i + 1] = 0.0;
    }
}
// r = b - (A x) from the SpMV of [x, 0]; X = [p r] = [r r]
__global__ void k_sstep_start(int64_t n, const double *b, const double *AX, double *X, double *r) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = b[i] - AX[2 * i];
        X[2 * i] = v;
        X[2 * i + 1] = v;
        r[i] = v;
    }
}

int ensure_kry(Plan *pl, size_t bytes) {
    if (pl->kry_bytes >= bytes) return MPK_OK;
    if (pl->d_kry) {
        cudaStreamSynchronize(pl->stream);
        cudaFree(pl->d_kry);
        pl->d_kry = nullptr;
        pl->kry_bytes = 0;
    }
    char *p = nullptr;
    int rc = dev_alloc<char>(nullptr, &p, bytes);
    if (rc) return rc;
    pl->d_kry = p;
    pl->kry_bytes = bytes;
    return MPK_OK;
}

unsigned grid_of(const Plan *pl, int64_t n) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)pl->num_sms * 8));
}

// Deterministic dot product a.b into dev_out (one double).
int dot(Plan *pl, const double *a, const double *b, double *partial, double *dev_out, cudaStream_t st) {
    const int nb = red_blocks(pl);
    k_dot_partial<<<nb, kRedThreads, 0, st>>>(pl->n, a, b, partial);
    k_sum_partials<<<1, 32, 0, st>>>(partial, nb, 1, dev_out);
    MPK_CUDA(cudaGetLastError());
    return MPK_OK;
}

// b and x (one FP64 column each) to level order (the plan-owned buffers
// bl, xl) unless permuted.  The reordering moves rows of nrhs elements, so a
// single column of 8-byte values goes as elements of 8 / nrhs bytes.
int to_level(Plan *pl, const double *b, const double *x, double *bl, double *xl, uint32_t flags, cudaStream_t st) {
    if (flags & MPK_IO_PERMUTED) {
        MPK_CUDA(cudaMemcpyAsync(bl, b, sizeof(double) * (size_t)pl->n, cudaMemcpyDeviceToDevice, st));
        MPK_CUDA(cudaMemcpyAsync(xl, x, sizeof(double) * (size_t)pl->n, cudaMemcpyDeviceToDevice, st));
        return MPK_OK;
    }
    int rc = permute_vectors(pl, b, bl, 1, 8 / pl->nrhs, 1, st);
    if (rc) return rc;
    return permute_vectors(pl, x, xl, 1, 8 / pl->nrhs, 1, st);
}
int from_level(Plan *pl, const double *xl, double *x, uint32_t flags, cudaStream_t st) {
    if (flags & MPK_IO_PERMUTED) {
        MPK_CUDA(cudaMemcpyAsync(x, xl, sizeof(double) * (size_t)pl->n, cudaMemcpyDeviceToDevice, st));
        return MPK_OK;
    }
    return permute_vectors(pl, xl, x, 1, 8 / pl->nrhs, 0, st);
}

}  // namespace
}  // namespace mpk

using namespace mpk;

extern "C" {

int mpk_cg(mpk_plan_t plan, const double *b, double *x, double tol, int32_t max_steps, int32_t *steps, double *relres,
           uint32_t flags) {
    if (!plan || !b || !x || !steps || !relres || !(tol >= 0.0) || max_steps < 0) return MPK_ERR_INVALID;
    Plan *pl = &plan->pl;
    if (pl->prec != MPK_F64 || pl->nrhs != 1) return MPK_ERR_INVALID;
    cudaStream_t st = pl->stream;
    const int64_t n = pl->n;
    const int nb = red_blocks(pl);
    // b, x, r, p, q (level order), the partial sums, the scalars
    int rc = ensure_kry(pl, sizeof(double) * ((size_t)5 * n + nb + 8));
    if (rc) return rc;
    double *bl = (double *)pl->d_kry, *xl = bl + n, *r = xl + n, *p = r + n, *q = p + n, *part = q + n,
           *sc = part + nb;
    if ((rc = to_level(pl, b, x, bl, xl, flags, st))) return rc;
    const unsigned g = grid_of(pl, n);
    double h[2];
    if ((rc = dot(pl, bl, bl, part, sc + 3, st))) return rc;
    if ((rc = launch_spmv1(pl, xl, q, st))) return rc;
    k_cg_start<<<g, 256, 0, st>>>(n, bl, q, r, p);
    if ((rc = dot(pl, r, r, part, sc, st))) return rc;
    MPK_CUDA(cudaMemcpyAsync(h, sc + 3, sizeof(double), cudaMemcpyDeviceToHost, st));
    MPK_CUDA(cudaMemcpyAsync(h + 1, sc, sizeof(double), cudaMemcpyDeviceToHost, st));
    MPK_CUDA(cudaStreamSynchronize(st));
    const double bn = std::sqrt(h[0]);
    double rr = h[1];
    int32_t it = 0;
    constexpr int32_t kCheck = 8;   // steps between reads of r.r (no sync inside)
    while (it < max_steps && !(std::sqrt(rr) <= tol * bn)) {
        const int32_t burst = std::min(kCheck, max_steps - it);
        for (int32_t j = 0; j < burst; j++) {
            if ((rc = launch_spmv1(pl, p, q, st))) return rc;
            if ((rc = dot(pl, p, q, part, sc + 1, st))) return rc;
            k_cg_step<<<g, 256, 0, st>>>(n, sc, xl, r, p, q);
            if ((rc = dot(pl, r, r, part, sc + 2, st))) return rc;
            k_cg_dir<<<g, 256, 0, st>>>(n, sc, r, p);
            k_cg_roll<<<1, 1, 0, st>>>(sc);
        }
        MPK_CUDA(cudaGetLastError());
        MPK_CUDA(cudaMemcpyAsync(h + 1, sc, sizeof(double), cudaMemcpyDeviceToHost, st));
        MPK_CUDA(cudaStreamSynchronize(st));
        rr = h[1];
        it += burst;
    }
    if ((rc = from_level(pl, xl, x, flags, st))) return rc;
    MPK_CUDA(cudaStreamSynchronize(st));
    *steps = it;
    *relres = bn > 0.0 ? std::sqrt(rr) / bn : 0.0;
    return MPK_OK;
}

int mpk_sstep_cg(mpk_plan_t plan, const double *b, double *x, double tol, int32_t max_steps, double rho,
                 int32_t *steps, double *relres, uint32_t flags) {
    if (!plan || !b || !x || !steps || !relres || !(tol >= 0.0) || max_steps < 0 || !(rho >= 0.0))
        return MPK_ERR_INVALID;
    Plan *pl = &plan->pl;
    if (pl->prec != MPK_F64 || pl->nrhs != 2 || pl->p > kMaxS) return MPK_ERR_INVALID;
    cudaStream_t st = pl->stream;
    const int64_t n = pl->n;
    const int32_t s = pl->p, m = 2 * s + 1, npairs = m * (m + 1) / 2;
    const int nb = red_blocks(pl);
    if (rho == 0.0) {   // the basis scale: the Gershgorin bound of A
        double lo = 0.0, hi = 0.0;
        int rc0 = mpk_gershgorin(plan, &lo, &hi);
        if (rc0) return rc0;
        rho = std::max(std::fabs(lo), std::fabs(hi));
        if (!(rho > 0.0)) rho = 1.0;
    }
    // b, x, r (level order), X = [p r] (n x 2), Y (s x n x 2), partial Gram, G
    const size_t need = sizeof(double) * ((size_t)3 * n + 2 * n + (size_t)2 * n * s + (size_t)nb * npairs + npairs + 8);
    int rc = ensure_kry(pl, need);
    if (rc) return rc;
    double *bl = (double *)pl->d_kry, *xl = bl + n, *r = xl + n, *X = r + n, *Y = X + 2 * n, *part = Y + 2 * n * s,
           *Gd = part + (size_t)nb * npairs, *sc = Gd + npairs;
    if ((rc = to_level(pl, b, x, bl, xl, flags, st))) return rc;
    const unsigned g = grid_of(pl, n);
    // r = b - A x: one SpMV of [x, 0] with the plan's (block width 2) kernel
    k_interleave_x<<<g, 256, 0, st>>>(n, xl, X);
    if ((rc = launch_spmv1(pl, X, Y, st))) return rc;
    k_sstep_start<<<g, 256, 0, st>>>(n, bl, Y, X, r);
    if ((rc = dot(pl, bl, bl, part, sc, st))) return rc;
    if ((rc = dot(pl, r, r, part, sc + 1, st))) return rc;
    double h[2];
    MPK_CUDA(cudaMemcpyAsync(h, sc, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    MPK_CUDA(cudaStreamSynchronize(st));
    const double bn = std::sqrt(h[0]);
    double rr = h[1];
    Basis V;
    V.X = X;
    V.Y = Y;
    V.n = n;
    V.s = s;
    for (int32_t k = 0; k <= kMaxS; k++) V.scale[k] = k <= s ? std::pow(rho, -(double)k) : 0.0;
    std::vector<double> Gu((size_t)npairs), G((size_t)m * m);
    int32_t done = 0;
    while (done < max_steps && !(std::sqrt(rr) <= tol * bn)) {
        // the basis: one level-blocked MPK of [p r]
        if ((rc = launch_wavefront(pl, X, Y, st))) return rc;
        k_gram_partial<<<nb, kRedThreads, 0, st>>>(V, m, part);
        k_sum_partials<<<(npairs + 127) / 128, 128, 0, st>>>(part, nb, npairs, Gd);
        MPK_CUDA(cudaGetLastError());
        MPK_CUDA(cudaMemcpyAsync(Gu.data(), Gd, sizeof(double) * npairs, cudaMemcpyDeviceToHost, st));
        if ((rc = read_device_error(pl, st))) return rc;   // synchronises the stream
        for (int32_t a = 0, q = 0; a < m; a++)
            for (int32_t c = a; c < m; c++, q++) G[(size_t)a * m + c] = G[(size_t)c * m + a] = Gu[q];
        // s steps of CG on the coordinates (B: the matrix of A in the basis)
        Coords cc;
        for (int32_t a = 0; a < kMaxCols; a++) cc.x[a] = cc.r[a] = cc.p[a] = 0.0;
        cc.p[0] = 1.0;
        cc.r[s + 1] = 1.0;
        auto quad = [&](const double *u, const double *v) {   // u^T G v
            double t = 0.0;
            for (int32_t a = 0; a < m; a++) {
                double w = 0.0;
                for (int32_t c = 0; c < m; c++) w += G[(size_t)a * m + c] * v[c];
                t += u[a] * w;
            }
            return t;
        };
        for (int32_t j = 0; j < s && done < max_steps && !(std::sqrt(rr) <= tol * bn); j++) {
            double w[kMaxCols] = {}, r2[kMaxCols];
            for (int32_t a = 0; a < s; a++) w[a + 1] += rho * cc.p[a];
            for (int32_t a = 0; a < s - 1; a++) w[s + 2 + a] += rho * cc.p[s + 1 + a];
            const double rGr = quad(cc.r, cc.r), pGw = quad(cc.p, w);
            if (!(rGr > 0.0) || !(pGw != 0.0)) {   // the residual vanished in the basis
                rr = 0.0;
                break;
            }
            const double alpha = rGr / pGw;
            for (int32_t a = 0; a < m; a++) {
                cc.x[a] += alpha * cc.p[a];
                r2[a] = cc.r[a] - alpha * w[a];
            }
            const double rGr2 = quad(r2, r2);
            const double beta = rGr2 / rGr;
            for (int32_t a = 0; a < m; a++) {
                cc.p[a] = r2[a] + beta * cc.p[a];
                cc.r[a] = r2[a];
            }
            rr = rGr2 > 0.0 ? rGr2 : 0.0;
            done++;
        }
        k_sstep_update<<<g, 256, 0, st>>>(V, m, cc, xl, X);
        MPK_CUDA(cudaGetLastError());
    }
    if ((rc = from_level(pl, xl, x, flags, st))) return rc;
    MPK_CUDA(cudaStreamSynchronize(st));
    *steps = done;
    *relres = bn > 0.0 ? std::sqrt(rr) / bn : 0.0;
    return MPK_OK;
}

}  // extern "C"
