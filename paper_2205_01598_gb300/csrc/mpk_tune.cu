// Autotuner of the level-blocked MPK (the tuning of Sec. 6.1: p_m, C and the
// split of a power k into sweeps, Sec. 5.1), measured on the GPU.  A
// candidate with sweeps of q < k powers is one plan with mpk_opts.sweep = q
// (all sweeps in one launch), except on the resident schedule, which runs
// one plan per sweep.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "mpk_internal.cuh"

namespace mpk {
namespace {

// Mean time of one mpk_run of `plan` (level order), repeated until min_time_s
// (at least 3 runs after 2 warm-up runs); x and Y are device scratch large
// enough for the plan.
int time_plan(mpk_plan_t plan, void *x, void *Y, double min_time_s, double *ms) {
    Plan *pl = &plan->pl;
    cudaStream_t st = pl->stream;
    for (int w = 0; w < 2; w++) {
        int rc = mpk_run(plan, x, Y, MPK_IO_PERMUTED | MPK_ASYNC);
        if (rc) return rc;
    }
    int rc = mpk_run(plan, x, Y, MPK_IO_PERMUTED);   // surfaces device-side errors
    if (rc) return rc;
    cudaEvent_t e0, e1;
    MPK_CUDA(cudaEventCreate(&e0));
    MPK_CUDA(cudaEventCreate(&e1));
    int reps = 0;
    double total = 0;
    const auto t_start = std::chrono::steady_clock::now();
    do {
        const int batch = reps == 0 ? 3 : std::max(1, reps);
        cudaEventRecord(e0, st);
        for (int r = 0; r < batch && rc == MPK_OK; r++) rc = mpk_run(plan, x, Y, MPK_IO_PERMUTED | MPK_ASYNC);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float f = 0;
        cudaEventElapsedTime(&f, e0, e1);
        total += f;
        reps += batch;
    } while (rc == MPK_OK &&
             std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count() < min_time_s);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    if ((rc = read_device_error(pl, st))) return rc;
    *ms = total / reps;
    return MPK_OK;
}

}  // namespace
}  // namespace mpk

using namespace mpk;

extern "C" {

int mpk_tune_default_grid(int32_t k, mpk_tune_candidate *out, int32_t max, int32_t *count) {
    if (!out || !count || k < 1) return MPK_ERR_INVALID;
    std::vector<mpk_tune_candidate> g;
    auto add = [&](int32_t t, double f, int32_t q, uint32_t tune = 0) {
        mpk_tune_candidate r{};
        r.tile_rows = t;
        r.safety_f = f;
        r.tune = tune;
        r.p_sweep = q;
        r.ms = -1;
        r.status = 0;
        g.push_back(r);
    };
    add(0, 0.5, k);   // the library's default options
    std::vector<int32_t> sweeps = {k};
    if (k >= 4) sweeps.push_back((k + 1) / 2);
    for (int32_t q : sweeps) add(0, 0.5, q, MPK_TUNE_RESIDENT);   // tiles sized to the stage
    if (k >= 2) sweeps.push_back(1);
    const int32_t tiles[] = {64, 128, 256, 512, 1024};
    const double fs[] = {0.25, 0.5};
    for (int32_t q : sweeps)
        for (double f : fs)
            for (int32_t t : tiles) add(t, f, q);
    const int32_t c = (int32_t)g.size();
    for (int32_t i = 0; i < std::min(c, max); i++) out[i] = g[i];
    *count = std::min(c, max);
    return c <= max ? MPK_OK : MPK_ERR_INVALID;
}

int mpk_autotune(const mpk_csr *A, int32_t k, const mpk_opts *base, double min_time_s, mpk_tune_candidate *cand,
                 int32_t n_cand, int32_t *best) {
    if (!A || !base || !cand || !best || n_cand < 1 || k < 1 || k > kMaxP) return MPK_ERR_INVALID;
    *best = -1;
    const size_t eb = is_f64_vec(base->prec) ? 8 : 4;
    const size_t vec = (size_t)A->n * (size_t)std::max(1, base->nrhs) * eb;
    char *x = nullptr, *Y = nullptr;
    int rc = dev_alloc<char>(nullptr, &x, vec);
    if (!rc) rc = dev_alloc<char>(nullptr, &Y, vec * (size_t)k);
    if (!rc && cudaMemset(x, 0, vec) != cudaSuccess) rc = MPK_ERR_CUDA;
    double best_ms = INFINITY;
    for (int32_t c = 0; c < n_cand && !rc; c++) {
        mpk_tune_candidate &cd = cand[c];
        const int32_t q = std::min(std::max(1, cd.p_sweep), k);
        mpk_opts o = *base;
        o.tile_rows = cd.tile_rows;
        o.safety_f = cd.safety_f;
        o.tune = cd.tune;
        double ms = 0, t = 0;
        int st = MPK_OK;
        if (!(cd.tune & MPK_TUNE_RESIDENT)) {
            // the work-list schedule runs the sweeps in one launch
            o.sweep = q;
            mpk_plan_t plan = nullptr;
            st = mpk_plan(A, k, &o, &plan);
            if (st == MPK_OK) st = time_plan(plan, x, Y, min_time_s, &ms);
            if (plan) mpk_plan_destroy(plan);
        } else {
            // the resident schedule owns tiles for all powers of a launch:
            // one launch per sweep, and one for the remainder
            const int32_t sweeps = k / q, rem = k % q;
            for (int32_t part = 0; part < 2 && st == MPK_OK; part++) {
                const int32_t pw = part == 0 ? q : rem;
                const int32_t times = part == 0 ? sweeps : (rem ? 1 : 0);
                if (!times) continue;
                mpk_plan_t plan = nullptr;
                st = mpk_plan(A, pw, &o, &plan);
                if (st == MPK_OK) st = time_plan(plan, x, Y, min_time_s, &t);
                if (plan) mpk_plan_destroy(plan);
                ms += times * t;
            }
        }
        cd.status = st;
        cd.ms = st == MPK_OK ? ms : -1.0;
        if (st == MPK_OK && ms < best_ms) {
            best_ms = ms;
            *best = c;
        }
        if (st == MPK_ERR_CUDA) rc = st;   // a CUDA error ends the search
    }
    if (x) cudaFree(x);
    if (Y) cudaFree(Y);
    if (rc) return rc;
    return *best >= 0 ? MPK_OK : MPK_ERR_UNSUPPORTED;
}

}  // extern "C"
