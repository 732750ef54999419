/* Reported CPU baseline of the benchmark, beside the oracle (TEST AND
 * BENCHMARK INFRASTRUCTURE ONLY): p back-to-back FP64 CRS SpMVs, the rows of
 * each split statically across the host's OpenMP threads -- the paper's
 * baseline MPK (Sec. 3.1, Fig. 1) run as its multicore comparator
 * (Sec. 6, static OpenMP schedule).  Each row is summed in stored order
 * without FMA contraction, like the sequential oracle, so the two agree bit
 * for bit.  Compiled separately with -fopenmp; it is not part of the
 * oracle's reference arithmetic. */
#include <omp.h>
#include <stddef.h>

int omp_pxspmv_threads(void) { return omp_get_max_threads(); }

void omp_pxspmv(int n, const int *rowptr, const int *col, const double *val, int p, const double *x,
                double *Y) {
    for (int k = 0; k < p; k++) {
        const double *in = k == 0 ? x : Y + (size_t)(k - 1) * (size_t)n;
        double *out = Y + (size_t)k * (size_t)n;
#pragma omp parallel for schedule(static)
        for (int i = 0; i < n; i++) {
            double s = 0.0;
            for (int j = rowptr[i]; j < rowptr[i + 1]; j++) s += val[j] * in[col[j]];
            out[i] = s;
        }
    }
}
