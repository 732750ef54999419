// Chebyshev propagation with the input and the result in HOST memory: the
// vectors are staged through stream-ordered device allocations of the
// plan's stream around the device entry points.
#include "mpk_internal.cuh"

using namespace mpk;

namespace {

int cheb_host(mpk_plan_t plan, const double *coef, int32_t M, double c, double r, const void *x_host,
              double *y_host, uint32_t flags, int G,
              int (*run)(mpk_plan_t, const double *, int32_t, double, double, const void *, double *, uint32_t)) {
    if (!plan || !x_host || !y_host) return MPK_ERR_INVALID;
    Plan *pl = &plan->pl;
    if (pl->nrhs != G) return MPK_ERR_INVALID;
    cudaStream_t st = pl->stream;
    const size_t xb = (size_t)pl->n * G * elem_bytes_of(pl), yb = (size_t)pl->n * G * sizeof(double);
    void *dx = nullptr, *dy = nullptr;
    if (cudaMallocAsync(&dx, std::max<size_t>(xb, 16), st) != cudaSuccess) {
        (void)cudaGetLastError();
        return MPK_ERR_OOM;
    }
    if (cudaMallocAsync(&dy, std::max<size_t>(yb, 16), st) != cudaSuccess) {
        (void)cudaGetLastError();
        cudaFreeAsync(dx, st);
        return MPK_ERR_OOM;
    }
    int rc = MPK_OK;
    if (cudaMemcpyAsync(dx, x_host, xb, cudaMemcpyHostToDevice, st) != cudaSuccess) rc = MPK_ERR_CUDA;
    if (rc == MPK_OK) rc = run(plan, coef, M, c, r, dx, (double *)dy, flags | MPK_ASYNC);
    if (rc == MPK_OK && cudaMemcpyAsync(y_host, dy, yb, cudaMemcpyDeviceToHost, st) != cudaSuccess) rc = MPK_ERR_CUDA;
    cudaFreeAsync(dx, st);
    cudaFreeAsync(dy, st);
    if (rc != MPK_OK || (flags & MPK_ASYNC)) return rc;
    return read_device_error(pl, st);
}

}  // namespace

extern "C" {

int mpk_cheb_host(mpk_plan_t plan, const double *coef, int32_t M, double c, double r, const void *x_host,
                  double *y_host, uint32_t flags) {
    return cheb_host(plan, coef, M, c, r, x_host, y_host, flags, 2, mpk_cheb);
}

int mpk_cheb_real_host(mpk_plan_t plan, const double *coef, int32_t M, double c, double r, const void *x_host,
                       double *y_host, uint32_t flags) {
    return cheb_host(plan, coef, M, c, r, x_host, y_host, flags, 1, mpk_cheb_real);
}

}  // extern "C"
