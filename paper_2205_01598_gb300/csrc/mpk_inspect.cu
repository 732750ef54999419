// Read-only views of a plan's schedule for tests and tools: the issue order
// of the work items and the dependency range of every tile (Sec. 4.3
// conditions at tile granularity).
#include <cstring>

#include "mpk_internal.cuh"

using namespace mpk;

extern "C" {

int mpk_plan_schedule(mpk_plan_t plan, int32_t *work, int32_t *dep_lo, int32_t *dep_hi) {
    if (!plan || !work || !dep_lo || !dep_hi) return MPK_ERR_INVALID;
    const Plan *pl = &plan->pl;
    std::vector<int32_t> w;
    const int rc = work_to_host(pl, w);
    if (rc != MPK_OK) return rc;
    std::memcpy(work, w.data(), sizeof(int32_t) * w.size());
    MPK_CUDA(cudaMemcpy(dep_lo, pl->d_dep_lo, sizeof(int32_t) * (size_t)pl->n_tiles, cudaMemcpyDeviceToHost));
    std::memcpy(dep_hi, pl->h_dep_hi.data(), sizeof(int32_t) * (size_t)pl->n_tiles);
    return MPK_OK;
}

}  // extern "C"
