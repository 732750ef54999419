// Batched level-blocked MPK: several plans (matrices of different sizes,
// block widths and powers) run in ONE persistent wavefront launch, which can
// be captured in a CUDA graph and replayed.
#include <algorithm>
#include <cstring>

#include "mpk_internal.cuh"

namespace mpk {

struct Batch {
    std::vector<Plan *> plans;
    int32_t count = 0, prec = MPK_F32, n_items = 0, grid = 0;
    cudaStream_t stream = nullptr;
    std::vector<ExecArgs> h_table;
    ExecArgs *d_table = nullptr;
    int32_t *d_work = nullptr, *d_wplan = nullptr, *d_ctl = nullptr;
    int32_t **d_plan_ctl = nullptr;
    BatchArgs args{};
    cudaStream_t capture_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

void free_batch(Batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
    void *ps[] = {b->d_table, b->d_work, b->d_wplan, b->d_ctl, b->d_plan_ctl};
    for (void *p : ps)
        if (p) cudaFree(p);
}

// Issue order of the batch: the plans' own orders merged by relative
// position (item j of a plan with n items sits at (j + 1/2) / n), so each
// plan keeps its order (its dependencies stay earlier) and all plans advance
// together through the launch: while one plan's items wait for the previous
// power, the CTAs hold items of the others.  (Plans one after another, the
// largest first, measured 213 vs 209 ms on the 64-matrix Zipf batch and
// 322 vs 287 ms with the default options.)
int merge_orders(const std::vector<Plan *> &plans, std::vector<int32_t> &work, std::vector<int32_t> &wplan) {
    std::vector<std::vector<int32_t>> own(plans.size());
    for (size_t m = 0; m < plans.size(); m++) {
        const int rc = work_to_host(plans[m], own[m]);
        if (rc != MPK_OK) return rc;
    }
    struct Ref { double pos; int32_t m, j; };
    std::vector<Ref> refs;
    size_t total = 0;
    for (const auto &w : own) total += w.size();
    refs.reserve(total);
    for (int32_t m = 0; m < (int32_t)plans.size(); m++) {
        const double n = (double)own[m].size();
        for (int32_t j = 0; j < (int32_t)own[m].size(); j++) refs.push_back({(j + 0.5) / n, m, j});
    }
    std::sort(refs.begin(), refs.end(), [](const Ref &a, const Ref &b) {
        return a.pos != b.pos ? a.pos < b.pos : (a.m != b.m ? a.m < b.m : a.j < b.j);
    });
    work.resize(total);
    wplan.resize(total);
    for (size_t i = 0; i < total; i++) {
        work[i] = own[refs[i].m][refs[i].j];
        wplan[i] = refs[i].m;
    }
    return MPK_OK;
}

int upload_table(Batch *b, const void *const *xs, void *const *Ys, cudaStream_t st) {
    for (int32_t m = 0; m < b->count; m++) {
        b->h_table[m].x = xs[m];
        b->h_table[m].Y = Ys[m];
    }
    MPK_CUDA(cudaMemcpyAsync(b->d_table, b->h_table.data(), sizeof(ExecArgs) * b->count, cudaMemcpyHostToDevice, st));
    return MPK_OK;
}

int launch_batch(Batch *b, cudaStream_t st) {
    void *a[] = {(void *)&b->args};
    return launch_coop(batch_kernel(b->prec), b->grid, 0, a, st);
}

int batch_error(Batch *b, cudaStream_t st) {
    int32_t w[CTL_WORDS];
    MPK_CUDA(cudaMemcpyAsync(w, b->d_ctl, sizeof(w), cudaMemcpyDeviceToHost, st));
    MPK_CUDA(cudaStreamSynchronize(st));
    if (w[CTL_ERR] != 0) {
        MPK_CUDA(cudaMemsetAsync(b->d_ctl + CTL_ERR, 0, 3 * sizeof(int32_t), st));
        MPK_CUDA(cudaStreamSynchronize(st));
        return w[CTL_ERR];
    }
    return MPK_OK;
}

#define MPK_TRYB(x)                    \
    do {                               \
        int _rc = (x);                 \
        if (_rc != MPK_OK) return _rc; \
    } while (0)

int build_batch(Batch *b, const mpk_plan_t *plans, int32_t count) {
    b->count = count;
    for (int32_t m = 0; m < count; m++) {
        Plan *pl = &plans[m]->pl;
        if (pl->has_diag || pl->prec == MPK_F64_DF || pl->prec != plans[0]->pl.prec ||
            pl->device != plans[0]->pl.device)
            return MPK_ERR_UNSUPPORTED;
        b->plans.push_back(pl);
    }
    b->prec = b->plans[0]->prec;
    b->stream = b->plans[0]->stream;
    std::vector<int32_t> work, wplan;
    MPK_TRYB(merge_orders(b->plans, work, wplan));
    b->n_items = (int32_t)work.size();
    MPK_TRYB(dev_alloc<int32_t>(nullptr, &b->d_work, work.size()));
    MPK_TRYB(dev_alloc<int32_t>(nullptr, &b->d_wplan, wplan.size()));
    MPK_TRYB(dev_alloc<ExecArgs>(nullptr, &b->d_table, (size_t)count));
    MPK_TRYB(dev_alloc<int32_t *>(nullptr, &b->d_plan_ctl, (size_t)count));
    MPK_TRYB(dev_alloc<int32_t>(nullptr, &b->d_ctl, CTL_WORDS));
    cudaStream_t st = b->stream;
    std::vector<int32_t *> ctls;
    b->h_table.resize(count);
    double timeout = 0;
    for (int32_t m = 0; m < count; m++) {
        b->h_table[m] = exec_args(b->plans[m], nullptr, nullptr);
        b->h_table[m].ctl = b->d_ctl;   // abort / error words are batch-wide
        ctls.push_back(b->plans[m]->d_ctl);
        timeout = std::max(timeout, b->plans[m]->timeout_s);
    }
    MPK_CUDA(cudaMemcpyAsync(b->d_work, work.data(), work.size() * 4, cudaMemcpyHostToDevice, st));
    MPK_CUDA(cudaMemcpyAsync(b->d_wplan, wplan.data(), wplan.size() * 4, cudaMemcpyHostToDevice, st));
    MPK_CUDA(cudaMemcpyAsync(b->d_table, b->h_table.data(), sizeof(ExecArgs) * count, cudaMemcpyHostToDevice, st));
    MPK_CUDA(cudaMemcpyAsync(b->d_plan_ctl, ctls.data(), sizeof(int32_t *) * count, cudaMemcpyHostToDevice, st));
    MPK_CUDA(cudaMemsetAsync(b->d_ctl, 0, sizeof(int32_t) * CTL_WORDS, st));
    MPK_CUDA(cudaStreamSynchronize(st));
    int occ = 0;
    const void *fn = batch_kernel(b->prec);
    MPK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kWaveThreads, 0));
    if (occ < 1) return MPK_ERR_CUDA;
    b->grid = (int32_t)std::max<int64_t>(
        1, std::min<int64_t>((int64_t)b->plans[0]->num_sms * occ, (int64_t)b->n_items));
    ExecArgs g = {};
    g.work = b->d_work;
    g.n_items = b->n_items;
    g.ctl = b->d_ctl;
    g.timeout_ns = (uint64_t)(timeout * 1e9);
    g.drop_tile = g.drop_k = -1;
    b->args = BatchArgs{g, b->d_table, b->d_wplan, b->d_plan_ctl, count};
    return MPK_OK;
}

}  // namespace

}  // namespace mpk

struct mpk_batch_s {
    mpk::Batch b;
};

using namespace mpk;

extern "C" {

int mpk_batch_create(const mpk_plan_t *plans, int32_t count, mpk_batch_t *out) {
    if (!out) return MPK_ERR_INVALID;
    *out = nullptr;
    if (!plans || count < 1 || count > kMaxBatch) return MPK_ERR_INVALID;
    for (int32_t m = 0; m < count; m++)
        if (!plans[m]) return MPK_ERR_INVALID;
    mpk_batch_s *h = new (std::nothrow) mpk_batch_s();
    if (!h) return MPK_ERR_OOM;
    int rc = build_batch(&h->b, plans, count);
    if (rc != MPK_OK) {
        free_batch(&h->b);
        delete h;
        return rc;
    }
    *out = h;
    return MPK_OK;
}

int mpk_batch_info(mpk_batch_t batch, int32_t *n_items, int32_t *grid_ctas) {
    if (!batch) return MPK_ERR_INVALID;
    if (n_items) *n_items = batch->b.n_items;
    if (grid_ctas) *grid_ctas = batch->b.grid;
    return MPK_OK;
}

int mpk_batch_run(mpk_batch_t batch, const void *const *xs, void *const *Ys, uint32_t flags) {
    if (!batch || !xs || !Ys) return MPK_ERR_INVALID;
    Batch *b = &batch->b;
    for (int32_t m = 0; m < b->count; m++)
        if (!xs[m] || !Ys[m]) return MPK_ERR_INVALID;
    int rc = upload_table(b, xs, Ys, b->stream);
    if (rc) return rc;
    if ((rc = launch_batch(b, b->stream))) return rc;
    MPK_CUDA(cudaGetLastError());
    if (flags & MPK_ASYNC) return MPK_OK;
    return batch_error(b, b->stream);
}

int mpk_batch_graph_capture(mpk_batch_t batch, const void *const *xs, void *const *Ys) {
    if (!batch || !xs || !Ys) return MPK_ERR_INVALID;
    Batch *b = &batch->b;
    for (int32_t m = 0; m < b->count; m++)
        if (!xs[m] || !Ys[m]) return MPK_ERR_INVALID;
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    if (b->graph) {
        cudaGraphDestroy(b->graph);
        b->graph = nullptr;
    }
    int rc = upload_table(b, xs, Ys, b->stream);
    if (rc) return rc;
    MPK_CUDA(cudaStreamSynchronize(b->stream));
    if (!b->capture_stream) MPK_CUDA(cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking));
    MPK_CUDA(cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal));
    rc = launch_batch(b, b->capture_stream);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->capture_stream, &graph);
    if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return cuda_status(e, "cudaStreamEndCapture", __LINE__);
    b->graph = graph;
    MPK_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0));
    return MPK_OK;
}

int mpk_batch_graph_launch(mpk_batch_t batch, uint32_t flags) {
    if (!batch || !batch->b.exec) return MPK_ERR_INVALID;
    Batch *b = &batch->b;
    MPK_CUDA(cudaGraphLaunch(b->exec, b->stream));
    if (flags & MPK_ASYNC) return MPK_OK;
    return batch_error(b, b->stream);
}

int mpk_batch_destroy(mpk_batch_t batch) {
    if (!batch) return MPK_OK;
    cudaStreamSynchronize(batch->b.stream);
    free_batch(&batch->b);
    delete batch;
    return MPK_OK;
}

}  // extern "C"
