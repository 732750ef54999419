// Small multilayer perceptron of the learned planner: n_in -> h -> h -> n_out
// (ReLU on the hidden layers, linear output), trained with a masked
// mean-squared error and Adam.  Forward, backward and update are plain CUDA
// kernels (the layers are a few dozen wide; tensor cores would not pay off).
#include <cmath>
#include <vector>

#include "mpk_internal.cuh"

namespace mpk {
namespace {

// out[b, j] = act(sum_i W[j, i] * in[b, i] + bias[j])
__global__ void k_dense(int32_t B, int32_t ni, int32_t no, const float *in, const float *W, const float *bias,
                        float *out, int relu) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (int64_t)B * no) return;
    const int32_t b = (int32_t)(g / no), j = (int32_t)(g % no);
    float s = bias[j];
    for (int32_t i = 0; i < ni; i++) s = fmaf(W[(int64_t)j * ni + i], in[(int64_t)b * ni + i], s);
    out[g] = relu ? fmaxf(s, 0.0f) : s;
}

// din[b, i] = (sum_j W[j, i] * dout[b, j]) * relu'(act[b, i])
__global__ void k_dense_bwd_in(int32_t B, int32_t ni, int32_t no, const float *dout, const float *W, const float *act,
                               float *din) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (int64_t)B * ni) return;
    const int32_t b = (int32_t)(g / ni), i = (int32_t)(g % ni);
    float s = 0.0f;
    for (int32_t j = 0; j < no; j++) s = fmaf(W[(int64_t)j * ni + i], dout[(int64_t)b * no + j], s);
    din[g] = act[g] > 0.0f ? s : 0.0f;
}

// gW[j, i] = sum_b dout[b, j] * in[b, i]; gb[j] = sum_b dout[b, j] (thread per (j, i|bias))
__global__ void k_dense_bwd_w(int32_t B, int32_t ni, int32_t no, const float *dout, const float *in, float *gW,
                              float *gb) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (int64_t)no * (ni + 1)) return;
    const int32_t j = (int32_t)(g / (ni + 1)), i = (int32_t)(g % (ni + 1));
    float s = 0.0f;
    if (i < ni) {
        for (int32_t b = 0; b < B; b++) s = fmaf(dout[(int64_t)b * no + j], in[(int64_t)b * ni + i], s);
        gW[(int64_t)j * ni + i] = s;
    } else {
        for (int32_t b = 0; b < B; b++) s += dout[(int64_t)b * no + j];
        gb[j] = s;
    }
}

// acc[0] += sum M, acc[1] += sum M (Y - T)^2
__global__ void k_mse_sums(int64_t n, const float *Y, const float *T, const float *M, double *acc) {
    __shared__ double s0[8], s1[8];
    double a = 0, b = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double m = M[i], d = (double)Y[i] - (double)T[i];
        a += m;
        b += m * d * d;
    }
    for (int o = 16; o; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { s0[w] = a; s1[w] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < (int)(blockDim.x >> 5); i++) { s0[0] += s0[i]; s1[0] += s1[i]; }
        atomicAdd(&acc[0], s0[0]);
        atomicAdd(&acc[1], s1[0]);
    }
}

// dY = 2 M (Y - T) / sum M
__global__ void k_mse_grad(int64_t n, const float *Y, const float *T, const float *M, const double *acc, float *dY) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dY[i] = (float)(2.0 * (double)M[i] * ((double)Y[i] - (double)T[i]) / fmax(acc[0], 1e-30));
}

__global__ void k_adam(int64_t n, float *w, const float *g, float *m, float *v, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

inline unsigned nb(int64_t n, int t = 256) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

uint64_t splitmix_next(uint64_t &s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace

struct Mlp {
    int32_t ni = 0, nh = 0, no = 0, batch_cap = 0;
    int64_t np = 0;
    cudaStream_t stream = nullptr;
    float *params = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    float *h1 = nullptr, *h2 = nullptr, *y = nullptr, *dy = nullptr, *dh2 = nullptr, *dh1 = nullptr;
    double *acc = nullptr;
    int64_t step = 0;
    // offsets of W1, b1, W2, b2, W3, b3 in the flat parameter vector
    int64_t oW1 = 0, ob1 = 0, oW2 = 0, ob2 = 0, oW3 = 0, ob3 = 0;
};

namespace {

void free_mlp(Mlp *n) {
    void *ps[] = {n->params, n->grad, n->m, n->v, n->h1, n->h2, n->y, n->dy, n->dh2, n->dh1, n->acc};
    for (void *p : ps)
        if (p) cudaFree(p);
}

int ensure_batch(Mlp *n, int32_t B) {
    if (B <= n->batch_cap) return MPK_OK;
    float *bufs[] = {n->h1, n->h2, n->y, n->dy, n->dh2, n->dh1};
    for (float *b : bufs)
        if (b) cudaFree(b);
    n->h1 = n->h2 = n->y = n->dy = n->dh2 = n->dh1 = nullptr;
    n->batch_cap = 0;
    int rc = 0;
    if (!rc) rc = dev_alloc<float>(nullptr, &n->h1, (size_t)B * n->nh);
    if (!rc) rc = dev_alloc<float>(nullptr, &n->h2, (size_t)B * n->nh);
    if (!rc) rc = dev_alloc<float>(nullptr, &n->y, (size_t)B * n->no);
    if (!rc) rc = dev_alloc<float>(nullptr, &n->dy, (size_t)B * n->no);
    if (!rc) rc = dev_alloc<float>(nullptr, &n->dh2, (size_t)B * n->nh);
    if (!rc) rc = dev_alloc<float>(nullptr, &n->dh1, (size_t)B * n->nh);
    if (!rc) n->batch_cap = B;
    return rc;
}

void forward(Mlp *n, const float *X, int32_t B, float *Y) {
    cudaStream_t st = n->stream;
    const float *P = n->params;
    k_dense<<<nb((int64_t)B * n->nh), 256, 0, st>>>(B, n->ni, n->nh, X, P + n->oW1, P + n->ob1, n->h1, 1);
    k_dense<<<nb((int64_t)B * n->nh), 256, 0, st>>>(B, n->nh, n->nh, n->h1, P + n->oW2, P + n->ob2, n->h2, 1);
    k_dense<<<nb((int64_t)B * n->no), 256, 0, st>>>(B, n->nh, n->no, n->h2, P + n->oW3, P + n->ob3, Y, 0);
}

}  // namespace
}  // namespace mpk

struct mpk_mlp_s {
    mpk::Mlp n;
};

using namespace mpk;

extern "C" {

int mpk_mlp_create(int32_t n_in, int32_t n_hidden, int32_t n_out, uint64_t seed, void *stream, mpk_mlp_t *out) {
    if (!out) return MPK_ERR_INVALID;
    *out = nullptr;
    if (n_in < 1 || n_hidden < 1 || n_out < 1 || n_in > 4096 || n_hidden > 4096 || n_out > 4096) return MPK_ERR_INVALID;
    mpk_mlp_s *h = new (std::nothrow) mpk_mlp_s();
    if (!h) return MPK_ERR_OOM;
    Mlp *n = &h->n;
    n->ni = n_in;
    n->nh = n_hidden;
    n->no = n_out;
    n->stream = (cudaStream_t)stream;
    n->oW1 = 0;
    n->ob1 = n->oW1 + (int64_t)n_hidden * n_in;
    n->oW2 = n->ob1 + n_hidden;
    n->ob2 = n->oW2 + (int64_t)n_hidden * n_hidden;
    n->oW3 = n->ob2 + n_hidden;
    n->ob3 = n->oW3 + (int64_t)n_out * n_hidden;
    n->np = n->ob3 + n_out;
    int rc = dev_alloc<float>(nullptr, &n->params, (size_t)n->np);
    if (!rc) rc = dev_alloc<float>(nullptr, &n->grad, (size_t)n->np);
    if (!rc) rc = dev_alloc<float>(nullptr, &n->m, (size_t)n->np);
    if (!rc) rc = dev_alloc<float>(nullptr, &n->v, (size_t)n->np);
    if (!rc) rc = dev_alloc<double>(nullptr, &n->acc, 2);
    if (!rc) {
        // Glorot-uniform weights from SplitMix64, zero biases
        std::vector<float> w((size_t)n->np, 0.0f);
        uint64_t s = seed;
        auto fill = [&](int64_t off, int32_t fo, int32_t fi) {
            const double a = std::sqrt(6.0 / (fi + fo));
            for (int64_t i = 0; i < (int64_t)fo * fi; i++) {
                const double u = (double)(splitmix_next(s) >> 11) * (1.0 / 9007199254740992.0);
                w[off + i] = (float)((2.0 * u - 1.0) * a);
            }
        };
        fill(n->oW1, n_hidden, n_in);
        fill(n->oW2, n_hidden, n_hidden);
        fill(n->oW3, n_out, n_hidden);
        if (cudaMemcpy(n->params, w.data(), sizeof(float) * w.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemset(n->m, 0, sizeof(float) * n->np) != cudaSuccess ||
            cudaMemset(n->v, 0, sizeof(float) * n->np) != cudaSuccess)
            rc = MPK_ERR_CUDA;
    }
    if (rc) {
        free_mlp(n);
        delete h;
        return rc;
    }
    *out = h;
    return MPK_OK;
}

int32_t mpk_mlp_num_params(mpk_mlp_t net) { return net ? (int32_t)net->n.np : MPK_ERR_INVALID; }

int mpk_mlp_get_params(mpk_mlp_t net, float *host, int32_t count) {
    if (!net || !host || count != net->n.np) return MPK_ERR_INVALID;
    MPK_CUDA(cudaMemcpyAsync(host, net->n.params, sizeof(float) * count, cudaMemcpyDeviceToHost, net->n.stream));
    MPK_CUDA(cudaStreamSynchronize(net->n.stream));
    return MPK_OK;
}

int mpk_mlp_set_params(mpk_mlp_t net, const float *host, int32_t count) {
    if (!net || !host || count != net->n.np) return MPK_ERR_INVALID;
    MPK_CUDA(cudaMemcpyAsync(net->n.params, host, sizeof(float) * count, cudaMemcpyHostToDevice, net->n.stream));
    MPK_CUDA(cudaMemsetAsync(net->n.m, 0, sizeof(float) * count, net->n.stream));
    MPK_CUDA(cudaMemsetAsync(net->n.v, 0, sizeof(float) * count, net->n.stream));
    MPK_CUDA(cudaStreamSynchronize(net->n.stream));
    net->n.step = 0;
    return MPK_OK;
}

int mpk_mlp_forward(mpk_mlp_t net, const float *X, int32_t batch, float *Y) {
    if (!net || !X || !Y || batch < 1) return MPK_ERR_INVALID;
    Mlp *n = &net->n;
    int rc = ensure_batch(n, batch);
    if (rc) return rc;
    forward(n, X, batch, Y);
    MPK_CUDA(cudaGetLastError());
    return MPK_OK;
}

int mpk_mlp_loss_grad(mpk_mlp_t net, const float *X, const float *T, const float *M, int32_t batch, double *loss,
                      float *grad_host) {
    if (!net || !X || !T || !M || batch < 1) return MPK_ERR_INVALID;
    Mlp *n = &net->n;
    int rc = ensure_batch(n, batch);
    if (rc) return rc;
    cudaStream_t st = n->stream;
    const int64_t ny = (int64_t)batch * n->no;
    forward(n, X, batch, n->y);
    MPK_CUDA(cudaMemsetAsync(n->acc, 0, 2 * sizeof(double), st));
    k_mse_sums<<<std::min<unsigned>(nb(ny), 1024), 256, 0, st>>>(ny, n->y, T, M, n->acc);
    k_mse_grad<<<nb(ny), 256, 0, st>>>(ny, n->y, T, M, n->acc, n->dy);
    float *G = n->grad;
    const float *P = n->params;
    k_dense_bwd_w<<<nb((int64_t)n->no * (n->nh + 1)), 256, 0, st>>>(batch, n->nh, n->no, n->dy, n->h2, G + n->oW3,
                                                                    G + n->ob3);
    k_dense_bwd_in<<<nb((int64_t)batch * n->nh), 256, 0, st>>>(batch, n->nh, n->no, n->dy, P + n->oW3, n->h2, n->dh2);
    k_dense_bwd_w<<<nb((int64_t)n->nh * (n->nh + 1)), 256, 0, st>>>(batch, n->nh, n->nh, n->dh2, n->h1, G + n->oW2,
                                                                    G + n->ob2);
    k_dense_bwd_in<<<nb((int64_t)batch * n->nh), 256, 0, st>>>(batch, n->nh, n->nh, n->dh2, P + n->oW2, n->h1, n->dh1);
    k_dense_bwd_w<<<nb((int64_t)n->nh * (n->ni + 1)), 256, 0, st>>>(batch, n->ni, n->nh, n->dh1, X, G + n->oW1,
                                                                    G + n->ob1);
    MPK_CUDA(cudaGetLastError());
    double h_acc[2];
    MPK_CUDA(cudaMemcpyAsync(h_acc, n->acc, sizeof(h_acc), cudaMemcpyDeviceToHost, st));
    if (grad_host) MPK_CUDA(cudaMemcpyAsync(grad_host, G, sizeof(float) * n->np, cudaMemcpyDeviceToHost, st));
    MPK_CUDA(cudaStreamSynchronize(st));
    if (loss) *loss = h_acc[1] / std::max(h_acc[0], 1e-30);
    return MPK_OK;
}

int mpk_mlp_adam_step(mpk_mlp_t net, float lr, float beta1, float beta2, float eps) {
    if (!net || !(lr > 0)) return MPK_ERR_INVALID;
    Mlp *n = &net->n;
    n->step++;
    const float c1 = 1.0f - std::pow(beta1, (float)n->step), c2 = 1.0f - std::pow(beta2, (float)n->step);
    k_adam<<<nb(n->np), 256, 0, n->stream>>>(n->np, n->params, n->grad, n->m, n->v, lr, beta1, beta2, eps, c1, c2);
    MPK_CUDA(cudaGetLastError());
    return MPK_OK;
}

int mpk_mlp_destroy(mpk_mlp_t net) {
    if (!net) return MPK_OK;
    cudaStreamSynchronize(net->n.stream);
    free_mlp(&net->n);
    delete net;
    return MPK_OK;
}

}  // extern "C"
