// Parameter-predicting MLP: float32 forward, backward and Adam kernels, and
// the C ABI around them (dacp_mlp_*). The network maps features of one
// realization (size, coupling statistics, the first Chebyshev moments of a
// random vector) to the method's three tuning knobs: the window ratio, the
// filter-order constant and the basis ratio. It is trained on runs of the
// method itself; the paper picks these by hand (Sec. III).
//
// Layers: z_l = W_l a_{l-1} + b_l, a_l = relu(z_l) for hidden layers, y = z_L.
// Loss: sum (y - t)^2 / (2 B) on standardised inputs and targets.
// Adam (Kingma & Ba 2015) with bias correction.

#include <float.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <random>
#include <string>
#include <vector>

#include "../../include/dacp.h"
#include "common.cuh"
#include "ops.h"

namespace dacp {

constexpr int kTile = 16;

// C[M x N] = op(A)[M x K] op(B)[K x N] (+ bias[N]) (relu), row-major.
// op(A) = A (A is M x K, lda) or A^T (A is K x M, lda); likewise for B.
template <bool TA, bool TB>
__global__ void sgemm_kernel(int M, int N, int K, const float* __restrict__ A, int lda,
                             const float* __restrict__ B, int ldb, float* __restrict__ C, int ldc,
                             const float* __restrict__ bias, int relu, int accumulate) {
    __shared__ float As[kTile][kTile + 1];
    __shared__ float Bs[kTile][kTile + 1];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int row = blockIdx.y * kTile + ty;
    const int col = blockIdx.x * kTile + tx;
    float acc = 0.f;
    for (int k0 = 0; k0 < K; k0 += kTile) {
        const int ka = k0 + tx;   // A tile: rows of C, k along x
        if (row < M && ka < K) As[ty][tx] = TA ? A[static_cast<int64_t>(ka) * lda + row] : A[static_cast<int64_t>(row) * lda + ka];
        else As[ty][tx] = 0.f;
        const int kb = k0 + ty;   // B tile: k along y, cols of C
        if (kb < K && col < N) Bs[ty][tx] = TB ? B[static_cast<int64_t>(col) * ldb + kb] : B[static_cast<int64_t>(kb) * ldb + col];
        else Bs[ty][tx] = 0.f;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kTile; ++k) acc = fmaf(As[ty][k], Bs[k][tx], acc);
        __syncthreads();
    }
    if (row < M && col < N) {
        if (bias) acc += bias[col];
        if (relu) acc = fmaxf(acc, 0.f);
        float* c = C + static_cast<int64_t>(row) * ldc + col;
        *c = accumulate ? *c + acc : acc;
    }
}

// delta = (y - t) / B, loss partials = (y - t)^2 / (2B)
__global__ void mse_grad_kernel(const float* __restrict__ y, const float* __restrict__ t, int n, float inv_b,
                                float* __restrict__ delta, double* __restrict__ loss) {
    __shared__ double red[256];
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float r = y[i] - t[i];
        delta[i] = r * inv_b;
        acc += 0.5 * static_cast<double>(r) * r * inv_b;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, red[0]);
}

// delta_prev *= relu'(z_prev): z_prev > 0 <=> a_prev > 0
__global__ void relu_mask_kernel(float* __restrict__ d, const float* __restrict__ a, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        if (!(a[i] > 0.f)) d[i] = 0.f;
}

// db[j] = sum_b delta[b][j]
__global__ void colsum_kernel(const float* __restrict__ d, int B, int N, float* __restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    float s = 0.f;
    for (int b = 0; b < B; ++b) s += d[static_cast<int64_t>(b) * N + j];
    out[j] = s;
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// x_out[b][f] = (x[idx[b]][f] - mean[f]) / std[f]; idx may be NULL (identity)
__global__ void gather_norm_kernel(const float* __restrict__ x, const int* __restrict__ idx, int B, int F,
                                   const float* __restrict__ mean, const float* __restrict__ sd,
                                   float* __restrict__ out) {
    const int n = B * F;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int b = i / F, f = i % F;
        const int src = idx ? idx[b] : b;
        out[i] = (x[static_cast<int64_t>(src) * F + f] - mean[f]) / sd[f];
    }
}

// y = clamp(z * std + mean, lo, hi)
__global__ void denorm_kernel(const float* __restrict__ z, int B, int F, const float* __restrict__ mean,
                              const float* __restrict__ sd, const float* __restrict__ lo,
                              const float* __restrict__ hi, float* __restrict__ y) {
    const int n = B * F;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int f = i % F;
        y[i] = fminf(fmaxf(z[i] * sd[f] + mean[f], lo[f]), hi[f]);
    }
}

template <bool TA, bool TB>
static void sgemm(int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* C, int ldc,
                  const float* bias, int relu, int acc, cudaStream_t st) {
    dim3 blk(kTile, kTile), grid((N + kTile - 1) / kTile, (M + kTile - 1) / kTile);
    sgemm_kernel<TA, TB><<<grid, blk, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, relu, acc);
}

static int grid1(int64_t n) { return static_cast<int>(std::min<int64_t>((n + 255) / 256, 4096)); }

}  // namespace dacp

using namespace dacp;

struct dacp_mlp_ctx {
    std::vector<int> sizes;              // n_in, hidden..., n_out
    std::vector<int64_t> woff, boff;     // offsets into the flat parameter vector
    int64_t nparam = 0;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    int device = 0;
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
    float *in_mean = nullptr, *in_std = nullptr, *out_mean = nullptr, *out_std = nullptr;
    float *out_lo = nullptr, *out_hi = nullptr;   // range the outputs are clamped to
    std::vector<float*> act;             // activations per layer, capacity cap_b rows
    float* delta[2] = {nullptr, nullptr};
    float *xb = nullptr, *tb = nullptr, *yb = nullptr;
    double* loss_d = nullptr;
    int cap_b = 0;
    int adam_t = 0;
    int64_t launches = 0;
    std::string err;
};

namespace {

dacp_status mfail(dacp_mlp_ctx* c, dacp_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return s;
}

#define MCK(call)                                                                                   \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) return mfail(c, DACP_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

int max_width(const dacp_mlp_ctx* c) {
    int w = 0;
    for (int s : c->sizes) w = std::max(w, s);
    return w;
}

dacp_status ensure_batch(dacp_mlp_ctx* c, int B) {
    if (B <= c->cap_b) return DACP_OK;
    for (float* a : c->act) cudaFree(a);
    cudaFree(c->delta[0]);
    cudaFree(c->delta[1]);
    cudaFree(c->xb);
    cudaFree(c->tb);
    cudaFree(c->yb);
    c->act.assign(c->sizes.size(), nullptr);
    const int W = max_width(c);
    for (size_t l = 0; l < c->sizes.size(); ++l) MCK(cudaMalloc(&c->act[l], sizeof(float) * B * c->sizes[l]));
    MCK(cudaMalloc(&c->delta[0], sizeof(float) * B * W));
    MCK(cudaMalloc(&c->delta[1], sizeof(float) * B * W));
    MCK(cudaMalloc(&c->xb, sizeof(float) * B * c->sizes.front()));
    MCK(cudaMalloc(&c->tb, sizeof(float) * B * c->sizes.back()));
    MCK(cudaMalloc(&c->yb, sizeof(float) * B * c->sizes.back()));
    c->cap_b = B;
    return DACP_OK;
}

// act[0] = normalised inputs (already there); act[l] = layer outputs; act[L] = linear output
void forward_dev(dacp_mlp_ctx* c, int B) {
    const int L = static_cast<int>(c->sizes.size()) - 1;
    for (int l = 0; l < L; ++l) {
        const int in = c->sizes[l], out = c->sizes[l + 1];
        sgemm<false, true>(B, out, in, c->act[l], in, c->p + c->woff[l], in, c->act[l + 1], out,
                           c->p + c->boff[l], l < L - 1 ? 1 : 0, 0, c->st);
    }
    c->launches += L;
}

// gradients into c->g given normalised targets tb; returns loss via loss_d
void backward_dev(dacp_mlp_ctx* c, int B) {
    const int L = static_cast<int>(c->sizes.size()) - 1;
    const int nout = c->sizes.back();
    cudaMemsetAsync(c->loss_d, 0, sizeof(double), c->st);
    mse_grad_kernel<<<grid1(B * nout), 256, 0, c->st>>>(c->act[L], c->tb, B * nout, 1.f / B, c->delta[0], c->loss_d);
    c->launches += 1;
    int cur = 0;
    for (int l = L - 1; l >= 0; --l) {
        const int in = c->sizes[l], out = c->sizes[l + 1];
        // dW_l [out x in] = delta^T [out x B] * a_l [B x in]
        sgemm<true, false>(out, in, B, c->delta[cur], out, c->act[l], in, c->g + c->woff[l], in, nullptr, 0, 0, c->st);
        colsum_kernel<<<(out + 255) / 256, 256, 0, c->st>>>(c->delta[cur], B, out, c->g + c->boff[l]);
        c->launches += 2;
        if (l > 0) {
            // delta_prev [B x in] = delta [B x out] * W_l [out x in], masked by relu'
            sgemm<false, false>(B, in, out, c->delta[cur], out, c->p + c->woff[l], in, c->delta[1 - cur], in, nullptr,
                                0, 0, c->st);
            relu_mask_kernel<<<grid1(B * in), 256, 0, c->st>>>(c->delta[1 - cur], c->act[l], B * in);
            c->launches += 2;
            cur = 1 - cur;
        }
    }
}

}  // namespace

extern "C" {

dacp_status dacp_mlp_create(dacp_mlp* out, int n_in, int n_hidden, int hidden_layers, int n_out,
                            const float* weights, uint64_t seed, void* stream) {
    if (!out) return DACP_ERR_ARG;
    *out = nullptr;
    if (n_in < 1 || n_hidden < 1 || hidden_layers < 0 || hidden_layers > 8 || n_out < 1 || n_in > 4096 ||
        n_hidden > 4096 || n_out > 4096)
        return DACP_ERR_ARG;
    dacp_mlp_ctx* c = new dacp_mlp_ctx();
    cudaGetDevice(&c->device);
    c->sizes.push_back(n_in);
    for (int i = 0; i < hidden_layers; ++i) c->sizes.push_back(n_hidden);
    c->sizes.push_back(n_out);
    int64_t o = 0;
    for (size_t l = 0; l + 1 < c->sizes.size(); ++l) {
        c->woff.push_back(o);
        o += static_cast<int64_t>(c->sizes[l]) * c->sizes[l + 1];
        c->boff.push_back(o);
        o += c->sizes[l + 1];
    }
    c->nparam = o;
    auto bail = [&](dacp_status s) {
        dacp_mlp_destroy(c);
        return s;
    };
    if (stream) {
        c->st = static_cast<cudaStream_t>(stream);
    } else {
        if (cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking) != cudaSuccess) return bail(DACP_ERR_CUDA);
        c->own_stream = true;
    }
    std::vector<float> h(static_cast<size_t>(o), 0.f);
    if (weights) {
        memcpy(h.data(), weights, sizeof(float) * o);
    } else {
        std::mt19937_64 rng(seed);
        for (size_t l = 0; l + 1 < c->sizes.size(); ++l) {
            const float lim = sqrtf(6.f / c->sizes[l]);
            std::uniform_real_distribution<float> U(-lim, lim);
            for (int64_t i = 0; i < static_cast<int64_t>(c->sizes[l]) * c->sizes[l + 1]; ++i) h[c->woff[l] + i] = U(rng);
        }
    }
    const size_t pb = sizeof(float) * o;
    if (cudaMalloc(&c->p, pb) != cudaSuccess || cudaMalloc(&c->g, pb) != cudaSuccess ||
        cudaMalloc(&c->m, pb) != cudaSuccess || cudaMalloc(&c->v, pb) != cudaSuccess ||
        cudaMalloc(&c->in_mean, sizeof(float) * n_in) != cudaSuccess ||
        cudaMalloc(&c->in_std, sizeof(float) * n_in) != cudaSuccess ||
        cudaMalloc(&c->out_mean, sizeof(float) * n_out) != cudaSuccess ||
        cudaMalloc(&c->out_std, sizeof(float) * n_out) != cudaSuccess ||
        cudaMalloc(&c->out_lo, sizeof(float) * n_out) != cudaSuccess ||
        cudaMalloc(&c->out_hi, sizeof(float) * n_out) != cudaSuccess ||
        cudaMalloc(&c->loss_d, sizeof(double)) != cudaSuccess)
        return bail(DACP_ERR_NOMEM);
    std::vector<float> zeros_in(n_in, 0.f), ones_in(n_in, 1.f), zeros_out(n_out, 0.f), ones_out(n_out, 1.f);
    std::vector<float> lo_out(n_out, -FLT_MAX), hi_out(n_out, FLT_MAX);
    bool ok = cudaMemcpy(c->p, h.data(), pb, cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemset(c->m, 0, pb) == cudaSuccess && cudaMemset(c->v, 0, pb) == cudaSuccess &&
              cudaMemcpy(c->in_mean, zeros_in.data(), 4 * n_in, cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemcpy(c->in_std, ones_in.data(), 4 * n_in, cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemcpy(c->out_mean, zeros_out.data(), 4 * n_out, cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemcpy(c->out_std, ones_out.data(), 4 * n_out, cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemcpy(c->out_lo, lo_out.data(), 4 * n_out, cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemcpy(c->out_hi, hi_out.data(), 4 * n_out, cudaMemcpyHostToDevice) == cudaSuccess;
    if (!ok) return bail(DACP_ERR_CUDA);
    *out = c;
    return DACP_OK;
}

void dacp_mlp_destroy(dacp_mlp c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->st) cudaStreamSynchronize(c->st);
    for (float* a : c->act) cudaFree(a);
    for (void* q : {static_cast<void*>(c->p), static_cast<void*>(c->g), static_cast<void*>(c->m),
                    static_cast<void*>(c->v), static_cast<void*>(c->in_mean), static_cast<void*>(c->in_std),
                    static_cast<void*>(c->out_mean), static_cast<void*>(c->out_std), static_cast<void*>(c->out_lo),
                    static_cast<void*>(c->out_hi), static_cast<void*>(c->delta[0]),
                    static_cast<void*>(c->delta[1]), static_cast<void*>(c->xb), static_cast<void*>(c->tb),
                    static_cast<void*>(c->yb), static_cast<void*>(c->loss_d)})
        cudaFree(q);
    if (c->own_stream && c->st) cudaStreamDestroy(c->st);
    delete c;
}

const char* dacp_mlp_last_error(dacp_mlp c) { return c ? c->err.c_str() : "NULL handle"; }

dacp_status dacp_mlp_get_weights(dacp_mlp c, float* w, int64_t cap, int64_t* count) {
    if (!c) return DACP_ERR_ARG;
    if (count) *count = c->nparam;
    if (!w || cap < c->nparam) return mfail(c, DACP_ERR_ARG, "capacity %lld < %lld", (long long)cap, (long long)c->nparam);
    cudaSetDevice(c->device);
    MCK(cudaMemcpyAsync(w, c->p, sizeof(float) * c->nparam, cudaMemcpyDeviceToHost, c->st));
    MCK(cudaStreamSynchronize(c->st));
    return DACP_OK;
}

dacp_status dacp_mlp_set_weights(dacp_mlp c, const float* w, int64_t count) {
    if (!c || !w || count != c->nparam) return mfail(c, DACP_ERR_ARG, "expected %lld weights", c ? (long long)c->nparam : 0LL);
    cudaSetDevice(c->device);
    MCK(cudaMemcpyAsync(c->p, w, sizeof(float) * count, cudaMemcpyHostToDevice, c->st));
    MCK(cudaMemsetAsync(c->m, 0, sizeof(float) * count, c->st));
    MCK(cudaMemsetAsync(c->v, 0, sizeof(float) * count, c->st));
    MCK(cudaStreamSynchronize(c->st));
    c->adam_t = 0;
    return DACP_OK;
}

dacp_status dacp_mlp_set_normalization(dacp_mlp c, const float* in_mean, const float* in_std,
                                       const float* out_mean, const float* out_std) {
    if (!c || !in_mean || !in_std || !out_mean || !out_std) return DACP_ERR_ARG;
    cudaSetDevice(c->device);
    const int ni = c->sizes.front(), no = c->sizes.back();
    for (int i = 0; i < ni; ++i)
        if (!(in_std[i] > 0.f)) return mfail(c, DACP_ERR_ARG, "in_std[%d] <= 0", i);
    for (int i = 0; i < no; ++i)
        if (!(out_std[i] > 0.f)) return mfail(c, DACP_ERR_ARG, "out_std[%d] <= 0", i);
    MCK(cudaMemcpyAsync(c->in_mean, in_mean, 4 * ni, cudaMemcpyHostToDevice, c->st));
    MCK(cudaMemcpyAsync(c->in_std, in_std, 4 * ni, cudaMemcpyHostToDevice, c->st));
    MCK(cudaMemcpyAsync(c->out_mean, out_mean, 4 * no, cudaMemcpyHostToDevice, c->st));
    MCK(cudaMemcpyAsync(c->out_std, out_std, 4 * no, cudaMemcpyHostToDevice, c->st));
    MCK(cudaStreamSynchronize(c->st));
    return DACP_OK;
}

dacp_status dacp_mlp_set_output_range(dacp_mlp c, const float* lo, const float* hi) {
    if (!c || !lo || !hi) return DACP_ERR_ARG;
    cudaSetDevice(c->device);
    const int no = c->sizes.back();
    for (int i = 0; i < no; ++i)
        if (!(lo[i] <= hi[i])) return mfail(c, DACP_ERR_ARG, "output range %d: lo > hi or NaN", i);
    MCK(cudaMemcpyAsync(c->out_lo, lo, 4 * no, cudaMemcpyHostToDevice, c->st));
    MCK(cudaMemcpyAsync(c->out_hi, hi, 4 * no, cudaMemcpyHostToDevice, c->st));
    MCK(cudaStreamSynchronize(c->st));
    return DACP_OK;
}

dacp_status dacp_mlp_forward(dacp_mlp c, const float* x, int batch, float* y) {
    if (!c || !x || !y || batch < 1) return DACP_ERR_ARG;
    cudaSetDevice(c->device);
    dacp_status s = ensure_batch(c, batch);
    if (s != DACP_OK) return s;
    const int ni = c->sizes.front(), no = c->sizes.back(), L = static_cast<int>(c->sizes.size()) - 1;
    MCK(cudaMemcpyAsync(c->xb, x, sizeof(float) * batch * ni, cudaMemcpyHostToDevice, c->st));
    gather_norm_kernel<<<grid1(batch * ni), 256, 0, c->st>>>(c->xb, nullptr, batch, ni, c->in_mean, c->in_std, c->act[0]);
    forward_dev(c, batch);
    denorm_kernel<<<grid1(batch * no), 256, 0, c->st>>>(c->act[L], batch, no, c->out_mean, c->out_std, c->out_lo,
                                                         c->out_hi, c->yb);
    c->launches += 2;
    MCK(cudaGetLastError());
    MCK(cudaMemcpyAsync(y, c->yb, sizeof(float) * batch * no, cudaMemcpyDeviceToHost, c->st));
    MCK(cudaStreamSynchronize(c->st));
    return DACP_OK;
}

dacp_status dacp_mlp_gradients(dacp_mlp c, const float* x, const float* t, int batch, float* grad, double* loss) {
    if (!c || !x || !t || !grad || batch < 1) return DACP_ERR_ARG;
    cudaSetDevice(c->device);
    dacp_status s = ensure_batch(c, batch);
    if (s != DACP_OK) return s;
    const int ni = c->sizes.front(), no = c->sizes.back();
    MCK(cudaMemcpyAsync(c->xb, x, sizeof(float) * batch * ni, cudaMemcpyHostToDevice, c->st));
    MCK(cudaMemcpyAsync(c->yb, t, sizeof(float) * batch * no, cudaMemcpyHostToDevice, c->st));
    gather_norm_kernel<<<grid1(batch * ni), 256, 0, c->st>>>(c->xb, nullptr, batch, ni, c->in_mean, c->in_std, c->act[0]);
    gather_norm_kernel<<<grid1(batch * no), 256, 0, c->st>>>(c->yb, nullptr, batch, no, c->out_mean, c->out_std, c->tb);
    c->launches += 2;
    forward_dev(c, batch);
    backward_dev(c, batch);
    MCK(cudaGetLastError());
    MCK(cudaMemcpyAsync(grad, c->g, sizeof(float) * c->nparam, cudaMemcpyDeviceToHost, c->st));
    double l = 0.0;
    MCK(cudaMemcpyAsync(&l, c->loss_d, sizeof(double), cudaMemcpyDeviceToHost, c->st));
    MCK(cudaStreamSynchronize(c->st));
    if (loss) *loss = l;
    return DACP_OK;
}

dacp_status dacp_mlp_train(dacp_mlp c, const float* x, const float* t, int n_samples, int batch, int epochs,
                           float lr, uint64_t seed, double* final_loss) {
    if (!c || !x || !t || n_samples < 1 || batch < 1 || epochs < 1 || !(lr > 0.f)) return DACP_ERR_ARG;
    cudaSetDevice(c->device);
    batch = std::min(batch, n_samples);
    dacp_status s = ensure_batch(c, batch);
    if (s != DACP_OK) return s;
    const int ni = c->sizes.front(), no = c->sizes.back();
    float *xd = nullptr, *td = nullptr;
    int* idx_d = nullptr;
    double* epoch_loss = nullptr;
    auto cleanup = [&]() {
        cudaFree(xd);
        cudaFree(td);
        cudaFree(idx_d);
        cudaFree(epoch_loss);
    };
    if (cudaMalloc(&xd, sizeof(float) * n_samples * ni) != cudaSuccess ||
        cudaMalloc(&td, sizeof(float) * n_samples * no) != cudaSuccess ||
        cudaMalloc(&idx_d, sizeof(int) * n_samples) != cudaSuccess ||
        cudaMalloc(&epoch_loss, sizeof(double)) != cudaSuccess) {
        cleanup();
        return mfail(c, DACP_ERR_NOMEM, "training buffers");
    }
    cudaMemcpyAsync(xd, x, sizeof(float) * n_samples * ni, cudaMemcpyHostToDevice, c->st);
    cudaMemcpyAsync(td, t, sizeof(float) * n_samples * no, cudaMemcpyHostToDevice, c->st);
    std::mt19937_64 rng(seed);
    std::vector<int> perm(n_samples);
    for (int i = 0; i < n_samples; ++i) perm[i] = i;
    const int steps_per_epoch = n_samples / batch;
    double last = 0.0;
    for (int ep = 0; ep < epochs; ++ep) {
        std::shuffle(perm.begin(), perm.end(), rng);
        cudaMemcpyAsync(idx_d, perm.data(), sizeof(int) * n_samples, cudaMemcpyHostToDevice, c->st);
        cudaMemsetAsync(epoch_loss, 0, sizeof(double), c->st);
        for (int sidx = 0; sidx < steps_per_epoch; ++sidx) {
            const int* ib = idx_d + sidx * batch;
            gather_norm_kernel<<<grid1(batch * ni), 256, 0, c->st>>>(xd, ib, batch, ni, c->in_mean, c->in_std, c->act[0]);
            gather_norm_kernel<<<grid1(batch * no), 256, 0, c->st>>>(td, ib, batch, no, c->out_mean, c->out_std, c->tb);
            c->launches += 2;
            forward_dev(c, batch);
            backward_dev(c, batch);
            ++c->adam_t;
            const float c1 = 1.f - powf(0.9f, static_cast<float>(c->adam_t));
            const float c2 = 1.f - powf(0.999f, static_cast<float>(c->adam_t));
            adam_kernel<<<grid1(c->nparam), 256, 0, c->st>>>(c->p, c->g, c->m, c->v, static_cast<int>(c->nparam), lr, 0.9f,
                                                              0.999f, 1e-8f, c1, c2);
            c->launches += 1;
        }
        if (ep == epochs - 1) {
            cudaMemcpyAsync(&last, c->loss_d, sizeof(double), cudaMemcpyDeviceToHost, c->st);
        }
    }
    cudaError_t e = cudaStreamSynchronize(c->st);
    cleanup();
    if (e != cudaSuccess) return mfail(c, DACP_ERR_CUDA, "training: %s", cudaGetErrorString(e));
    if (final_loss) *final_loss = last;
    return DACP_OK;
}

dacp_status dacp_mlp_get_launch_count(dacp_mlp c, int64_t* count) {
    if (!c || !count) return DACP_ERR_ARG;
    *count = c->launches;
    return DACP_OK;
}

}  // extern "C"

// Device-side forward for the DACP handle: features already normalised in
// `in` (B x n_in on the device); raw outputs (denormalised) into `out`.
namespace dacp {
cudaError_t mlp_forward_device(dacp_mlp c, const float* feats, int B, float* out, cudaStream_t st, int64_t* launches) {
    if (ensure_batch(c, B) != DACP_OK) return cudaErrorMemoryAllocation;
    const int ni = c->sizes.front(), no = c->sizes.back(), L = static_cast<int>(c->sizes.size()) - 1;
    cudaStream_t keep = c->st;
    c->st = st;
    gather_norm_kernel<<<grid1(B * ni), 256, 0, st>>>(feats, nullptr, B, ni, c->in_mean, c->in_std, c->act[0]);
    forward_dev(c, B);
    denorm_kernel<<<grid1(B * no), 256, 0, st>>>(c->act[L], B, no, c->out_mean, c->out_std, c->out_lo, c->out_hi,
                                                 out);
    c->st = keep;
    if (launches) *launches += L + 2;
    return cudaGetLastError();
}
int mlp_n_in(dacp_mlp c) { return c->sizes.front(); }
int mlp_n_out(dacp_mlp c) { return c->sizes.back(); }
}  // namespace dacp
