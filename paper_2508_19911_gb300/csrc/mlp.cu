// Learned smoothness indicator: training of the per-(cell, variable) MLP
// on the GPU, and its C-ABI.
//
// Network: x (the 63-entry CGKS-5th data vector) -> xh = x/(max|x| + delta)
// -> z = W1 xh + b1 (kMlpHidden = 8) -> h = max(z, 0) -> logit = w2 . h + b2,
// p = sigmoid(logit) = probability that GENO's chi equals 1 (within the
// label tolerance), i.e. that the nonlinear reconstruction is the linear P4.
// Loss: mean over the batch of w_y (softplus(logit) - y logit), w_0 = the
// weight of the "keep GENO" class, w_1 = 1.
//
// Training step (deterministic, no floating-point atomics):
//   forward kernel, one thread per sample of the batch: stores xh, h, the
//     back-propagated dL/dz and dL/dlogit;
//   gradient kernel, one thread per parameter: sums over the batch in
//     sample order;
//   Adam kernel, one thread per parameter.
#include <cmath>
#include <cstring>
#include <new>

#include "basis.h"
#include "common.cuh"
#include "../../include/gks.h"

namespace gks {
namespace {

constexpr int H = kMlpHidden;
constexpr int D = kNumData;
constexpr int NP = kMlpParams;
constexpr int kOffB1 = H * D, kOffW2 = H * D + H, kOffB2 = H * D + 2 * H;

struct Work {
    float *xh;    // [B][D]
    float *h;     // [B][H]
    float *dz;    // [B][H]
    float *dl;    // [B]
    float *loss;  // [B]
    float *grad;  // [NP]
    float *m, *v; // Adam moments [NP]
    float *lsum;  // [1]
};

__device__ __forceinline__ long long sample_index(long long k, long long stride, long long offset,
                                                  long long n) {
    return (k * stride + offset) % n;
}

__global__ void __launch_bounds__(128) mlp_forward_kernel(const float *__restrict__ params,
                                                          const float *__restrict__ x,
                                                          const float *__restrict__ y,
                                                          long long ld, long long n, int B,
                                                          long long first, long long stride,
                                                          long long offset, float w0, Work w) {
    const int sb = blockIdx.x * blockDim.x + threadIdx.x;
    if (sb >= B) return;
    const long long s = sample_index(first + sb, stride, offset, n);
    float xs[D];
    float m = 0.0f;
#pragma unroll
    for (int c = 0; c < D; ++c) {
        xs[c] = x[(long long)c * ld + s];
        m = fmaxf(m, fabsf(xs[c]));
    }
    const float inv = 1.0f / (m + kMlpDelta);
#pragma unroll
    for (int c = 0; c < D; ++c) {
        xs[c] *= inv;
        w.xh[(long long)sb * D + c] = xs[c];
    }
    float logit = params[kOffB2];
    float hz[H];
#pragma unroll
    for (int j = 0; j < H; ++j) {
        float z = params[kOffB1 + j];
#pragma unroll
        for (int c = 0; c < D; ++c) z = fmaf(params[j * D + c], xs[c], z);
        hz[j] = z;
        const float hj = fmaxf(z, 0.0f);
        w.h[(long long)sb * H + j] = hj;
        logit = fmaf(params[kOffW2 + j], hj, logit);
    }
    const float yy = y[s];
    const float wt = yy > 0.5f ? 1.0f : w0;
    // softplus(logit) - y logit, written stably
    const float sp = fmaxf(logit, 0.0f) + log1pf(expf(-fabsf(logit)));
    w.loss[sb] = wt * (sp - yy * logit);
    const float p = 1.0f / (1.0f + expf(-logit));
    const float dl = wt * (p - yy) / (float)B;
    w.dl[sb] = dl;
#pragma unroll
    for (int j = 0; j < H; ++j) w.dz[(long long)sb * H + j] = hz[j] > 0.0f ? dl * params[kOffW2 + j] : 0.0f;
}

__global__ void __launch_bounds__(128) mlp_grad_kernel(int B, Work w) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > NP) return;
    float s = 0.0f;
    if (p == NP) {  // mean loss of the batch
        for (int b = 0; b < B; ++b) s += w.loss[b];
        *w.lsum = s / (float)B;
        return;
    }
    if (p < kOffB1) {
        const int j = p / D, c = p % D;
        for (int b = 0; b < B; ++b) s = fmaf(w.dz[(long long)b * H + j], w.xh[(long long)b * D + c], s);
    } else if (p < kOffW2) {
        const int j = p - kOffB1;
        for (int b = 0; b < B; ++b) s += w.dz[(long long)b * H + j];
    } else if (p < kOffB2) {
        const int j = p - kOffW2;
        for (int b = 0; b < B; ++b) s = fmaf(w.dl[b], w.h[(long long)b * H + j], s);
    } else {
        for (int b = 0; b < B; ++b) s += w.dl[b];
    }
    w.grad[p] = s;
}

__global__ void mlp_adam_kernel(float *params, Work w, float lr, float b1, float b2, float eps,
                                float bc1, float bc2) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NP) return;
    const float g = w.grad[p];
    const float m = b1 * w.m[p] + (1.0f - b1) * g;
    const float v = b2 * w.v[p] + (1.0f - b2) * g * g;
    w.m[p] = m;
    w.v[p] = v;
    params[p] -= lr * (m / bc1) / (sqrtf(v / bc2) + eps);
}

__global__ void copy_loss_kernel(const float *lsum, float *dst, float scale, int accumulate) {
    if (accumulate) *dst += scale * *lsum;
    else *dst = scale * *lsum;
}

int alloc_work(Work *w, int B) {
    std::memset(w, 0, sizeof(*w));
    const size_t floats = (size_t)B * (D + 2 * H + 2) + 3 * NP + 1;
    float *base = nullptr;
    if (cudaMalloc((void **)&base, floats * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return GKS_ERR_NOMEM;
    }
    w->xh = base;
    w->h = w->xh + (size_t)B * D;
    w->dz = w->h + (size_t)B * H;
    w->dl = w->dz + (size_t)B * H;
    w->loss = w->dl + B;
    w->grad = w->loss + B;
    w->m = w->grad + NP;
    w->v = w->m + NP;
    w->lsum = w->v + NP;
    return GKS_OK;
}

__global__ void labels_kernel(const float *chi, float *y, long long m, float eps) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) y[i] = chi[i] >= 1.0f - eps ? 1.0f : 0.0f;
}

}  // namespace

int launch_labels(const float *chi, float *y, long long m, float eps, cudaStream_t s) {
    labels_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(chi, y, m, eps);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

}  // namespace gks

using namespace gks;

extern "C" int gks_mlp_nparams(void) { return NP; }

extern "C" int gks_mlp_loss_grad(const float *params, const float *x, const float *y, int n,
                                 long long ld, float neg_weight, float *loss, float *grad,
                                 void *cuda_stream) {
    if (!params || !x || !y || !loss || !grad || n <= 0 || ld < n || !(neg_weight > 0.0f))
        return GKS_ERR_ARG;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    Work w;
    int rc = alloc_work(&w, n);
    if (rc) return rc;
    mlp_forward_kernel<<<(n + 127) / 128, 128, 0, s>>>(params, x, y, ld, n, n, 0, 1, 0,
                                                       neg_weight, w);
    mlp_grad_kernel<<<(NP + 1 + 127) / 128, 128, 0, s>>>(n, w);
    cudaMemcpyAsync(grad, w.grad, sizeof(float) * NP, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(loss, w.lsum, sizeof(float), cudaMemcpyDeviceToDevice, s);
    const cudaError_t e = cudaStreamSynchronize(s);
    cudaFree(w.xh);
    return e == cudaSuccess && cudaGetLastError() == cudaSuccess ? GKS_OK : GKS_ERR_CUDA;
}

extern "C" int gks_mlp_train(float *params, const float *x, const float *y, int n, long long ld,
                             int epochs, int batch, float lr, float neg_weight, unsigned seed,
                             float *loss_hist, void *cuda_stream) {
    if (!params || !x || !y || n <= 0 || ld < n || epochs < 0 || batch <= 0 || batch > n ||
        !(lr > 0.0f) || !(neg_weight > 0.0f))
        return GKS_ERR_ARG;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    Work w;
    int rc = alloc_work(&w, batch);
    if (rc) return rc;
    cudaMemsetAsync(w.m, 0, sizeof(float) * 2 * NP, s);
    // sample order: k -> (k * stride + offset) mod n with stride coprime to n
    // (a fresh stride and offset per epoch from a small LCG on the seed)
    unsigned long long st = 0x9E3779B97F4A7C15ull ^ seed;
    auto next = [&st]() {
        st = st * 6364136223846793005ull + 1442695040888963407ull;
        return st >> 17;
    };
    auto gcd = [](long long a, long long b) {
        while (b) { const long long t = a % b; a = b; b = t; }
        return a;
    };
    const long long steps_per_epoch = n / batch;
    long long t = 0;
    const float b1 = 0.9f, b2 = 0.999f;
    for (int ep = 0; ep < epochs; ++ep) {
        long long stride = (long long)(next() % (unsigned long long)n);
        if (stride == 0) stride = 1;
        while (gcd(stride, n) != 1) stride = stride % n + 1;
        const long long offset = (long long)(next() % (unsigned long long)n);
        for (long long k = 0; k < steps_per_epoch; ++k) {
            ++t;
            mlp_forward_kernel<<<(batch + 127) / 128, 128, 0, s>>>(params, x, y, ld, n, batch,
                                                                   k * batch, stride, offset,
                                                                   neg_weight, w);
            mlp_grad_kernel<<<(NP + 1 + 127) / 128, 128, 0, s>>>(batch, w);
            mlp_adam_kernel<<<(NP + 127) / 128, 128, 0, s>>>(
                params, w, lr, b1, b2, 1e-8f, 1.0f - powf(b1, (float)t), 1.0f - powf(b2, (float)t));
            if (loss_hist)
                copy_loss_kernel<<<1, 1, 0, s>>>(w.lsum, loss_hist + ep, 1.0f / steps_per_epoch,
                                                 k > 0);
        }
    }
    const cudaError_t e = cudaStreamSynchronize(s);
    cudaFree(w.xh);
    return e == cudaSuccess && cudaGetLastError() == cudaSuccess ? GKS_OK : GKS_ERR_CUDA;
}
