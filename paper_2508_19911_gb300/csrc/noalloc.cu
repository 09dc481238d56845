// gks_diagnostics_noalloc: the diagnostics reduction for callers that must
// not allocate device memory.
//
// Who needs it: a monitor that samples E_k, the dissipation rates and the
// positivity of a running simulation from outside the solver -- a host
// thread, a checkpoint hook, a library that only receives device pointers.
// A large run (CGKS-5th at 256^3 keeps ~80 GB of state and workspace)
// leaves little free HBM, so a cudaMalloc made just to sample diagnostics
// can fail or evict the simulation's own buffers, and a caller without a
// gks_ctx has no workspace to borrow. This entry point allocates nothing:
// its scratch (one block of partial sums per chunk of cells) is the
// file-scope device array below, which every GPU that loads the library
// holds (3 MB) until the process exits.
//
// The results equal gks_diagnostics' up to the order of the floating-point
// sums (a different partition of the cells into blocks).
#include <cmath>
#include <mutex>

#include "common.cuh"
#include "../../include/gks.h"

namespace gks {
namespace {

constexpr int kNaBlock = 256;
constexpr long long kNaChunk = 4096;       // cells per block
constexpr int kNaMaxChunks = 32768;        // => at most 2^27 cells (512^3)
constexpr int kNaSlots = 12;

// 32768 chunks x 12 partial results x 8 bytes = 3 MiB
static __device__ __align__(256) double g_noalloc_partials[kNaMaxChunks * kNaSlots];

__device__ __forceinline__ double na_combine(int s, double a, double b) {
    if (s == 3 || s == 4) return fmin(a, b);
    if (s == 11) return fmax(a, b);
    return a + b;
}

__device__ __forceinline__ double na_identity(int s) {
    return (s == 3 || s == 4) ? INFINITY : 0.0;
}

__device__ void na_block_reduce(double acc[kNaSlots], double *dst) {
    __shared__ double sh[kNaSlots][kNaBlock];
#pragma unroll
    for (int s = 0; s < kNaSlots; ++s) sh[s][threadIdx.x] = acc[s];
    __syncthreads();
    for (int w = kNaBlock / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
#pragma unroll
            for (int s = 0; s < kNaSlots; ++s)
                sh[s][threadIdx.x] = na_combine(s, sh[s][threadIdx.x], sh[s][threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
#pragma unroll
        for (int s = 0; s < kNaSlots; ++s) dst[s] = sh[s][0];
    }
}

// One block per chunk of kNaChunk cells; block b writes its 12 results to
// partials[12 b .. 12 b + 11] (every slot a later kernel reads is written by
// this call, so nothing has to be cleared beforehand).
__global__ void __launch_bounds__(kNaBlock) na_partial_kernel(GridDesc g, PhysParams P,
                                                              const double *__restrict__ Q,
                                                              const double *__restrict__ G,
                                                              double *partials) {
    const long long n = g.n;
    const double vol = g.h[0] * g.h[1] * g.h[2];
    double acc[kNaSlots];
#pragma unroll
    for (int s = 0; s < kNaSlots; ++s) acc[s] = na_identity(s);
    const long long begin = (long long)blockIdx.x * kNaChunk;
    const long long end = begin + kNaChunk < n ? begin + kNaChunk : n;
    for (long long c = begin + threadIdx.x; c < end; c += blockDim.x) {
        double W[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) {
            W[v] = Q[(long long)v * n + c];
            acc[5 + v] += W[v] * vol;
        }
        const double rho = W[0];
        const double vel[3] = {W[1] / rho, W[2] / rho, W[3] / rho};
        const double p = (P.gamma - 1.0) *
                         (W[4] - 0.5 * rho * (vel[0] * vel[0] + vel[1] * vel[1] + vel[2] * vel[2]));
        bool ok = rho > 0.0 && p > 0.0;
#pragma unroll
        for (int v = 0; v < 5; ++v) ok = ok && isfinite(W[v]);
        if (!ok) {
            acc[10] += 1.0;
            continue;
        }
        acc[3] = fmin(acc[3], rho);
        acc[4] = fmin(acc[4], p);
        const double cs = sqrt(P.gamma * p / rho);
#pragma unroll
        for (int d = 0; d < 3; ++d) acc[11] = fmax(acc[11], fabs(vel[d]) + cs);
        acc[0] += 0.5 * rho * (vel[0] * vel[0] + vel[1] * vel[1] + vel[2] * vel[2]) * vol;
        const int i = (int)(c % g.nx);
        const int j = (int)((c / g.nx) % g.ny);
        const int k = (int)(c / ((long long)g.nx * g.ny));
        double dQ[4][3];
#pragma unroll
        for (int v = 0; v < 4; ++v)
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                if (G) {
                    dQ[v][d] = G[((long long)v * 3 + d) * n + c];
                } else {
                    const long long hi = cell_index(g, d == 0 ? wrap(i + 1, g.nx) : i,
                                                    d == 1 ? wrap(j + 1, g.ny) : j,
                                                    d == 2 ? wrap(k + 1, g.nz) : k);
                    const long long lo = cell_index(g, d == 0 ? wrap(i - 1, g.nx) : i,
                                                    d == 1 ? wrap(j - 1, g.ny) : j,
                                                    d == 2 ? wrap(k - 1, g.nz) : k);
                    dQ[v][d] = (Q[(long long)v * n + hi] - Q[(long long)v * n + lo]) / (2.0 * g.h[d]);
                }
            }
        double du[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int d = 0; d < 3; ++d) du[a][d] = (dQ[1 + a][d] - vel[a] * dQ[0][d]) / rho;
        const double wx = du[2][1] - du[1][2], wy = du[0][2] - du[2][0], wz = du[1][0] - du[0][1];
        const double div = du[0][0] + du[1][1] + du[2][2];
        const double mu = viscosity(P, rho, p);
        acc[1] += mu * (wx * wx + wy * wy + wz * wz) * vol;
        acc[2] += 4.0 / 3.0 * mu * div * div * vol;
    }
    na_block_reduce(acc, partials + (long long)blockIdx.x * kNaSlots);
}

__global__ void __launch_bounds__(kNaBlock) na_final_kernel(const double *partials, int nchunks,
                                                            double volume, double *out) {
    double acc[kNaSlots];
#pragma unroll
    for (int s = 0; s < kNaSlots; ++s) acc[s] = na_identity(s);
    for (int b = threadIdx.x; b < nchunks; b += blockDim.x)
#pragma unroll
        for (int s = 0; s < kNaSlots; ++s)
            acc[s] = na_combine(s, acc[s], partials[(long long)b * kNaSlots + s]);
    __shared__ double res[kNaSlots];
    na_block_reduce(acc, res);
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int s = 0; s < kNaSlots; ++s) out[s] = res[s];
        out[0] /= volume;
        out[1] /= volume;
        out[2] /= volume;
    }
}

// Device address of g_noalloc_partials, looked up once per device (with that
// device current). In host code the symbol is only a host-side stand-in.
constexpr int kMaxDevices = 64;
std::mutex g_na_mutex;
double *g_na_ptr[kMaxDevices] = {nullptr};

int na_scratch(int dev, double **ptr) {
    if (dev < 0 || dev >= kMaxDevices) return GKS_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return GKS_ERR_CUDA;
        }
        g_na_ptr[dev] = (double *)p;
    }
    *ptr = g_na_ptr[dev];
    return GKS_OK;
}

}  // namespace
}  // namespace gks

extern "C" int gks_diagnostics_noalloc(const double *Q, const double *gradQ, int nx, int ny,
                                       int nz, double Lx, double Ly, double Lz, double gamma,
                                       double mu, int mu_law, double T_ref, double *out_dev,
                                       void *cuda_stream) {
    using namespace gks;
    if (!Q || !out_dev) return GKS_ERR_ARG;
    if (nx < 1 || ny < 1 || nz < 1 || !(Lx > 0.0) || !(Ly > 0.0) || !(Lz > 0.0)) return GKS_ERR_ARG;
    if (!(gamma > 1.0) || !(mu >= 0.0) || mu_law < 0 || mu_law > 1 || !(T_ref > 0.0))
        return GKS_ERR_ARG;
    const long long n = (long long)nx * ny * nz;
    const long long nchunks = (n + kNaChunk - 1) / kNaChunk;
    if (nchunks > kNaMaxChunks) return GKS_ERR_ARG;  // more than 2^27 cells
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return GKS_ERR_CUDA;
    double *scratch = nullptr;
    const int rc = na_scratch(dev, &scratch);
    if (rc) return rc;
    GridDesc g;
    g.nx = nx; g.ny = ny; g.nz = nz; g.n = n;
    g.h[0] = Lx / nx; g.h[1] = Ly / ny; g.h[2] = Lz / nz;
    PhysParams P = {};
    P.gamma = gamma;
    P.mu0 = mu;
    P.mu_law = mu_law;
    P.T_ref = T_ref;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    na_partial_kernel<<<(unsigned)nchunks, kNaBlock, 0, s>>>(g, P, Q, gradQ, scratch);
    na_final_kernel<<<1, kNaBlock, 0, s>>>(scratch, (int)nchunks,
                                           g.h[0] * g.h[1] * g.h[2] * (double)n, out_dev);
    return cudaGetLastError() == cudaSuccess ? GKS_OK : GKS_ERR_CUDA;
}
