// gks_diagnostics_noalloc: the diagnostics reduction for callers that must
// not allocate device memory.
//
// Who needs it: a monitor that samples E_k, the dissipation rates and the
// positivity of a running simulation from outside the solver -- a host
// thread, a checkpoint hook, a library that only receives device pointers.
// A large run (CGKS-5th at 512^3 keeps ~230 GB of state and workspace)
// leaves little free HBM, so a cudaMalloc made just to sample diagnostics
// can fail or evict the simulation's own buffers, and a caller without a
// gks_ctx has no workspace to borrow. This entry point allocates nothing:
// its scratch (the partial results of the reduction's blocks) is the
// file-scope device array below, which every GPU that loads the library
// holds (57 KB) until the process exits.
//
// The kernels are the context's own (launch_diagnostics in update.cu) with
// the same block count, so the results equal gks_diagnostics' bit for bit.
#include <mutex>

#include "common.cuh"
#include "../../include/gks.h"

namespace gks {
namespace {

// kDiagMaxBlocks blocks x kDiagSlots partial results x 8 bytes = 57 KiB
static __device__ __align__(256) double g_noalloc_partials[kDiagMaxBlocks * kDiagSlots];

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
    if (n > (1LL << 31)) return GKS_ERR_ARG;  // the grid limit of gks_init
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return GKS_ERR_CUDA;
    double *scratch = nullptr;
    const int rc = na_scratch(dev, &scratch);
    if (rc) return rc;
    GridDesc g = {};  // uniform, periodic: the general-grid fields stay zero
    g.nx = nx; g.ny = ny; g.nz = nz; g.n = n;
    g.h[0] = Lx / nx; g.h[1] = Ly / ny; g.h[2] = Lz / nz;
    PhysParams P = {};
    P.gamma = gamma;
    P.mu0 = mu;
    P.mu_law = mu_law;
    P.T_ref = T_ref;
    // every slot the final block reads is written by the partial blocks of
    // this call, so the shared scratch needs no clearing
    return launch_diagnostics(g, P, Q, gradQ, scratch, diagnostics_blocks(g), out_dev,
                              (cudaStream_t)cuda_stream)
               ? GKS_ERR_CUDA
               : GKS_OK;
}
