// Shared device-side definitions of the GB300 CGKS-5th / GKS-2nd path.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace gks {

// status word bits (gks_status)
constexpr int kStatusNonphysical = 1;
constexpr int kStatusNonfinite = 2;

struct GridDesc {
    int nx, ny, nz;
    long long n;     // cells
    double h[3];     // cell sizes
};

struct PhysParams {
    double gamma, Pr, mu0, cfl, C_tau, eps_tau, T_ref;
    double Nint;     // internal degrees of freedom (5 - 3 gamma)/(gamma - 1)
    int mu_law, inviscid, nonlinear, scheme;
};

__host__ __device__ __forceinline__ long long cell_index(const GridDesc &g, int i, int j, int k) {
    return ((long long)k * g.ny + j) * g.nx + i;
}

__device__ __forceinline__ int wrap(int i, int n) {
    return i < 0 ? i + n : (i >= n ? i - n : i);
}

// dynamic viscosity: constant, or the Sutherland law of Sec. 4.2 with the
// temperature T = p/rho normalised by T_ref
__device__ __forceinline__ double viscosity(const PhysParams &P, double rho, double p) {
    if (P.mu_law == 0) return P.mu0;
    const double th = (p / rho) / P.T_ref;
    return P.mu0 * 1.4042 * th * sqrt(th) / (th + 0.4042);
}

__device__ __forceinline__ void flag_status(int *status, int bits) {
    if (status) atomicOr(status, bits);
}

// Kernel launch helpers (defined in the .cu files)
int launch_recon5(const GridDesc &g, const PhysParams &P, const double *Q, const double *G,
                  double *fs, cudaStream_t s);
int launch_recon2(const GridDesc &g, const PhysParams &P, const double *Q, double *fs,
                  cudaStream_t s);
int upload_recon_tables(void);
int launch_flux_faces(const GridDesc &g, const PhysParams &P, const double *fs,
                      const double *dt_dev, double *frec, int *status, cudaStream_t s);
int launch_flux_faces_mixed(const GridDesc &g, const PhysParams &P, const float *fs,
                            const double *Q, const double *dt_dev, double *frec, int *status,
                            cudaStream_t s);
int launch_recon5_mixed(const GridDesc &g, const PhysParams &P, const double *Q, const double *G,
                        float *fs, cudaStream_t s);
int launch_recon2_mixed(const GridDesc &g, const PhysParams &P, const double *Q, float *fs,
                        cudaStream_t s);
int launch_flux_points(const PhysParams &P, const double *sl, const double *sr, int n,
                       const double *dt_dev, double *out, int *status, cudaStream_t s);
int launch_dt(const GridDesc &g, const PhysParams &P, const double *Q, double *red,
              double *dt_dev, double *t_dev, double t_stop, cudaStream_t s);
// stage: 0 GKS-2nd single stage, 1 CGKS first stage, 2 CGKS second stage
int launch_update(const GridDesc &g, const PhysParams &P, int stage, const double *frec,
                  const double *dt_dev, double *Q, double *G, double *Qs, double *Gs,
                  double *Acc, double *S1, int *status, cudaStream_t s);
int launch_diagnostics(const GridDesc &g, const PhysParams &P, const double *Q,
                       const double *G, double *partials, int nblocks, double *out_dev,
                       cudaStream_t s);
int diagnostics_blocks(const GridDesc &g);

}  // namespace gks
