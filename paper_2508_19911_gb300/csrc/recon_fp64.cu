// FP64 reconstruction kernels (Sec. 3.2 CGKS-5th, Sec. 3.3 GKS-2nd), the
// FP64 ensemble reconstruction and the upload of the FP64 tables. Compiled
// with the default multiply-add contraction.
//
// CGKS-5th, one thread per (cell, conserved variable): the data vector
// orbit by orbit, a = R d by parity-class blocks, GENO, and the 24 face
// Gauss points by a Walsh-Hadamard transform of the class sums (see
// recon.cu). GKS-2nd, one thread per cell: central least-squares gradient,
// the Venkatakrishnan limiter phi0 = min over the six faces, midpoint states.
#include "recon_fp64_device.cuh"

namespace gks {
namespace {

template <bool GEN>
__global__ void __launch_bounds__(128) recon5_kernel(GridDesc g, Slab S, int nonlinear,
                                                     const double *__restrict__ Q,
                                                     const double *__restrict__ G,
                                                     double *__restrict__ fs) {
    const long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (l < S.nb)
        recon5_cell<GEN>(g, nonlinear, Q, G, fs, slab_global(g, S, l), (int)blockIdx.y, S.nb, l);
}

template <bool GEN>
__global__ void __launch_bounds__(128) recon2_kernel(GridDesc g, Slab S, int nonlinear,
                                                     double eps2, const double *__restrict__ Q,
                                                     double *__restrict__ fs) {
    const long long n = g.n;
    const long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= S.nb) return;
    const long long c = slab_global(g, S, l);
    const int i = (int)(c % g.nx);
    const int j = (int)((c / g.nx) % g.ny);
    const int k = (int)(c / ((long long)g.nx * g.ny));
    long long nb[6];
    int fl[6];
    double h[3] = {g.h[0], g.h[1], g.h[2]};
    if constexpr (!GEN) {
#pragma unroll
        for (int m = 0; m < 6; ++m)
            nb[m] = cell_index(g, wrap(i + face_off(m, 0), g.nx), wrap(j + face_off(m, 1), g.ny),
                               wrap(k + face_off(m, 2), g.nz));
    } else {
        // mirror ghosts across non-periodic axes; this cell's sizes and the
        // limiter's eps^2 = h^3 from its own volume (reading R9)
        const int c0[3] = {i, j, k};
#pragma unroll
        for (int m = 0; m < 6; ++m) {
            int cc[3];
            fl[m] = 0;
#pragma unroll
            for (int a = 0; a < 3; ++a) cc[a] = nb_coord(g, a, c0[a] + face_off(m, a), fl[m]);
            nb[m] = cell_index(g, cc[0], cc[1], cc[2]);
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) h[a] = cell_h(g, a, c0[a]);
        const double hv = cbrt(h[0] * h[1] * h[2]);
        eps2 = hv * hv * hv;
    }
#pragma unroll 1
    for (int v = 0; v < 5; ++v) {
        const double *Qv = Q + (long long)v * n;
        const double q0 = __ldg(Qv + c);
        double qn[6];
#pragma unroll
        for (int m = 0; m < 6; ++m) {
            qn[m] = __ldg(Qv + nb[m]);
            if constexpr (GEN) qn[m] = neg_if(qn[m], ghost_neg(g, v, fl[m]));
        }
        // least-squares gradient of the face-neighbour averages on a uniform
        // grid: the central difference (normalised units; on a stretched
        // mesh those of the reference cell)
        double b[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) b[d] = 0.5 * (qn[2 * d + 1] - qn[2 * d]);
        double phi = 1.0;
        if (nonlinear) {
            double qmax = q0, qmin = q0;
#pragma unroll
            for (int m = 0; m < 6; ++m) {
                qmax = fmax(qmax, qn[m]);
                qmin = fmin(qmin, qn[m]);
            }
#pragma unroll
            for (int f = 0; f < 6; ++f) {
                const double d2 = (f & 1) ? 0.5 * b[f / 2] : -0.5 * b[f / 2];
                if (d2 != 0.0) {
                    const double dp = d2 > 0.0 ? qmax - q0 : qmin - q0;
                    const double pf = (dp * dp + eps2 + 2.0 * d2 * dp) /
                                      (dp * dp + 2.0 * d2 * d2 + d2 * dp + eps2);
                    phi = fmin(phi, pf);
                }
            }
        }
#pragma unroll
        for (int f = 0; f < 6; ++f) {
            const int d = f / 2;
            const int cmp = frame_comp(v, d);
            double *o = fs + ((long long)f * 20) * S.nb + l;
            o[(long long)cmp * S.nb] = q0 + phi * ((f & 1) ? 0.5 : -0.5) * b[d];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const int jf = (q - d + 3) % 3;
                o[(long long)(5 + 5 * jf + cmp) * S.nb] = phi * b[q] / h[q];
            }
        }
    }
}

__global__ void __launch_bounds__(128) recon5_ens_fp64_kernel(const EnsInst *__restrict__ inst,
                                                              const EnsItem *__restrict__ items,
                                                              int nitems,
                                                              const double *__restrict__ Qa,
                                                              const double *__restrict__ Ga,
                                                              double *__restrict__ fsa) {
    for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
        const EnsItem it = items[w];
        const EnsInst I = inst[it.inst];
        const double *Q = Qa + 5 * I.off;
        const double *G = Ga + 15 * I.off;
        const long long T = it.c1 - it.c0;
        for (long long t = threadIdx.x; t < 5 * T; t += blockDim.x)
            recon5_cell<false>(I.g, I.P.nonlinear, Q, G, fsa + 480 * I.off, it.c0 + t % T, (int)(t / T),
                        I.g.n, it.c0 + t % T);
    }
}

}  // namespace

int upload_recon_tables_fp64(const ReconTables &t) {
    if (cudaMemcpyToSymbol(cR, t.R, sizeof(t.R)) != cudaSuccess) return -2;
    if (cudaMemcpyToSymbol(cRs, t.Rs, sizeof(t.Rs)) != cudaSuccess) return -2;
    if (cudaMemcpyToSymbol(cBs, t.Bs, sizeof(t.Bs)) != cudaSuccess) return -2;
    if (cudaMemcpyToSymbol(cMean, t.mean, sizeof(t.mean)) != cudaSuccess) return -2;
    if (cudaMemcpyToSymbol(cMval, t.mval, sizeof(t.mval)) != cudaSuccess) return -2;
    if (cudaMemcpyToSymbol(cMder, t.mder, sizeof(t.mder)) != cudaSuccess) return -2;
    return 0;
}

int launch_recon5_ens_fp64(const EnsInst *inst, const EnsItem *items, int nitems, int blocks,
                           const double *Qa, const double *Ga, double *fsa, cudaStream_t s) {
    recon5_ens_fp64_kernel<<<blocks, 128, 0, s>>>(inst, items, nitems, Qa, Ga, fsa);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int launch_recon5(const GridDesc &g, const Slab &S, const PhysParams &P, const double *Q,
                  const double *G, double *fs, cudaStream_t s) {
    const int block = 128;
    const long long grid = (S.nb + block - 1) / block;
    if (g.general)
        recon5_kernel<true><<<dim3((unsigned)grid, 5), block, 0, s>>>(g, S, P.nonlinear, Q, G, fs);
    else
        recon5_kernel<false><<<dim3((unsigned)grid, 5), block, 0, s>>>(g, S, P.nonlinear, Q, G, fs);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int launch_recon2(const GridDesc &g, const Slab &S, const PhysParams &P, const double *Q,
                  double *fs, cudaStream_t s) {
    const double hv = cbrt(g.h[0] * g.h[1] * g.h[2]);
    const double eps2 = hv * hv * hv;  // (K h)^3 with K = 1
    const int block = 128;
    const long long grid = (S.nb + block - 1) / block;
    if (g.general)
        recon2_kernel<true><<<(unsigned)grid, block, 0, s>>>(g, S, P.nonlinear, eps2, Q, fs);
    else
        recon2_kernel<false><<<(unsigned)grid, block, 0, s>>>(g, S, P.nonlinear, eps2, Q, fs);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

}  // namespace gks
