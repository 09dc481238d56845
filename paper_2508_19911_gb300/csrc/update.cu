// Time step, cell update and diagnostics kernels.
//
//   dt (Sec. 4): dt = CFL min(min_{cells,d} h_d/(|U_d| + c), h_min^2/(3 nu_max));
//     warp-shuffle and block reductions of max (|U_d| + c)/h_d and max nu,
//     combined across blocks with atomicMax on the bit patterns of the
//     (non-negative) doubles, then one thread forms dt, clamps it to the
//     remaining time and advances t on the device.
//   update (Sec. 2 Eq. semi, Sec. 3.1, Sec. 3.4): L = -sum_d (F_d(i+1/2) -
//     F_d(i-1/2))/h_d from the face-averaged fluxes, the same for dL/dt;
//     GKS-2nd: Q += dt L + dt^2/2 dL/dt. CGKS-5th: stage 1 writes
//     Q* = Q + dt/2 L + dt^2/8 dL/dt, grad Q* from the interface values
//     (Gauss's theorem, Sec. 3.1) advanced by dt/2, and keeps
//     A = Q + dt L + dt^2/6 dL/dt and S1 = Gauss sum of Q_G^n; stage 2 writes
//     Q^{n+1} = A + dt^2/3 dL*/dt and grad Q^{n+1} = S1 + dt Gauss sum of
//     dQ_G*/dt.
//   diagnostics (Sec. 4.1/4.2): per-block partial sums/minima/maxima
//     (warp shuffles, then across the block's warps), then one block
//     reduces the partials the same way; a fixed order throughout
//     (deterministic, no floating-point atomics).
#include <cmath>

#include "update_device.cuh"

namespace gks {
namespace {

constexpr int kBlock = 256;

__global__ void __launch_bounds__(kBlock) dt_reduce_kernel(GridDesc g, PhysParams P,
                                                           const double *__restrict__ Q,
                                                           unsigned long long *red) {
    const long long n = g.n;
    double rate = 0.0, numax = 0.0;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x) {
        cell_rates(g, P, Q, c, rate, numax);
    }
    block_max_to<kBlock>(rate, numax, red);
}

__global__ void dt_finalize_kernel(GridDesc g, PhysParams P, unsigned long long *red,
                                   double *dt_dev, double *t_dev, double t_stop) {
    const double rate = __longlong_as_double((long long)red[0]);
    const double numax = __longlong_as_double((long long)red[1]);
    double dt = dt_from_rates(g, P, rate, numax);
    if (t_dev) {
        const double rem = t_stop - *t_dev;
        if (dt > rem) dt = rem;
        if (!(dt > 0.0)) dt = 0.0;
        *t_dev += dt;
    }
    if (!(dt > 0.0) || !isfinite(dt)) dt = 0.0;
    *dt_dev = dt;
    red[0] = 0ull;
    red[1] = 0ull;
}

template <int STAGE>
__global__ void __launch_bounds__(kBlock) update_kernel(GridDesc g, PhysParams P,
                                                        const double *__restrict__ fr,
                                                        const double *__restrict__ dt_dev,
                                                        double *__restrict__ Q, double *__restrict__ G,
                                                        double *__restrict__ Qs, double *__restrict__ Gs,
                                                        double *__restrict__ Acc,
                                                        double *__restrict__ S1, int *status) {
    const double dt = *dt_dev;
    if (!(dt > 0.0)) return;
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < g.n) update_cell<STAGE>(g, P, fr, dt, Q, G, Qs, Gs, Acc, S1, status, c);
}

// ---- persistent ensemble kernels (instances of uneven size) -------------
__global__ void __launch_bounds__(kBlock) dt_reduce_ens_kernel(const EnsInst *__restrict__ inst,
                                                               const EnsItem *__restrict__ items,
                                                               int nitems, const double *__restrict__ Qa,
                                                               unsigned long long *red) {
    for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
        const EnsItem it = items[w];
        const EnsInst I = inst[it.inst];
        double rate = 0.0, numax = 0.0;
        for (long long c = it.c0 + threadIdx.x; c < it.c1; c += blockDim.x)
            cell_rates(I.g, I.P, Qa + 5 * I.off, c, rate, numax);
        block_max_to<kBlock>(rate, numax, red + 2 * it.inst);
    }
}

// one thread per instance: dt_i, clamped to t_stop - t_i, t_i advanced
__global__ void dt_finalize_ens_kernel(const EnsInst *__restrict__ inst, int ninst,
                                       unsigned long long *red, double *dt_arr, double *t_arr,
                                       double t_stop) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ninst) return;
    const EnsInst I = inst[i];
    double dt = dt_from_rates(I.g, I.P, __longlong_as_double((long long)red[2 * i]),
                              __longlong_as_double((long long)red[2 * i + 1]));
    const double rem = t_stop - t_arr[i];
    if (dt > rem) dt = rem;
    if (!(dt > 0.0) || !isfinite(dt)) dt = 0.0;
    t_arr[i] += dt;
    dt_arr[i] = dt;
    red[2 * i] = 0ull;
    red[2 * i + 1] = 0ull;
}

template <int STAGE>
__global__ void __launch_bounds__(kBlock) update_ens_kernel(const EnsInst *__restrict__ inst,
                                                            const EnsItem *__restrict__ items,
                                                            int nitems, const double *__restrict__ fra,
                                                            const double *__restrict__ dt_arr,
                                                            double *Qa, double *Ga, double *Qsa,
                                                            double *Gsa, double *Acca, double *S1a,
                                                            int *status) {
    for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
        const EnsItem it = items[w];
        const EnsInst I = inst[it.inst];
        const double dt = dt_arr[it.inst];
        if (!(dt > 0.0)) continue;
        const long long o = I.off;
        for (long long c = it.c0 + threadIdx.x; c < it.c1; c += blockDim.x)
            update_cell<STAGE>(I.g, I.P, fra + 90 * o, dt, Qa + 5 * o, Ga + 15 * o, Qsa + 5 * o,
                               Gsa + 15 * o, Acca + 5 * o, S1a + 15 * o, status, c);
    }
}

// ---- diagnostics ---------------------------------------------------------
// slots: 0 ek, 1 eps_S, 2 eps_D, 3 min rho, 4 min p, 5..9 sum Q, 10 bad,
// 11 max speed; 3, 4 are minima, 11 a maximum, the rest sums
constexpr int kDiag = kDiagSlots;

__device__ __forceinline__ double neg_val(const GridDesc &g, int v, int flip, double x) {
    return ghost_neg(g, v, flip) ? -x : x;
}

__device__ __forceinline__ double combine(int s, double a, double b) {
    if (s == 3 || s == 4) return fmin(a, b);
    if (s == 11) return fmax(a, b);
    return a + b;
}

__device__ __forceinline__ double identity_of(int s) {
    if (s == 3 || s == 4) return INFINITY;
    if (s == 11) return 0.0;
    return 0.0;
}

// block reduction of the 12 slots: each warp combines its 32 lanes with
// shuffles (a fixed butterfly: deterministic), warp leaders meet in shared
// memory, warp 0 combines the kBlock/32 warp results; thread 0 writes dst
__device__ void block_reduce_store(double acc[kDiag], double *dst) {
    constexpr int kWarps = kBlock / 32;
    __shared__ double sh[kDiag][kWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int s = 0; s < kDiag; ++s) {
        double v = acc[s];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = combine(s, v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0) sh[s][warp] = v;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int s = 0; s < kDiag; ++s) {
            double v = lane < kWarps ? sh[s][lane] : identity_of(s);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v = combine(s, v, __shfl_xor_sync(0xffffffffu, v, o));
            if (lane == 0) dst[s] = v;
        }
    }
}

__global__ void __launch_bounds__(kBlock) diag_partial_kernel(GridDesc g, PhysParams P,
                                                              const double *__restrict__ Q,
                                                              const double *__restrict__ G,
                                                              double *partials) {
    const long long n = g.n;
    const double vol_u = g.h[0] * g.h[1] * g.h[2];
    double acc[kDiag];
#pragma unroll
    for (int s = 0; s < kDiag; ++s) acc[s] = identity_of(s);
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(c % g.nx);
        const int j = (int)((c / g.nx) % g.ny);
        const int k = (int)(c / ((long long)g.nx * g.ny));
        const double vol = g.general ? cell_h(g, 0, i) * cell_h(g, 1, j) * cell_h(g, 2, k) : vol_u;
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
        double dQ[4][3];  // d(rho), d(rho U), d(rho V), d(rho W)
#pragma unroll
        for (int v = 0; v < 4; ++v)
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                if (G) {
                    dQ[v][d] = G[((long long)v * 3 + d) * n + c];
                } else if (g.general) {
                    // the two neighbours (mirror ghosts at a boundary), their
                    // centres h_c + (h_hi + h_lo)/2 apart
                    const int cc[3] = {i, j, k};
                    int fh = 0, fl = 0, ch[3], cl[3];
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        ch[a] = a == d ? nb_coord(g, a, cc[a] + 1, fh) : cc[a];
                        cl[a] = a == d ? nb_coord(g, a, cc[a] - 1, fl) : cc[a];
                    }
                    const double qh = neg_val(g, v, fh, Q[(long long)v * n + cell_index(g, ch[0], ch[1], ch[2])]);
                    const double ql = neg_val(g, v, fl, Q[(long long)v * n + cell_index(g, cl[0], cl[1], cl[2])]);
                    const double dist = cell_h(g, d, cc[d]) +
                                        0.5 * (cell_h(g, d, ch[d]) + cell_h(g, d, cl[d]));
                    dQ[v][d] = (qh - ql) / dist;
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
        double du[3][3];  // du[a][d] = dU_a/dx_d
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
    block_reduce_store(acc, partials + (long long)blockIdx.x * kDiag);
}

__global__ void __launch_bounds__(kBlock) diag_final_kernel(const double *partials, int nblocks,
                                                            double volume, double *out) {
    double acc[kDiag];
#pragma unroll
    for (int s = 0; s < kDiag; ++s) acc[s] = identity_of(s);
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
        for (int s = 0; s < kDiag; ++s) acc[s] = combine(s, acc[s], partials[(long long)b * kDiag + s]);
    __shared__ double res[kDiag];
    block_reduce_store(acc, res);
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int s = 0; s < kDiag; ++s) out[s] = res[s];
        out[0] /= volume;
        out[1] /= volume;
        out[2] /= volume;
    }
}

}  // namespace

int launch_dt(const GridDesc &g, const PhysParams &P, const double *Q, double *red,
              double *dt_dev, double *t_dev, double t_stop, cudaStream_t s) {
    long long blocks = (g.n + kBlock - 1) / kBlock;
    if (blocks > 152 * 8) blocks = 152 * 8;
    dt_reduce_kernel<<<(unsigned)blocks, kBlock, 0, s>>>(g, P, Q, (unsigned long long *)red);
    dt_finalize_kernel<<<1, 1, 0, s>>>(g, P, (unsigned long long *)red, dt_dev, t_dev, t_stop);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int launch_update(const GridDesc &g, const PhysParams &P, int stage, const double *frec,
                  const double *dt_dev, double *Q, double *G, double *Qs, double *Gs,
                  double *Acc, double *S1, int *status, cudaStream_t s) {
    const long long blocks = (g.n + kBlock - 1) / kBlock;
    if (stage == 0)
        update_kernel<0><<<(unsigned)blocks, kBlock, 0, s>>>(g, P, frec, dt_dev, Q, G, Qs, Gs, Acc, S1, status);
    else if (stage == 1)
        update_kernel<1><<<(unsigned)blocks, kBlock, 0, s>>>(g, P, frec, dt_dev, Q, G, Qs, Gs, Acc, S1, status);
    else
        update_kernel<2><<<(unsigned)blocks, kBlock, 0, s>>>(g, P, frec, dt_dev, Q, G, Qs, Gs, Acc, S1, status);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int launch_dt_ens(const EnsInst *inst, int ninst, const EnsItem *items, int nitems, int blocks,
                  const double *Qa, double *red, double *dt_arr, double *t_arr, double t_stop,
                  cudaStream_t s) {
    dt_reduce_ens_kernel<<<blocks, kBlock, 0, s>>>(inst, items, nitems, Qa,
                                                   (unsigned long long *)red);
    dt_finalize_ens_kernel<<<(ninst + 63) / 64, 64, 0, s>>>(inst, ninst, (unsigned long long *)red,
                                                            dt_arr, t_arr, t_stop);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int launch_update_ens(const EnsInst *inst, const EnsItem *items, int nitems, int blocks, int stage,
                      const double *fra, const double *dt_arr, double *Qa, double *Ga, double *Qsa,
                      double *Gsa, double *Acca, double *S1a, int *status, cudaStream_t s) {
    if (stage == 1)
        update_ens_kernel<1><<<blocks, kBlock, 0, s>>>(inst, items, nitems, fra, dt_arr, Qa, Ga, Qsa,
                                                       Gsa, Acca, S1a, status);
    else
        update_ens_kernel<2><<<blocks, kBlock, 0, s>>>(inst, items, nitems, fra, dt_arr, Qa, Ga, Qsa,
                                                       Gsa, Acca, S1a, status);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int diagnostics_blocks(const GridDesc &g) {
    long long blocks = (g.n + kBlock - 1) / kBlock;
    if (blocks > kDiagMaxBlocks) blocks = kDiagMaxBlocks;
    return (int)blocks;
}

int launch_diagnostics(const GridDesc &g, const PhysParams &P, const double *Q, const double *G,
                       double *partials, int nblocks, double *out_dev, cudaStream_t s) {
    diag_partial_kernel<<<nblocks, kBlock, 0, s>>>(g, P, Q, G, partials);
    const double volume = g.general ? g.volume : g.h[0] * g.h[1] * g.h[2] * (double)g.n;
    diag_final_kernel<<<1, kBlock, 0, s>>>(partials, nblocks, volume, out_dev);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

}  // namespace gks
