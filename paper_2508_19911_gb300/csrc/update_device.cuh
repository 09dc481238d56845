// Device code of the time step (Sec. 4) and of the cell update (Sec. 2
// Eq. semi, Sec. 3.1, Sec. 3.4): per-cell rates and the block reduction of
// dt, and update_cell. Included by update.cu (the kernels) and by the
// single-launch ensemble step. See update.cu.
#pragma once
#include <cmath>

#include "common.cuh"

namespace gks {
namespace {

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// max over the cell of (|U_d| + c)/h_d and the kinematic viscosity
__device__ __forceinline__ void cell_rates(const GridDesc &g, const PhysParams &P,
                                           const double *__restrict__ Q, long long c,
                                           double &rate, double &numax) {
    const long long n = g.n;
    const double rho = Q[c];
    const double ir = 1.0 / rho;
    const double U = Q[n + c] * ir, V = Q[2 * n + c] * ir, W = Q[3 * n + c] * ir;
    const double p = (P.gamma - 1.0) * (Q[4 * n + c] - 0.5 * rho * (U * U + V * V + W * W));
    const double cs = sqrt(P.gamma * p * ir);
    double h[3] = {g.h[0], g.h[1], g.h[2]};
    if (g.general) {
        const long long nxy = (long long)g.nx * g.ny;
        h[0] = cell_h(g, 0, (int)(c % g.nx));
        h[1] = cell_h(g, 1, (int)((c % nxy) / g.nx));
        h[2] = cell_h(g, 2, (int)(c / nxy));
    }
    rate = fmax(rate, (fabs(U) + cs) / h[0]);
    rate = fmax(rate, (fabs(V) + cs) / h[1]);
    rate = fmax(rate, (fabs(W) + cs) / h[2]);
    numax = fmax(numax, viscosity(P, rho, p) * ir);
}

// block-wide max of (rate, numax) over NT threads, combined into red[0],
// red[1] by atomicMax on the bit patterns (all values non-negative)
template <int NT>
__device__ __forceinline__ void block_max_to(double rate, double numax, unsigned long long *red) {
    rate = warp_max(rate);
    numax = warp_max(numax);
    __shared__ double sr[NT / 32], sn[NT / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { sr[wid] = rate; sn[wid] = numax; }
    __syncthreads();
    if (wid == 0) {
        rate = lane < NT / 32 ? sr[lane] : 0.0;
        numax = lane < NT / 32 ? sn[lane] : 0.0;
        rate = warp_max(rate);
        numax = warp_max(numax);
        if (lane == 0) {
            atomicMax(red, (unsigned long long)__double_as_longlong(rate));
            atomicMax(red + 1, (unsigned long long)__double_as_longlong(numax));
        }
    }
    __syncthreads();
}

__device__ __forceinline__ double dt_from_rates(const GridDesc &g, const PhysParams &P,
                                                double rate, double numax) {
    double dt = P.cfl / rate;
    if (!P.inviscid && numax > 0.0) {
        const double hmin = g.general ? g.hmin : fmin(g.h[0], fmin(g.h[1], g.h[2]));
        dt = fmin(dt, P.cfl * hmin * hmin / (3.0 * numax));
    }
    return dt;
}

template <int STAGE>
__device__ __forceinline__ void update_cell(const GridDesc &g, const PhysParams &P,
                                            const double *__restrict__ fr, double dt,
                                            double *__restrict__ Q, double *__restrict__ G,
                                            double *__restrict__ Qs, double *__restrict__ Gs,
                                            double *__restrict__ Acc, double *__restrict__ S1,
                                            int *status, long long c) {
    const long long n = g.n;
    const int i = (int)(c % g.nx);
    const int j = (int)((c / g.nx) % g.ny);
    const int k = (int)(c / ((long long)g.nx * g.ny));
    long long hi[3] = {cell_index(g, wrap(i + 1, g.nx), j, k),
                       cell_index(g, i, wrap(j + 1, g.ny), k),
                       cell_index(g, i, j, wrap(k + 1, g.nz))};
    // records of the faces on the high side: strides n (the next cell's low
    // face) or np (a high boundary face of a non-periodic axis)
    const double *Fh[3] = {fr, fr + 30 * n, fr + 60 * n};
    long long hs[3] = {n, n, n};
    const double dt2 = dt * dt;
    // 1/h once per thread (FP64 division is a multi-instruction sequence)
    double ih[3] = {1.0 / g.h[0], 1.0 / g.h[1], 1.0 / g.h[2]};
    if (g.general) {
        const int cc[3] = {i, j, k};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            ih[d] = 1.0 / cell_h(g, d, cc[d]);
            if (g.bc[d] && cc[d] == axis_len(g, d) - 1) {
                Fh[d] = fr + 90 * n + (long long)d * 30 * g.np;
                hs[d] = g.np;
                hi[d] = plane_pos(g, d, i, j, k);
            }
        }
    }
    constexpr double kSixth = 1.0 / 6.0, kThird = 1.0 / 3.0;
    double out[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
        double L = 0.0, Lt = 0.0;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double *F = fr + (long long)d * 30 * n;
            L += (Fh[d][(long long)v * hs[d] + hi[d]] - F[(long long)v * n + c]) * ih[d];
            Lt += (Fh[d][(long long)(5 + v) * hs[d] + hi[d]] - F[(long long)(5 + v) * n + c]) * ih[d];
        }
        L = -L;
        Lt = -Lt;
        const long long qi = (long long)v * n + c;
        if (STAGE == 0) {
            out[v] = Q[qi] + dt * L + 0.5 * dt2 * Lt;
            Q[qi] = out[v];
        } else if (STAGE == 1) {
            const double q = Q[qi];
            out[v] = q + 0.5 * dt * L + 0.125 * dt2 * Lt;
            Qs[qi] = out[v];
            Acc[qi] = q + dt * L + dt2 * kSixth * Lt;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const double *F = fr + (long long)d * 30 * n;
                const double ql = Fh[d][(long long)(10 + v) * hs[d] + hi[d]];
                const double qlt = Fh[d][(long long)(15 + v) * hs[d] + hi[d]];
                const double qr = F[(long long)(20 + v) * n + c];
                const double qrt = F[(long long)(25 + v) * n + c];
                const long long gi = ((long long)v * 3 + d) * n + c;
                Gs[gi] = ((ql + 0.5 * dt * qlt) - (qr + 0.5 * dt * qrt)) * ih[d];
                S1[gi] = (ql - qr) * ih[d];
            }
        } else {
            out[v] = Acc[qi] + dt2 * kThird * Lt;
            Q[qi] = out[v];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const double *F = fr + (long long)d * 30 * n;
                const double qlt = Fh[d][(long long)(15 + v) * hs[d] + hi[d]];
                const double qrt = F[(long long)(25 + v) * n + c];
                const long long gi = ((long long)v * 3 + d) * n + c;
                G[gi] = S1[gi] + dt * (qlt - qrt) * ih[d];
            }
        }
    }
    // status word: non-physical or non-finite new state
    const double rho = out[0];
    const double ke = 0.5 * (out[1] * out[1] + out[2] * out[2] + out[3] * out[3]) / rho;
    const double p = (P.gamma - 1.0) * (out[4] - ke);
    bool finite = true;
#pragma unroll
    for (int v = 0; v < 5; ++v) finite = finite && isfinite(out[v]);
    if (!finite) flag_status(status, kStatusNonfinite);
    else if (!(rho > 0.0 && p > 0.0)) flag_status(status, kStatusNonphysical);
}

}  // namespace
}  // namespace gks
