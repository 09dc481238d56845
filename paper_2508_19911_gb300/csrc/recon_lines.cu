// CGKS-5th with reading B of the target cell's data (the paper's S^0 of
// S^data-5th, Sec. 3.1-3.2): the state carries, per conserved variable,
// the 12 line-averaged derivatives L[4a + k] (along axis a, between the
// face Gauss points k of the cell's two faces normal to a) instead of the
// averaged gradient. FP64, periodic grids (uniform or stretched).
//
//   reconstruction: the 72-entry data vector (the neighbours' averages, the
//     face neighbours' averaged gradients and the edge neighbours'
//     tangential derivatives from their lines' means, the own 12 lines),
//     a = R d with the 34 x 72 matrix of the constrained least squares in
//     the reflection-symmetrised data basis, GENO (Eq. weno-new; the
//     sub-stencil slopes' tangential parts from the own lines' means, chi
//     from the misfit of the 54 weighted derivative rows), the quartic and
//     its derivatives at the 24 face Gauss points from its parity-class
//     sums;
//   flux: the Gauss-point flux of flux_device.cuh; F^n and F_t^n averaged
//     over the face's 4 points, the interface values kept per point;
//   update: Q as with gradients; each line from the interface values at
//     its two face Gauss points (the two-stage update point by point).
#include <mutex>

#include "recon_common.cuh"
#include "flux_device.cuh"

namespace gks {
namespace {

constexpr int kRecL = 90;  // record values per face: F^n, F_t^n, then 4 x 20 interface values

__constant__ double cRsL[kNumDataL][kMaxClass];  // R in the symmetrised data basis
__constant__ double cBsL[kNumDataL][kMaxClass];  // weighted derivative rows, same basis
__constant__ double cMeanL[kNumBasis];
__constant__ double cMvalL[3][kNumBasis];
__constant__ double cMderL[3][3][kNumBasis];

// values and derivatives at the 8 Gauss points of the two faces normal to
// axis D from the quartic's parity-class sums (a monomial's value at the
// point is its magnitude times the sign pattern of its class; the
// Walsh-Hadamard transform turns the 8 class sums into the 8 points).
// GENO's blend is folded in by the caller: a scaled by chi, base =
// q0 - chi K, and P1's slopes w = (1 - chi) bbar added to the classes of
// one odd axis (value: w_j |x_j|, |x_D| = 1/2, |x_T| = g) and to class 0
// of the derivatives.
template <int D>
__device__ __forceinline__ void eval_faces_lines(double *__restrict__ fs, long long n, long long c,
                                                 int v, const double a[kNumBasis], double base,
                                                 const double w[3], bool blend, const double ih[3]) {
    constexpr int T1 = (D + 1) % 3, T2 = (D + 2) % 3;
    double S[8], Dq[3][8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        S[k] = 0.0;
        Dq[0][k] = Dq[1][k] = Dq[2][k] = 0.0;
    }
    static_for<kNumBasis>([&](auto I) {
        constexpr int i = decltype(I)::value;
        S[basis_class(i)] = fma(a[i], cMvalL[D][i], S[basis_class(i)]);
        static_for<3>([&](auto Qc) {
            constexpr int q = decltype(Qc)::value;
            if constexpr (has_deriv(i, q))
                Dq[q][deriv_class(i, q)] = fma(a[i], cMderL[D][q][i], Dq[q][deriv_class(i, q)]);
        });
    });
    if (blend) {
        S[1 << D] = fma(0.5, w[D], S[1 << D]);
        S[1 << T1] = fma(kG, w[T1], S[1 << T1]);
        S[1 << T2] = fma(kG, w[T2], S[1 << T2]);
#pragma unroll
        for (int q = 0; q < 3; ++q) Dq[q][0] += w[q];
    }
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
        for (int k = 0; k < 8; ++k) Dq[q][k] *= ih[q];
    class_to_points(S);
    class_to_points(Dq[0]);
    class_to_points(Dq[1]);
    class_to_points(Dq[2]);
    const int cmp = frame_comp(v, D);
#pragma unroll
    for (int side = 0; side < 2; ++side)
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            const int p = (side << D) | ((kk & 1) << T1) | (((kk >> 1) & 1) << T2);
            double *o = fs + ((long long)((2 * D + side) * 4 + kk) * 20) * n + c;
            o[(long long)cmp * n] = base + S[p];
#pragma unroll
            for (int q = 0; q < 3; ++q) o[(long long)(5 + 5 * ((q - D + 3) % 3) + cmp) * n] = Dq[q][p];
        }
}

// averaged gradient along axis a of variable v in cell nb: the mean of its
// four lines
__device__ __forceinline__ double line_mean(const double *__restrict__ Lv, long long n, int a,
                                            long long nb) {
    return 0.25 * (__ldg(Lv + (long long)(4 * a) * n + nb) + __ldg(Lv + (long long)(4 * a + 1) * n + nb) +
                   __ldg(Lv + (long long)(4 * a + 2) * n + nb) + __ldg(Lv + (long long)(4 * a + 3) * n + nb));
}

// Value of line-form data column K for one (cell, variable): the
// neighbours' averages minus q0, their gradients as their lines' means
// (times h), the own lines (times h)
// hm[a][o + 1]: the cell size along axis a of the cells at offset o = -1,
// 0, 1 (a stretched mesh takes each neighbour's gradient in its own index
// coordinates, as the reference-cell mapping of the averaged-gradient form)
template <int K>
__device__ __forceinline__ double data_col_l(const double *__restrict__ Qv,
                                             const double *__restrict__ Lv, long long n, long long c,
                                             const long long nbF[6], const long long nbE[12],
                                             double q0, const double hm[3][3]) {
    if constexpr (K < kColEdge) {
        return __ldg(Qv + nbF[K]) - q0;
    } else if constexpr (K < kColFaceGrad) {
        return __ldg(Qv + nbE[K - kColEdge]) - q0;
    } else if constexpr (K < kColEdgeGrad) {
        constexpr int m = (K - kColFaceGrad) / 3, j = (K - kColFaceGrad) % 3;
        return hm[j][face_off(m, j) + 1] * line_mean(Lv, n, j, nbF[m]);
    } else if constexpr (K < kColLines) {
        constexpr int e = (K - kColEdgeGrad) / 2;
        constexpr int ea = edge_axis_a(e), eb = edge_axis_b(e), ee = edge_axis_e(e);
        if constexpr ((K - kColEdgeGrad) % 2 == 0) {
            constexpr double oa = edge_off(e, ea), ob = edge_off(e, eb);
            const double da = hm[ea][edge_off(e, ea) + 1] * line_mean(Lv, n, ea, nbE[e]);
            const double db = hm[eb][edge_off(e, eb) + 1] * line_mean(Lv, n, eb, nbE[e]);
            return (oa * da - ob * db) * kRs2;
        } else {
            return hm[ee][1] * line_mean(Lv, n, ee, nbE[e]);
        }
    } else {
        constexpr int a = (K - kColLines) / 4;
        return hm[a][1] * __ldg(Lv + (long long)(K - kColLines) * n + c);
    }
}

// One (cell, variable) per thread (blockIdx.y = variable), periodic grid
// (uniform or stretched). a = R d orbit by orbit in the symmetrised data basis
// (kSymL: 330 products instead of 34 x 72), GENO's misfit the same way.
__global__ void __launch_bounds__(128) recon5_lines_kernel(GridDesc g, int nonlinear,
                                                           const double *__restrict__ Q,
                                                           const double *__restrict__ L,
                                                           double *__restrict__ fs) {
    const long long n = g.n;
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const int v = (int)blockIdx.y;
    const int i = (int)(c % g.nx);
    const int j = (int)((c / g.nx) % g.ny);
    const int k = (int)(c / ((long long)g.nx * g.ny));
    const int c0[3] = {i, j, k};
    long long nbF[6], nbE[12];
#pragma unroll
    for (int m = 0; m < 6; ++m)
        nbF[m] = cell_index(g, wrap(i + face_off(m, 0), g.nx), wrap(j + face_off(m, 1), g.ny),
                            wrap(k + face_off(m, 2), g.nz));
#pragma unroll
    for (int e = 0; e < 12; ++e)
        nbE[e] = cell_index(g, wrap(i + edge_off(e, 0), g.nx), wrap(j + edge_off(e, 1), g.ny),
                            wrap(k + edge_off(e, 2), g.nz));
    double hm[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int o = 0; o < 3; ++o) hm[a][o] = cell_h(g, a, wrap(c0[a] + o - 1, axis_len(g, a)));
    const double ih[3] = {1.0 / hm[0][1], 1.0 / hm[1][1], 1.0 / hm[2][1]};
    const double *Qv = Q + (long long)v * n;
    const double *Lv = L + (long long)v * 12 * n;
    const double q0 = __ldg(Qv + c);

    double a[kNumBasis];
#pragma unroll
    for (int ii = 0; ii < kNumBasis; ++ii) a[ii] = 0.0;
    double dface[6], g0[3] = {0.0, 0.0, 0.0};
    double norm2 = 0.0;  // |d_C|^2 + |W d_B|^2 for GENO's misfit
    double ov[8];
    static_for<kNumDataL>([&](auto Rr) {
        constexpr int r = decltype(Rr)::value;
        constexpr int nm = kSymL.nm[r];
        if constexpr (kSymL.orbit[r] == r) {
            static_for<nm>([&](auto Qq) {
                constexpr int q = decltype(Qq)::value;
                constexpr int col = kSymL.mem[r][q];
                ov[q] = data_col_l<col>(Qv, Lv, n, c, nbF, nbE, q0, hm);
                constexpr double wc = col_weight(col);
                norm2 = fma(wc * wc * ov[q], ov[q], norm2);
                if constexpr (col < kColEdge) dface[col] = ov[q];
                if constexpr (col >= kColLines) g0[(col - kColLines) / 4] += 0.25 * ov[q];
            });
        }
        double ds = kSymL.sgn[r][0] > 0 ? ov[0] : -ov[0];
        static_for<nm - 1>([&](auto Qq) {
            constexpr int q = decltype(Qq)::value + 1;
            if constexpr (kSymL.sgn[r][q] > 0) ds += ov[q];
            else ds -= ov[q];
        });
        constexpr int cls = kSymL.cls[r];
        static_for<kClass.n[cls]>([&](auto J) {
            constexpr int jj = decltype(J)::value;
            constexpr int ib = kClass.member[cls][jj];
            a[ib] = fma(cRsL[r][jj], ds, a[ib]);
        });
    });
    double K = 0.0;
    static_for<kNumBasis>([&](auto I) {
        constexpr int ii = decltype(I)::value;
        if constexpr (basis_class(ii) == 0) K = fma(a[ii], cMeanL[ii], K);
    });

    double chi = 1.0, bbar[3] = {0.0, 0.0, 0.0};
    if (nonlinear) {
        const double eps = 1e-15;
        double w[6], wsum = 0.0;
#pragma unroll
        for (int m = 0; m < 6; ++m) {
            const int ax = m / 2;
            const double bn = (m & 1) ? dface[m] : -dface[m];
            double s = bn * bn;
#pragma unroll
            for (int q = 0; q < 3; ++q)
                if (q != ax) s = fma(g0[q], g0[q], s);
            const double t = s + eps, t2 = t * t;
            w[m] = (1.0 / 6.0) / (t2 * t2 * t);
            wsum += w[m];
        }
#pragma unroll
        for (int m = 0; m < 6; ++m) w[m] /= wsum;
#pragma unroll
        for (int q = 0; q < 3; ++q)
            bbar[q] = (1.0 - w[2 * q] - w[2 * q + 1]) * g0[q] - w[2 * q] * dface[2 * q] +
                      w[2 * q + 1] * dface[2 * q + 1];
        // GENO's misfit (reading R5): |W (B a - d_B)|^2 over the 54 weighted
        // derivative rows, orbit by orbit (sum of res_r^2 / nm), the
        // derivative columns loaded again
        double res2 = 0.0;
        static_for<kNumDataL>([&](auto Rr) {
            constexpr int r = decltype(Rr)::value;
            constexpr int nm = kSymL.nm[r];
            if constexpr (kSymL.mem[r][0] >= kColFaceGrad) {
                if constexpr (kSymL.orbit[r] == r) {
                    static_for<nm>([&](auto Qq) {
                        constexpr int q = decltype(Qq)::value;
                        constexpr int col = kSymL.mem[r][q];
                        ov[q] = data_col_l<col>(Qv, Lv, n, c, nbF, nbE, q0, hm);
                    });
                }
                double ds = kSymL.sgn[r][0] > 0 ? ov[0] : -ov[0];
                static_for<nm - 1>([&](auto Qq) {
                    constexpr int q = decltype(Qq)::value + 1;
                    if constexpr (kSymL.sgn[r][q] > 0) ds += ov[q];
                    else ds -= ov[q];
                });
                constexpr int cls = kSymL.cls[r];
                constexpr double wr = col_weight(kSymL.mem[r][0]);
                double res = -wr * ds;
                static_for<kClass.n[cls]>([&](auto J) {
                    constexpr int jj = decltype(J)::value;
                    constexpr int ib = kClass.member[cls][jj];
                    res = fma(cBsL[r][jj], a[ib], res);
                });
                res2 = fma(res * (1.0 / nm), res, res2);
            }
        });
        const double r0 = __ldg(Q + c), e0 = __ldg(Q + 4 * n + c);
        const double S = v == 0 ? r0 : (v == 4 ? e0 : sqrt(fabs(r0 * e0)));
        const double sig = res2 / (norm2 + kGenoKappa * kGenoKappa * S * S + eps);
        const double s = sig * (1.0 / kGenoSigma0);
        chi = 1.0 / (1.0 + s + s * s);
    }
    double w[3] = {0.0, 0.0, 0.0}, base = q0 - K;
    if (nonlinear) {
#pragma unroll
        for (int ii = 0; ii < kNumBasis; ++ii) a[ii] *= chi;
        base = fma(-chi, K, q0);
#pragma unroll
        for (int q = 0; q < 3; ++q) w[q] = (1.0 - chi) * bbar[q];
    }
    eval_faces_lines<0>(fs, n, c, v, a, base, w, nonlinear, ih);
    eval_faces_lines<1>(fs, n, c, v, a, base, w, nonlinear, ih);
    eval_faces_lines<2>(fs, n, c, v, a, base, w, nonlinear, ih);
}

// The Gauss-point flux of every face (periodic): four adjacent lanes hold
// the four points of a face; F^n and F_t^n are averaged by a butterfly,
// each lane keeps its point's interface values. Records per axis d and
// cell c (the face on c's low side): [0..9] F^n, F_t^n, [10 + 20 p + 5 b +
// component] Q^l, dQ^l/dt, Q^r, dQ^r/dt (b = 0..3) of point p, global frame.
__global__ void __launch_bounds__(128, 1) flux_faces_lines_kernel(GridDesc g, PhysParams P,
                                                                 const double *__restrict__ fs,
                                                                 const double *__restrict__ dt_dev,
                                                                 double *__restrict__ frec,
                                                                 int *status) {
    const double dt = *dt_dev;
    if (!(dt > 0.0)) return;  // same for every thread of the grid
    const long long n = g.n;
    const long long total = 12 * n;
    long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = gid < total;
    if (!valid) gid = total - 1;  // groups of four lanes are entirely in or out
    const int kq = (int)(gid & 3);
    const long long fc = gid >> 2;
    const int d = (int)(fc / n);
    const long long c = fc - (long long)d * n;
    const int i = (int)(c % g.nx);
    const int j = (int)((c / g.nx) % g.ny);
    const int k = (int)(c / ((long long)g.nx * g.ny));
    const long long left = cell_index(g, d == 0 ? wrap(i - 1, g.nx) : i, d == 1 ? wrap(j - 1, g.ny) : j,
                                      d == 2 ? wrap(k - 1, g.nz) : k);
    double sl[20], sr[20], out[30];
    const double *pl = fs + ((long long)((2 * d + 1) * 4 + kq) * 20) * n + left;
    const double *pr = fs + ((long long)((2 * d) * 4 + kq) * 20) * n + c;
#pragma unroll
    for (int q = 0; q < 20; ++q) {
        sl[q] = __ldg(pl + (long long)q * n);
        sr[q] = __ldg(pr + (long long)q * n);
    }
    flux_point<true>(P, sl, sr, dt, out, valid ? status : nullptr);
#pragma unroll
    for (int q = 0; q < 10; ++q) {
        double s = out[q] + __shfl_xor_sync(0xffffffffu, out[q], 1);
        s = s + __shfl_xor_sync(0xffffffffu, s, 2);
        out[q] = 0.25 * s;
    }
    if (!valid) return;
#pragma unroll
    for (int q = 0; q < 10; ++q) {
        if (q % 4 != kq) continue;
        const int blk = q / 5, cmp = q % 5;
        frec[((long long)d * kRecL + blk * 5 + global_var(cmp, d)) * n + c] = out[q];
    }
#pragma unroll
    for (int q = 10; q < 30; ++q) {
        const int blk = (q - 10) / 5, cmp = q % 5;
        frec[((long long)d * kRecL + 10 + 20 * kq + blk * 5 + global_var(cmp, d)) * n + c] = out[q];
    }
}

// one stage of the update with lines (see the file comment)
template <int STAGE>
__global__ void __launch_bounds__(256) update_lines_kernel(GridDesc g, PhysParams P,
                                                           const double *__restrict__ fr,
                                                           const double *__restrict__ dt_dev,
                                                           double *__restrict__ Q, double *__restrict__ L,
                                                           double *__restrict__ Qs, double *__restrict__ Ls,
                                                           double *__restrict__ Acc, double *__restrict__ S1,
                                                           int *status) {
    const double dt = *dt_dev;
    if (!(dt > 0.0)) return;
    const long long n = g.n;
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const int i = (int)(c % g.nx);
    const int j = (int)((c / g.nx) % g.ny);
    const int k = (int)(c / ((long long)g.nx * g.ny));
    const long long hi[3] = {cell_index(g, wrap(i + 1, g.nx), j, k),
                             cell_index(g, i, wrap(j + 1, g.ny), k),
                             cell_index(g, i, j, wrap(k + 1, g.nz))};
    const double ih[3] = {1.0 / cell_h(g, 0, i), 1.0 / cell_h(g, 1, j), 1.0 / cell_h(g, 2, k)};
    const double dt2 = dt * dt;
    double out[5];
#pragma unroll 1
    for (int v = 0; v < 5; ++v) {
        double Lq = 0.0, Lt = 0.0;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double *F = fr + (long long)d * kRecL * n;
            Lq += (F[(long long)v * n + hi[d]] - F[(long long)v * n + c]) * ih[d];
            Lt += (F[(long long)(5 + v) * n + hi[d]] - F[(long long)(5 + v) * n + c]) * ih[d];
        }
        Lq = -Lq;
        Lt = -Lt;
        const long long qi = (long long)v * n + c;
        if (STAGE == 1) {
            const double q = Q[qi];
            out[v] = q + 0.5 * dt * Lq + 0.125 * dt2 * Lt;
            Qs[qi] = out[v];
            Acc[qi] = q + dt * Lq + dt2 * (1.0 / 6.0) * Lt;
        } else {
            out[v] = Acc[qi] + dt2 * (1.0 / 3.0) * Lt;
            Q[qi] = out[v];
        }
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double *F = fr + (long long)d * kRecL * n;
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                const double *Fp = F + (long long)(10 + 20 * p) * n;
                const long long li = ((long long)v * 12 + 4 * d + p) * n + c;
                const double qlt = Fp[(long long)(5 + v) * n + hi[d]];
                const double qrt = Fp[(long long)(15 + v) * n + c];
                if (STAGE == 1) {
                    const double ql = Fp[(long long)v * n + hi[d]];
                    const double qr = Fp[(long long)(10 + v) * n + c];
                    Ls[li] = ((ql + 0.5 * dt * qlt) - (qr + 0.5 * dt * qrt)) * ih[d];
                    S1[li] = (ql - qr) * ih[d];
                } else {
                    L[li] = S1[li] + dt * (qlt - qrt) * ih[d];
                }
            }
        }
    }
    const double rho = out[0];
    const double ke = 0.5 * (out[1] * out[1] + out[2] * out[2] + out[3] * out[3]) / rho;
    const double p = (P.gamma - 1.0) * (out[4] - ke);
    bool finite = true;
#pragma unroll
    for (int v = 0; v < 5; ++v) finite = finite && isfinite(out[v]);
    if (!finite) flag_status(status, kStatusNonfinite);
    else if (!(rho > 0.0 && p > 0.0)) flag_status(status, kStatusNonphysical);
}

// the averaged gradients [5][3][cells] of a lines state (for the diagnostics)
__global__ void lines_to_grad_kernel(long long n, const double *__restrict__ L,
                                     double *__restrict__ G) {
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < 15 * n;
         t += (long long)gridDim.x * blockDim.x) {
        const long long c = t % n, va = t / n;  // va = 3 v + a
        const int v = (int)(va / 3), a = (int)(va % 3);
        const double *Lv = L + (long long)v * 12 * n;
        G[t] = 0.25 * (Lv[(long long)(4 * a) * n + c] + Lv[(long long)(4 * a + 1) * n + c] +
                       Lv[(long long)(4 * a + 2) * n + c] + Lv[(long long)(4 * a + 3) * n + c]);
    }
}

}  // namespace

int upload_recon_tables_lines(void) {
    static std::mutex mu;  // contexts may be used from several threads
    std::lock_guard<std::mutex> lock(mu);
    static ReconTablesLines t;
    static int built = 0;
    if (!built) {
        if (build_recon_tables_lines(&t)) return -1;
        built = 1;
    }
    if (cudaMemcpyToSymbol(cRsL, t.Rs, sizeof(t.Rs)) != cudaSuccess) return -2;
    if (cudaMemcpyToSymbol(cBsL, t.Bs, sizeof(t.Bs)) != cudaSuccess) return -2;
    if (cudaMemcpyToSymbol(cMeanL, t.mean, sizeof(t.mean)) != cudaSuccess) return -2;
    if (cudaMemcpyToSymbol(cMvalL, t.mval, sizeof(t.mval)) != cudaSuccess) return -2;
    if (cudaMemcpyToSymbol(cMderL, t.mder, sizeof(t.mder)) != cudaSuccess) return -2;
    return 0;
}

int launch_recon5_lines(const GridDesc &g, const PhysParams &P, const double *Q, const double *L,
                        double *fs, cudaStream_t s) {
    const long long blocks = (g.n + 127) / 128;
    recon5_lines_kernel<<<dim3((unsigned)blocks, 5), 128, 0, s>>>(g, P.nonlinear, Q, L, fs);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int launch_flux_faces_lines(const GridDesc &g, const PhysParams &P, const double *fs,
                            const double *dt_dev, double *frec, int *status, cudaStream_t s) {
    const long long blocks = (12 * g.n + 127) / 128;
    flux_faces_lines_kernel<<<(unsigned)blocks, 128, 0, s>>>(g, P, fs, dt_dev, frec, status);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int launch_update_lines(const GridDesc &g, const PhysParams &P, int stage, const double *frec,
                        const double *dt_dev, double *Q, double *L, double *Qs, double *Ls,
                        double *Acc, double *S1, int *status, cudaStream_t s) {
    const long long blocks = (g.n + 255) / 256;
    if (stage == 1)
        update_lines_kernel<1><<<(unsigned)blocks, 256, 0, s>>>(g, P, frec, dt_dev, Q, L, Qs, Ls,
                                                                Acc, S1, status);
    else
        update_lines_kernel<2><<<(unsigned)blocks, 256, 0, s>>>(g, P, frec, dt_dev, Q, L, Qs, Ls,
                                                                Acc, S1, status);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int launch_lines_to_grad(long long n, const double *L, double *G, cudaStream_t s) {
    const long long blocks = (15 * n + 255) / 256;
    lines_to_grad_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(n, L, G);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

}  // namespace gks
