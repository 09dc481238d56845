// Device code of the FP64 CGKS-5th reconstruction (Sec. 3.2): the FP64
// tables (constant memory; every includer has its own copy and uploads it),
// the data vector, GENO and the evaluation at the face Gauss points
// (recon5_cell). Included by recon_fp64.cu (the reconstruction kernels)
// and by the single-launch ensemble step. See recon_fp64.cu.
#pragma once
#include "recon_common.cuh"

namespace gks {
namespace {


__constant__ double cR[kNumBasis][kNumData];
__constant__ double cRs[kNumData][kMaxClass];  // R in the symmetrised data basis
__constant__ double cBs[kNumData][kMaxClass];  // weighted derivative rows, same basis
__constant__ double cMean[kNumBasis];
__constant__ double cMval[3][kNumBasis];
__constant__ double cMder[3][3][kNumBasis];
// Value of data column K for one (cell, variable) (layout in basis.h); on a
// general grid (GEN) the neighbours' gradients are scaled by their own cell
// sizes and a mirror ghost's averages and derivatives carry their signs
template <int K, bool GEN>
__device__ __forceinline__ double data_col(const double *__restrict__ Qv,
                                           const double *__restrict__ Gv, long long n, long long c,
                                           const long long nbF[6], const long long nbE[12],
                                           double q0, const double h[3], const NbGeo &geo) {
    if constexpr (K < kColEdge) {
        const double x = __ldg(Qv + nbF[K]);
        if constexpr (GEN) return neg_if(x, (geo.fF[K] >> 3) & 1) - q0;
        else return x - q0;
    } else if constexpr (K < kColFaceGrad) {
        const double x = __ldg(Qv + nbE[K - kColEdge]);
        if constexpr (GEN) return neg_if(x, (geo.fE[K - kColEdge] >> 3) & 1) - q0;
        else return x - q0;
    } else if constexpr (K < kColEdgeGrad) {
        constexpr int m = (K - kColFaceGrad) / 3, j = (K - kColFaceGrad) % 3;
        if constexpr (GEN)
            return geo.hm[j][face_off(m, j) + 1] *
                   neg_if(__ldg(Gv + j * n + nbF[m]), der_neg(geo.fF[m], j));
        else return h[j] * __ldg(Gv + j * n + nbF[m]);
    } else if constexpr (K < kColCentreGrad) {
        constexpr int e = (K - kColEdgeGrad) / 2;
        constexpr int ea = edge_axis_a(e), eb = edge_axis_b(e), ee = edge_axis_e(e);
        if constexpr ((K - kColEdgeGrad) % 2 == 0) {
            constexpr double oa = edge_off(e, ea), ob = edge_off(e, eb);
            double da, db;
            if constexpr (GEN) {
                da = geo.hm[ea][edge_off(e, ea) + 1] *
                     neg_if(__ldg(Gv + ea * n + nbE[e]), der_neg(geo.fE[e], ea));
                db = geo.hm[eb][edge_off(e, eb) + 1] *
                     neg_if(__ldg(Gv + eb * n + nbE[e]), der_neg(geo.fE[e], eb));
            } else {
                da = h[ea] * __ldg(Gv + ea * n + nbE[e]);
                db = h[eb] * __ldg(Gv + eb * n + nbE[e]);
            }
            return (oa * da - ob * db) * kRs2;
        } else {
            if constexpr (GEN)
                return geo.hm[ee][1] * neg_if(__ldg(Gv + ee * n + nbE[e]), der_neg(geo.fE[e], ee));
            else return h[ee] * __ldg(Gv + ee * n + nbE[e]);
        }
    } else {
        constexpr int j = K - kColCentreGrad;
        return h[j] * __ldg(Gv + j * n + c);
    }
}

// P4 (and, blended, P1) at the 8 Gauss points of the two faces normal to
// axis D. GENO's blend chi P4 + (1 - chi) P1 is applied to the class sums
// before the transform: the caller scales a by chi (and base to
// q0 - chi K); P1's slopes w = (1 - chi) bbar each sit in the class of one
// odd axis (class sum w_j |x_j|, |x_D| = 1/2, |x_T| = g) and, for the
// derivatives, in class 0. The derivatives are scaled by 1/h before the
// transform too (it is linear).
template <int D>
__device__ __forceinline__ void eval_faces(double *__restrict__ fs, long long n, long long c,
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
        constexpr int cls = basis_class(i);
        S[cls] = fma(a[i], cMval[D][i], S[cls]);
        static_for<3>([&](auto Qc) {
            constexpr int q = decltype(Qc)::value;
            if constexpr (has_deriv(i, q)) {
                constexpr int dc = deriv_class(i, q);
                Dq[q][dc] = fma(a[i], cMder[D][q][i], Dq[q][dc]);
            }
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
            for (int q = 0; q < 3; ++q) {
                const int jf = (q - D + 3) % 3;
                o[(long long)(5 + 5 * jf + cmp) * n] = Dq[q][p];
            }
        }
}

// cell c (global), variable v; face states to buffer position l (stride nb)
template <bool GEN>
__device__ __forceinline__ void recon5_cell(const GridDesc &g, int nonlinear,
                                            const double *__restrict__ Q,
                                            const double *__restrict__ G,
                                            double *__restrict__ fs, long long c, int v,
                                            long long nb, long long l) {
    const long long n = g.n;
    const int i = (int)(c % g.nx);
    const int j = (int)((c / g.nx) % g.ny);
    const int k = (int)(c / ((long long)g.nx * g.ny));
    long long nbF[6], nbE[12];
    NbGeo geo;
    stencil<GEN>(g, i, j, k, v, nbF, nbE, geo);
    double h[3] = {g.h[0], g.h[1], g.h[2]};
    if constexpr (GEN) {
        h[0] = geo.hm[0][1];
        h[1] = geo.hm[1][1];
        h[2] = geo.hm[2][1];
    }
    const double ih[3] = {1.0 / h[0], 1.0 / h[1], 1.0 / h[2]};

    const double *Qv = Q + (long long)v * n;
    const double *Gv = G + (long long)v * 3 * n;
    const double q0 = __ldg(Qv + c);
    double a[kNumBasis];
#pragma unroll
    for (int ii = 0; ii < kNumBasis; ++ii) a[ii] = 0.0;
    double dface[6], dctr[3];
    double norm2 = 0.0;  // |d_C|^2 + |W d_B|^2 for GENO's misfit
    // a = R d orbit by orbit: load the orbit's columns, form its symmetrised
    // combinations, multiply each with its class block of R
    double ov[8];
    static_for<kNumData>([&](auto Rr) {
        constexpr int r = decltype(Rr)::value;
        constexpr int nm = kSym.nm[r];
        if constexpr (kSym.orbit[r] == r) {
            static_for<nm>([&](auto Qq) {
                constexpr int q = decltype(Qq)::value;
                constexpr int col = kSym.mem[r][q];
                ov[q] = data_col<col, GEN>(Qv, Gv, n, c, nbF, nbE, q0, h, geo);
                constexpr double wc = col_weight(col);
                norm2 = fma(wc * wc * ov[q], ov[q], norm2);
                if constexpr (col < kColEdge) dface[col] = ov[q];
                if constexpr (col >= kColCentreGrad) dctr[col - kColCentreGrad] = ov[q];
            });
        }
        double ds = kSym.sgn[r][0] > 0 ? ov[0] : -ov[0];
        static_for<nm - 1>([&](auto Qq) {
            constexpr int q = decltype(Qq)::value + 1;
            if constexpr (kSym.sgn[r][q] > 0) ds += ov[q];
            else ds -= ov[q];
        });
        constexpr int cls = kSym.cls[r];
        static_for<kClass.n[cls]>([&](auto J) {
            constexpr int jj = decltype(J)::value;
            constexpr int ib = kClass.member[cls][jj];
            a[ib] = fma(cRs[r][jj], ds, a[ib]);
        });
    });

    // P4(x) = Q0 - sum_i a_i mean_i + sum_i a_i x^{e_i}/e_i!
    double K = 0.0;
    static_for<kNumBasis>([&](auto I) {
        constexpr int ii = decltype(I)::value;
        if constexpr (basis_class(ii) == 0) K = fma(a[ii], cMean[ii], K);
    });
    const double base = q0 - K;

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
                if (q != ax) s = fma(dctr[q], dctr[q], s);
            const double t = s + eps, t2 = t * t;
            w[m] = (1.0 / 6.0) / (t2 * t2 * t);
            wsum += w[m];
        }
#pragma unroll
        for (int m = 0; m < 6; ++m) w[m] /= wsum;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            // sum_m w_m b^m_q: tangential slopes from the own gradient,
            // the normal one from the neighbour difference
            bbar[q] = (1.0 - w[2 * q] - w[2 * q + 1]) * dctr[q] - w[2 * q] * dface[2 * q] +
                      w[2 * q + 1] * dface[2 * q + 1];
        }
        // GENO's misfit: |W (B a - d_B)|^2 orbit by orbit in the symmetrised
        // basis (sum over an orbit's combinations of res_r^2 / nm), the
        // derivative columns loaded again (they were read moments ago)
        double res2 = 0.0;
        static_for<kNumData>([&](auto Rr) {
            constexpr int r = decltype(Rr)::value;
            constexpr int nm = kSym.nm[r];
            if constexpr (kSym.mem[r][0] >= kColFaceGrad) {
                if constexpr (kSym.orbit[r] == r) {
                    static_for<nm>([&](auto Qq) {
                        constexpr int q = decltype(Qq)::value;
                        constexpr int col = kSym.mem[r][q];
                        ov[q] = data_col<col, GEN>(Qv, Gv, n, c, nbF, nbE, q0, h, geo);
                    });
                }
                double ds = kSym.sgn[r][0] > 0 ? ov[0] : -ov[0];
                static_for<nm - 1>([&](auto Qq) {
                    constexpr int q = decltype(Qq)::value + 1;
                    if constexpr (kSym.sgn[r][q] > 0) ds += ov[q];
                    else ds -= ov[q];
                });
                constexpr int cls = kSym.cls[r];
                constexpr double wr = col_weight(kSym.mem[r][0]);
                double res = -wr * ds;
                static_for<kClass.n[cls]>([&](auto J) {
                    constexpr int jj = decltype(J)::value;
                    constexpr int ib = kClass.member[cls][jj];
                    res = fma(cBs[r][jj], a[ib], res);
                });
                res2 = fma(res * (1.0 / nm), res, res2);
            }
        });
        // the cell's own magnitude: rho, rho E, sqrt(rho rho E) for momenta
        const double r0 = __ldg(Q + c), e0 = __ldg(Q + 4 * n + c);
        const double S = v == 0 ? r0 : (v == 4 ? e0 : sqrt(fabs(r0 * e0)));
        const double sig = res2 / (norm2 + kGenoKappa * kGenoKappa * S * S + eps);
        const double s = sig * (1.0 / kGenoSigma0);
        chi = 1.0 / (1.0 + s + s * s);
    }
    double w[3] = {0.0, 0.0, 0.0};
    double bse = base;
    if (nonlinear) {
        // chi P4 + (1 - chi) P1 (Eq. weno-new), folded into the evaluation
#pragma unroll
        for (int ii = 0; ii < kNumBasis; ++ii) a[ii] *= chi;
        bse = fma(-chi, K, q0);
        const double omc = 1.0 - chi;
#pragma unroll
        for (int q = 0; q < 3; ++q) w[q] = omc * bbar[q];
    }
    eval_faces<0>(fs, nb, l, v, a, bse, w, nonlinear, ih);
    eval_faces<1>(fs, nb, l, v, a, bse, w, nonlinear, ih);
    eval_faces<2>(fs, nb, l, v, a, bse, w, nonlinear, ih);
}

}  // namespace
}  // namespace gks
