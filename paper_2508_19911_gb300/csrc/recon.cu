// Spatial reconstruction kernels (Sec. 3.2 CGKS-5th, Sec. 3.3 GKS-2nd).
//
// CGKS-5th, one thread per cell, per conserved variable:
//   1. gather the 63 entries of S^data-5th (neighbour averages minus Q0,
//      neighbour and own cell-averaged gradients scaled by h) and
//      accumulate a = R d column by column; R (34 x 63, the constrained
//      least squares of Eq. compact-big-5) sits in constant memory and
//      every index is a compile-time constant, so each FMA reads a uniform
//      constant-bank operand;
//   2. GENO (Eq. weno-new): the six sub-stencil slopes b^m (Eq.
//      compact-sub-2), IS_m = |b^m|^2, w_m = d_m/(IS_m + eps)^5 normalised,
//      IS_H = a^T H a (H block-diagonal by parity class),
//      chi = 1/(1 + (r/0.1)^3), r = |IS_H - IS_L|/(IS_H + IS_L + eps);
//   3. evaluate P4 and its gradient at the 24 face Gauss points: the
//      points of the faces normal to axis d are (+-1/2, +-g, +-g) up to a
//      permutation, so the 34 monomials are first summed into 8 parity
//      classes (one magnitude factor per monomial) and every point value
//      is a signed sum of the 8 class sums.
// GKS-2nd, one thread per cell: central least-squares gradient, the
// Venkatakrishnan limiter phi0 = min over the six faces, midpoint states.
#include <cmath>
#include <type_traits>
#include <utility>

#include "basis.h"
#include "common.cuh"

namespace gks {
namespace {

// Compile-time loop: f(std::integral_constant<int, I>) for I = 0..N-1, so
// that every table index below is a constant expression of the front end.
template <typename F, int... I>
__device__ __forceinline__ void static_for_impl(F &&f, std::integer_sequence<int, I...>) {
    (f(std::integral_constant<int, I>{}), ...);
}
template <int N, typename F>
__device__ __forceinline__ void static_for(F &&f) {
    static_for_impl(f, std::make_integer_sequence<int, N>{});
}

__constant__ double cR[kNumBasis][kNumData];
__constant__ double cH[kNumBasis][kNumBasis];
__constant__ double cMean[kNumBasis];
__constant__ double cMval[3][kNumBasis];
__constant__ double cMder[3][3][kNumBasis];
// FP32 copies for the mixed-precision kernels
__constant__ float cRf[kNumBasis][kNumData];
__constant__ float cHf[kNumBasis][kNumBasis];
__constant__ float cMeanf[kNumBasis];
__constant__ float cMvalf[3][kNumBasis];
__constant__ float cMderf[3][3][kNumBasis];

constexpr double kG = 0.28867513459481288225;     // 1/(2 sqrt 3)
constexpr double kRs2 = 0.70710678118654752440;   // 1/sqrt 2

template <int COL>
__device__ __forceinline__ void add_column(double a[kNumBasis], double x) {
#pragma unroll
    for (int i = 0; i < kNumBasis; ++i) a[i] = fma(cR[i][COL], x, a[i]);
}

// face-frame component of conserved variable v on a face normal to axis d
__device__ __forceinline__ int frame_comp(int v, int d) {
    return (v == 0 || v == 4) ? v : 1 + (v - 1 - d + 3) % 3;
}

template <int D, int SIDE, int KK>
__device__ __forceinline__ void write_point(double *__restrict__ fs, long long n, long long c,
                                            int v, const double S[8], const double Dq[3][8],
                                            double base, double chi, const double bbar[3],
                                            double q0, bool nonlinear, const double h[3]) {
    constexpr int T1 = (D + 1) % 3, T2 = (D + 2) % 3;
    constexpr double sD = SIDE ? 1.0 : -1.0;
    constexpr double s1 = (KK & 1) ? 1.0 : -1.0;
    constexpr double s2 = (KK & 2) ? 1.0 : -1.0;
    double sg[3];
    sg[D] = sD;
    sg[T1] = s1;
    sg[T2] = s2;
    double val = base, der[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int cls = 0; cls < 8; ++cls) {
        const double sign = ((cls & 1) ? sg[0] : 1.0) * ((cls & 2) ? sg[1] : 1.0) *
                            ((cls & 4) ? sg[2] : 1.0);
        val += sign * S[cls];
#pragma unroll
        for (int q = 0; q < 3; ++q) der[q] += sign * Dq[q][cls];
    }
    if (nonlinear) {
        double x[3];
        x[D] = 0.5 * sD;
        x[T1] = kG * s1;
        x[T2] = kG * s2;
        const double p1 = q0 + bbar[0] * x[0] + bbar[1] * x[1] + bbar[2] * x[2];
        val = chi * val + (1.0 - chi) * p1;
#pragma unroll
        for (int q = 0; q < 3; ++q) der[q] = chi * der[q] + (1.0 - chi) * bbar[q];
    }
    constexpr int f = 2 * D + SIDE;
    const int cmp = frame_comp(v, D);
    double *o = fs + ((long long)(f * 4 + KK) * 20) * n + c;
    o[(long long)cmp * n] = val;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const int jf = (q - D + 3) % 3;
        o[(long long)(5 + 5 * jf + cmp) * n] = der[q] / h[q];
    }
}

template <int D>
__device__ __forceinline__ void eval_faces(double *__restrict__ fs, long long n, long long c,
                                           int v, const double a[kNumBasis], double base,
                                           double chi, const double bbar[3], double q0,
                                           bool nonlinear, const double h[3]) {
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
    write_point<D, 0, 0>(fs, n, c, v, S, Dq, base, chi, bbar, q0, nonlinear, h);
    write_point<D, 0, 1>(fs, n, c, v, S, Dq, base, chi, bbar, q0, nonlinear, h);
    write_point<D, 0, 2>(fs, n, c, v, S, Dq, base, chi, bbar, q0, nonlinear, h);
    write_point<D, 0, 3>(fs, n, c, v, S, Dq, base, chi, bbar, q0, nonlinear, h);
    write_point<D, 1, 0>(fs, n, c, v, S, Dq, base, chi, bbar, q0, nonlinear, h);
    write_point<D, 1, 1>(fs, n, c, v, S, Dq, base, chi, bbar, q0, nonlinear, h);
    write_point<D, 1, 2>(fs, n, c, v, S, Dq, base, chi, bbar, q0, nonlinear, h);
    write_point<D, 1, 3>(fs, n, c, v, S, Dq, base, chi, bbar, q0, nonlinear, h);
}

__global__ void __launch_bounds__(128) recon5_kernel(GridDesc g, int nonlinear,
                                                     const double *__restrict__ Q,
                                                     const double *__restrict__ G,
                                                     double *__restrict__ fs) {
    const long long n = g.n;
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const int i = (int)(c % g.nx);
    const int j = (int)((c / g.nx) % g.ny);
    const int k = (int)(c / ((long long)g.nx * g.ny));
    long long nbF[6], nbE[12];
#pragma unroll
    for (int m = 0; m < 6; ++m)
        nbF[m] = cell_index(g, wrap(i + face_off(m, 0), g.nx), wrap(j + face_off(m, 1), g.ny),
                            wrap(k + face_off(m, 2), g.nz));
#pragma unroll
    for (int e = 0; e < 12; ++e)
        nbE[e] = cell_index(g, wrap(i + edge_off(e, 0), g.nx), wrap(j + edge_off(e, 1), g.ny),
                            wrap(k + edge_off(e, 2), g.nz));
    const double h[3] = {g.h[0], g.h[1], g.h[2]};

#pragma unroll 1
    for (int v = 0; v < 5; ++v) {
        const double *Qv = Q + (long long)v * n;
        const double *Gv = G + (long long)v * 3 * n;
        const double q0 = __ldg(Qv + c);
        double a[kNumBasis];
#pragma unroll
        for (int ii = 0; ii < kNumBasis; ++ii) a[ii] = 0.0;
        double dface[6], dctr[3];
        // face neighbours
#define FACE_COLS(M)                                                               \
        {                                                                          \
            const double dq = __ldg(Qv + nbF[M]) - q0;                             \
            dface[M] = dq;                                                         \
            add_column<kColFace + M>(a, dq);                                       \
            add_column<kColFaceGrad + 3 * M + 0>(a, h[0] * __ldg(Gv + nbF[M]));     \
            add_column<kColFaceGrad + 3 * M + 1>(a, h[1] * __ldg(Gv + n + nbF[M])); \
            add_column<kColFaceGrad + 3 * M + 2>(a, h[2] * __ldg(Gv + 2 * n + nbF[M])); \
        }
        FACE_COLS(0) FACE_COLS(1) FACE_COLS(2) FACE_COLS(3) FACE_COLS(4) FACE_COLS(5)
#undef FACE_COLS
        // edge neighbours: in-plane direction orthogonal to the offset, and
        // the edge direction
#define EDGE_COLS(E)                                                                   \
        {                                                                              \
            constexpr int ea = edge_axis_a(E), eb = edge_axis_b(E), ee = edge_axis_e(E); \
            constexpr double oa = edge_off(E, ea), ob = edge_off(E, eb);              \
            add_column<kColEdge + E>(a, __ldg(Qv + nbE[E]) - q0);                      \
            const double da = h[ea] * __ldg(Gv + ea * n + nbE[E]);                     \
            const double db = h[eb] * __ldg(Gv + eb * n + nbE[E]);                     \
            add_column<kColEdgeGrad + 2 * E>(a, (oa * da - ob * db) * kRs2);           \
            add_column<kColEdgeGrad + 2 * E + 1>(a, h[ee] * __ldg(Gv + ee * n + nbE[E])); \
        }
        EDGE_COLS(0) EDGE_COLS(1) EDGE_COLS(2) EDGE_COLS(3) EDGE_COLS(4) EDGE_COLS(5)
        EDGE_COLS(6) EDGE_COLS(7) EDGE_COLS(8) EDGE_COLS(9) EDGE_COLS(10) EDGE_COLS(11)
#undef EDGE_COLS
        // own gradient
        dctr[0] = h[0] * __ldg(Gv + c);
        dctr[1] = h[1] * __ldg(Gv + n + c);
        dctr[2] = h[2] * __ldg(Gv + 2 * n + c);
        add_column<kColCentreGrad + 0>(a, dctr[0]);
        add_column<kColCentreGrad + 1>(a, dctr[1]);
        add_column<kColCentreGrad + 2>(a, dctr[2]);

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
            double w[6], IS[6], wsum = 0.0;
#pragma unroll
            for (int m = 0; m < 6; ++m) {
                const int ax = m / 2;
                const double bn = (m & 1) ? dface[m] : -dface[m];
                double s = bn * bn;
#pragma unroll
                for (int q = 0; q < 3; ++q)
                    if (q != ax) s += dctr[q] * dctr[q];
                IS[m] = s;
                const double t = s + eps, t2 = t * t;
                w[m] = (1.0 / 6.0) / (t2 * t2 * t);
                wsum += w[m];
            }
            double ISL = 0.0;
#pragma unroll
            for (int m = 0; m < 6; ++m) {
                w[m] /= wsum;
                ISL += w[m] * IS[m];
            }
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                // sum_m w_m b^m_q: tangential slopes from the own gradient,
                // the normal one from the neighbour difference
                bbar[q] = (1.0 - w[2 * q] - w[2 * q + 1]) * dctr[q] - w[2 * q] * dface[2 * q] +
                          w[2 * q + 1] * dface[2 * q + 1];
            }
            double ISH = 0.0;
            static_for<kNumBasis>([&](auto I) {
                constexpr int ii = decltype(I)::value;
                double t = 0.0;
                static_for<kNumBasis>([&](auto J) {
                    constexpr int jj = decltype(J)::value;
                    if constexpr (basis_class(ii) == basis_class(jj)) t = fma(cH[ii][jj], a[jj], t);
                });
                ISH = fma(a[ii], t, ISH);
            });
            const double r = fabs(ISH - ISL) / (ISH + ISL + eps);
            const double rr = r * 10.0;
            chi = 1.0 / (1.0 + rr * rr * rr);
        }
        eval_faces<0>(fs, n, c, v, a, base, chi, bbar, q0, nonlinear, h);
        eval_faces<1>(fs, n, c, v, a, base, chi, bbar, q0, nonlinear, h);
        eval_faces<2>(fs, n, c, v, a, base, chi, bbar, q0, nonlinear, h);
    }
}

__global__ void __launch_bounds__(128) recon2_kernel(GridDesc g, int nonlinear, double eps2,
                                                     const double *__restrict__ Q,
                                                     double *__restrict__ fs) {
    const long long n = g.n;
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const int i = (int)(c % g.nx);
    const int j = (int)((c / g.nx) % g.ny);
    const int k = (int)(c / ((long long)g.nx * g.ny));
    long long nb[6];
#pragma unroll
    for (int m = 0; m < 6; ++m)
        nb[m] = cell_index(g, wrap(i + face_off(m, 0), g.nx), wrap(j + face_off(m, 1), g.ny),
                           wrap(k + face_off(m, 2), g.nz));
#pragma unroll 1
    for (int v = 0; v < 5; ++v) {
        const double *Qv = Q + (long long)v * n;
        const double q0 = __ldg(Qv + c);
        double qn[6];
#pragma unroll
        for (int m = 0; m < 6; ++m) qn[m] = __ldg(Qv + nb[m]);
        // least-squares gradient of the face-neighbour averages on a uniform
        // grid: the central difference (normalised units)
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
            double *o = fs + ((long long)f * 20) * n + c;
            o[(long long)cmp * n] = q0 + phi * ((f & 1) ? 0.5 : -0.5) * b[d];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const int jf = (q - d + 3) % 3;
                o[(long long)(5 + 5 * jf + cmp) * n] = phi * b[q] / g.h[q];
            }
        }
    }
}

// ---- mixed precision: FP32 reconstruction of the offsets W - Q0 ----------
// The data entries are formed in FP64 (neighbour average minus own average,
// h times gradient) and rounded once to FP32; the least-squares product, the
// GENO weights and the Gauss-point evaluation run in FP32 and the face state
// is stored as the FP32 offset from the cell's own FP64 average, so that the
// flux kernel restores W = Q0 + offset without losing the small fluctuations
// of large fields (rho E ~ 180 at Ma 0.1).
template <int COL>
__device__ __forceinline__ void add_column_f(float a[kNumBasis], float x) {
#pragma unroll
    for (int i = 0; i < kNumBasis; ++i) a[i] = fmaf(cRf[i][COL], x, a[i]);
}

template <int D, int SIDE, int KK>
__device__ __forceinline__ void write_point_f(float *__restrict__ fs, long long n, long long c,
                                              int v, const float S[8], const float Dq[3][8],
                                              float base, float chi, const float bbar[3],
                                              bool nonlinear, const float ih[3]) {
    constexpr int T1 = (D + 1) % 3, T2 = (D + 2) % 3;
    constexpr float sD = SIDE ? 1.0f : -1.0f;
    constexpr float s1 = (KK & 1) ? 1.0f : -1.0f;
    constexpr float s2 = (KK & 2) ? 1.0f : -1.0f;
    float sg[3];
    sg[D] = sD;
    sg[T1] = s1;
    sg[T2] = s2;
    float val = base, der[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int cls = 0; cls < 8; ++cls) {
        const float sign = ((cls & 1) ? sg[0] : 1.0f) * ((cls & 2) ? sg[1] : 1.0f) *
                           ((cls & 4) ? sg[2] : 1.0f);
        val += sign * S[cls];
#pragma unroll
        for (int q = 0; q < 3; ++q) der[q] += sign * Dq[q][cls];
    }
    if (nonlinear) {
        float x[3];
        x[D] = 0.5f * sD;
        x[T1] = (float)kG * s1;
        x[T2] = (float)kG * s2;
        const float p1 = bbar[0] * x[0] + bbar[1] * x[1] + bbar[2] * x[2];
        val = chi * val + (1.0f - chi) * p1;
#pragma unroll
        for (int q = 0; q < 3; ++q) der[q] = chi * der[q] + (1.0f - chi) * bbar[q];
    }
    constexpr int f = 2 * D + SIDE;
    const int cmp = frame_comp(v, D);
    float *o = fs + ((long long)(f * 4 + KK) * 20) * n + c;
    o[(long long)cmp * n] = val;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const int jf = (q - D + 3) % 3;
        o[(long long)(5 + 5 * jf + cmp) * n] = der[q] * ih[q];
    }
}

template <int D>
__device__ __forceinline__ void eval_faces_f(float *__restrict__ fs, long long n, long long c, int v,
                                             const float a[kNumBasis], float base, float chi,
                                             const float bbar[3], bool nonlinear,
                                             const float ih[3]) {
    float S[8], Dq[3][8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        S[k] = 0.0f;
        Dq[0][k] = Dq[1][k] = Dq[2][k] = 0.0f;
    }
    static_for<kNumBasis>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int cls = basis_class(i);
        S[cls] = fmaf(a[i], cMvalf[D][i], S[cls]);
        static_for<3>([&](auto Qc) {
            constexpr int q = decltype(Qc)::value;
            if constexpr (has_deriv(i, q)) {
                constexpr int dc = deriv_class(i, q);
                Dq[q][dc] = fmaf(a[i], cMderf[D][q][i], Dq[q][dc]);
            }
        });
    });
    write_point_f<D, 0, 0>(fs, n, c, v, S, Dq, base, chi, bbar, nonlinear, ih);
    write_point_f<D, 0, 1>(fs, n, c, v, S, Dq, base, chi, bbar, nonlinear, ih);
    write_point_f<D, 0, 2>(fs, n, c, v, S, Dq, base, chi, bbar, nonlinear, ih);
    write_point_f<D, 0, 3>(fs, n, c, v, S, Dq, base, chi, bbar, nonlinear, ih);
    write_point_f<D, 1, 0>(fs, n, c, v, S, Dq, base, chi, bbar, nonlinear, ih);
    write_point_f<D, 1, 1>(fs, n, c, v, S, Dq, base, chi, bbar, nonlinear, ih);
    write_point_f<D, 1, 2>(fs, n, c, v, S, Dq, base, chi, bbar, nonlinear, ih);
    write_point_f<D, 1, 3>(fs, n, c, v, S, Dq, base, chi, bbar, nonlinear, ih);
}

__global__ void __launch_bounds__(128) recon5_mixed_kernel(GridDesc g, int nonlinear,
                                                           const double *__restrict__ Q,
                                                           const double *__restrict__ G,
                                                           float *__restrict__ fs) {
    const long long n = g.n;
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const int i = (int)(c % g.nx);
    const int j = (int)((c / g.nx) % g.ny);
    const int k = (int)(c / ((long long)g.nx * g.ny));
    long long nbF[6], nbE[12];
#pragma unroll
    for (int m = 0; m < 6; ++m)
        nbF[m] = cell_index(g, wrap(i + face_off(m, 0), g.nx), wrap(j + face_off(m, 1), g.ny),
                            wrap(k + face_off(m, 2), g.nz));
#pragma unroll
    for (int e = 0; e < 12; ++e)
        nbE[e] = cell_index(g, wrap(i + edge_off(e, 0), g.nx), wrap(j + edge_off(e, 1), g.ny),
                            wrap(k + edge_off(e, 2), g.nz));
    const double h[3] = {g.h[0], g.h[1], g.h[2]};
    const float ih[3] = {(float)(1.0 / g.h[0]), (float)(1.0 / g.h[1]), (float)(1.0 / g.h[2])};

#pragma unroll 1
    for (int v = 0; v < 5; ++v) {
        const double *Qv = Q + (long long)v * n;
        const double *Gv = G + (long long)v * 3 * n;
        const double q0 = __ldg(Qv + c);
        float a[kNumBasis];
#pragma unroll
        for (int ii = 0; ii < kNumBasis; ++ii) a[ii] = 0.0f;
        float dface[6], dctr[3];
#define FACE_COLS_F(M)                                                                       \
        {                                                                                    \
            const float dq = (float)(__ldg(Qv + nbF[M]) - q0);                               \
            dface[M] = dq;                                                                   \
            add_column_f<kColFace + M>(a, dq);                                               \
            add_column_f<kColFaceGrad + 3 * M + 0>(a, (float)(h[0] * __ldg(Gv + nbF[M])));   \
            add_column_f<kColFaceGrad + 3 * M + 1>(a, (float)(h[1] * __ldg(Gv + n + nbF[M]))); \
            add_column_f<kColFaceGrad + 3 * M + 2>(a, (float)(h[2] * __ldg(Gv + 2 * n + nbF[M]))); \
        }
        FACE_COLS_F(0) FACE_COLS_F(1) FACE_COLS_F(2) FACE_COLS_F(3) FACE_COLS_F(4) FACE_COLS_F(5)
#undef FACE_COLS_F
#define EDGE_COLS_F(E)                                                                       \
        {                                                                                    \
            constexpr int ea = edge_axis_a(E), eb = edge_axis_b(E), ee = edge_axis_e(E);     \
            constexpr double oa = edge_off(E, ea), ob = edge_off(E, eb);                     \
            add_column_f<kColEdge + E>(a, (float)(__ldg(Qv + nbE[E]) - q0));                 \
            const double da = h[ea] * __ldg(Gv + ea * n + nbE[E]);                           \
            const double db = h[eb] * __ldg(Gv + eb * n + nbE[E]);                           \
            add_column_f<kColEdgeGrad + 2 * E>(a, (float)((oa * da - ob * db) * kRs2));      \
            add_column_f<kColEdgeGrad + 2 * E + 1>(a, (float)(h[ee] * __ldg(Gv + ee * n + nbE[E]))); \
        }
        EDGE_COLS_F(0) EDGE_COLS_F(1) EDGE_COLS_F(2) EDGE_COLS_F(3) EDGE_COLS_F(4) EDGE_COLS_F(5)
        EDGE_COLS_F(6) EDGE_COLS_F(7) EDGE_COLS_F(8) EDGE_COLS_F(9) EDGE_COLS_F(10) EDGE_COLS_F(11)
#undef EDGE_COLS_F
        dctr[0] = (float)(h[0] * __ldg(Gv + c));
        dctr[1] = (float)(h[1] * __ldg(Gv + n + c));
        dctr[2] = (float)(h[2] * __ldg(Gv + 2 * n + c));
        add_column_f<kColCentreGrad + 0>(a, dctr[0]);
        add_column_f<kColCentreGrad + 1>(a, dctr[1]);
        add_column_f<kColCentreGrad + 2>(a, dctr[2]);

        float K = 0.0f;
        static_for<kNumBasis>([&](auto I) {
            constexpr int ii = decltype(I)::value;
            if constexpr (basis_class(ii) == 0) K = fmaf(a[ii], cMeanf[ii], K);
        });
        const float base = -K;  // offset of P4 from Q0, before the class sums

        float chi = 1.0f, bbar[3] = {0.0f, 0.0f, 0.0f};
        if (nonlinear) {
            const float eps = 1e-15f;
            float w[6], IS[6], t[6];
#pragma unroll
            for (int m = 0; m < 6; ++m) {
                const int ax = m / 2;
                const float bn = (m & 1) ? dface[m] : -dface[m];
                float s = bn * bn;
#pragma unroll
                for (int q = 0; q < 3; ++q)
                    if (q != ax) s = fmaf(dctr[q], dctr[q], s);
                IS[m] = s;
                t[m] = s + eps;
            }
            // w_m = (1/(IS_m + eps)^5) / sum_k (1/(IS_k + eps)^5), written with
            // ratios so that no power over- or underflows in FP32
            float ISL = 0.0f;
#pragma unroll
            for (int m = 0; m < 6; ++m) {
                float sum = 0.0f;
#pragma unroll
                for (int kq = 0; kq < 6; ++kq) {
                    const float r = t[m] / t[kq];
                    const float r2 = r * r;
                    sum += r2 * r2 * r;
                }
                w[m] = 1.0f / sum;
                ISL = fmaf(w[m], IS[m], ISL);
            }
#pragma unroll
            for (int q = 0; q < 3; ++q)
                bbar[q] = (1.0f - w[2 * q] - w[2 * q + 1]) * dctr[q] - w[2 * q] * dface[2 * q] +
                          w[2 * q + 1] * dface[2 * q + 1];
            float ISH = 0.0f;
            static_for<kNumBasis>([&](auto I) {
                constexpr int ii = decltype(I)::value;
                float tt = 0.0f;
                static_for<kNumBasis>([&](auto J) {
                    constexpr int jj = decltype(J)::value;
                    if constexpr (basis_class(ii) == basis_class(jj)) tt = fmaf(cHf[ii][jj], a[jj], tt);
                });
                ISH = fmaf(a[ii], tt, ISH);
            });
            const float r = fabsf(ISH - ISL) / (ISH + ISL + eps);
            const float rr = r * 10.0f;
            chi = 1.0f / (1.0f + rr * rr * rr);
        }
        eval_faces_f<0>(fs, n, c, v, a, base, chi, bbar, nonlinear, ih);
        eval_faces_f<1>(fs, n, c, v, a, base, chi, bbar, nonlinear, ih);
        eval_faces_f<2>(fs, n, c, v, a, base, chi, bbar, nonlinear, ih);
    }
}

__global__ void __launch_bounds__(128) recon2_mixed_kernel(GridDesc g, int nonlinear, float eps2,
                                                           const double *__restrict__ Q,
                                                           float *__restrict__ fs) {
    const long long n = g.n;
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const int i = (int)(c % g.nx);
    const int j = (int)((c / g.nx) % g.ny);
    const int k = (int)(c / ((long long)g.nx * g.ny));
    long long nb[6];
#pragma unroll
    for (int m = 0; m < 6; ++m)
        nb[m] = cell_index(g, wrap(i + face_off(m, 0), g.nx), wrap(j + face_off(m, 1), g.ny),
                           wrap(k + face_off(m, 2), g.nz));
    const float ih[3] = {(float)(1.0 / g.h[0]), (float)(1.0 / g.h[1]), (float)(1.0 / g.h[2])};
#pragma unroll 1
    for (int v = 0; v < 5; ++v) {
        const double *Qv = Q + (long long)v * n;
        const double q0 = __ldg(Qv + c);
        float dn[6];  // neighbour minus own average, FP64 difference
#pragma unroll
        for (int m = 0; m < 6; ++m) dn[m] = (float)(__ldg(Qv + nb[m]) - q0);
        float b[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) b[d] = 0.5f * (dn[2 * d + 1] - dn[2 * d]);
        float phi = 1.0f;
        if (nonlinear) {
            float dmax = 0.0f, dmin = 0.0f;
#pragma unroll
            for (int m = 0; m < 6; ++m) {
                dmax = fmaxf(dmax, dn[m]);
                dmin = fminf(dmin, dn[m]);
            }
#pragma unroll
            for (int f = 0; f < 6; ++f) {
                const float d2 = (f & 1) ? 0.5f * b[f / 2] : -0.5f * b[f / 2];
                if (d2 != 0.0f) {
                    const float dp = d2 > 0.0f ? dmax : dmin;
                    const float pf = (dp * dp + eps2 + 2.0f * d2 * dp) /
                                     (dp * dp + 2.0f * d2 * d2 + d2 * dp + eps2);
                    phi = fminf(phi, pf);
                }
            }
        }
#pragma unroll
        for (int f = 0; f < 6; ++f) {
            const int d = f / 2;
            const int cmp = frame_comp(v, d);
            float *o = fs + ((long long)f * 20) * n + c;
            o[(long long)cmp * n] = phi * ((f & 1) ? 0.5f : -0.5f) * b[d];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const int jf = (q - d + 3) % 3;
                o[(long long)(5 + 5 * jf + cmp) * n] = phi * b[q] * ih[q];
            }
        }
    }
}

}  // namespace

int upload_recon_tables(void) {
    static ReconTables t;
    static int built = 0;
    if (!built) {
        if (build_recon_tables(&t)) return -1;
        built = 1;
    }
    if (cudaMemcpyToSymbol(cR, t.R, sizeof(t.R)) != cudaSuccess) return -2;
    if (cudaMemcpyToSymbol(cH, t.H, sizeof(t.H)) != cudaSuccess) return -2;
    if (cudaMemcpyToSymbol(cMean, t.mean, sizeof(t.mean)) != cudaSuccess) return -2;
    if (cudaMemcpyToSymbol(cMval, t.mval, sizeof(t.mval)) != cudaSuccess) return -2;
    if (cudaMemcpyToSymbol(cMder, t.mder, sizeof(t.mder)) != cudaSuccess) return -2;
    static float fR[kNumBasis][kNumData], fH[kNumBasis][kNumBasis], fMean[kNumBasis],
        fMval[3][kNumBasis], fMder[3][3][kNumBasis];
    for (int i = 0; i < kNumBasis; ++i) {
        for (int c = 0; c < kNumData; ++c) fR[i][c] = (float)t.R[i][c];
        for (int c = 0; c < kNumBasis; ++c) fH[i][c] = (float)t.H[i][c];
        fMean[i] = (float)t.mean[i];
        for (int d = 0; d < 3; ++d) {
            fMval[d][i] = (float)t.mval[d][i];
            for (int q = 0; q < 3; ++q) fMder[d][q][i] = (float)t.mder[d][q][i];
        }
    }
    if (cudaMemcpyToSymbol(cRf, fR, sizeof(fR)) != cudaSuccess) return -2;
    if (cudaMemcpyToSymbol(cHf, fH, sizeof(fH)) != cudaSuccess) return -2;
    if (cudaMemcpyToSymbol(cMeanf, fMean, sizeof(fMean)) != cudaSuccess) return -2;
    if (cudaMemcpyToSymbol(cMvalf, fMval, sizeof(fMval)) != cudaSuccess) return -2;
    if (cudaMemcpyToSymbol(cMderf, fMder, sizeof(fMder)) != cudaSuccess) return -2;
    return 0;
}

int launch_recon5_mixed(const GridDesc &g, const PhysParams &P, const double *Q, const double *G,
                        float *fs, cudaStream_t s) {
    const int block = 128;
    const long long grid = (g.n + block - 1) / block;
    recon5_mixed_kernel<<<(unsigned)grid, block, 0, s>>>(g, P.nonlinear, Q, G, fs);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int launch_recon2_mixed(const GridDesc &g, const PhysParams &P, const double *Q, float *fs,
                        cudaStream_t s) {
    const double hv = cbrt(g.h[0] * g.h[1] * g.h[2]);
    const float eps2 = (float)(hv * hv * hv);
    const int block = 128;
    const long long grid = (g.n + block - 1) / block;
    recon2_mixed_kernel<<<(unsigned)grid, block, 0, s>>>(g, P.nonlinear, eps2, Q, fs);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int launch_recon5(const GridDesc &g, const PhysParams &P, const double *Q, const double *G,
                  double *fs, cudaStream_t s) {
    const int block = 128;
    const long long grid = (g.n + block - 1) / block;
    recon5_kernel<<<(unsigned)grid, block, 0, s>>>(g, P.nonlinear, Q, G, fs);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int launch_recon2(const GridDesc &g, const PhysParams &P, const double *Q, double *fs,
                  cudaStream_t s) {
    const double hv = cbrt(g.h[0] * g.h[1] * g.h[2]);
    const double eps2 = hv * hv * hv;  // (K h)^3 with K = 1
    const int block = 128;
    const long long grid = (g.n + block - 1) / block;
    recon2_kernel<<<(unsigned)grid, block, 0, s>>>(g, P.nonlinear, eps2, Q, fs);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

}  // namespace gks
