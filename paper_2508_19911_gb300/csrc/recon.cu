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
// FP32 tables of the mixed-precision kernels, one device array that every
// block stages into shared memory (vector loads, one per four FMAs; read
// from constant memory, the per-FMA loads throttled the kernel). Layout in
// floats, each section 16-byte aligned; kPad pads the 34 basis
// coefficients to a multiple of four.
constexpr int kPad = 36;
constexpr int kTabR = 0;                                  // [63][kPad]: column c of R
constexpr int kTabMval = kTabR + kNumData * kPad;         // [3][kPad]
constexpr int kTabMder = kTabMval + 3 * kPad;             // [3][3][kPad]
constexpr int kTabH = kTabMder + 9 * kPad;                // [34][kPad]
constexpr int kTabMean = kTabH + kNumBasis * kPad;        // [kPad]
constexpr int kTabW1 = kTabMean + kPad;                   // [63][kMlpHidden]: column c of W1
constexpr int kTabB1 = kTabW1 + kNumData * kMlpHidden;    // [kMlpHidden]
constexpr int kTabW2 = kTabB1 + kMlpHidden;               // [kMlpHidden]
constexpr int kTabB2 = kTabW2 + kMlpHidden;               // b2, logit(theta), 2 unused
constexpr int kTabFloats = kTabB2 + 4;
static_assert(kTabMval % 4 == 0 && kTabMder % 4 == 0 && kTabH % 4 == 0 && kTabMean % 4 == 0 &&
                  kTabW1 % 4 == 0 && kMlpHidden % 4 == 0 && kTabFloats % 4 == 0,
              "sections of the FP32 table must be float4 aligned");
// the learned smoothness indicator's network lives in the same table (one
// network per device)
__device__ __align__(16) float gTabF[kTabFloats];

__device__ __forceinline__ float4 ld4(const float *T, int off) {
    return *reinterpret_cast<const float4 *>(T + off);
}

__device__ __forceinline__ float f4(const float4 &w, int k) {
    return k == 0 ? w.x : k == 1 ? w.y : k == 2 ? w.z : w.w;
}

// copy the table into this block's shared memory (all threads take part)
__device__ __forceinline__ void stage_tables(float *sT) {
    const float4 *src = reinterpret_cast<const float4 *>(gTabF);
    float4 *dst = reinterpret_cast<float4 *>(sT);
    for (int i = threadIdx.x; i < kTabFloats / 4; i += blockDim.x) dst[i] = src[i];
    __syncthreads();
}

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

__device__ __forceinline__ void recon5_cell(const GridDesc &g, int nonlinear,
                                            const double *__restrict__ Q,
                                            const double *__restrict__ G,
                                            double *__restrict__ fs, long long c, int v) {
    const long long n = g.n;
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

    {
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

__global__ void __launch_bounds__(128, 3) recon5_kernel(GridDesc g, int nonlinear,
                                                     const double *__restrict__ Q,
                                                     const double *__restrict__ G,
                                                     double *__restrict__ fs) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < g.n) recon5_cell(g, nonlinear, Q, G, fs, c, (int)blockIdx.y);
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
// recon5_mixed_kernel modes
constexpr int kModePlain = 0;      // full GENO
constexpr int kModeIndicator = 1;  // GENO skipped where the network is confident
constexpr int kModeDump = 2;       // write the data vector and chi, no face states

template <int COL, int MODE>
__device__ __forceinline__ void add_column_f(const float *T, float a[kNumBasis],
                                             float hid[kMlpHidden], float &amax, float x) {
    static_for<kPad / 4>([&](auto I4) {
        constexpr int i4 = decltype(I4)::value;
        const float4 w = ld4(T, kTabR + COL * kPad + 4 * i4);
        static_for<4>([&](auto K) {
            constexpr int i = 4 * i4 + decltype(K)::value;
            if constexpr (i < kNumBasis) a[i] = fmaf(f4(w, decltype(K)::value), x, a[i]);
        });
    });
    if (MODE == kModeIndicator) {
        static_for<kMlpHidden / 4>([&](auto J4) {
            constexpr int j4 = decltype(J4)::value;
            const float4 w = ld4(T, kTabW1 + COL * kMlpHidden + 4 * j4);
            hid[4 * j4 + 0] = fmaf(w.x, x, hid[4 * j4 + 0]);
            hid[4 * j4 + 1] = fmaf(w.y, x, hid[4 * j4 + 1]);
            hid[4 * j4 + 2] = fmaf(w.z, x, hid[4 * j4 + 2]);
            hid[4 * j4 + 3] = fmaf(w.w, x, hid[4 * j4 + 3]);
        });
        amax = fmaxf(amax, fabsf(x));
    }
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
__device__ __forceinline__ void eval_faces_f(const float *T, float *__restrict__ fs,
                                             long long n, long long c, int v,
                                             const float a[kNumBasis], float base, float chi,
                                             const float bbar[3], bool nonlinear,
                                             const float ih[3]) {
    float S[8], Dq[3][8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        S[k] = 0.0f;
        Dq[0][k] = Dq[1][k] = Dq[2][k] = 0.0f;
    }
    static_for<kPad / 4>([&](auto I4) {
        constexpr int i4 = decltype(I4)::value;
        const float4 mv = ld4(T, kTabMval + D * kPad + 4 * i4);
        const float4 m0 = ld4(T, kTabMder + (3 * D + 0) * kPad + 4 * i4);
        const float4 m1 = ld4(T, kTabMder + (3 * D + 1) * kPad + 4 * i4);
        const float4 m2 = ld4(T, kTabMder + (3 * D + 2) * kPad + 4 * i4);
        static_for<4>([&](auto K) {
            constexpr int kk = decltype(K)::value;
            constexpr int i = 4 * i4 + kk;
            if constexpr (i < kNumBasis) {
                constexpr int cls = basis_class(i);
                S[cls] = fmaf(a[i], f4(mv, kk), S[cls]);
                if constexpr (has_deriv(i, 0)) {
                    constexpr int dc = deriv_class(i, 0);
                    Dq[0][dc] = fmaf(a[i], f4(m0, kk), Dq[0][dc]);
                }
                if constexpr (has_deriv(i, 1)) {
                    constexpr int dc = deriv_class(i, 1);
                    Dq[1][dc] = fmaf(a[i], f4(m1, kk), Dq[1][dc]);
                }
                if constexpr (has_deriv(i, 2)) {
                    constexpr int dc = deriv_class(i, 2);
                    Dq[2][dc] = fmaf(a[i], f4(m2, kk), Dq[2][dc]);
                }
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

template <int MODE>
__device__ __forceinline__ void recon5_mixed_cell(const float *T,
                                                  const GridDesc &g, int nonlinear,
                                                  const double *__restrict__ Q,
                                                  const double *__restrict__ G,
                                                  float *__restrict__ fs,
                                                  float *__restrict__ dump_x,
                                                  float *__restrict__ dump_chi,
                                                  unsigned long long *skips, long long c,
                                                  long long dump_ld, long long dump_base, int v) {
    const long long n = g.n;
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
    // h and 1/h in FP32: the gradient entries h G are rounded to FP32 anyway
    // (only the differences of averages need FP64, for their cancellation)
    const float hf[3] = {(float)g.h[0], (float)g.h[1], (float)g.h[2]};
    const float ih[3] = {1.0f / hf[0], 1.0f / hf[1], 1.0f / hf[2]};

{
        const double *Qv = Q + (long long)v * n;
        const double *Gv = G + (long long)v * 3 * n;
        const double q0 = __ldg(Qv + c);
        float a[kNumBasis], hid[kMlpHidden], amax = 0.0f;
#pragma unroll
        for (int ii = 0; ii < kNumBasis; ++ii) a[ii] = 0.0f;
#pragma unroll
        for (int jj = 0; jj < kMlpHidden; ++jj) hid[jj] = 0.0f;
        float dface[6], dctr[3];
        // dump mode: data entry COL of (cell, variable) ->
        // dump_x[COL * dump_ld + dump_base + 5 c + v]
#define DUMP(COL, X)                                                                         \
        if (MODE == kModeDump) dump_x[(long long)(COL) * dump_ld + dump_base + 5 * c + v] = (X);
#define FACE_COLS_F(M)                                                                       \
        {                                                                                    \
            const float dq = (float)(__ldg(Qv + nbF[M]) - q0);                               \
            const float g0 = hf[0] * (float)__ldg(Gv + nbF[M]);                              \
            const float g1 = hf[1] * (float)__ldg(Gv + n + nbF[M]);                          \
            const float g2 = hf[2] * (float)__ldg(Gv + 2 * n + nbF[M]);                      \
            dface[M] = dq;                                                                   \
            add_column_f<kColFace + M, MODE>(T, a, hid, amax, dq);                              \
            add_column_f<kColFaceGrad + 3 * M + 0, MODE>(T, a, hid, amax, g0);                  \
            add_column_f<kColFaceGrad + 3 * M + 1, MODE>(T, a, hid, amax, g1);                  \
            add_column_f<kColFaceGrad + 3 * M + 2, MODE>(T, a, hid, amax, g2);                  \
            DUMP(kColFace + M, dq) DUMP(kColFaceGrad + 3 * M, g0)                            \
            DUMP(kColFaceGrad + 3 * M + 1, g1) DUMP(kColFaceGrad + 3 * M + 2, g2)            \
        }
        FACE_COLS_F(0) FACE_COLS_F(1) FACE_COLS_F(2) FACE_COLS_F(3) FACE_COLS_F(4) FACE_COLS_F(5)
#undef FACE_COLS_F
#define EDGE_COLS_F(E)                                                                       \
        {                                                                                    \
            constexpr int ea = edge_axis_a(E), eb = edge_axis_b(E), ee = edge_axis_e(E);     \
            constexpr float oa = edge_off(E, ea), ob = edge_off(E, eb);                      \
            const float dq = (float)(__ldg(Qv + nbE[E]) - q0);                               \
            const float da = hf[ea] * (float)__ldg(Gv + ea * n + nbE[E]);                    \
            const float db = hf[eb] * (float)__ldg(Gv + eb * n + nbE[E]);                    \
            const float t0 = (oa * da - ob * db) * (float)kRs2;                              \
            const float t1 = hf[ee] * (float)__ldg(Gv + ee * n + nbE[E]);                    \
            add_column_f<kColEdge + E, MODE>(T, a, hid, amax, dq);                              \
            add_column_f<kColEdgeGrad + 2 * E, MODE>(T, a, hid, amax, t0);                      \
            add_column_f<kColEdgeGrad + 2 * E + 1, MODE>(T, a, hid, amax, t1);                  \
            DUMP(kColEdge + E, dq) DUMP(kColEdgeGrad + 2 * E, t0)                            \
            DUMP(kColEdgeGrad + 2 * E + 1, t1)                                               \
        }
        EDGE_COLS_F(0) EDGE_COLS_F(1) EDGE_COLS_F(2) EDGE_COLS_F(3) EDGE_COLS_F(4) EDGE_COLS_F(5)
        EDGE_COLS_F(6) EDGE_COLS_F(7) EDGE_COLS_F(8) EDGE_COLS_F(9) EDGE_COLS_F(10) EDGE_COLS_F(11)
#undef EDGE_COLS_F
        dctr[0] = hf[0] * (float)__ldg(Gv + c);
        dctr[1] = hf[1] * (float)__ldg(Gv + n + c);
        dctr[2] = hf[2] * (float)__ldg(Gv + 2 * n + c);
        add_column_f<kColCentreGrad + 0, MODE>(T, a, hid, amax, dctr[0]);
        add_column_f<kColCentreGrad + 1, MODE>(T, a, hid, amax, dctr[1]);
        add_column_f<kColCentreGrad + 2, MODE>(T, a, hid, amax, dctr[2]);
        DUMP(kColCentreGrad, dctr[0]) DUMP(kColCentreGrad + 1, dctr[1])
        DUMP(kColCentreGrad + 2, dctr[2])
#undef DUMP
        // learned indicator: the network sees d / (max|d| + delta); by
        // linearity the hidden pre-activations were accumulated on the raw d
        bool geno = nonlinear != 0;
        if (MODE == kModeIndicator && geno) {
            const float inv = 1.0f / (amax + kMlpDelta);
            float logit = T[kTabB2];
#pragma unroll
            for (int jj = 0; jj < kMlpHidden; ++jj)
                logit = fmaf(T[kTabW2 + jj], fmaxf(fmaf(hid[jj], inv, T[kTabB1 + jj]), 0.0f), logit);
            if (logit >= T[kTabB2 + 1]) {
                geno = false;  // confident that chi = 1: the linear P4 alone
                if (skips) atomicAdd(skips, 1ull);
            }
        }

        float K = 0.0f;
        static_for<kNumBasis>([&](auto I) {
            constexpr int ii = decltype(I)::value;
            if constexpr (basis_class(ii) == 0) K = fmaf(a[ii], T[kTabMean + ii], K);
        });
        const float base = -K;  // offset of P4 from Q0, before the class sums

        float chi = 1.0f, bbar[3] = {0.0f, 0.0f, 0.0f};
        if (geno) {
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
            // w_m = (1/t_m^5) / sum_k (1/t_k^5) with t = IS + eps, written with
            // u_k = t_min / t_k in (0, 1] so that no power overflows in FP32
            // (at least one u_k is 1, so the sum is >= 1)
            float tmin = t[0];
#pragma unroll
            for (int m = 1; m < 6; ++m) tmin = fminf(tmin, t[m]);
            float u5[6], usum = 0.0f;
#pragma unroll
            for (int m = 0; m < 6; ++m) {
                const float u = tmin / t[m];
                const float u2 = u * u;
                u5[m] = u2 * u2 * u;
                usum += u5[m];
            }
            const float iusum = 1.0f / usum;
            float ISL = 0.0f;
#pragma unroll
            for (int m = 0; m < 6; ++m) {
                w[m] = u5[m] * iusum;
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
                    if constexpr (basis_class(ii) == basis_class(jj)) tt = fmaf(T[kTabH + ii * kPad + jj], a[jj], tt);
                });
                ISH = fmaf(a[ii], tt, ISH);
            });
            const float r = fabsf(ISH - ISL) / (ISH + ISL + eps);
            const float rr = r * 10.0f;
            chi = 1.0f / (1.0f + rr * rr * rr);
        }
        if (MODE == kModeDump) {
            dump_chi[dump_base + 5 * c + v] = chi;
            return;
        }
        eval_faces_f<0>(T, fs, n, c, v, a, base, chi, bbar, geno, ih);
        eval_faces_f<1>(T, fs, n, c, v, a, base, chi, bbar, geno, ih);
        eval_faces_f<2>(T, fs, n, c, v, a, base, chi, bbar, geno, ih);
    }
}

// Persistent: each block stages the FP32 table once, then strides over
// tiles of 128 cells x one conserved variable (the five variables of a cell
// block are adjacent tiles). The empty asm with a memory clobber at the top
// of each tile keeps the compiler from hoisting table loads out of the tile
// loop into registers (which spills).
template <int MODE>
__global__ void __launch_bounds__(128) recon5_mixed_kernel(GridDesc g, int nonlinear,
                                                           const double *__restrict__ Q,
                                                           const double *__restrict__ G,
                                                           float *__restrict__ fs,
                                                           float *__restrict__ dump_x,
                                                           float *__restrict__ dump_chi,
                                                           unsigned long long *skips) {
    __shared__ __align__(16) float sT[kTabFloats];
    stage_tables(sT);
    const long long ntiles = 5 * ((g.n + 127) / 128);
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        asm volatile("" ::: "memory");
        const long long c = (t / 5) * 128 + threadIdx.x;
        if (c < g.n)
            recon5_mixed_cell<MODE>(sT, g, nonlinear, Q, G, fs, dump_x, dump_chi, skips, c,
                                    5 * g.n, 0, (int)(t % 5));
    }
}

// Persistent ensemble reconstruction: blocks stride over the work items of
// all instances; MIXED selects the FP32 kernel (MODE as above).
template <bool MIXED, int MODE>
__global__ void __launch_bounds__(128) recon5_ens_kernel(const EnsInst *__restrict__ inst,
                                                         const EnsItem *__restrict__ items,
                                                         int nitems, const double *__restrict__ Qa,
                                                         const double *__restrict__ Ga,
                                                         void *__restrict__ fsa,
                                                         float *__restrict__ dump_x,
                                                         float *__restrict__ dump_chi,
                                                         unsigned long long *skips,
                                                         long long dump_ld) {
    __shared__ __align__(16) float sT[MIXED ? kTabFloats : 4];
    if constexpr (MIXED) stage_tables(sT);
    for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
        const EnsItem it = items[w];
        const EnsInst I = inst[it.inst];
        const double *Q = Qa + 5 * I.off;
        const double *G = Ga + 15 * I.off;
        const long long T = it.c1 - it.c0;
        for (long long t = threadIdx.x; t < 5 * T; t += blockDim.x) {
            asm volatile("" ::: "memory");
            if constexpr (MIXED)
                recon5_mixed_cell<MODE>(sT, I.g, I.P.nonlinear, Q, G,
                                        fsa ? (float *)fsa + 480 * I.off : nullptr, dump_x,
                                        dump_chi, skips, it.c0 + t % T, dump_ld, 5 * I.off,
                                        (int)(t / T));
            else
                recon5_cell(I.g, I.P.nonlinear, Q, G, (double *)fsa + 480 * I.off, it.c0 + t % T,
                            (int)(t / T));
        }
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
    // FP32 sections of the staged table (the network's sections are left
    // as they are)
    static float tab[kTabW1];
    for (int i = 0; i < kTabW1; ++i) tab[i] = 0.0f;
    for (int i = 0; i < kNumBasis; ++i) {
        for (int c = 0; c < kNumData; ++c) tab[kTabR + c * kPad + i] = (float)t.R[i][c];
        for (int j = 0; j < kNumBasis; ++j) tab[kTabH + i * kPad + j] = (float)t.H[i][j];
        tab[kTabMean + i] = (float)t.mean[i];
        for (int d = 0; d < 3; ++d) {
            tab[kTabMval + d * kPad + i] = (float)t.mval[d][i];
            for (int q = 0; q < 3; ++q) tab[kTabMder + (3 * d + q) * kPad + i] = (float)t.mder[d][q][i];
        }
    }
    if (cudaMemcpyToSymbol(gTabF, tab, sizeof(tab)) != cudaSuccess) return -2;
    return 0;
}

// grid of a persistent kernel: the blocks that fit on the device at once
// (occupancy of this kernel: registers, 18 KB of shared memory), capped by
// the number of tiles
template <typename K>
static unsigned persistent_blocks(K kernel, long long tiles) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 128, 0) != cudaSuccess ||
        sms <= 0 || per_sm <= 0) {
        sms = 152;
        per_sm = 2;
    }
    const long long b = (long long)per_sm * sms;
    return (unsigned)(tiles < b ? tiles : b);
}

int launch_recon5_mixed(const GridDesc &g, const PhysParams &P, const double *Q, const double *G,
                        float *fs, cudaStream_t s, int indicator, unsigned long long *skips) {
    const long long tiles = 5 * ((g.n + 127) / 128);
    if (indicator)
        recon5_mixed_kernel<kModeIndicator>
            <<<persistent_blocks(recon5_mixed_kernel<kModeIndicator>, tiles), 128, 0, s>>>(
                g, P.nonlinear, Q, G, fs, nullptr, nullptr, skips);
    else
        recon5_mixed_kernel<kModePlain>
            <<<persistent_blocks(recon5_mixed_kernel<kModePlain>, tiles), 128, 0, s>>>(
                g, P.nonlinear, Q, G, fs, nullptr, nullptr, nullptr);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int launch_indicator_dump(const GridDesc &g, const double *Q, const double *G, float *x,
                          float *chi, cudaStream_t s) {
    const long long tiles = 5 * ((g.n + 127) / 128);
    recon5_mixed_kernel<kModeDump><<<persistent_blocks(recon5_mixed_kernel<kModeDump>, tiles), 128,
                                     0, s>>>(g, 1, Q, G, nullptr, x, chi, nullptr);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int launch_recon5_ens(const EnsInst *inst, const EnsItem *items, int nitems, int blocks,
                      int mixed, int indicator, const double *Qa, const double *Ga, void *fsa,
                      unsigned long long *skips, cudaStream_t s) {
    if (!mixed)
        recon5_ens_kernel<false, kModePlain><<<blocks, 128, 0, s>>>(inst, items, nitems, Qa, Ga, fsa,
                                                                    nullptr, nullptr, nullptr, 0);
    else if (indicator)
        recon5_ens_kernel<true, kModeIndicator><<<blocks, 128, 0, s>>>(inst, items, nitems, Qa, Ga,
                                                                       fsa, nullptr, nullptr, skips, 0);
    else
        recon5_ens_kernel<true, kModePlain><<<blocks, 128, 0, s>>>(inst, items, nitems, Qa, Ga, fsa,
                                                                   nullptr, nullptr, nullptr, 0);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int launch_indicator_dump_ens(const EnsInst *inst, const EnsItem *items, int nitems, int blocks,
                              const double *Qa, const double *Ga, float *x, float *chi,
                              long long total_cells, cudaStream_t s) {
    recon5_ens_kernel<true, kModeDump><<<blocks, 128, 0, s>>>(inst, items, nitems, Qa, Ga, nullptr,
                                                              x, chi, nullptr, 5 * total_cells);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int upload_indicator(const float *params, float theta) {
    // params: W1 [kMlpHidden][63] row major, b1, w2, b2 (kMlpParams floats,
    // host); stored with W1 transposed so that one column is contiguous
    static float net[kTabFloats - kTabW1];
    for (int j = 0; j < kMlpHidden; ++j)
        for (int c = 0; c < kNumData; ++c) net[c * kMlpHidden + j] = params[j * kNumData + c];
    for (int j = 0; j < kMlpHidden; ++j) {
        net[kTabB1 - kTabW1 + j] = params[kMlpHidden * kNumData + j];
        net[kTabW2 - kTabW1 + j] = params[kMlpHidden * kNumData + kMlpHidden + j];
    }
    net[kTabB2 - kTabW1] = params[kMlpHidden * kNumData + 2 * kMlpHidden];
    // skip when sigmoid(logit) >= theta, i.e. logit >= log(theta / (1 - theta))
    net[kTabB2 - kTabW1 + 1] = theta >= 1.0f ? INFINITY : logf(theta / (1.0f - theta));
    net[kTabB2 - kTabW1 + 2] = net[kTabB2 - kTabW1 + 3] = 0.0f;
    if (cudaMemcpyToSymbol(gTabF, net, sizeof(net), sizeof(float) * kTabW1) != cudaSuccess)
        return -2;
    return 0;
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
    recon5_kernel<<<dim3((unsigned)grid, 5), block, 0, s>>>(g, P.nonlinear, Q, G, fs);
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
