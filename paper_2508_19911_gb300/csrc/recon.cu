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
__constant__ double cRs[kNumData][kMaxClass];  // R in the symmetrised data basis
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
constexpr int kPadS = 12;                                 // kMaxClass padded to a float4 multiple
constexpr int kTabRs = 0;                                 // [63][kPadS]: class block of R per combination
constexpr int kTabMval = kTabRs + kNumData * kPadS;       // [3][kPad]
constexpr int kTabMder = kTabMval + 3 * kPad;             // [3][3][kPad]
constexpr int kTabH = kTabMder + 9 * kPad;                // [34][kPad]
constexpr int kTabMean = kTabH + kNumBasis * kPad;        // [kPad]
constexpr int kTabW1 = kTabMean + kPad;                   // [63][kMlpHidden]: column c of W1
constexpr int kTabB1 = kTabW1 + kNumData * kMlpHidden;    // [kMlpHidden]
constexpr int kTabW2 = kTabB1 + kMlpHidden;               // [kMlpHidden]
constexpr int kTabB2 = kTabW2 + kMlpHidden;               // b2, logit(theta), 2 unused
constexpr int kTabFloats = kTabB2 + 4;
static_assert(kMaxClass <= kPadS && kPadS % 4 == 0, "class block padding");
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

// face-frame component of conserved variable v on a face normal to axis d
__device__ __forceinline__ int frame_comp(int v, int d) {
    return (v == 0 || v == 4) ? v : 1 + (v - 1 - d + 3) % 3;
}

// Value of data column K for one (cell, variable) (layout in basis.h)
template <int K>
__device__ __forceinline__ double data_col(const double *__restrict__ Qv,
                                           const double *__restrict__ Gv, long long n, long long c,
                                           const long long nbF[6], const long long nbE[12],
                                           double q0, const double h[3]) {
    if constexpr (K < kColEdge) {
        return __ldg(Qv + nbF[K]) - q0;
    } else if constexpr (K < kColFaceGrad) {
        return __ldg(Qv + nbE[K - kColEdge]) - q0;
    } else if constexpr (K < kColEdgeGrad) {
        constexpr int m = (K - kColFaceGrad) / 3, j = (K - kColFaceGrad) % 3;
        return h[j] * __ldg(Gv + j * n + nbF[m]);
    } else if constexpr (K < kColCentreGrad) {
        constexpr int e = (K - kColEdgeGrad) / 2;
        constexpr int ea = edge_axis_a(e), eb = edge_axis_b(e), ee = edge_axis_e(e);
        if constexpr ((K - kColEdgeGrad) % 2 == 0) {
            constexpr double oa = edge_off(e, ea), ob = edge_off(e, eb);
            const double da = h[ea] * __ldg(Gv + ea * n + nbE[e]);
            const double db = h[eb] * __ldg(Gv + eb * n + nbE[e]);
            return (oa * da - ob * db) * kRs2;
        } else {
            return h[ee] * __ldg(Gv + ee * n + nbE[e]);
        }
    } else {
        constexpr int j = K - kColCentreGrad;
        return h[j] * __ldg(Gv + j * n + c);
    }
}

// In-place Walsh-Hadamard transform over the three axis bits: from class
// sums X[cls] to the values at the eight points (+-x, +-y, +-z); afterwards
// X[p] is the value where axis j has sign + if bit j of p is set, else -.
template <typename T>
__device__ __forceinline__ void class_to_points(T X[8]) {
#pragma unroll
    for (int b = 1; b < 8; b <<= 1)
#pragma unroll
        for (int p = 0; p < 8; ++p)
            if (!(p & b)) {
                const T lo = X[p], hi = X[p | b];
                X[p] = lo - hi;
                X[p | b] = lo + hi;
            }
}

template <int D>
__device__ __forceinline__ void eval_faces(double *__restrict__ fs, long long n, long long c,
                                           int v, const double a[kNumBasis], double base,
                                           double chi, const double bbar[3], double q0,
                                           bool nonlinear, const double ih[3]) {
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
            double val = base + S[p], der[3] = {Dq[0][p], Dq[1][p], Dq[2][p]};
            if (nonlinear) {
                double x[3];
                x[D] = side ? 0.5 : -0.5;
                x[T1] = (kk & 1) ? kG : -kG;
                x[T2] = (kk & 2) ? kG : -kG;
                const double p1 = fma(bbar[0], x[0], fma(bbar[1], x[1], fma(bbar[2], x[2], q0)));
                val = fma(chi, val - p1, p1);  // chi P4 + (1 - chi) P1
#pragma unroll
                for (int q = 0; q < 3; ++q) der[q] = fma(chi, der[q] - bbar[q], bbar[q]);
            }
            double *o = fs + ((long long)((2 * D + side) * 4 + kk) * 20) * n + c;
            o[(long long)cmp * n] = val;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const int jf = (q - D + 3) % 3;
                o[(long long)(5 + 5 * jf + cmp) * n] = der[q] * ih[q];
            }
        }
}

// cell c (global), variable v; face states to buffer position l (stride nb)
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
#pragma unroll
    for (int m = 0; m < 6; ++m)
        nbF[m] = cell_index(g, wrap(i + face_off(m, 0), g.nx), wrap(j + face_off(m, 1), g.ny),
                            wrap(k + face_off(m, 2), g.nz));
#pragma unroll
    for (int e = 0; e < 12; ++e)
        nbE[e] = cell_index(g, wrap(i + edge_off(e, 0), g.nx), wrap(j + edge_off(e, 1), g.ny),
                            wrap(k + edge_off(e, 2), g.nz));
    const double h[3] = {g.h[0], g.h[1], g.h[2]};
    const double ih[3] = {1.0 / h[0], 1.0 / h[1], 1.0 / h[2]};

    const double *Qv = Q + (long long)v * n;
    const double *Gv = G + (long long)v * 3 * n;
    const double q0 = __ldg(Qv + c);
    double a[kNumBasis];
#pragma unroll
    for (int ii = 0; ii < kNumBasis; ++ii) a[ii] = 0.0;
    double dface[6], dctr[3];
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
                ov[q] = data_col<col>(Qv, Gv, n, c, nbF, nbE, q0, h);
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
        double w[6], IS[6], wsum = 0.0;
#pragma unroll
        for (int m = 0; m < 6; ++m) {
            const int ax = m / 2;
            const double bn = (m & 1) ? dface[m] : -dface[m];
            double s = bn * bn;
#pragma unroll
            for (int q = 0; q < 3; ++q)
                if (q != ax) s = fma(dctr[q], dctr[q], s);
            IS[m] = s;
            const double t = s + eps, t2 = t * t;
            w[m] = (1.0 / 6.0) / (t2 * t2 * t);
            wsum += w[m];
        }
        double ISL = 0.0;
#pragma unroll
        for (int m = 0; m < 6; ++m) {
            w[m] /= wsum;
            ISL = fma(w[m], IS[m], ISL);
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
    eval_faces<0>(fs, nb, l, v, a, base, chi, bbar, q0, nonlinear, ih);
    eval_faces<1>(fs, nb, l, v, a, base, chi, bbar, q0, nonlinear, ih);
    eval_faces<2>(fs, nb, l, v, a, base, chi, bbar, q0, nonlinear, ih);
}

__global__ void __launch_bounds__(128) recon5_kernel(GridDesc g, Slab S, int nonlinear,
                                                     const double *__restrict__ Q,
                                                     const double *__restrict__ G,
                                                     double *__restrict__ fs) {
    const long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (l < S.nb)
        recon5_cell(g, nonlinear, Q, G, fs, slab_global(g, S, l), (int)blockIdx.y, S.nb, l);
}

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
            double *o = fs + ((long long)f * 20) * S.nb + l;
            o[(long long)cmp * S.nb] = q0 + phi * ((f & 1) ? 0.5 : -0.5) * b[d];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const int jf = (q - d + 3) % 3;
                o[(long long)(5 + 5 * jf + cmp) * S.nb] = phi * b[q] / g.h[q];
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

// learned indicator: hidden pre-activations from data column COL
template <int COL>
__device__ __forceinline__ void add_hidden_f(const float *T, float hid[kMlpHidden], float &amax,
                                             float x) {
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

// FP32 data column K: differences of averages in FP64, rounded once; the
// gradient entries h G in FP32. The products are __fmul_rn (never fused
// into a later sum), so that every kernel that inlines this rounds them the
// same way, whatever else uses the value (network, dump).
// FP32 data column K: differences of averages in FP64, rounded once; the
// gradient entries h G in FP32, G either converted here or read from an
// FP32 copy Gf (VIEW; the same values). The products are __fmul_rn (never
// fused into a later sum), so that every kernel that inlines this rounds
// them the same way, whatever else uses the value (network, dump).
template <bool VIEW>
__device__ __forceinline__ float gval(const double *__restrict__ Gv, const float *__restrict__ Gfv,
                                      long long idx) {
    if constexpr (VIEW) return __ldg(Gfv + idx);
    else return (float)__ldg(Gv + idx);
}

template <int K, bool VIEW>
__device__ __forceinline__ float data_col_f(const double *__restrict__ Qv,
                                            const double *__restrict__ Gv,
                                            const float *__restrict__ Gfv, long long n,
                                            long long c, const long long nbF[6],
                                            const long long nbE[12], double q0, const float hf[3]) {
    if constexpr (K < kColEdge) {
        return (float)(__ldg(Qv + nbF[K]) - q0);
    } else if constexpr (K < kColFaceGrad) {
        return (float)(__ldg(Qv + nbE[K - kColEdge]) - q0);
    } else if constexpr (K < kColEdgeGrad) {
        constexpr int m = (K - kColFaceGrad) / 3, j = (K - kColFaceGrad) % 3;
        return __fmul_rn(hf[j], gval<VIEW>(Gv, Gfv, j * n + nbF[m]));
    } else if constexpr (K < kColCentreGrad) {
        constexpr int e = (K - kColEdgeGrad) / 2;
        constexpr int ea = edge_axis_a(e), eb = edge_axis_b(e), ee = edge_axis_e(e);
        if constexpr ((K - kColEdgeGrad) % 2 == 0) {
            const float da = __fmul_rn(hf[ea], gval<VIEW>(Gv, Gfv, ea * n + nbE[e]));
            const float db = __fmul_rn(hf[eb], gval<VIEW>(Gv, Gfv, eb * n + nbE[e]));
            // o_a d_a - o_b d_b with o = +-1
            constexpr bool same = edge_off(e, ea) == edge_off(e, eb);
            const float t = same ? __fsub_rn(da, db) : __fadd_rn(da, db);
            return __fmul_rn(edge_off(e, ea) > 0 ? t : -t, (float)kRs2);
        } else {
            return __fmul_rn(hf[ee], gval<VIEW>(Gv, Gfv, ee * n + nbE[e]));
        }
    } else {
        constexpr int j = K - kColCentreGrad;
        return __fmul_rn(hf[j], gval<VIEW>(Gv, Gfv, j * n + c));
    }
}

template <int D>
__device__ __forceinline__ void eval_faces_f(const float *T, float *__restrict__ fs,
                                             long long n, long long c, int v,
                                             const float a[kNumBasis], float base, float chi,
                                             const float bbar[3], bool nonlinear,
                                             const float ih[3]) {
    constexpr int T1 = (D + 1) % 3, T2 = (D + 2) % 3;
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
            float val = base + S[p], der[3] = {Dq[0][p], Dq[1][p], Dq[2][p]};
            if (nonlinear) {
                float x[3];
                x[D] = side ? 0.5f : -0.5f;
                x[T1] = (kk & 1) ? (float)kG : -(float)kG;
                x[T2] = (kk & 2) ? (float)kG : -(float)kG;
                const float p1 = fmaf(bbar[0], x[0], fmaf(bbar[1], x[1], bbar[2] * x[2]));
                val = fmaf(chi, val - p1, p1);  // chi P4 + (1 - chi) P1
#pragma unroll
                for (int q = 0; q < 3; ++q) der[q] = fmaf(chi, der[q] - bbar[q], bbar[q]);
            }
            float *o = fs + ((long long)((2 * D + side) * 4 + kk) * 20) * n + c;
            o[(long long)cmp * n] = val;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const int jf = (q - D + 3) % 3;
                o[(long long)(5 + 5 * jf + cmp) * n] = der[q] * ih[q];
            }
        }
}

template <int MODE, bool VIEW>
__device__ __forceinline__ void recon5_mixed_cell(const float *T,
                                                  const GridDesc &g, int nonlinear,
                                                  const double *__restrict__ Q,
                                                  const double *__restrict__ G,
                                                  const float *__restrict__ Gf,
                                                  float *__restrict__ fs,
                                                  float *__restrict__ dump_x,
                                                  float *__restrict__ dump_chi,
                                                  unsigned long long *skips, long long c,
                                                  long long dump_ld, long long dump_base, int v,
                                                  long long nb, long long l) {
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
        const double *Gv = VIEW ? nullptr : G + (long long)v * 3 * n;
        const float *Gfv = VIEW ? Gf + (long long)v * 3 * n : nullptr;
        const double q0 = __ldg(Qv + c);
        float a[kNumBasis], hid[kMlpHidden], amax = 0.0f;
#pragma unroll
        for (int ii = 0; ii < kNumBasis; ++ii) a[ii] = 0.0f;
#pragma unroll
        for (int jj = 0; jj < kMlpHidden; ++jj) hid[jj] = 0.0f;
        float dface[6], dctr[3];
        // a = R d orbit by orbit (see recon5_cell); the network and the dump
        // see the raw columns as they are loaded. Dump mode: data entry COL
        // of (cell, variable) -> dump_x[COL * dump_ld + dump_base + 5 c + v]
        float ov[8];
        static_for<kNumData>([&](auto Rr) {
            constexpr int r = decltype(Rr)::value;
            constexpr int nm = kSym.nm[r];
            if constexpr (kSym.orbit[r] == r) {
                static_for<nm>([&](auto Qq) {
                    constexpr int q = decltype(Qq)::value;
                    constexpr int col = kSym.mem[r][q];
                    ov[q] = data_col_f<col, VIEW>(Qv, Gv, Gfv, n, c, nbF, nbE, q0, hf);
                    if constexpr (col < kColEdge) dface[col] = ov[q];
                    if constexpr (col >= kColCentreGrad) dctr[col - kColCentreGrad] = ov[q];
                    if constexpr (MODE == kModeIndicator) add_hidden_f<col>(T, hid, amax, ov[q]);
                    if constexpr (MODE == kModeDump)
                        dump_x[(long long)col * dump_ld + dump_base + 5 * c + v] = ov[q];
                });
            }
            float ds = kSym.sgn[r][0] > 0 ? ov[0] : -ov[0];
            static_for<nm - 1>([&](auto Qq) {
                constexpr int q = decltype(Qq)::value + 1;
                if constexpr (kSym.sgn[r][q] > 0) ds += ov[q];
                else ds -= ov[q];
            });
            constexpr int cls = kSym.cls[r];
            static_for<(kClass.n[cls] + 3) / 4>([&](auto J4) {
                constexpr int j4 = decltype(J4)::value;
                const float4 w = ld4(T, kTabRs + r * kPadS + 4 * j4);
                static_for<4>([&](auto K) {
                    constexpr int jj = 4 * j4 + decltype(K)::value;
                    if constexpr (jj < kClass.n[cls]) {
                        constexpr int ib = kClass.member[cls][jj];
                        a[ib] = fmaf(f4(w, decltype(K)::value), ds, a[ib]);
                    }
                });
            });
        });
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
        eval_faces_f<0>(T, fs, nb, l, v, a, base, chi, bbar, geno, ih);
        eval_faces_f<1>(T, fs, nb, l, v, a, base, chi, bbar, geno, ih);
        eval_faces_f<2>(T, fs, nb, l, v, a, base, chi, bbar, geno, ih);
    }
}

// Persistent: each block stages the FP32 table once, then strides over
// tiles of 128 cells x one conserved variable (the five variables of a cell
// block are adjacent tiles). The empty asm with a memory clobber at the top
// of each tile keeps the compiler from hoisting table loads out of the tile
// loop into registers (which spills).
template <int MODE, bool VIEW>
__global__ void __launch_bounds__(128) recon5_mixed_kernel(GridDesc g, Slab S, int nonlinear,
                                                           const double *__restrict__ Q,
                                                           const double *__restrict__ G,
                                                           const float *__restrict__ Gf,
                                                           float *__restrict__ fs,
                                                           float *__restrict__ dump_x,
                                                           float *__restrict__ dump_chi,
                                                           unsigned long long *skips) {
    __shared__ __align__(16) float sT[kTabFloats];
    stage_tables(sT);
    const long long ntiles = 5 * ((S.nb + 127) / 128);
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        asm volatile("" ::: "memory");
        const long long l = (t / 5) * 128 + threadIdx.x;
        if (l < S.nb)
            recon5_mixed_cell<MODE, VIEW>(sT, g, nonlinear, Q, G, Gf, fs, dump_x, dump_chi, skips,
                                          slab_global(g, S, l), 5 * g.n, 0, (int)(t % 5), S.nb,
                                          l);
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
                recon5_mixed_cell<MODE, false>(sT, I.g, I.P.nonlinear, Q, G, nullptr,
                                        fsa ? (float *)fsa + 480 * I.off : nullptr, dump_x,
                                        dump_chi, skips, it.c0 + t % T, dump_ld, 5 * I.off,
                                        (int)(t / T), I.g.n, it.c0 + t % T);
            else
                recon5_cell(I.g, I.P.nonlinear, Q, G, (double *)fsa + 480 * I.off, it.c0 + t % T,
                            (int)(t / T), I.g.n, it.c0 + t % T);
        }
    }
}

__global__ void __launch_bounds__(128) recon2_mixed_kernel(GridDesc g, Slab S, int nonlinear,
                                                           float eps2, const double *__restrict__ Q,
                                                           float *__restrict__ fs) {
    const long long n = g.n;
    const long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= S.nb) return;
    const long long c = slab_global(g, S, l);
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
            float *o = fs + ((long long)f * 20) * S.nb + l;
            o[(long long)cmp * S.nb] = phi * ((f & 1) ? 0.5f : -0.5f) * b[d];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const int jf = (q - d + 3) % 3;
                o[(long long)(5 + 5 * jf + cmp) * S.nb] = phi * b[q] * ih[q];
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
    if (cudaMemcpyToSymbol(cRs, t.Rs, sizeof(t.Rs)) != cudaSuccess) return -2;
    if (cudaMemcpyToSymbol(cH, t.H, sizeof(t.H)) != cudaSuccess) return -2;
    if (cudaMemcpyToSymbol(cMean, t.mean, sizeof(t.mean)) != cudaSuccess) return -2;
    if (cudaMemcpyToSymbol(cMval, t.mval, sizeof(t.mval)) != cudaSuccess) return -2;
    if (cudaMemcpyToSymbol(cMder, t.mder, sizeof(t.mder)) != cudaSuccess) return -2;
    // FP32 sections of the staged table (the network's sections are left
    // as they are)
    static float tab[kTabW1];
    for (int i = 0; i < kTabW1; ++i) tab[i] = 0.0f;
    for (int r = 0; r < kNumData; ++r)
        for (int j = 0; j < kMaxClass; ++j) tab[kTabRs + r * kPadS + j] = (float)t.Rs[r][j];
    for (int i = 0; i < kNumBasis; ++i) {
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

// FP32 copy of the cell gradients (15 per cell), read by the mixed
// reconstruction instead of converting each G value at every stencil use
__global__ void g_to_f32_kernel(const double *__restrict__ G, float *__restrict__ Gf, long long m) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (long long)gridDim.x * blockDim.x)
        Gf[i] = (float)G[i];
}

int launch_g_to_f32(const GridDesc &g, const double *G, float *Gf, cudaStream_t s) {
    const long long m = 15 * g.n;
    const long long blocks = (m + 255) / 256;
    g_to_f32_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(G, Gf, m);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

// Gf: the FP32 gradient copy of this stage (launch_g_to_f32)
int launch_recon5_mixed(const GridDesc &g, const Slab &S, const PhysParams &P, const double *Q,
                        const float *Gf, float *fs, cudaStream_t s, int indicator,
                        unsigned long long *skips) {
    if (!Gf) return -1;
    const long long tiles = 5 * ((S.nb + 127) / 128);
    if (indicator)
        recon5_mixed_kernel<kModeIndicator, true>
            <<<persistent_blocks(recon5_mixed_kernel<kModeIndicator, true>, tiles), 128, 0, s>>>(
                g, S, P.nonlinear, Q, nullptr, Gf, fs, nullptr, nullptr, skips);
    else
        recon5_mixed_kernel<kModePlain, true>
            <<<persistent_blocks(recon5_mixed_kernel<kModePlain, true>, tiles), 128, 0, s>>>(
                g, S, P.nonlinear, Q, nullptr, Gf, fs, nullptr, nullptr, nullptr);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

// Gf: FP32 gradient buffer of a mixed context, or nullptr (FP64 context:
// each G value is converted where it is used; the same values)
int launch_indicator_dump(const GridDesc &g, const double *Q, const double *G, float *Gf, float *x,
                          float *chi, cudaStream_t s) {
    const long long tiles = 5 * ((g.n + 127) / 128);
    const Slab S = whole_grid(g);
    if (Gf) {
        if (launch_g_to_f32(g, G, Gf, s)) return -2;
        recon5_mixed_kernel<kModeDump, true>
            <<<persistent_blocks(recon5_mixed_kernel<kModeDump, true>, tiles), 128, 0, s>>>(
                g, S, 1, Q, nullptr, Gf, nullptr, x, chi, nullptr);
    } else {
        recon5_mixed_kernel<kModeDump, false>
            <<<persistent_blocks(recon5_mixed_kernel<kModeDump, false>, tiles), 128, 0, s>>>(
                g, S, 1, Q, G, nullptr, nullptr, x, chi, nullptr);
    }
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

int launch_recon2_mixed(const GridDesc &g, const Slab &S, const PhysParams &P, const double *Q,
                        float *fs, cudaStream_t s) {
    const double hv = cbrt(g.h[0] * g.h[1] * g.h[2]);
    const float eps2 = (float)(hv * hv * hv);
    const int block = 128;
    const long long grid = (S.nb + block - 1) / block;
    recon2_mixed_kernel<<<(unsigned)grid, block, 0, s>>>(g, S, P.nonlinear, eps2, Q, fs);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int launch_recon5(const GridDesc &g, const Slab &S, const PhysParams &P, const double *Q,
                  const double *G, double *fs, cudaStream_t s) {
    const int block = 128;
    const long long grid = (S.nb + block - 1) / block;
    recon5_kernel<<<dim3((unsigned)grid, 5), block, 0, s>>>(g, S, P.nonlinear, Q, G, fs);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int launch_recon2(const GridDesc &g, const Slab &S, const PhysParams &P, const double *Q,
                  double *fs, cudaStream_t s) {
    const double hv = cbrt(g.h[0] * g.h[1] * g.h[2]);
    const double eps2 = hv * hv * hv;  // (K h)^3 with K = 1
    const int block = 128;
    const long long grid = (S.nb + block - 1) / block;
    recon2_kernel<<<(unsigned)grid, block, 0, s>>>(g, S, P.nonlinear, eps2, Q, fs);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

}  // namespace gks
