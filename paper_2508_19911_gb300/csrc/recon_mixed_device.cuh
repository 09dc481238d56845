// Device code of the mixed-precision CGKS-5th reconstruction (Sec. 3.2 in
// FP32): the FP32 table (a __device__ array staged into shared memory;
// every includer has its own copy and uploads it), the data vector with the
// float-float differences of averages, GENO, the learned indicator's
// inference and the evaluation at the face Gauss points
// (recon5_mixed_cell). Included by recon.cu (compiled without implicit
// multiply-add contraction) and by the single-launch ensemble step. See
// recon.cu.
#pragma once
#include "recon_common.cuh"

namespace gks {
namespace {


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
constexpr int kTabBs = kTabMder + 9 * kPad;               // [63][kPadS]: class block of W B
constexpr int kTabMean = kTabBs + kNumData * kPadS;       // [kPad]
constexpr int kTabW1 = kTabMean + kPad;                   // [63][kMlpHidden]: column c of W1
constexpr int kTabB1 = kTabW1 + kNumData * kMlpHidden;    // [kMlpHidden]
constexpr int kTabW2 = kTabB1 + kMlpHidden;               // [kMlpHidden]
constexpr int kTabB2 = kTabW2 + kMlpHidden;               // b2, logit(theta), 2 unused
constexpr int kTabFloats = kTabB2 + 4;
static_assert(kMaxClass <= kPadS && kPadS % 4 == 0, "class block padding");
static_assert(kTabMval % 4 == 0 && kTabMder % 4 == 0 && kTabBs % 4 == 0 && kTabMean % 4 == 0 &&
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

// FP32 data column K. VIEW (mixed contexts and the ensemble): the
// difference of two averages from their float-float splits,
// (hi_k - hi_0) + (lo_k - lo_0) (the hi difference is exact where the two
// averages are within a factor of two), and the gradients from the FP32
// copy Gf; otherwise (an FP64 context's dump) the FP64 difference rounded
// once and each G converted here. The products are __fmul_rn (never fused
// into a later sum), so that every kernel that inlines this rounds them the
// same way, whatever else uses the value (network, dump).
template <bool VIEW>
__device__ __forceinline__ float gval(const double *__restrict__ Gv, const float *__restrict__ Gfv,
                                      long long idx) {
    if constexpr (VIEW) return __ldg(Gfv + idx);
    else return (float)__ldg(Gv + idx);
}

// GEN: a general grid (mirror ghosts, per-cell sizes; see recon_fp64.cu)
template <int K, bool VIEW, bool GEN>
__device__ __forceinline__ float data_col_f(const double *__restrict__ Qv,
                                            const double *__restrict__ Gv,
                                            const float *__restrict__ qh,
                                            const float *__restrict__ ql,
                                            const float *__restrict__ Gfv, long long n,
                                            long long c, const long long nbF[6],
                                            const long long nbE[12], double q0, float h0,
                                            float l0, const float hf[3], const NbGeo &geo) {
    if constexpr (K < kColFaceGrad) {
        const long long nb = K < kColEdge ? nbF[K] : nbE[K - kColEdge];
        bool neg = false;
        if constexpr (GEN) neg = ((K < kColEdge ? geo.fF[K] : geo.fE[K - kColEdge]) >> 3) & 1;
        if constexpr (VIEW)
            return __fadd_rn(__fsub_rn(neg_if(__ldg(qh + nb), neg), h0),
                             __fsub_rn(neg_if(__ldg(ql + nb), neg), l0));
        else
            return (float)(neg_if(__ldg(Qv + nb), neg) - q0);
    } else if constexpr (K < kColEdgeGrad) {
        constexpr int m = (K - kColFaceGrad) / 3, j = (K - kColFaceGrad) % 3;
        if constexpr (GEN)
            return __fmul_rn((float)geo.hm[j][face_off(m, j) + 1],
                             neg_if(gval<VIEW>(Gv, Gfv, j * n + nbF[m]), der_neg(geo.fF[m], j)));
        else return __fmul_rn(hf[j], gval<VIEW>(Gv, Gfv, j * n + nbF[m]));
    } else if constexpr (K < kColCentreGrad) {
        constexpr int e = (K - kColEdgeGrad) / 2;
        constexpr int ea = edge_axis_a(e), eb = edge_axis_b(e), ee = edge_axis_e(e);
        if constexpr ((K - kColEdgeGrad) % 2 == 0) {
            float da, db;
            if constexpr (GEN) {
                da = __fmul_rn((float)geo.hm[ea][edge_off(e, ea) + 1],
                               neg_if(gval<VIEW>(Gv, Gfv, ea * n + nbE[e]), der_neg(geo.fE[e], ea)));
                db = __fmul_rn((float)geo.hm[eb][edge_off(e, eb) + 1],
                               neg_if(gval<VIEW>(Gv, Gfv, eb * n + nbE[e]), der_neg(geo.fE[e], eb)));
            } else {
                da = __fmul_rn(hf[ea], gval<VIEW>(Gv, Gfv, ea * n + nbE[e]));
                db = __fmul_rn(hf[eb], gval<VIEW>(Gv, Gfv, eb * n + nbE[e]));
            }
            // o_a d_a - o_b d_b with o = +-1
            constexpr bool same = edge_off(e, ea) == edge_off(e, eb);
            const float t = same ? __fsub_rn(da, db) : __fadd_rn(da, db);
            return __fmul_rn(edge_off(e, ea) > 0 ? t : -t, (float)kRs2);
        } else {
            if constexpr (GEN)
                return __fmul_rn((float)geo.hm[ee][1],
                                 neg_if(gval<VIEW>(Gv, Gfv, ee * n + nbE[e]), der_neg(geo.fE[e], ee)));
            else return __fmul_rn(hf[ee], gval<VIEW>(Gv, Gfv, ee * n + nbE[e]));
        }
    } else {
        constexpr int j = K - kColCentreGrad;
        return __fmul_rn(hf[j], gval<VIEW>(Gv, Gfv, j * n + c));
    }
}

// the FP32 evaluation at the Gauss points, GENO's blend folded into the
// class sums as in recon_fp64.cu (a scaled by chi, base = -chi K for the
// offset from Q0, w = (1 - chi) bbar)
template <int D>
__device__ __forceinline__ void eval_faces_f(const float *T, float *__restrict__ fs,
                                             long long n, long long c, int v,
                                             const float a[kNumBasis], float base,
                                             const float w[3], bool blend, const float ih[3]) {
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
    if (blend) {
        S[1 << D] = fmaf(0.5f, w[D], S[1 << D]);
        S[1 << T1] = fmaf((float)kG, w[T1], S[1 << T1]);
        S[1 << T2] = fmaf((float)kG, w[T2], S[1 << T2]);
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
            float *o = fs + ((long long)((2 * D + side) * 4 + kk) * 20) * n + c;
            o[(long long)cmp * n] = base + S[p];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const int jf = (q - D + 3) % 3;
                o[(long long)(5 + 5 * jf + cmp) * n] = Dq[q][p];
            }
        }
}

template <int MODE, bool VIEW, bool GEN = false>
__device__ __forceinline__ void recon5_mixed_cell(const float *T,
                                                  const GridDesc &g, int nonlinear,
                                                  const double *__restrict__ Q,
                                                  const double *__restrict__ G,
                                                  const float *__restrict__ Gf,
                                                  const float *__restrict__ Qhi,
                                                  const float *__restrict__ Qlo,
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
    NbGeo geo;
    stencil<GEN>(g, i, j, k, v, nbF, nbE, geo);
    // h and 1/h in FP32: the gradient entries h G are rounded to FP32 anyway
    // (only the differences of averages need FP64, for their cancellation)
    float hf[3] = {(float)g.h[0], (float)g.h[1], (float)g.h[2]};
    if constexpr (GEN) {
        hf[0] = (float)geo.hm[0][1];
        hf[1] = (float)geo.hm[1][1];
        hf[2] = (float)geo.hm[2][1];
    }
    const float ih[3] = {1.0f / hf[0], 1.0f / hf[1], 1.0f / hf[2]};

{
        const double *Qv = VIEW ? nullptr : Q + (long long)v * n;
        const double *Gv = VIEW ? nullptr : G + (long long)v * 3 * n;
        const float *Gfv = VIEW ? Gf + (long long)v * 3 * n : nullptr;
        const float *qh = VIEW ? Qhi + (long long)v * n : nullptr;
        const float *ql = VIEW ? Qlo + (long long)v * n : nullptr;
        const double q0 = VIEW ? 0.0 : __ldg(Qv + c);
        const float h0 = VIEW ? __ldg(qh + c) : 0.0f, l0 = VIEW ? __ldg(ql + c) : 0.0f;
        float a[kNumBasis], hid[kMlpHidden], amax = 0.0f;
#pragma unroll
        for (int ii = 0; ii < kNumBasis; ++ii) a[ii] = 0.0f;
#pragma unroll
        for (int jj = 0; jj < kMlpHidden; ++jj) hid[jj] = 0.0f;
        float dface[6], dctr[3];
        float norm2 = 0.0f;  // |d_C|^2 + |W d_B|^2 for GENO's misfit
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
                    ov[q] = data_col_f<col, VIEW, GEN>(Qv, Gv, qh, ql, Gfv, n, c, nbF, nbE, q0,
                                                       h0, l0, hf, geo);
                    constexpr float wc = (float)(col_weight(col) * col_weight(col));
                    norm2 = fmaf(wc * ov[q], ov[q], norm2);
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
            float w[6], t[6];
#pragma unroll
            for (int m = 0; m < 6; ++m) {
                const int ax = m / 2;
                const float bn = (m & 1) ? dface[m] : -dface[m];
                float s = bn * bn;
#pragma unroll
                for (int q = 0; q < 3; ++q)
                    if (q != ax) s = fmaf(dctr[q], dctr[q], s);
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
#pragma unroll
            for (int m = 0; m < 6; ++m) w[m] = u5[m] * iusum;
#pragma unroll
            for (int q = 0; q < 3; ++q)
                bbar[q] = (1.0f - w[2 * q] - w[2 * q + 1]) * dctr[q] - w[2 * q] * dface[2 * q] +
                          w[2 * q + 1] * dface[2 * q + 1];
            // GENO's misfit (see recon_fp64.cu), derivative columns reloaded
            float res2 = 0.0f;
            static_for<kNumData>([&](auto Rr) {
                constexpr int r = decltype(Rr)::value;
                constexpr int nm = kSym.nm[r];
                if constexpr (kSym.mem[r][0] >= kColFaceGrad) {
                    if constexpr (kSym.orbit[r] == r) {
                        static_for<nm>([&](auto Qq) {
                            constexpr int q = decltype(Qq)::value;
                            constexpr int col = kSym.mem[r][q];
                            ov[q] = data_col_f<col, VIEW, GEN>(Qv, Gv, qh, ql, Gfv, n, c, nbF,
                                                               nbE, q0, h0, l0, hf, geo);
                        });
                    }
                    float ds = kSym.sgn[r][0] > 0 ? ov[0] : -ov[0];
                    static_for<nm - 1>([&](auto Qq) {
                        constexpr int q = decltype(Qq)::value + 1;
                        if constexpr (kSym.sgn[r][q] > 0) ds += ov[q];
                        else ds -= ov[q];
                    });
                    constexpr int cls = kSym.cls[r];
                    constexpr float wr = (float)col_weight(kSym.mem[r][0]);
                    float res = -wr * ds;
                    static_for<(kClass.n[cls] + 3) / 4>([&](auto J4) {
                        constexpr int j4 = decltype(J4)::value;
                        const float4 bw = ld4(T, kTabBs + r * kPadS + 4 * j4);
                        static_for<4>([&](auto K) {
                            constexpr int jj = 4 * j4 + decltype(K)::value;
                            if constexpr (jj < kClass.n[cls]) {
                                constexpr int ib = kClass.member[cls][jj];
                                res = fmaf(f4(bw, decltype(K)::value), a[ib], res);
                            }
                        });
                    });
                    res2 = fmaf(res * (1.0f / nm), res, res2);
                }
            });
            // the cell's own magnitude: rho, rho E, sqrt(rho rho E) for momenta
            float r0, e0;
            if constexpr (VIEW) {
                r0 = __ldg(Qhi + c);
                e0 = __ldg(Qhi + 4 * n + c);
            } else {
                r0 = (float)__ldg(Q + c);
                e0 = (float)__ldg(Q + 4 * n + c);
            }
            const float S = v == 0 ? r0 : (v == 4 ? e0 : sqrtf(fabsf(r0 * e0)));
            const float kap = (float)kGenoKappa;
            const float sig = res2 / (norm2 + kap * kap * S * S + eps);
            const float s = sig * (float)(1.0 / kGenoSigma0);
            chi = 1.0f / (1.0f + s + s * s);
        }
        if (MODE == kModeDump) {
            dump_chi[dump_base + 5 * c + v] = chi;
            return;
        }
        float w[3] = {0.0f, 0.0f, 0.0f};
        float bse = base;
        if (geno) {
            // chi P4 + (1 - chi) P1 (Eq. weno-new), folded into the evaluation
#pragma unroll
            for (int ii = 0; ii < kNumBasis; ++ii) a[ii] *= chi;
            bse = -chi * K;
            const float omc = 1.0f - chi;
#pragma unroll
            for (int q = 0; q < 3; ++q) w[q] = omc * bbar[q];
        }
        eval_faces_f<0>(T, fs, nb, l, v, a, bse, w, geno, ih);
        eval_faces_f<1>(T, fs, nb, l, v, a, bse, w, geno, ih);
        eval_faces_f<2>(T, fs, nb, l, v, a, bse, w, geno, ih);
    }
}

}  // namespace
}  // namespace gks
