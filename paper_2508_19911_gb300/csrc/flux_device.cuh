// Device code of the gas-kinetic flux at one Gauss point (Sec. 2 of the
// paper) and of one face's Gauss points: the FP64 path (flux_point), the
// mixed path (float-float shell, FP32 core: flux_point_mixed) and the
// per-face driver (flux_face_point). Included by flux.cu (the flux kernels)
// and by the translation units whose persistent kernels run a whole time
// step (the ensemble's single-launch step); every includer gets its own
// copy of the constant tables below. See flux.cu for the method.
#pragma once
#include <cmath>

#include "common.cuh"
#include "ff.cuh"

namespace gks {
namespace {


constexpr int kNU = 7;  // <u^0..u^6>
constexpr int kNV = 6;  // <v^0..v^5>

template <int N, typename T>
__device__ __forceinline__ void full_line(T C, T inv2l, T *m) {
    m[0] = 1.0;
    m[1] = C;
#pragma unroll
    for (int k = 0; k + 2 < N; ++k) m[k + 2] = C * m[k + 1] + (k + 1) * inv2l * m[k];
}

// starting values of the half-line moments: sgn = +1 for u > 0, -1 for u < 0.
// With y = sgn sqrt(lam) C and E = exp(-y^2) (which the edge term needs
// anyway), erfc(-y) = erfcx(|y|) E for y <= 0 and 2 - erfcx(|y|) E for
// y > 0 (no cancellation either way): one exponential instead of two.
__device__ __forceinline__ void half_start(double C, double lam, double sgn, double &m0, double &m1) {
    const double rsl = rsqrt(lam), sl = lam * rsl;
    const double y = sgn * sl * C;
    const double E = exp(-lam * C * C);
    const double ec = erfcx(fabs(y)) * E;  // erfc(|y|)
    m0 = 0.5 * (y > 0.0 ? 2.0 - ec : ec);
    const double edge = 0.28209479177387814347 * E * rsl;  // 1/(2 sqrt(pi))
    m1 = C * m0 + sgn * edge;
}

template <int N, typename T>
__device__ __forceinline__ void half_line(T C, T inv2l, T m0, T m1, T *m) {
    m[0] = m0;
    m[1] = m1;
#pragma unroll
    for (int k = 0; k + 2 < N; ++k) m[k + 2] = C * m[k + 1] + (k + 1) * inv2l * m[k];
}

// <u^A v^B w^D psi>
template <int A, int B, int D, typename T>
__device__ __forceinline__ void psi_m(const T *u, const T *v, const T *w, T x2, T o[5]) {
    const T vw = v[B] * w[D];
    const T b = u[A] * vw;
    o[0] = b;
    o[1] = u[A + 1] * vw;
    o[2] = u[A] * v[B + 1] * w[D];
    o[3] = u[A] * v[B] * w[D + 1];
    o[4] = T(0.5) * (u[A + 2] * vw + u[A] * (v[B + 2] * w[D] + v[B] * w[D + 2]) + b * x2);
}

// The symmetric moment matrix G[i][k] = <u^A v^B w^D psi_i psi_k> of one
// Maxwellian (u, v, w its 1D moments, x2 = <xi^2>, x4 = <xi^4>), packed
// (00 01 02 03 04 11 12 13 14 22 23 24 33 34 44). Built once and applied to
// every slope vector that meets the same weight u^A v^B w^D (the three
// directional slopes and A of one side share several), instead of
// re-deriving its entries in every contraction.
template <typename T>
struct Sym5 {
    T g[15];
};

template <int A, int B, int D, typename T>
__device__ __forceinline__ Sym5<T> mom_matrix(const T *u, const T *v, const T *w, T x2, T x4);

__device__ __forceinline__ double mad(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float mad(float a, float b, float c) { return fmaf(a, b, c); }

// The entries with psi_4 = (u^2 + s)/2, s = v^2 + w^2 + xi^2, are
// composed from pieces shared by every matrix of the same Maxwellian (the
// compiler merges identical subexpressions): <v^b w^d s> = sig(b, d) and
// <s^2>, and the half and quarter u-moments, so that
//   <u^a v^b w^d psi_4> = (1/2) u_{a+2} vw_{bd} + (1/2) u_a sig_{bd},
//   <psi_4^2>           = (1/4) u_4 vw + (1/2) u_2 sig + (1/4) u_0 <s^2>.
template <int A, int B, int D, typename T>
__device__ __forceinline__ Sym5<T> mom_matrix(const T *u, const T *v, const T *w, T x2, T x4) {
    auto vw = [&](int b, int d) { return v[B + b] * w[D + d]; };
    auto m = [&](int a, int b, int d) { return u[A + a] * vw(b, d); };
    auto hu = [&](int a) { return T(0.5) * u[A + a]; };
    auto qu = [&](int a) { return T(0.25) * u[A + a]; };
    auto sig = [&](int b, int d) { return mad(x2, vw(b, d), vw(b + 2, d) + vw(b, d + 2)); };
    auto E = [&](int a, int b, int d) { return mad(hu(a + 2), vw(b, d), hu(a) * sig(b, d)); };
    Sym5<T> M;
    M.g[0] = m(0, 0, 0);
    M.g[1] = m(1, 0, 0);
    M.g[2] = m(0, 1, 0);
    M.g[3] = m(0, 0, 1);
    M.g[4] = E(0, 0, 0);
    M.g[5] = m(2, 0, 0);
    M.g[6] = m(1, 1, 0);
    M.g[7] = m(1, 0, 1);
    M.g[8] = E(1, 0, 0);
    M.g[9] = m(0, 2, 0);
    M.g[10] = m(0, 1, 1);
    M.g[11] = E(0, 1, 0);
    M.g[12] = m(0, 0, 2);
    M.g[13] = E(0, 0, 1);
    const T s2 = mad(x4, vw(0, 0),
                     mad(T(2) * x2, vw(2, 0) + vw(0, 2), vw(4, 0) + vw(0, 4) + T(2) * vw(2, 2)));
    M.g[14] = mad(qu(4), vw(0, 0), mad(hu(2), sig(0, 0), qu(0) * s2));
    return M;
}

// acc += G b, one fused multiply-add per matrix entry (the caller scales b:
// the density-weighted slopes are formed once and shared by every matrix
// they meet)
template <typename T>
__device__ __forceinline__ void sym_acc(const Sym5<T> &M, const T b[5], T acc[5]) {
    const T *g = M.g;
    acc[0] = mad(g[4], b[4], mad(g[3], b[3], mad(g[2], b[2], mad(g[1], b[1], mad(g[0], b[0], acc[0])))));
    acc[1] = mad(g[8], b[4], mad(g[7], b[3], mad(g[6], b[2], mad(g[5], b[1], mad(g[1], b[0], acc[1])))));
    acc[2] = mad(g[11], b[4], mad(g[10], b[3], mad(g[9], b[2], mad(g[6], b[1], mad(g[2], b[0], acc[2])))));
    acc[3] = mad(g[13], b[4], mad(g[12], b[3], mad(g[10], b[2], mad(g[7], b[1], mad(g[3], b[0], acc[3])))));
    acc[4] = mad(g[14], b[4], mad(g[13], b[3], mad(g[11], b[2], mad(g[8], b[1], mad(g[4], b[0], acc[4])))));
}

// Slope of a Maxwellian (U, V, W, lam; il = 1/(2 lam)) with N internal
// degrees of freedom: the a with <(a.psi) psi> = d, solved in closed form.
// c4 = 4/(N + 3).
template <typename T>
__device__ __forceinline__ void maxwell_slope(const T d[5], T U, T V, T W, T lam, T il, T N,
                                              T c4, T a[5]) {
    // the state's own factors (shared by every slope of the same state)
    const T q2K = U * U + V * V + W * W + (N + T(3)) * il;
    const T m2U = T(-2) * U, m2V = T(-2) * V, m2W = T(-2) * W;
    const T R1 = d[1] - U * d[0], R2 = d[2] - V * d[0], R3 = d[3] - W * d[0];
    const T R4 = T(2) * d[4] - q2K * d[0];
    a[4] = c4 * lam * lam * mad(m2U, R1, mad(m2V, R2, mad(m2W, R3, R4)));
    a[1] = T(2) * lam * R1 - U * a[4];
    a[2] = T(2) * lam * R2 - V * a[4];
    a[3] = T(2) * lam * R3 - W * a[4];
    a[0] = d[0] - U * a[1] - V * a[2] - W * a[3] - (T(0.5) * q2K) * a[4];
}

// heat flux 1/2 <(u-U0)((u-U0)^2+(v-V0)^2+(w-W0)^2+xi^2)> of a term from its
// flux moments X and conserved moments Y
template <typename T>
__device__ __forceinline__ T heat(const T X[5], const T Y[5], T U0, T V0, T W0) {
    return (X[4] - U0 * Y[4]) - U0 * (X[1] - U0 * Y[1]) - V0 * (X[2] - U0 * Y[2]) -
           W0 * (X[3] - U0 * Y[3]) + T(0.5) * (U0 * U0 + V0 * V0 + W0 * W0) * (X[0] - U0 * Y[0]);
}

// integrals over [0, T] of the six time functions of Eq. flux (see the
// kernel comment in flux_point); the Taylor series below x = T/tau = 1
__device__ __forceinline__ void time_integrals(double T, double tau, double c[6]) {
    if (!(tau > 0.0)) {
        c[0] = T; c[1] = 0.0; c[2] = 0.5 * T * T; c[3] = 0.0; c[4] = 0.0; c[5] = 0.0;
        return;
    }
    const double x = T / tau;
    const double E = -expm1(-x);
    const double t2 = tau * tau;
    if (x < 1.0) {
        // terms to n = 20: x^21/21! < 2e-20 of the smallest sum for x < 1;
        // each step multiplies by the rounded reciprocal 1/n (an FP64
        // division is a multi-instruction sequence, 18 of them per call)
        double term = 0.5 * x * x;  // (-1)^n x^n / n! at n = 2
        double s1 = term, s2 = 0.0, s3 = 0.0;
#pragma unroll
        for (int n = 3; n <= 20; ++n) {
            term *= -x * (1.0 / n);  // 1/n folds to a constant once unrolled
            s1 += term;
            s2 += (n - 2) * term;
            s3 -= term;
        }
        c[0] = tau * s1;
        c[1] = t2 * s2;
        c[2] = t2 * s3;
    } else {
        c[0] = T - tau * E;
        c[1] = 2.0 * t2 * E - tau * T * (2.0 - E);
        c[2] = 0.5 * T * T - tau * T + t2 * E;
    }
    c[3] = tau * E;
    c[4] = -2.0 * t2 * E + tau * T * (1.0 - E);
    c[5] = -t2 * E;
}


// Coefficients of terms 2..6 (k = 1..5) in F^n = sum_k al_k X_k and
// F_t = sum_k be_k X_k, al_k = (4 C_k(dt/2) - C_k(dt))/dt, be_k =
// 4 (C_k(dt) - 2 C_k(dt/2))/dt^2, written out in b = exp(-dt/(2 tau)) and
// a = 1 - b, e.g. al_4 = tau a (3 - b)/dt, be_4 = -4 tau a^2/dt^2, for
// dt >= x_min tau; below, from the time integrals (Taylor series). For small
// x = dt/tau the closed forms of al_1, al_2 cancel to O(x^2) of their terms
// (relative error ~ 1e-16/x^2): x_min = 2 keeps FP64 accuracy, x_min = 0.01
// (1e-12) suffices where the coefficients are rounded to FP32.
__device__ __forceinline__ void time_coefficients(double dt, double tau, double al[6], double be[6],
                                                  double x_min) {
    if (tau > 0.0 && dt >= x_min * tau) {
        const double a = -expm1(-0.5 * dt / tau), b = 1.0 - a;
        const double idt = 1.0 / dt;
        const double t2 = tau * tau;
        const double g = a * (3.0 - b) * idt;          // (4 E_h - E)/dt
        const double h = 4.0 * a * a * idt * idt;      // -4 (E - 2 E_h)/dt^2
        al[1] = 2.0 * t2 * g - tau * (1.0 + 2.0 * b - b * b);
        be[1] = 4.0 * tau * a * (b * dt - 2.0 * tau * a) * idt * idt;
        al[2] = t2 * g - tau;
        be[2] = 1.0 - t2 * h;
        al[3] = tau * g;
        be[3] = -tau * h;
        al[4] = tau * b * (2.0 - b) - 2.0 * t2 * g;
        be[4] = -be[1];
        al[5] = -t2 * g;
        be[5] = t2 * h;
    } else {
        double cA[6], cH[6];
        time_integrals(dt, tau, cA);
        time_integrals(0.5 * dt, tau, cH);
        const double idt = 1.0 / dt, idt2 = idt * idt;
#pragma unroll
        for (int k = 1; k < 6; ++k) {
            al[k] = (4.0 * cH[k] - cA[k]) * idt;
            be[k] = 4.0 * (cA[k] - 2.0 * cH[k]) * idt2;
        }
    }
}

// The closed forms above in FP32 (for the mixed flux, whose coefficients
// meet FP32 moments): for x = dt/tau >= 1/2 their error is at most
// ~1e-7 tau (tau^2/dt for be), FP32 rounding of the coefficients' own
// scale, checked against a 50-digit reference (relative errors of the
// small al_1, al_2 reach 8e-6 at x = 1/2 and grow like 1/x^2 below it).
__device__ __forceinline__ void time_coefficients_f(float dt, float tau, float al[6], float be[6]) {
    const float a = -expm1f(-0.5f * dt / tau), b = 1.0f - a;
    const float idt = 1.0f / dt;
    const float t2 = tau * tau;
    const float g = a * (3.0f - b) * idt;
    const float h = 4.0f * a * a * idt * idt;
    al[1] = 2.0f * t2 * g - tau * (1.0f + 2.0f * b - b * b);
    be[1] = 4.0f * tau * a * (b * dt - 2.0f * tau * a) * idt * idt;
    al[2] = t2 * g - tau;
    be[2] = 1.0f - t2 * h;
    al[3] = tau * g;
    be[3] = -tau * h;
    al[4] = tau * b * (2.0f - b) - 2.0f * t2 * g;
    be[4] = -be[1];
    al[5] = -t2 * g;
    be[5] = t2 * h;
}

template <typename T>
struct PrimT {
    T rho, U, V, W, p, lam;
};
using Prim = PrimT<double>;

__device__ __forceinline__ Prim to_prim(const double *s, double gamma) {
    Prim P;
    P.rho = s[0];
    const double ir = 1.0 / s[0];
    P.U = s[1] * ir;
    P.V = s[2] * ir;
    P.W = s[3] * ir;
    P.p = (gamma - 1.0) * (s[4] - 0.5 * P.rho * (P.U * P.U + P.V * P.V + P.W * P.W));
    P.lam = 0.5 * P.rho / P.p;
    return P;
}

// sum_j <u_j (a_j.psi) psi> of a Maxwellian whose slopes a_j carry the
// derivatives dW/dx_j (ds: d/dn, d/dt1, d/dt2 of the five conserved
// variables): <u_j psi g> is the Euler flux F_j(W), so the sum is
// (1/rho) sum_j dF_j/dW dW/dx_j, written with the flux Jacobians of the
// face frame (velocity (U, V, W), total enthalpy H, gm1 = gamma - 1 =
// 2/(N + 3)) instead of three contractions of full-line moment matrices.
// acc += dF_j/dW d: the Euler flux Jacobian along face-frame direction j
// (velocity vel, k2 = |vel|^2/2, total enthalpy H, gm1 = gamma - 1)
template <typename T>
__device__ __forceinline__ void euler_jac_acc(const T *d, int j, const T vel[3], T k2, T H, T gm1,
                                              T acc[5]) {
    const T c = vel[j];
    const T dp = gm1 * mad(k2, d[0], d[4] - vel[0] * d[1] - vel[1] * d[2] - vel[2] * d[3]);
    const T dmj = d[1 + j];
    acc[0] += dmj;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        acc[1 + i] = mad(vel[i], dmj, mad(c, d[1 + i], mad(-(vel[i] * c), d[0], acc[1 + i])));
        if (i == j) acc[1 + i] += dp;
    }
    acc[4] = mad(c, d[4] + dp, mad(H, mad(-c, d[0], dmj), acc[4]));
}

// sum_j <u_j (a_j.psi) psi> of a Maxwellian whose slopes a_j carry the
// derivatives dW/dx_j (ds: d/dn, d/dt1, d/dt2 of the five conserved
// variables): <u_j psi g> is the Euler flux F_j(W), so the sum is
// (1/rho) sum_j dF_j/dW dW/dx_j, written with the flux Jacobians of the
// face frame (gm1 = gamma - 1 = 2/(N + 3)) instead of three contractions
// of full-line moment matrices.
template <typename T>
__device__ __forceinline__ void euler_rate(const T *ds, T ir, T U, T V, T W, T H, T gm1,
                                           T out[5]) {
    const T vel[3] = {U, V, W};
    const T k2 = T(0.5) * (U * U + V * V + W * W);
    T acc[5] = {0, 0, 0, 0, 0};
#pragma unroll
    for (int j = 0; j < 3; ++j) euler_jac_acc(ds + 5 * j, j, vel, k2, H, gm1, acc);
#pragma unroll
    for (int i = 0; i < 5; ++i) out[i] = acc[i] * ir;
}

// Contribution of one side (SGN = +1: left state over u > 0; -1: right
// state over u < 0) to W0's slopes and to terms 4-6 of Eq. flux.
// ds: the 15 derivatives d/dn, d/dt1, d/dt2 of the 5 conserved variables.
template <int SGN, typename T>
__device__ __forceinline__ void side_terms(const T *ds, const PrimT<T> &S, T N, T c4, T uh0, T uh1,
                                           T U0, T V0, T W0, T dW0[3][5], T X4[5], T X5acc[5],
                                           T X6[5], T q[3], T dtW[5]) {
    const T ir = T(1) / S.rho;
    const T inv2l = S.p * ir;  // 1/(2 lam)
    T uh[kNU], v[kNV], w[kNV];
    half_line<kNU>(S.U, inv2l, uh0, uh1, uh);
    full_line<kNV>(S.V, inv2l, v);
    full_line<kNV>(S.W, inv2l, w);
    const T x2 = N * inv2l, x4 = (N * N + T(2) * N) * inv2l * inv2l;
    // one-sided Maxwellian slopes a_j
    T a[3][5];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        T d[5];
#pragma unroll
        for (int i = 0; i < 5; ++i) d[i] = ds[5 * j + i] * ir;
        maxwell_slope(d, S.U, S.V, S.W, S.lam, inv2l, N, c4, a[j]);
    }
    // A from the compatibility condition: <(A.psi) psi> = -<(a.u) psi>
    // (full line): the Euler flux Jacobians applied to the derivatives
    T Tv[5], A[5];
    euler_rate(ds, ir, S.U, S.V, S.W, mad(T(0.5) * (N + T(5)), inv2l,
                                          T(0.5) * (S.U * S.U + S.V * S.V + S.W * S.W)),
               T(0.5) * c4, Tv);
    {
        T mT[5];
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            mT[i] = -Tv[i];
            dtW[i] = -S.rho * Tv[i];  // Euler time derivative of W_s
        }
        maxwell_slope(mT, S.U, S.V, S.W, S.lam, inv2l, N, c4, A);
    }
    // every later contraction weighs the slopes with rho: scale them once
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        a[0][i] *= S.rho;
        a[1][i] *= S.rho;
        a[2][i] *= S.rho;
        A[i] *= S.rho;
    }
    // half line, weight 1: the slopes of the interface equilibrium (collected
    // from both sides), term 4 (g_s: rows 1 and 0 of its matrix are
    // <u psi>, <psi>) and term 6's conserved moments <(A.psi) psi>
    T X[5], Y[5], X5[5] = {0, 0, 0, 0, 0}, Y5[5] = {0, 0, 0, 0, 0}, Y6[5] = {0, 0, 0, 0, 0};
    {
        const Sym5<T> H = mom_matrix<0, 0, 0>(uh, v, w, x2, x4);
#pragma unroll
        for (int j = 0; j < 3; ++j) sym_acc(H, a[j], dW0[j]);
        sym_acc(H, A, Y6);
        const T r1[5] = {H.g[1], H.g[5], H.g[6], H.g[7], H.g[8]};
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            X[i] = S.rho * r1[i];
            Y[i] = S.rho * H.g[i];
            X4[i] += X[i];
        }
        q[0] += heat(X, Y, U0, V0, W0);
    }
    // weight u: term 6's flux moments <(A.psi) u psi> and the first
    // directional part of term 5's conserved moments
#pragma unroll
    for (int i = 0; i < 5; ++i) X[i] = T(0);
    {
        const Sym5<T> H = mom_matrix<1, 0, 0>(uh, v, w, x2, x4);
        sym_acc(H, A, X);
        sym_acc(H, a[0], Y5);
    }
#pragma unroll
    for (int i = 0; i < 5; ++i) X6[i] += X[i];
    q[2] += heat(X, Y6, U0, V0, W0);
    // term 5: (a.u) g_s = sum_j (a_j.psi) c_j g_s
    sym_acc(mom_matrix<0, 1, 0>(uh, v, w, x2, x4), a[1], Y5);
    sym_acc(mom_matrix<0, 0, 1>(uh, v, w, x2, x4), a[2], Y5);
    sym_acc(mom_matrix<2, 0, 0>(uh, v, w, x2, x4), a[0], X5);
    sym_acc(mom_matrix<1, 1, 0>(uh, v, w, x2, x4), a[1], X5);
    sym_acc(mom_matrix<1, 0, 1>(uh, v, w, x2, x4), a[2], X5);
    q[1] += heat(X5, Y5, U0, V0, W0);
#pragma unroll
    for (int i = 0; i < 5; ++i) X5acc[i] += X5[i];
}

// Equilibrium part: abar from the collided slopes dW0, Abar by
// compatibility; X1..X3 (term 1 only if kTerm1), q1..q3, dW0/dt.
template <bool kTerm1, typename T>
__device__ __forceinline__ void equilibrium_terms(const PrimT<T> &Z, T N, T c4, const T dW0[3][5],
                                                  T X[6][5], T q[6], T dtW0[5]) {
    const T ir = T(1) / Z.rho;
    const T inv2l = Z.p * ir;  // 1/(2 lam)
    T u[kNU], v[kNV], w[kNV];
    full_line<kNU>(Z.U, inv2l, u);
    full_line<kNV>(Z.V, inv2l, v);
    full_line<kNV>(Z.W, inv2l, w);
    const T x2 = N * inv2l, x4 = (N * N + T(2) * N) * inv2l * inv2l;
    T ab[3][5];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        T d[5];
#pragma unroll
        for (int i = 0; i < 5; ++i) d[i] = dW0[j][i] * ir;
        maxwell_slope(d, Z.U, Z.V, Z.W, Z.lam, inv2l, N, c4, ab[j]);
    }
    // T0 = sum_j <u_j (abar_j.psi) psi>: the Euler flux Jacobians of W0
    // applied to its collided slopes dW0 (see euler_rate)
    const T H0 = mad(T(0.5) * (N + T(5)), inv2l, T(0.5) * (Z.U * Z.U + Z.V * Z.V + Z.W * Z.W));
    T T0[5];
    euler_rate(&dW0[0][0], ir, Z.U, Z.V, Z.W, H0, T(0.5) * c4, T0);
    // rho0-weighted slopes for the flux moments of term 2
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        ab[0][i] *= Z.rho;
        ab[1][i] *= Z.rho;
        ab[2][i] *= Z.rho;
    }
    T Y[5];
    if (kTerm1) {
        // term 1: g0 (rows 1 and 0 of its moment matrix: <u psi>, <psi>)
        const Sym5<T> F0 = mom_matrix<0, 0, 0>(u, v, w, x2, x4);
        const T r1[5] = {F0.g[1], F0.g[5], F0.g[6], F0.g[7], F0.g[8]};
#pragma unroll
        for (int i = 0; i < 5; ++i) { X[0][i] = Z.rho * r1[i]; Y[i] = Z.rho * F0.g[i]; }
        q[0] = heat(X[0], Y, Z.U, Z.V, Z.W);
    }
    // term 2: (abar.u) g0; its conserved moments are rho0 T0
    sym_acc(mom_matrix<2, 0, 0>(u, v, w, x2, x4), ab[0], X[1]);
    sym_acc(mom_matrix<1, 1, 0>(u, v, w, x2, x4), ab[1], X[1]);
    sym_acc(mom_matrix<1, 0, 1>(u, v, w, x2, x4), ab[2], X[1]);
#pragma unroll
    for (int i = 0; i < 5; ++i) Y[i] = Z.rho * T0[i];
    q[1] = heat(X[1], Y, Z.U, Z.V, Z.W);
    // term 3: Abar g0 with <(Abar.psi) psi> = -T0 (compatibility): its
    // conserved moments are dW0/dt = -rho0 T0 and its flux moments
    // <u (Abar.psi) psi g0> = dF_n/dW dW0/dt (the normal flux Jacobian)
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        Y[i] = -Z.rho * T0[i];
        dtW0[i] = Y[i];
    }
    {
        const T vel[3] = {Z.U, Z.V, Z.W};
        euler_jac_acc(dtW0, 0, vel, T(0.5) * (Z.U * Z.U + Z.V * Z.V + Z.W * Z.W), H0,
                      T(0.5) * c4, X[2]);
    }
    q[2] = heat(X[2], Y, Z.U, Z.V, Z.W);
}

// W0 = rho_l <psi>_{u>0} + rho_r <psi>_{u<0} and the half-line starting
// moments of both sides
__device__ __forceinline__ void interface_state(const Prim &L, const Prim &R, double N,
                                                double W0[5], double &ul0, double &ul1,
                                                double &ur0, double &ur1) {
    half_start(L.U, L.lam, 1.0, ul0, ul1);
    half_start(R.U, R.lam, -1.0, ur0, ur1);
    double u[4], v[3], w[3], o[5];
    const double il = L.p * (1.0 / L.rho), ir = R.p * (1.0 / R.rho);  // 1/(2 lam)
    half_line<4>(L.U, il, ul0, ul1, u);
    full_line<3>(L.V, il, v);
    full_line<3>(L.W, il, w);
    psi_m<0, 0, 0>(u, v, w, N * il, o);
#pragma unroll
    for (int i = 0; i < 5; ++i) W0[i] = L.rho * o[i];
    half_line<4>(R.U, ir, ur0, ur1, u);
    full_line<3>(R.V, ir, v);
    full_line<3>(R.W, ir, w);
    psi_m<0, 0, 0>(u, v, w, N * ir, o);
#pragma unroll
    for (int i = 0; i < 5; ++i) W0[i] += R.rho * o[i];
}

// collision time (Sec. 4) and F^n, F_t^n from the six term moments: the
// coefficients al_k, be_k of time_coefficients (closed forms for
// dt >= 2 tau, the time-integral series below), with al_1 = 1 - al_4 and
// be_1 = -be_4 (the time functions of terms 1 and 4 add up to 1)
__device__ __forceinline__ void combine_terms(const PhysParams &P, const Prim &L, const Prim &R,
                                              const Prim &Z, double dt, const double X[6][5],
                                              const double q[6], double out[10], double &dpr) {
    dpr = fabs((L.p - R.p) / (L.p + R.p));
    const double tau = P.inviscid ? (P.eps_tau * dt + P.C_tau * dpr * dt)
                                  : (viscosity(P, Z.rho, Z.p) / Z.p + P.C_tau * dpr * dt);
    double al[6], be[6];
    time_coefficients(dt, tau, al, be, 2.0);
    al[0] = 1.0 - al[3];
    be[0] = -be[3];
    const double prfix = 1.0 / P.Pr - 1.0;
    double qn = 0.0, qt = 0.0;
#pragma unroll
    for (int i = 0; i < 10; ++i) out[i] = 0.0;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            out[i] += al[k] * X[k][i];
            out[5 + i] += be[k] * X[k][i];
        }
        qn += al[k] * q[k];
        qt += be[k] * q[k];
    }
    out[4] += prfix * qn;
    out[9] += prfix * qt;
}

// The gas-kinetic flux at one Gauss point, face frame.
//   out[0..4]  F^n, out[5..9] F_t^n,
//   out[10..29] (kInterface) Q^l, dQ^l/dt, Q^r, dQ^r/dt of Sec. 3.4.
// Eq. flux has six terms with time functions
//   c1 = 1 - e^{-t/tau} (g0), c2 = (t+tau) e^{-t/tau} - tau ((abar.u) g0),
//   c3 = t - tau + tau e^{-t/tau} (Abar g0), c4 = e^{-t/tau} (g_l H + g_r (1-H)),
//   c5 = -(tau+t) e^{-t/tau} ((a.u) g_{l,r}), c6 = -tau e^{-t/tau} (A g_{l,r});
// with X_k their flux moments, fbar(T) = sum_k C_k(T) X_k (C_k the time
// integrals) and F^n = (4 fbar(dt/2) - fbar(dt))/dt,
// F_t^n = 4 (fbar(dt) - 2 fbar(dt/2))/dt^2.
template <bool kInterface>
__device__ void flux_point(const PhysParams &P, const double *sl, const double *sr, double dt,
                           double out[30], int *status) {
    const double N = P.Nint;
    const Prim L = to_prim(sl, P.gamma), R = to_prim(sr, P.gamma);
    if (!(L.rho > 0.0 && L.p > 0.0 && R.rho > 0.0 && R.p > 0.0)) {
        flag_status(status, kStatusNonphysical);
#pragma unroll
        for (int i = 0; i < 30; ++i) out[i] = nan("");
        return;
    }
    double W0[5], ul0, ul1, ur0, ur1;
    interface_state(L, R, N, W0, ul0, ul1, ur0, ur1);
    const Prim Z = to_prim(W0, P.gamma);
    if (!(Z.rho > 0.0 && Z.p > 0.0)) {
        flag_status(status, kStatusNonphysical);
#pragma unroll
        for (int i = 0; i < 30; ++i) out[i] = nan("");
        return;
    }
    double dW0[3][5], X[6][5], q[6] = {0, 0, 0, 0, 0, 0}, dtWl[5], dtWr[5], dtW0[5];
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int i = 0; i < 5; ++i) dW0[j][i] = 0.0;
#pragma unroll
    for (int k = 0; k < 6; ++k)
#pragma unroll
        for (int i = 0; i < 5; ++i) X[k][i] = 0.0;
    const double c4 = 4.0 / (N + 3.0);
    side_terms<1>(sl + 5, L, N, c4, ul0, ul1, Z.U, Z.V, Z.W, dW0, X[3], X[4], X[5], q + 3, dtWl);
    side_terms<-1>(sr + 5, R, N, c4, ur0, ur1, Z.U, Z.V, Z.W, dW0, X[3], X[4], X[5], q + 3, dtWr);
    equilibrium_terms<true>(Z, N, c4, dW0, X, q, dtW0);
    double dpr;
    combine_terms(P, L, R, Z, dt, X, q, out, dpr);
    if (kInterface) {
        const double e = (P.C_tau * dpr > 0.0) ? exp(-1.0 / (P.C_tau * dpr)) : 0.0;
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            out[10 + i] = (1.0 - e) * W0[i] + e * sl[i];
            out[15 + i] = (1.0 - e) * dtW0[i] + e * dtWl[i];
            out[20 + i] = (1.0 - e) * W0[i] + e * sr[i];
            out[25 + i] = (1.0 - e) * dtW0[i] + e * dtWr[i];
        }
    }
}

// ---- mixed precision: float-float shell, FP32 core ----------------------
// Of the six terms of Eq. flux only three quantities need more than FP32:
// the interface equilibrium W0 (its pressure enters the Euler flux), the
// Euler flux X1 of W0 (term 1, which carries the pressure), and the
// difference D = X1 - X4 with X4 the half-space flux of the initial states
// (term 4): the time coefficients of terms 1 and 4 satisfy al1 + al4 = 1
// and be1 + be4 = 0 exactly (the time functions c1 + c4 integrate to T), so
//   F^n  = X1 - al4 D + sum_{k=2,3,5,6} al_k X_k,
//   F_t^n =    - be4 D + sum_{k=2,3,5,6} be_k X_k,
// and D is small where the flow is smooth. These three are computed in
// float-float arithmetic (ff.cuh) from W = Q0 + offset, with the half-line
// starting values erfc and exp from a float-float series (FP64 beyond its
// range); the slopes and moments of terms 2, 3, 5, 6 are the FP32 core
// shared with the FP64 kernel's templates. The float-float sums are the
// like-term form (error 2^-46 of the operands' magnitudes, not of the
// result): what matters here is the error against each quantity's own
// scale (rho, rho E, their fluxes), never relative to a small result of
// a cancellation, except 1 - erf (a half-space weight), which keeps the
// full float-float subtraction.
struct PrimFF {
    ff rho, U, V, W, p, lam, il;  // il = 1/(2 lam) = p/rho
};

__device__ __forceinline__ ff ff_half(ff a) { return ff_make(0.5f * a.hi, 0.5f * a.lo); }

__device__ __forceinline__ PrimFF to_prim_ff(const ff s[5], ff gm1) {
    PrimFF P;
    P.rho = s[0];
    const ff ir = ff_recip(s[0]);
    P.U = ff_mul(s[1], ir);
    P.V = ff_mul(s[2], ir);
    P.W = ff_mul(s[3], ir);
    const ff q2 = ff_add_like(ff_add_like(ff_mul(P.U, P.U), ff_mul(P.V, P.V)), ff_mul(P.W, P.W));
    P.p = ff_mul(gm1, ff_sub_like(s[4], ff_half(ff_mul(P.rho, q2))));
    P.il = ff_mul(P.p, ir);
    // lam only feeds the FP32 core (the half-line start uses il)
    P.lam = ff_make(__fdividef(0.5f * P.rho.hi, P.p.hi), 0.0f);
    return P;
}

// Half-line starting moments of one side (sgn = +1: u > 0; -1: u < 0):
// with y = sqrt(lam) U, m0 = (1 + sgn erf(y))/2 and m1 = U m0 + sgn
// e^{-y^2}/(2 sqrt(pi lam)). For |y| <= 2 (every state below a component
// Mach number of ~2.4) erf and the exponential come from one series in
// t_n = (-y^2)^n/n!: e^{-y^2} = sum t_n, erf(y) = 2y/sqrt(pi) sum t_n/(2n+1),
// in float-float (|t_n| <= 4^n/n!: 32 terms reach 2^-53; the largest term,
// 10.7 at n = 4, costs one digit to cancellation); otherwise the FP64 erfc
// and exp.
constexpr int kSeriesTerms = 32;
// 1/n and 1/(2n+1), n = 0..32, as float-float constants (the series loop is
// not unrolled: the kernel's instruction footprint, not its arithmetic,
// stalled the mixed flux)
__constant__ ffc cSeriesInv[kSeriesTerms + 1] = {
    ff_const(0.0), ff_const(1.0 / 1), ff_const(1.0 / 2), ff_const(1.0 / 3),
    ff_const(1.0 / 4), ff_const(1.0 / 5), ff_const(1.0 / 6), ff_const(1.0 / 7),
    ff_const(1.0 / 8), ff_const(1.0 / 9), ff_const(1.0 / 10), ff_const(1.0 / 11),
    ff_const(1.0 / 12), ff_const(1.0 / 13), ff_const(1.0 / 14), ff_const(1.0 / 15),
    ff_const(1.0 / 16), ff_const(1.0 / 17), ff_const(1.0 / 18), ff_const(1.0 / 19),
    ff_const(1.0 / 20), ff_const(1.0 / 21), ff_const(1.0 / 22), ff_const(1.0 / 23),
    ff_const(1.0 / 24), ff_const(1.0 / 25), ff_const(1.0 / 26), ff_const(1.0 / 27),
    ff_const(1.0 / 28), ff_const(1.0 / 29), ff_const(1.0 / 30), ff_const(1.0 / 31),
    ff_const(1.0 / 32)};
__constant__ ffc cSeriesInvOdd[kSeriesTerms + 1] = {
    ff_const(1.0 / 1), ff_const(1.0 / 3), ff_const(1.0 / 5), ff_const(1.0 / 7),
    ff_const(1.0 / 9), ff_const(1.0 / 11), ff_const(1.0 / 13), ff_const(1.0 / 15),
    ff_const(1.0 / 17), ff_const(1.0 / 19), ff_const(1.0 / 21), ff_const(1.0 / 23),
    ff_const(1.0 / 25), ff_const(1.0 / 27), ff_const(1.0 / 29), ff_const(1.0 / 31),
    ff_const(1.0 / 33), ff_const(1.0 / 35), ff_const(1.0 / 37), ff_const(1.0 / 39),
    ff_const(1.0 / 41), ff_const(1.0 / 43), ff_const(1.0 / 45), ff_const(1.0 / 47),
    ff_const(1.0 / 49), ff_const(1.0 / 51), ff_const(1.0 / 53), ff_const(1.0 / 55),
    ff_const(1.0 / 57), ff_const(1.0 / 59), ff_const(1.0 / 61), ff_const(1.0 / 63),
    ff_const(1.0 / 65)};

__device__ __forceinline__ void half_start_ff(const PrimFF &S, int sgn, ff &m0, ff &m1) {
    const ff isl = ff_sqrt(ff_make(2.0f * S.il.hi, 2.0f * S.il.lo));  // 1/sqrt(lam), exact doubling
    const ff y = ff_mul(S.U, ff_recip(isl));
    if (fabsf(y.hi) <= 2.0f) {
        const ff w = ff_neg(ff_mul(y, y));
        ff t = ff_make(1.0f, 0.0f), se = t, sf = t;
#pragma unroll 1
        for (int n = 1; n <= kSeriesTerms; ++n) {
            t = ff_mul(ff_mul(t, w), ff_of(cSeriesInv[n]));
            se = ff_add_like(se, t);
            sf = ff_add_like(sf, ff_mul(t, ff_of(cSeriesInvOdd[n])));
            if (fabsf(t.hi) < 1e-16f) break;
        }
        constexpr ffc k2rpi = ff_const(1.1283791670955125739);   // 2/sqrt(pi)
        constexpr ffc krpi = ff_const(0.56418958354775628695);   // 1/sqrt(pi)
        const ff erf = ff_mul(ff_mul(y, ff_of(k2rpi)), sf);
        m0 = ff_half(sgn > 0 ? ff_add_f(erf, 1.0f) : ff_sub(ff_make(1.0f, 0.0f), erf));
        const ff edge = ff_half(ff_mul(ff_mul(se, ff_of(krpi)), isl));
        m1 = sgn > 0 ? ff_add_like(ff_mul(S.U, m0), edge) : ff_sub_like(ff_mul(S.U, m0), edge);
    } else {
        double d0, d1;
        half_start(ff_to_double(S.U), 0.5 / ff_to_double(S.il), (double)sgn, d0, d1);
        m0 = ff_from_double(d0);
        m1 = ff_from_double(d1);
    }
}

// rho <psi> and rho <u psi> of one side over its half line, added to W0 and
// X4; returns the half-line starting moments for the FP32 core
__device__ __forceinline__ void half_side_ff(const PrimFF &S, int sgn, ff N, ff W0[5], ff X4[5],
                                             float &m0f, float &m1f) {
    ff u[4];
    half_start_ff(S, sgn, u[0], u[1]);
    m0f = u[0].hi;
    m1f = u[1].hi;
    const ff inv2l = S.il;
    u[2] = ff_add_like(ff_mul(S.U, u[1]), ff_mul(inv2l, u[0]));
    u[3] = ff_add_like(ff_mul(S.U, u[2]), ff_mul(ff_add_like(inv2l, inv2l), u[1]));
    // <v^2> + <w^2> + <xi^2> of the full lines
    const ff s2 = ff_add_like(ff_add_like(ff_mul(S.V, S.V), ff_mul(S.W, S.W)),
                         ff_mul(ff_add_f(N, 2.0f), inv2l));
#pragma unroll
    for (int A = 0; A < 2; ++A) {
        ff o[5];
        o[0] = u[A];
        o[1] = u[A + 1];
        o[2] = ff_mul(u[A], S.V);
        o[3] = ff_mul(u[A], S.W);
        o[4] = ff_half(ff_add_like(u[A + 2], ff_mul(u[A], s2)));
        ff *acc = A == 0 ? W0 : X4;
#pragma unroll
        for (int i = 0; i < 5; ++i) acc[i] = ff_add_like(acc[i], ff_mul(S.rho, o[i]));
    }
}

__device__ __forceinline__ PrimT<float> prim_f(const PrimFF &P) {
    PrimT<float> f;
    f.rho = P.rho.hi; f.U = P.U.hi; f.V = P.V.hi; f.W = P.W.hi; f.p = P.p.hi; f.lam = P.lam.hi;
    return f;
}

// One Gauss point's record in float-float: F^n, F_t^n and, with
// kInterface, Q^l, dQ^l/dt, Q^r, dQ^r/dt (out[0..29], face frame); the
// FP32 entries have lo = 0.
// Ql, Qr: the two cells' FP64 averages as float-float pairs (exact splits)
template <bool kInterface>
__device__ void flux_point_mixed(const PhysParams &P, const ff Ql[5], const float ol[5],
                                 const float dl[15], const ff Qr[5], const float orr[5],
                                 const float dr[15], double dt, ff out[30], int *status) {
    const ff gm1 = ff_from_double(P.gamma - 1.0);
    const ff N = ff_from_double(P.Nint);
    ff Wl[5], Wr[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        Wl[i] = ff_add_f(Ql[i], ol[i]);
        Wr[i] = ff_add_f(Qr[i], orr[i]);
    }
    const PrimFF L = to_prim_ff(Wl, gm1), R = to_prim_ff(Wr, gm1);
    if (!(L.rho.hi > 0.0f && L.p.hi > 0.0f && R.rho.hi > 0.0f && R.p.hi > 0.0f)) {
        flag_status(status, kStatusNonphysical);
#pragma unroll
        for (int i = 0; i < 30; ++i) out[i] = ff_make(nanf(""), 0.0f);
        return;
    }
    ff W0[5], X4[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) W0[i] = X4[i] = ff_make(0.0f, 0.0f);
    float ul0, ul1, ur0, ur1;
    half_side_ff(L, 1, N, W0, X4, ul0, ul1);
    half_side_ff(R, -1, N, W0, X4, ur0, ur1);
    const PrimFF Z = to_prim_ff(W0, gm1);
    if (!(Z.rho.hi > 0.0f && Z.p.hi > 0.0f)) {
        flag_status(status, kStatusNonphysical);
#pragma unroll
        for (int i = 0; i < 30; ++i) out[i] = ff_make(nanf(""), 0.0f);
        return;
    }
    // term 1: the Euler flux of W0; D = X1 - X4
    ff X1[5];
    X1[0] = W0[1];
    X1[1] = ff_add_like(ff_mul(W0[1], Z.U), Z.p);
    X1[2] = ff_mul(W0[2], Z.U);
    X1[3] = ff_mul(W0[3], Z.U);
    X1[4] = ff_mul(ff_add_like(W0[4], Z.p), Z.U);
    float D[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) D[i] = ff_sub_like(X1[i], X4[i]).hi;

    // FP32 core: slopes and the moments of terms 2, 3, 5, 6 (and the heat
    // fluxes for the Prandtl fix)
    const float Nf = N.hi, c4f = 4.0f / (Nf + 3.0f);
    const PrimT<float> Lf = prim_f(L), Rf = prim_f(R), Zf = prim_f(Z);
    float dW0[3][5], X[6][5], q[6] = {0, 0, 0, 0, 0, 0}, dtWl[5], dtWr[5], dtW0[5];
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int i = 0; i < 5; ++i) dW0[j][i] = 0.0f;
#pragma unroll
    for (int k = 0; k < 6; ++k)
#pragma unroll
        for (int i = 0; i < 5; ++i) X[k][i] = 0.0f;
    // both sides through one copy of the code (left, then right: the order
    // of two inlined calls); the kernel is bound by instruction issue and
    // fetch, and one copy of the side terms halves their footprint
#pragma unroll 1
    for (int side = 0; side < 2; ++side) {
        float ds[15], dtW[5];
#pragma unroll
        for (int i = 0; i < 15; ++i) ds[i] = side ? dr[i] : dl[i];
        const PrimT<float> S = side ? Rf : Lf;
        side_terms<1>(ds, S, Nf, c4f, side ? ur0 : ul0, side ? ur1 : ul1, Zf.U, Zf.V, Zf.W, dW0, X[3],
                      X[4], X[5], q + 3, dtW);
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            if (side) dtWr[i] = dtW[i];
            else dtWl[i] = dtW[i];
        }
    }
    equilibrium_terms<false>(Zf, Nf, c4f, dW0, X, q, dtW0);  // a Maxwellian carries no heat flux: q1 = 0

    // collision time (Sec. 4) in FP32; time coefficients in FP32 for
    // dt >= tau/2, else from the FP64 closed forms (dt >= tau/100) or series
    const float dpr = fabsf(ff_sub_like(L.p, R.p).hi / ff_add_like(L.p, R.p).hi);
    const float dtf = (float)dt;
    float tau;
    if (P.inviscid) {
        tau = ((float)P.eps_tau + (float)P.C_tau * dpr) * dtf;
    } else {
        float mu = (float)P.mu0;
        if (P.mu_law) {
            const float th = (Zf.p / Zf.rho) / (float)P.T_ref;
            mu *= 1.4042f * th * sqrtf(th) / (th + 0.4042f);
        }
        tau = mu / Zf.p + (float)P.C_tau * dpr * dtf;
    }
    float al[6], be[6];
    if (tau > 0.0f && dtf >= 0.5f * tau) {
        time_coefficients_f(dtf, tau, al, be);
    } else {
        double ald[6], bed[6];
        time_coefficients(dt, (double)tau, ald, bed, 0.01);
#pragma unroll
        for (int k = 1; k < 6; ++k) {
            al[k] = (float)ald[k];
            be[k] = (float)bed[k];
        }
    }
    const float prfix = (float)(1.0 / P.Pr - 1.0);
    float qn = 0.0f, qt = 0.0f;
#pragma unroll
    for (int k = 1; k < 6; ++k) {
        qn = fmaf(al[k], q[k], qn);
        qt = fmaf(be[k], q[k], qt);
    }
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        float cf = -al[3] * D[i], ct = -be[3] * D[i];
#pragma unroll
        for (int k = 1; k < 6; ++k) {
            if (k == 3) continue;
            cf = fmaf(al[k], X[k][i], cf);
            ct = fmaf(be[k], X[k][i], ct);
        }
        if (i == 4) {
            cf = fmaf(prfix, qn, cf);
            ct = fmaf(prfix, qt, ct);
        }
        out[i] = ff_add_f(X1[i], cf);
        out[5 + i] = ff_make(ct, 0.0f);
    }
    if (kInterface) {
        const float cd = (float)P.C_tau * dpr;
        const float e = cd > 0.0f ? expf(-1.0f / cd) : 0.0f;
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            out[10 + i] = ff_add_f(W0[i], e * ff_sub_like(Wl[i], W0[i]).hi);
            out[15 + i] = ff_make((1.0f - e) * dtW0[i] + e * dtWl[i], 0.0f);
            out[20 + i] = ff_add_f(W0[i], e * ff_sub_like(Wr[i], W0[i]).hi);
            out[25 + i] = ff_make((1.0f - e) * dtW0[i] + e * dtWr[i], 0.0f);
        }
    }
}

// face-frame component c of conserved variable v on a face normal to axis d
__device__ __forceinline__ int global_var(int c, int d) {
    return (c == 0 || c == 4) ? c : 1 + (d + c - 1) % 3;
}

// Flux at Gauss point k of the face on the low-d side of cell c, reduced
// over the face's K Gauss points (lanes 4m..4m+3 hold the points of one
// face; all 32 lanes of the warp must call this together) and written to
// the face records. MIXED: FP32 face-state offsets + FP64 averages Q.
// l: the right cell's position in the face-state buffer S (the face is its
// low face along d); face states are read at buffer positions (stride
// S.nb), the averages Q and the records at global cells (stride g.n).
// mixed: the averages as float-float pairs Qhi, Qlo ([5][n] each, written
// once per stage by q_to_ff_kernel)
// bmode (general grids): 0 an interior face; 1 the low boundary face of a
// non-periodic axis (the cell's own low face state and its mirror ghost);
// 2 the high boundary face of cell l (its high face state and its mirror),
// written to the boundary records after the [3][30][n] records.
template <bool kCGKS, bool MIXED>
__device__ __forceinline__ void flux_face_point(const GridDesc &g, const Slab &S,
                                                const PhysParams &P,
                                                const void *__restrict__ fsv,
                                                const float *__restrict__ Qhi,
                                                const float *__restrict__ Qlo, double dt,
                                                double *__restrict__ frec, int *status, int d,
                                                long long l, int k, bool valid, int bmode = 0) {
    constexpr int K = kCGKS ? 4 : 1;
    const long long n = g.n, nb = S.nb;
    const long long nxy = (long long)g.nx * g.ny;
    const int p = (int)(l / nxy);
    const long long ij = l - (long long)p * nxy;
    const int i = (int)(ij % g.nx), j = (int)(ij / g.nx);
    const int gz = (S.zb + p) % g.nz;
    const long long c = (long long)gz * nxy + ij;  // global right cell
    long long ll, left;                            // left cell: buffer position, global
    if (d == 0) {
        const long long o = (long long)j * g.nx + wrap(i - 1, g.nx);
        ll = (long long)p * nxy + o;
        left = (long long)gz * nxy + o;
    } else if (d == 1) {
        const long long o = (long long)wrap(j - 1, g.ny) * g.nx + i;
        ll = (long long)p * nxy + o;
        left = (long long)gz * nxy + o;
    } else {
        ll = (long long)(p > 0 ? p - 1 : S.nzb - 1) * nxy + ij;
        left = (long long)wrap(gz - 1, g.nz) * nxy + ij;
    }
    constexpr int NV = kCGKS ? 30 : 10;
    // the record's position: the right cell's low face, or a high boundary face
    const long long rec_base = bmode == 2 ? 90 * n + plane_pos(g, d, i, j, gz) : c;
    const long long rec_stride = bmode == 2 ? g.np : n;
    if (bmode == 2) ll = l;  // the face state on the cell's high side
    if (!MIXED) {
        double out[30];
        const double *fs = (const double *)fsv;
        double sl[20], sr[20];
        const double *pl = fs + ((long long)((2 * d + 1) * K + k) * 20) * nb + ll;
        const double *pr = fs + ((long long)((2 * d) * K + k) * 20) * nb + l;
#pragma unroll
        for (int q = 0; q < 20; ++q) {
            sl[q] = __ldg(pl + (long long)q * nb);
            sr[q] = __ldg(pr + (long long)q * nb);
        }
        if (bmode == 1) {
#pragma unroll
            for (int q = 0; q < 20; ++q) sl[q] = mirror_neg(q, g.bc[d]) ? -sr[q] : sr[q];
        } else if (bmode == 2) {
#pragma unroll
            for (int q = 0; q < 20; ++q) sr[q] = mirror_neg(q, g.bc[d]) ? -sl[q] : sl[q];
        }
        flux_point<kCGKS>(P, sl, sr, dt, out, valid ? status : nullptr);
        if (kCGKS) {
            // Gauss-point average: butterfly over the four lanes of the face
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                double s = out[q] + __shfl_xor_sync(0xffffffffu, out[q], 1);
                s = s + __shfl_xor_sync(0xffffffffu, s, 2);
                out[q] = 0.25 * s;
            }
        }
        if (!valid) return;
        // face frame -> global frame; lane k writes the values with q % K == k
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            if (q % K != k) continue;
            const int blk = q / 5, cmp = q % 5;
            frec[((long long)d * 30 + blk * 5 + global_var(cmp, d)) * rec_stride + rec_base] = out[q];
        }
    } else {
        ff out[30];
        const float *fs = (const float *)fsv;
        ff Ql[5], Qr[5];
        float ol[5], orr[5], dl[15], dr[15];
        const float *pl = fs + ((long long)((2 * d + 1) * K + k) * 20) * nb + ll;
        const float *pr = fs + ((long long)((2 * d) * K + k) * 20) * nb + l;
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            const int v = global_var(q, d);
            Ql[q] = ff_make(__ldg(Qhi + (long long)v * n + left), __ldg(Qlo + (long long)v * n + left));
            Qr[q] = ff_make(__ldg(Qhi + (long long)v * n + c), __ldg(Qlo + (long long)v * n + c));
            ol[q] = __ldg(pl + (long long)q * nb);
            orr[q] = __ldg(pr + (long long)q * nb);
        }
#pragma unroll
        for (int q = 0; q < 15; ++q) {
            dl[q] = __ldg(pl + (long long)(5 + q) * nb);
            dr[q] = __ldg(pr + (long long)(5 + q) * nb);
        }
        if (bmode == 2) {
            // the high face state belongs to the cell itself (global c)
#pragma unroll
            for (int q = 0; q < 5; ++q) Ql[q] = Qr[q];
        }
        if (bmode == 1) {
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                const bool ng = mirror_neg(q, g.bc[d]);
                Ql[q] = ng ? ff_neg(Qr[q]) : Qr[q];
                ol[q] = ng ? -orr[q] : orr[q];
            }
#pragma unroll
            for (int q = 0; q < 15; ++q) dl[q] = mirror_neg(5 + q, g.bc[d]) ? -dr[q] : dr[q];
        } else if (bmode == 2) {
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                const bool ng = mirror_neg(q, g.bc[d]);
                Qr[q] = ng ? ff_neg(Ql[q]) : Ql[q];
                orr[q] = ng ? -ol[q] : ol[q];
            }
#pragma unroll
            for (int q = 0; q < 15; ++q) dr[q] = mirror_neg(5 + q, g.bc[d]) ? -dl[q] : dl[q];
        }
        flux_point_mixed<kCGKS>(P, Ql, ol, dl, Qr, orr, dr, dt, out, valid ? status : nullptr);
        if (kCGKS) {
            // Gauss-point average: the time derivatives (blocks 1, 3, 5) are
            // FP32 values (lo = 0), summed in FP32; F^n and the interface
            // values in float-float. Both butterflies give every lane of a
            // face the same bits (the sums are commutative at each step).
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                if ((q / 5) & 1) {
                    float s = out[q].hi + __shfl_xor_sync(0xffffffffu, out[q].hi, 1);
                    s = s + __shfl_xor_sync(0xffffffffu, s, 2);
                    out[q] = ff_make(0.25f * s, 0.0f);
                } else {
                    ff s = ff_add_like(out[q], ff_make(__shfl_xor_sync(0xffffffffu, out[q].hi, 1),
                                                       __shfl_xor_sync(0xffffffffu, out[q].lo, 1)));
                    s = ff_add_like(s, ff_make(__shfl_xor_sync(0xffffffffu, s.hi, 2),
                                               __shfl_xor_sync(0xffffffffu, s.lo, 2)));
                    out[q] = ff_make(0.25f * s.hi, 0.25f * s.lo);  // exact
                }
            }
        }
        if (!valid) return;
        // lane k converts and writes the values q = 4j + k only (chosen with
        // selects, so that the four lanes of a face do not diverge)
#pragma unroll
        for (int jq = 0; jq < (NV + K - 1) / K; ++jq) {
            ff x = out[K * jq];
            int q = K * jq;
#pragma unroll
            for (int kq = 1; kq < K; ++kq) {
                if (K * jq + kq < NV && k == kq) {
                    x = out[K * jq + kq];
                    q = K * jq + kq;
                }
            }
            if (q < NV && (K == 1 || q % K == k)) {
                const int blk = q / 5, cmp = q % 5;
                frec[((long long)d * 30 + blk * 5 + global_var(cmp, d)) * rec_stride + rec_base] =
                    ff_to_double(x);
            }
        }
    }
}

}  // namespace
}  // namespace gks
