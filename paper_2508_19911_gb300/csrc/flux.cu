// Gas-kinetic interface flux at Gauss points (Sec. 2 of the paper).
//
// For the face frame (u along the face normal) and left/right reconstructed
// states W_l, W_r with their spatial derivatives, the distribution of
// Eq. flux is integrated over [0, dt] and [0, dt/2]; F^n and F_t^n follow
// from the linearisation f = f^n + t f_t^n (Eq. deri-t-f). Moments of the
// Maxwellians are evaluated in closed form:
//   <u^n> on the full line by <u^{n+2}> = U <u^{n+1}> + (n+1)/(2 lam) <u^n>,
//   on the half lines from erfc/exp starting values and the same recursion,
//   <xi^2> = N/(2 lam), <xi^4> = (N^2 + 2N)/(4 lam^2),
// composed into <(a.psi) u^A v^B w^D psi> with compile-time exponents; the
// Maxwellian slopes a (<(a.psi) psi> = dW/rho) are solved in closed form.
// One thread evaluates one Gauss point; the four Gauss points of a CGKS-5th
// face are four adjacent lanes reduced with a butterfly of shuffles.
#include <cmath>

#include "common.cuh"

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

// starting values of the half-line moments: sgn = +1 for u > 0, -1 for u < 0
__device__ __forceinline__ void half_start(double C, double lam, double sgn, double &m0, double &m1) {
    const double sl = sqrt(lam);
    m0 = 0.5 * erfc(-sgn * sl * C);
    const double edge = 0.5 * exp(-lam * C * C) / (sl * 1.7724538509055160273);  // sqrt(pi)
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

// <xi^2 u^A v^B w^D psi>
template <int A, int B, int D, typename T>
__device__ __forceinline__ void psixi_m(const T *u, const T *v, const T *w, T x2, T x4, T o[5]) {
    const T vw = v[B] * w[D];
    const T b = u[A] * vw;
    o[0] = x2 * b;
    o[1] = x2 * u[A + 1] * vw;
    o[2] = x2 * u[A] * v[B + 1] * w[D];
    o[3] = x2 * u[A] * v[B] * w[D + 1];
    o[4] = T(0.5) * (x2 * (u[A + 2] * vw + u[A] * (v[B + 2] * w[D] + v[B] * w[D + 2])) + x4 * b);
}

// acc += s * <(a.psi) u^A v^B w^D psi>
template <int A, int B, int D, typename T>
__device__ __forceinline__ void apsi_acc(const T a[5], const T *u, const T *v, const T *w, T x2,
                                         T x4, T s, T acc[5]) {
    T t[5], o[5], e[5];
    psi_m<A, B, D>(u, v, w, x2, o);
#pragma unroll
    for (int i = 0; i < 5; ++i) t[i] = a[0] * o[i];
    psi_m<A + 1, B, D>(u, v, w, x2, o);
#pragma unroll
    for (int i = 0; i < 5; ++i) t[i] += a[1] * o[i];
    psi_m<A, B + 1, D>(u, v, w, x2, o);
#pragma unroll
    for (int i = 0; i < 5; ++i) t[i] += a[2] * o[i];
    psi_m<A, B, D + 1>(u, v, w, x2, o);
#pragma unroll
    for (int i = 0; i < 5; ++i) t[i] += a[3] * o[i];
    psi_m<A + 2, B, D>(u, v, w, x2, e);
    psi_m<A, B + 2, D>(u, v, w, x2, o);
#pragma unroll
    for (int i = 0; i < 5; ++i) e[i] += o[i];
    psi_m<A, B, D + 2>(u, v, w, x2, o);
#pragma unroll
    for (int i = 0; i < 5; ++i) e[i] += o[i];
    psixi_m<A, B, D>(u, v, w, x2, x4, o);
#pragma unroll
    for (int i = 0; i < 5; ++i) acc[i] += s * (t[i] + T(0.5) * a[4] * (e[i] + o[i]));
}

// acc += s * sum_j <(a_j.psi) c_j u^E psi>, c = (u, v, w): the directional
// slope terms of Eq. flux (E = 1 for fluxes, 0 for conserved moments)
template <int E, typename T>
__device__ __forceinline__ void dir_acc(const T a[3][5], const T *u, const T *v, const T *w,
                                        T x2, T x4, T s, T acc[5]) {
    apsi_acc<1 + E, 0, 0>(a[0], u, v, w, x2, x4, s, acc);
    apsi_acc<E, 1, 0>(a[1], u, v, w, x2, x4, s, acc);
    apsi_acc<E, 0, 1>(a[2], u, v, w, x2, x4, s, acc);
}

// Slope of a Maxwellian (U, V, W, lam) with N internal degrees of freedom:
// the a with <(a.psi) psi> = d, solved in closed form.
template <typename T>
__device__ __forceinline__ void maxwell_slope(const T d[5], T U, T V, T W, T lam, T N, T a[5]) {
    const T q2 = U * U + V * V + W * W;
    const T K = (N + T(3)) / (T(2) * lam);
    const T R1 = d[1] - U * d[0], R2 = d[2] - V * d[0], R3 = d[3] - W * d[0];
    const T R4 = T(2) * d[4] - (q2 + K) * d[0];
    a[4] = T(4) * lam * lam / (N + T(3)) * (R4 - T(2) * (U * R1 + V * R2 + W * R3));
    a[1] = T(2) * lam * R1 - U * a[4];
    a[2] = T(2) * lam * R2 - V * a[4];
    a[3] = T(2) * lam * R3 - W * a[4];
    a[0] = d[0] - U * a[1] - V * a[2] - W * a[3] - T(0.5) * a[4] * (q2 + K);
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
        double term = 0.5 * x * x;  // (-1)^n x^n / n! at n = 2
        double s1 = term, s2 = 0.0, s3 = 0.0;
#pragma unroll
        for (int n = 3; n <= 26; ++n) {
            term *= -x / n;
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

// the closed forms above for E = 1 - e^{-x}, given E directly
__device__ __forceinline__ void time_integrals_closed(double T, double tau, double E, double c[6]) {
    const double t2 = tau * tau;
    c[0] = T - tau * E;
    c[1] = 2.0 * t2 * E - tau * T * (2.0 - E);
    c[2] = 0.5 * T * T - tau * T + t2 * E;
    c[3] = tau * E;
    c[4] = -2.0 * t2 * E + tau * T * (1.0 - E);
    c[5] = -t2 * E;
}

// both intervals [0, dt] and [0, dt/2]: when dt/(2 tau) >= 1 one exponential
// serves both (E = 1 - e_h^2, E_h = 1 - e_h, no cancellation for e_h <= 1/e)
__device__ __forceinline__ void time_integrals_pair(double dt, double tau, double cA[6],
                                                    double cH[6]) {
    if (tau > 0.0 && dt >= 2.0 * tau) {
        const double eh = exp(-0.5 * dt / tau);
        time_integrals_closed(dt, tau, 1.0 - eh * eh, cA);
        time_integrals_closed(0.5 * dt, tau, 1.0 - eh, cH);
    } else {
        time_integrals(dt, tau, cA);
        time_integrals(0.5 * dt, tau, cH);
    }
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

__device__ __forceinline__ PrimT<float> to_float(const Prim &P) {
    PrimT<float> f;
    f.rho = (float)P.rho; f.U = (float)P.U; f.V = (float)P.V; f.W = (float)P.W;
    f.p = (float)P.p; f.lam = (float)P.lam;
    return f;
}

// Contribution of one side (SGN = +1: left state over u > 0; -1: right
// state over u < 0) to W0's slopes and to terms 4-6 of Eq. flux.
// ds: the 15 derivatives d/dn, d/dt1, d/dt2 of the 5 conserved variables.
template <int SGN, typename T>
__device__ __forceinline__ void side_terms(const T *ds, const PrimT<T> &S, T N, T uh0, T uh1,
                                           T U0, T V0, T W0, T dW0[3][5], T X4[5], T X5[5],
                                           T X6[5], T q[3], T dtW[5]) {
    const T inv2l = T(0.5) / S.lam;
    T uf[kNU], uh[kNU], v[kNV], w[kNV];
    full_line<kNU>(S.U, inv2l, uf);
    half_line<kNU>(S.U, inv2l, uh0, uh1, uh);
    full_line<kNV>(S.V, inv2l, v);
    full_line<kNV>(S.W, inv2l, w);
    const T x2 = N * inv2l, x4 = (N * N + T(2) * N) * inv2l * inv2l;
    // one-sided Maxwellian slopes a_j
    T a[3][5];
    const T ir = T(1) / S.rho;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        T d[5];
#pragma unroll
        for (int i = 0; i < 5; ++i) d[i] = ds[5 * j + i] * ir;
        maxwell_slope(d, S.U, S.V, S.W, S.lam, N, a[j]);
    }
    // A from the compatibility condition: <(A.psi) psi> = -<(a.u) psi>
    T Tv[5] = {0, 0, 0, 0, 0}, A[5];
    dir_acc<0>(a, uf, v, w, x2, x4, T(1), Tv);
    {
        T mT[5];
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            mT[i] = -Tv[i];
            dtW[i] = -S.rho * Tv[i];  // Euler time derivative of W_s
        }
        maxwell_slope(mT, S.U, S.V, S.W, S.lam, N, A);
    }
    // slopes of the interface equilibrium, collected from both sides
#pragma unroll
    for (int j = 0; j < 3; ++j) apsi_acc<0, 0, 0>(a[j], uh, v, w, x2, x4, S.rho, dW0[j]);
    T X[5], Y[5];
    // term 4: g_s on its half line
    psi_m<1, 0, 0>(uh, v, w, x2, X);
    psi_m<0, 0, 0>(uh, v, w, x2, Y);
#pragma unroll
    for (int i = 0; i < 5; ++i) { X[i] *= S.rho; Y[i] *= S.rho; X4[i] += X[i]; }
    q[0] += heat(X, Y, U0, V0, W0);
    // term 5: (a.u) g_s
#pragma unroll
    for (int i = 0; i < 5; ++i) { X[i] = T(0); Y[i] = T(0); }
    dir_acc<1>(a, uh, v, w, x2, x4, S.rho, X);
    dir_acc<0>(a, uh, v, w, x2, x4, S.rho, Y);
#pragma unroll
    for (int i = 0; i < 5; ++i) X5[i] += X[i];
    q[1] += heat(X, Y, U0, V0, W0);
    // term 6: A g_s
#pragma unroll
    for (int i = 0; i < 5; ++i) { X[i] = T(0); Y[i] = T(0); }
    apsi_acc<1, 0, 0>(A, uh, v, w, x2, x4, S.rho, X);
    apsi_acc<0, 0, 0>(A, uh, v, w, x2, x4, S.rho, Y);
#pragma unroll
    for (int i = 0; i < 5; ++i) X6[i] += X[i];
    q[2] += heat(X, Y, U0, V0, W0);
}

// Equilibrium part: abar from the collided slopes dW0, Abar by
// compatibility; X1..X3 (term 1 only if kTerm1), q1..q3, dW0/dt.
template <bool kTerm1, typename T>
__device__ __forceinline__ void equilibrium_terms(const PrimT<T> &Z, T N, const T dW0[3][5],
                                                  T X[6][5], T q[6], T dtW0[5]) {
    const T inv2l = T(0.5) / Z.lam;
    T u[kNU], v[kNV], w[kNV];
    full_line<kNU>(Z.U, inv2l, u);
    full_line<kNV>(Z.V, inv2l, v);
    full_line<kNV>(Z.W, inv2l, w);
    const T x2 = N * inv2l, x4 = (N * N + T(2) * N) * inv2l * inv2l;
    T ab[3][5];
    const T ir = T(1) / Z.rho;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        T d[5];
#pragma unroll
        for (int i = 0; i < 5; ++i) d[i] = dW0[j][i] * ir;
        maxwell_slope(d, Z.U, Z.V, Z.W, Z.lam, N, ab[j]);
    }
    T T0[5] = {0, 0, 0, 0, 0}, Ab[5];
    dir_acc<0>(ab, u, v, w, x2, x4, T(1), T0);
    {
        T mT[5];
#pragma unroll
        for (int i = 0; i < 5; ++i) mT[i] = -T0[i];
        maxwell_slope(mT, Z.U, Z.V, Z.W, Z.lam, N, Ab);
    }
    T Y[5];
    if (kTerm1) {
        // term 1: g0
        psi_m<1, 0, 0>(u, v, w, x2, X[0]);
        psi_m<0, 0, 0>(u, v, w, x2, Y);
#pragma unroll
        for (int i = 0; i < 5; ++i) { X[0][i] *= Z.rho; Y[i] *= Z.rho; }
        q[0] = heat(X[0], Y, Z.U, Z.V, Z.W);
    }
    // term 2: (abar.u) g0; its conserved moments are rho0 T0
    dir_acc<1>(ab, u, v, w, x2, x4, Z.rho, X[1]);
#pragma unroll
    for (int i = 0; i < 5; ++i) Y[i] = Z.rho * T0[i];
    q[1] = heat(X[1], Y, Z.U, Z.V, Z.W);
    // term 3: Abar g0; its conserved moments are -rho0 T0 (compatibility)
    apsi_acc<1, 0, 0>(Ab, u, v, w, x2, x4, Z.rho, X[2]);
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        Y[i] = -Z.rho * T0[i];
        dtW0[i] = Y[i];
    }
    q[2] = heat(X[2], Y, Z.U, Z.V, Z.W);
}

// W0 = rho_l <psi>_{u>0} + rho_r <psi>_{u<0} (FP64), the half-line
// starting moments of both sides and, if asked, the term-4 flux moments
// X4 = rho_l <u psi>_{u>0} + rho_r <u psi>_{u<0} (FP64)
template <bool kX4>
__device__ __forceinline__ void interface_state(const Prim &L, const Prim &R, double N,
                                                double W0[5], double X4[5], double &ul0,
                                                double &ul1, double &ur0, double &ur1) {
    half_start(L.U, L.lam, 1.0, ul0, ul1);
    half_start(R.U, R.lam, -1.0, ur0, ur1);
    double u[4], v[3], w[3], o[5];
    const double il = 0.5 / L.lam, ir = 0.5 / R.lam;
    half_line<4>(L.U, il, ul0, ul1, u);
    full_line<3>(L.V, il, v);
    full_line<3>(L.W, il, w);
    psi_m<0, 0, 0>(u, v, w, N * il, o);
#pragma unroll
    for (int i = 0; i < 5; ++i) W0[i] = L.rho * o[i];
    if (kX4) {
        psi_m<1, 0, 0>(u, v, w, N * il, o);
#pragma unroll
        for (int i = 0; i < 5; ++i) X4[i] = L.rho * o[i];
    }
    half_line<4>(R.U, ir, ur0, ur1, u);
    full_line<3>(R.V, ir, v);
    full_line<3>(R.W, ir, w);
    psi_m<0, 0, 0>(u, v, w, N * ir, o);
#pragma unroll
    for (int i = 0; i < 5; ++i) W0[i] += R.rho * o[i];
    if (kX4) {
        psi_m<1, 0, 0>(u, v, w, N * ir, o);
#pragma unroll
        for (int i = 0; i < 5; ++i) X4[i] += R.rho * o[i];
    }
}

// collision time (Sec. 4) and F^n, F_t^n from the six term moments
// (X1, X4: optional FP64 replacements of terms 1 and 4, whose time
// coefficients are large and cancel in F_t: beta_1 + beta_4 = 0)
template <typename TX>
__device__ __forceinline__ void combine_terms(const PhysParams &P, const Prim &L, const Prim &R,
                                              const Prim &Z, double dt, const TX X[6][5],
                                              const TX q[6], const double X1[5], const double X4[5],
                                              double out[10], double &dpr) {
    dpr = fabs((L.p - R.p) / (L.p + R.p));
    const double tau = P.inviscid ? (P.eps_tau * dt + P.C_tau * dpr * dt)
                                  : (viscosity(P, Z.rho, Z.p) / Z.p + P.C_tau * dpr * dt);
    double cA[6], cH[6];
    time_integrals_pair(dt, tau, cA, cH);
    const double idt = 1.0 / dt, idt2 = idt * idt;
    const double prfix = 1.0 / P.Pr - 1.0;
    double qn = 0.0, qt = 0.0;
#pragma unroll
    for (int i = 0; i < 10; ++i) out[i] = 0.0;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const double al = (4.0 * cH[k] - cA[k]) * idt;
        const double be = 4.0 * (cA[k] - 2.0 * cH[k]) * idt2;
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            const double x = (k == 0 && X1) ? X1[i] : ((k == 3 && X4) ? X4[i] : (double)X[k][i]);
            out[i] += al * x;
            out[5 + i] += be * x;
        }
        qn += al * (double)q[k];
        qt += be * (double)q[k];
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
    interface_state<false>(L, R, N, W0, nullptr, ul0, ul1, ur0, ur1);
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
    side_terms<1>(sl + 5, L, N, ul0, ul1, Z.U, Z.V, Z.W, dW0, X[3], X[4], X[5], q + 3, dtWl);
    side_terms<-1>(sr + 5, R, N, ur0, ur1, Z.U, Z.V, Z.W, dW0, X[3], X[4], X[5], q + 3, dtWr);
    equilibrium_terms<true>(Z, N, dW0, X, q, dtW0);
    double dpr;
    combine_terms<double>(P, L, R, Z, dt, X, q, nullptr, nullptr, out, dpr);
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

// Mixed precision (FP32 core, FP64 shell): the states W_l, W_r, the
// interface equilibrium W0 with its half-line moments, the Euler flux of
// W0 (term 1) and the half-space fluxes of g_l, g_r (term 4) -- the two
// terms that carry the pressure and whose large time coefficients cancel
// in F_t -- the collision time, the time integrals, the combinations F^n,
// F_t^n and the interface values are FP64; the Maxwellian slopes and the
// moment compositions of terms 2, 3, 5, 6 (multiplied by coefficients of
// order tau or tau^2/dt^2) are FP32.
template <bool kInterface>
__device__ void flux_point_mixed(const PhysParams &P, const double Wl[5], const float dl[15],
                                 const double Wr[5], const float dr[15], double dt,
                                 double out[30], int *status) {
    const double N = P.Nint;
    const Prim L = to_prim(Wl, P.gamma), R = to_prim(Wr, P.gamma);
    if (!(L.rho > 0.0 && L.p > 0.0 && R.rho > 0.0 && R.p > 0.0)) {
        flag_status(status, kStatusNonphysical);
#pragma unroll
        for (int i = 0; i < 30; ++i) out[i] = nan("");
        return;
    }
    double W0[5], X4d[5], ul0, ul1, ur0, ur1;
    interface_state<true>(L, R, N, W0, X4d, ul0, ul1, ur0, ur1);
    const Prim Z = to_prim(W0, P.gamma);
    if (!(Z.rho > 0.0 && Z.p > 0.0)) {
        flag_status(status, kStatusNonphysical);
#pragma unroll
        for (int i = 0; i < 30; ++i) out[i] = nan("");
        return;
    }
    // term 1: the Euler flux of W0, FP64
    double X1[5];
    X1[0] = W0[1];
    X1[1] = W0[1] * Z.U + Z.p;
    X1[2] = W0[2] * Z.U;
    X1[3] = W0[3] * Z.U;
    X1[4] = (W0[4] + Z.p) * Z.U;
    const float Nf = (float)N;
    const PrimT<float> Lf = to_float(L), Rf = to_float(R), Zf = to_float(Z);
    float dW0[3][5], X[6][5], q[6] = {0, 0, 0, 0, 0, 0}, dtWl[5], dtWr[5], dtW0[5];
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int i = 0; i < 5; ++i) dW0[j][i] = 0.0f;
#pragma unroll
    for (int k = 0; k < 6; ++k)
#pragma unroll
        for (int i = 0; i < 5; ++i) X[k][i] = 0.0f;
    side_terms<1>(dl, Lf, Nf, (float)ul0, (float)ul1, Zf.U, Zf.V, Zf.W, dW0, X[3], X[4], X[5],
                  q + 3, dtWl);
    side_terms<-1>(dr, Rf, Nf, (float)ur0, (float)ur1, Zf.U, Zf.V, Zf.W, dW0, X[3], X[4], X[5],
                   q + 3, dtWr);
    equilibrium_terms<false>(Zf, Nf, dW0, X, q, dtW0);  // a Maxwellian carries no heat flux: q1 = 0
    double dpr;
    combine_terms<float>(P, L, R, Z, dt, X, q, X1, X4d, out, dpr);
    if (kInterface) {
        const double e = (P.C_tau * dpr > 0.0) ? exp(-1.0 / (P.C_tau * dpr)) : 0.0;
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            out[10 + i] = (1.0 - e) * W0[i] + e * Wl[i];
            out[15 + i] = (1.0 - e) * (double)dtW0[i] + e * (double)dtWl[i];
            out[20 + i] = (1.0 - e) * W0[i] + e * Wr[i];
            out[25 + i] = (1.0 - e) * (double)dtW0[i] + e * (double)dtWr[i];
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
template <bool kCGKS, bool MIXED>
__device__ __forceinline__ void flux_face_point(const GridDesc &g, const PhysParams &P,
                                                const void *__restrict__ fsv,
                                                const double *__restrict__ Q, double dt,
                                                double *__restrict__ frec, int *status, int d,
                                                long long c, int k, bool valid) {
    constexpr int K = kCGKS ? 4 : 1;
    const long long n = g.n;
    const int i = (int)(c % g.nx);
    const int j = (int)((c / g.nx) % g.ny);
    const int kk = (int)(c / ((long long)g.nx * g.ny));
    const long long left = cell_index(g, d == 0 ? wrap(i - 1, g.nx) : i,
                                      d == 1 ? wrap(j - 1, g.ny) : j,
                                      d == 2 ? wrap(kk - 1, g.nz) : kk);
    double out[30];
    if (!MIXED) {
        const double *fs = (const double *)fsv;
        double sl[20], sr[20];
        const double *pl = fs + ((long long)((2 * d + 1) * K + k) * 20) * n + left;
        const double *pr = fs + ((long long)((2 * d) * K + k) * 20) * n + c;
#pragma unroll
        for (int q = 0; q < 20; ++q) {
            sl[q] = __ldg(pl + (long long)q * n);
            sr[q] = __ldg(pr + (long long)q * n);
        }
        flux_point<kCGKS>(P, sl, sr, dt, out, valid ? status : nullptr);
    } else {
        const float *fs = (const float *)fsv;
        double Wl[5], Wr[5];
        float dl[15], dr[15];
        const float *pl = fs + ((long long)((2 * d + 1) * K + k) * 20) * n + left;
        const float *pr = fs + ((long long)((2 * d) * K + k) * 20) * n + c;
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            const int v = global_var(q, d);
            Wl[q] = __ldg(Q + (long long)v * n + left) + (double)__ldg(pl + (long long)q * n);
            Wr[q] = __ldg(Q + (long long)v * n + c) + (double)__ldg(pr + (long long)q * n);
        }
#pragma unroll
        for (int q = 0; q < 15; ++q) {
            dl[q] = __ldg(pl + (long long)(5 + q) * n);
            dr[q] = __ldg(pr + (long long)(5 + q) * n);
        }
        flux_point_mixed<kCGKS>(P, Wl, dl, Wr, dr, dt, out, valid ? status : nullptr);
    }
    constexpr int NV = kCGKS ? 30 : 10;
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
        frec[((long long)d * 30 + blk * 5 + global_var(cmp, d)) * n + c] = out[q];
    }
}

template <bool kCGKS, bool MIXED>
__global__ void __launch_bounds__(128) flux_faces_kernel(GridDesc g, PhysParams P,
                                                         const void *__restrict__ fs,
                                                         const double *__restrict__ Q,
                                                         const double *__restrict__ dt_dev,
                                                         double *__restrict__ frec, int *status) {
    const double dt = *dt_dev;
    if (!(dt > 0.0)) return;  // same for every thread of the grid
    constexpr int K = kCGKS ? 4 : 1;
    const long long n = g.n;
    const long long total = 3 * n * K;
    long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = gid < total;
    if (!valid) gid = total - 1;  // groups of K lanes are entirely in or out
    const int k = (int)(gid % K);
    const long long fc = gid / K;
    const int d = (int)(fc / n);
    const long long c = fc - (long long)d * n;
    flux_face_point<kCGKS, MIXED>(g, P, fs, Q, dt, frec, status, d, c, k, valid);
}

// Persistent ensemble flux (CGKS-5th): blocks stride over the work items
// of all instances; an item of T cells holds 3 x T faces x 4 Gauss points.
template <bool MIXED>
__global__ void __launch_bounds__(128) flux_ens_kernel(const EnsInst *__restrict__ inst,
                                                       const EnsItem *__restrict__ items,
                                                       int nitems, const void *__restrict__ fsa,
                                                       const double *__restrict__ Qa,
                                                       const double *__restrict__ dt_arr,
                                                       double *__restrict__ fra, int *status) {
    for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
        const EnsItem it = items[w];
        const EnsInst I = inst[it.inst];
        const double dt = dt_arr[it.inst];
        if (!(dt > 0.0)) continue;  // uniform across the block
        const long long T = it.c1 - it.c0;
        const long long total = 12 * T;
        const void *fs = MIXED ? (const void *)((const float *)fsa + 480 * I.off)
                               : (const void *)((const double *)fsa + 480 * I.off);
        for (long long t0 = 0; t0 < total; t0 += blockDim.x) {
            long long gid = t0 + threadIdx.x;
            const bool valid = gid < total;
            if (!valid) gid = total - 1;
            const int k = (int)(gid & 3);
            const long long rem = gid >> 2;
            const int d = (int)(rem / T);
            const long long c = it.c0 + rem % T;
            flux_face_point<true, MIXED>(I.g, I.P, fs, Qa + 5 * I.off, dt, fra + 90 * I.off,
                                         status, d, c, k, valid);
        }
    }
}

__global__ void __launch_bounds__(128) flux_points_kernel(PhysParams P, const double *__restrict__ sl_,
                                                          const double *__restrict__ sr_, int n,
                                                          const double *__restrict__ dt_dev,
                                                          double *__restrict__ out_, int *status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double dt = *dt_dev;
    double sl[20], sr[20], out[30];
#pragma unroll
    for (int q = 0; q < 20; ++q) {
        sl[q] = sl_[(long long)q * n + i];
        sr[q] = sr_[(long long)q * n + i];
    }
    flux_point<true>(P, sl, sr, dt, out, status);
#pragma unroll
    for (int q = 0; q < 30; ++q) out_[(long long)q * n + i] = out[q];
}

}  // namespace

int launch_flux_faces_mixed(const GridDesc &g, const PhysParams &P, const float *fs, const double *Q,
                            const double *dt_dev, double *frec, int *status, cudaStream_t s) {
    const int K = P.scheme ? 4 : 1;
    const long long total = 3 * g.n * K;
    const int block = 128;
    const long long grid = (total + block - 1) / block;
    if (P.scheme)
        flux_faces_kernel<true, true><<<(unsigned)grid, block, 0, s>>>(g, P, fs, Q, dt_dev, frec, status);
    else
        flux_faces_kernel<false, true><<<(unsigned)grid, block, 0, s>>>(g, P, fs, Q, dt_dev, frec, status);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int launch_flux_faces(const GridDesc &g, const PhysParams &P, const double *fs,
                      const double *dt_dev, double *frec, int *status, cudaStream_t s) {
    const int K = P.scheme ? 4 : 1;
    const long long total = 3 * g.n * K;
    const int block = 128;
    const long long grid = (total + block - 1) / block;
    if (P.scheme)
        flux_faces_kernel<true, false><<<(unsigned)grid, block, 0, s>>>(g, P, fs, nullptr, dt_dev, frec, status);
    else
        flux_faces_kernel<false, false><<<(unsigned)grid, block, 0, s>>>(g, P, fs, nullptr, dt_dev, frec, status);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int launch_flux_ens(const EnsInst *inst, const EnsItem *items, int nitems, int blocks, int mixed,
                    const void *fsa, const double *Qa, const double *dt_arr, double *fra,
                    int *status, cudaStream_t s) {
    if (mixed)
        flux_ens_kernel<true><<<blocks, 128, 0, s>>>(inst, items, nitems, fsa, Qa, dt_arr, fra, status);
    else
        flux_ens_kernel<false><<<blocks, 128, 0, s>>>(inst, items, nitems, fsa, Qa, dt_arr, fra, status);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int launch_flux_points(const PhysParams &P, const double *sl, const double *sr, int n,
                       const double *dt_dev, double *out, int *status, cudaStream_t s) {
    const int block = 128;
    flux_points_kernel<<<(n + block - 1) / block, block, 0, s>>>(P, sl, sr, n, dt_dev, out, status);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

}  // namespace gks
