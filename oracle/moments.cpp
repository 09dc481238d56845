/*
 * Oracle: Maxwellian moments (Sec. 2 of the paper: Maxwellian g, the
 * collision invariants psi, Eq. Q-macro and Eq. flux-macro).
 * Test infrastructure only (see oracle.h).
 *
 * g = rho (lam/pi)^{(N+3)/2} exp(-lam[(u-U)^2+(v-V)^2+(w-W)^2+xi^2]),
 * psi = (1, u, v, w, (u^2+v^2+w^2+xi^2)/2).
 * A rho-normalised moment <u^a v^b w^c (xi^2)^k> factorises into
 * one-dimensional moments; each entry of G^x_{ik} = <x psi_i psi_k> is
 * expanded monomial by monomial and integrated term by term.
 */
#include "oracle_internal.h"

#include <cmath>
#include <cstring>

namespace orc {

/* One-dimensional Gaussian moments <c^n> of exp(-lam (c-C)^2), normalised
 * to unit mass over the full line, over the full line (half = 0), c > 0
 * (half = +1) or c < 0 (half = -1). Recursion from integration by parts:
 * <c^{n+2}> = C <c^{n+1}> + (n+1)/(2 lam) <c^n>, valid on the half lines
 * too because the boundary term at c = 0 vanishes for n >= 0.           */
void gauss_moments_1d(double C, double lam, int half, int nmax, double *m) {
    if (half == 0) {
        m[0] = 1.0;
        m[1] = C;
    } else {
        const double s = std::sqrt(lam);
        const double edge = std::exp(-lam * C * C) / (2.0 * std::sqrt(M_PI * lam));
        if (half > 0) {
            m[0] = 0.5 * std::erfc(-s * C);
            m[1] = C * m[0] + edge;
        } else {
            m[0] = 0.5 * std::erfc(s * C);
            m[1] = C * m[0] - edge;
        }
    }
    for (int n = 0; n + 2 <= nmax; ++n)
        m[n + 2] = C * m[n + 1] + (double)(n + 1) / (2.0 * lam) * m[n];
}

void moment_tables(double U, double V, double W, double lam, double Nint,
                   int half, Tables *t) {
    gauss_moments_1d(U, lam, half, kMaxU, t->u);
    gauss_moments_1d(V, lam, 0, kMaxV, t->v);
    gauss_moments_1d(W, lam, 0, kMaxV, t->w);
    /* internal degrees of freedom: N independent Gaussians of variance
     * 1/(2 lam): <xi^2> = N/(2 lam), <xi^4> = (N^2 + 2N)/(4 lam^2).     */
    t->xi[0] = 1.0;
    t->xi[1] = Nint / (2.0 * lam);
    t->xi[2] = (Nint * Nint + 2.0 * Nint) / (4.0 * lam * lam);
}

namespace {
struct Mono { double c; int a, b, d, k; };
/* psi_i as lists of monomials u^a v^b w^d (xi^2)^k */
const Mono kPsi[5][4] = {
    {{1.0, 0, 0, 0, 0}},
    {{1.0, 1, 0, 0, 0}},
    {{1.0, 0, 1, 0, 0}},
    {{1.0, 0, 0, 1, 0}},
    {{0.5, 2, 0, 0, 0}, {0.5, 0, 2, 0, 0}, {0.5, 0, 0, 2, 0}, {0.5, 0, 0, 0, 1}},
};
const int kPsiTerms[5] = {1, 1, 1, 1, 4};
/* extra factor x of G^x: 1, u, v, w, uu, uv, uw */
const int kExtra[7][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1},
                          {2, 0, 0}, {1, 1, 0}, {1, 0, 1}};
}  // namespace

double monomial_moment(const Tables &t, int a, int b, int d, int k) {
    return t.u[a] * t.v[b] * t.w[d] * t.xi[k];
}

void g_matrix(const Tables &t, int which, double G[5][5]) {
    const int *x = kExtra[which];
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) {
            double s = 0.0;
            for (int p = 0; p < kPsiTerms[i]; ++p)
                for (int q = 0; q < kPsiTerms[j]; ++q) {
                    const Mono &A = kPsi[i][p], &B = kPsi[j][q];
                    s += A.c * B.c *
                         monomial_moment(t, A.a + B.a + x[0], A.b + B.b + x[1],
                                         A.d + B.d + x[2], A.k + B.k);
                }
            G[i][j] = s;
        }
}

void all_g(const Tables &t, GSet *g) {
    for (int w = 0; w < 7; ++w) g_matrix(t, w, g->m[w]);
}

/* Generic dense solve A x = b by Gaussian elimination with partial
 * pivoting; A and b are copied. Returns 0 on success, -1 if singular.   */
int solve_dense(int n, const double *A_in, const double *b_in, double *x) {
    double A[kMaxSolve * kMaxSolve], b[kMaxSolve];
    std::memcpy(A, A_in, sizeof(double) * n * n);
    std::memcpy(b, b_in, sizeof(double) * n);
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
        if (A[piv * n + c] == 0.0) return -1;
        if (piv != c) {
            for (int j = 0; j < n; ++j) std::swap(A[c * n + j], A[piv * n + j]);
            std::swap(b[c], b[piv]);
        }
        for (int r = c + 1; r < n; ++r) {
            const double f = A[r * n + c] / A[c * n + c];
            for (int j = c; j < n; ++j) A[r * n + j] -= f * A[c * n + j];
            b[r] -= f * b[c];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        double s = b[r];
        for (int j = r + 1; j < n; ++j) s -= A[r * n + j] * x[j];
        x[r] = s / A[r * n + r];
    }
    return 0;
}

void matvec5(const double G[5][5], const double *a, double *y) {
    for (int i = 0; i < 5; ++i) {
        double s = 0.0;
        for (int j = 0; j < 5; ++j) s += G[i][j] * a[j];
        y[i] = s;
    }
}

/* Primitive variables of a conserved state (R = 1, T = p/rho).         */
Prim primitive(const double *Wc, double gamma) {
    Prim p;
    p.rho = Wc[0];
    p.U = Wc[1] / Wc[0];
    p.V = Wc[2] / Wc[0];
    p.W = Wc[3] / Wc[0];
    const double kin = 0.5 * p.rho * (p.U * p.U + p.V * p.V + p.W * p.W);
    p.p = (gamma - 1.0) * (Wc[4] - kin);
    p.lam = p.rho / (2.0 * p.p);
    return p;
}

double internal_dof(double gamma) { return (5.0 - 3.0 * gamma) / (gamma - 1.0); }

/* Slope of a Maxwellian: solve <(a.psi) psi> = dW/rho with the generic
 * moment matrix G^1 of the full-space Maxwellian.                       */
int slope(const Prim &p, double Nint, const double *dW, double *a) {
    Tables t;
    moment_tables(p.U, p.V, p.W, p.lam, Nint, 0, &t);
    double G[5][5];
    g_matrix(t, 0, G);
    double rhs[5];
    for (int i = 0; i < 5; ++i) rhs[i] = dW[i] / p.rho;
    return solve_dense(5, &G[0][0], rhs, a);
}

}  // namespace orc

extern "C" int orc_moment_matrix(double U, double V, double W, double lam,
                                 double Nint, int half, int which,
                                 double *out25) {
    if (which < 0 || which > 6 || lam <= 0.0) return -1;
    orc::Tables t;
    orc::moment_tables(U, V, W, lam, Nint, half, &t);
    double G[5][5];
    orc::g_matrix(t, which, G);
    std::memcpy(out25, &G[0][0], sizeof(G));
    return 0;
}

extern "C" int orc_slope(const double *Wc, const double *dW, double gamma,
                         double *a) {
    orc::Prim p = orc::primitive(Wc, gamma);
    if (!(p.rho > 0.0) || !(p.p > 0.0)) return -1;
    return orc::slope(p, orc::internal_dof(gamma), dW, a);
}
