/*
 * Oracle: spatial reconstruction (Sec. 3.2 CGKS-5th, Sec. 3.3 GKS-2nd).
 * Test infrastructure only (see oracle.h).
 *
 * All polynomials live in normalised cell coordinates
 * delta = (x - x0)/h per axis (Eq. base), the target cell being
 * [-1/2, 1/2]^3. Neighbour offsets, in this order:
 *   face neighbours Omega_{1,m}, m = 0..5:  -x, +x, -y, +y, -z, +z;
 *   edge neighbours Omega_{2,n}, n = 0..11: (-1,-1,0) (+1,-1,0) (-1,+1,0)
 *     (+1,+1,0) (-1,0,-1) (+1,0,-1) (-1,0,+1) (+1,0,+1) (0,-1,-1)
 *     (0,+1,-1) (0,-1,+1) (0,+1,+1).
 * Per-variable data vector d (63 entries) of the CGKS-5th stencil
 * (S^data-5th with readings R1, R2 of oracle.h):
 *   d[m]          Q_{1,m} - Q_0                      (m = 0..5)
 *   d[6+n]        Q_{2,n} - Q_0                      (n = 0..11)
 *   d[18+3m+j]    h_j dQ/dx_j averaged over Omega_{1,m}
 *   d[36+2n+t]    h dQ/dtau_t averaged over Omega_{2,n}: tau_0 is the unit
 *                 in-plane direction (o_a e_a - o_b e_b)/sqrt(2) orthogonal
 *                 to the centre-to-centre offset o (a < b its non-zero
 *                 axes), tau_1 the edge direction (the axis where o = 0)
 *   d[60+j]       h_j dQ/dx_j averaged over Omega_0.
 * Reading B of S^0 (row N2, reading R17): the own cell's data are its 12
 * line-averaged derivatives instead of its averaged gradient, d has 72
 * entries and
 *   d[60+4a+k]    h_a (Q(x_a = +h_a/2) - Q(x_a = -h_a/2))/h_a along the line
 *                 through the cell parallel to axis a at the tangential
 *                 position of face Gauss point k (k as face_gauss_point);
 * the neighbours' gradients are their cell averages (the mean of their four
 * line derivatives per axis), and P1_m's tangential slopes come from the
 * own averaged gradient, the mean of its four lines per axis.
 */
#include "oracle_internal.h"

#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

namespace orc {

int frame_axis(int d, int j) { return (d + j) % 3; }

void face_gauss_point(int f, int k, double x[3]) {
    const int d = f / 2;
    const double g = 0.5 / std::sqrt(3.0);  /* 2-point Gauss on [-1/2, 1/2] */
    x[d] = (f % 2) ? 0.5 : -0.5;
    x[frame_axis(d, 1)] = (k & 1) ? g : -g;
    x[frame_axis(d, 2)] = (k & 2) ? g : -g;
}

namespace {

typedef long double ld;

const int kFace[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0},
                         {0, 1, 0},  {0, 0, -1}, {0, 0, 1}};
const int kEdge[12][3] = {{-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 1, 0},
                          {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1}, {1, 0, 1},
                          {0, -1, -1}, {0, 1, -1}, {0, -1, 1}, {0, 1, 1}};

struct Basis { int d[34][3]; };

Basis make_basis() {
    Basis b;
    int n = 0;
    for (int deg = 1; deg <= 4; ++deg)
        for (int i = deg; i >= 0; --i)
            for (int j = deg - i; j >= 0; --j) {
                b.d[n][0] = i; b.d[n][1] = j; b.d[n][2] = deg - i - j;
                ++n;
            }
    return b;
}

ld fact(int n) { ld f = 1; for (int i = 2; i <= n; ++i) f *= i; return f; }
ld ipow(ld x, int n) { ld r = 1; for (int i = 0; i < n; ++i) r *= x; return r; }

/* average of x^n over [o - 1/2, o + 1/2] */
ld avg1(int o, int n) {
    return (ipow(o + 0.5L, n + 1) - ipow(o - 0.5L, n + 1)) / (n + 1);
}
/* average over the unit cell at offset o of delta^e / e! (e may have a
 * negative entry: then the derivative vanished and the value is 0)     */
ld avg_mono(const int o[3], const int e[3]) {
    for (int j = 0; j < 3; ++j) if (e[j] < 0) return 0;
    return avg1(o[0], e[0]) * avg1(o[1], e[1]) * avg1(o[2], e[2]) /
           (fact(e[0]) * fact(e[1]) * fact(e[2]));
}
/* average over offset o of p_d (zero mean over the target cell) */
ld avg_p(const int o[3], const int d[3]) {
    static const int z[3] = {0, 0, 0};
    return avg_mono(o, d) - avg_mono(z, d);
}
/* average over offset o of d p_d / d delta_j */
ld avg_dp(const int o[3], const int d[3], int j) {
    int e[3] = {d[0], d[1], d[2]};
    e[j] -= 1;
    return avg_mono(o, e);
}

/* Gauss-Jordan elimination with partial pivoting on an n x (n + m)
 * augmented long-double matrix (row major). Returns -1 if singular.    */
int gauss_jordan(int n, int m, std::vector<ld> &A) {
    const int w = n + m;
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs((double)A[r * w + c]) > std::fabs((double)A[piv * w + c])) piv = r;
        if (A[piv * w + c] == 0) return -1;
        if (piv != c)
            for (int j = 0; j < w; ++j) std::swap(A[c * w + j], A[piv * w + j]);
        const ld inv = 1 / A[c * w + c];
        for (int j = 0; j < w; ++j) A[c * w + j] *= inv;
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            const ld f = A[r * w + c];
            if (f == 0) continue;
            for (int j = 0; j < w; ++j) A[r * w + j] -= f * A[c * w + j];
        }
    }
    return 0;
}

struct Recon5Tables {
    double R[34][72];          /* coefficients a = R d (nd columns)         */
    double B[54][34];          /* derivative rows of Eq. compact-big-5
                                  (unweighted; nB of them)                  */
    double wq[54];             /* their least-squares weights (R3)          */
    double mean0[34];          /* mean of delta^d/d! over the target cell   */
    int nd, nB;                /* 63, 45 (reading A); 72, 54 (reading B)   */
    int ok;
};

/* value of delta^d/d! at x (normalised coordinates) */
ld mono_at(const ld x[3], const int d[3]) {
    return ipow(x[0], d[0]) * ipow(x[1], d[1]) * ipow(x[2], d[2]) /
           (fact(d[0]) * fact(d[1]) * fact(d[2]));
}

Recon5Tables build_tables(int variant) {
    Recon5Tables T;
    std::memset(&T, 0, sizeof(T));
    const Basis b = make_basis();
    static const int z[3] = {0, 0, 0};
    /* constrained least squares of Eq. compact-big-5:
     *   C a = d_C  (cell averages of the 18 neighbours, exact),
     *   B a ~ d_B  (45 derivative equations, weighted least squares R3).
     * KKT system [B^T B  C^T; C  0] [a; lambda] = [B^T d_B; d_C].        */
    const int nB = variant ? 54 : 45, nd = 18 + nB;
    ld C[18][34], B[54][34];
    for (int k = 0; k < 18; ++k) {
        const int *o = (k < 6) ? kFace[k] : kEdge[k - 6];
        for (int i = 0; i < 34; ++i) C[k][i] = avg_p(o, b.d[i]);
    }
    int r = 0;
    for (int m = 0; m < 6; ++m)
        for (int j = 0; j < 3; ++j, ++r)
            for (int i = 0; i < 34; ++i) B[r][i] = avg_dp(kFace[m], b.d[i], j);
    for (int n = 0; n < 12; ++n) {
        const int *o = kEdge[n];
        int axes[2], na = 0, ez = 0;
        for (int j = 0; j < 3; ++j) {
            if (o[j] != 0) axes[na++] = j; else ez = j;
        }
        const ld rs2 = 1 / std::sqrt(2.0L);
        for (int i = 0; i < 34; ++i)
            B[r][i] = rs2 * (o[axes[0]] * avg_dp(o, b.d[i], axes[0]) -
                             o[axes[1]] * avg_dp(o, b.d[i], axes[1]));
        ++r;
        for (int i = 0; i < 34; ++i) B[r][i] = avg_dp(o, b.d[i], ez);
        ++r;
    }
    if (!variant) {
        for (int j = 0; j < 3; ++j, ++r)
            for (int i = 0; i < 34; ++i) B[r][i] = avg_dp(z, b.d[i], j);
    } else {
        /* the 12 line-averaged derivatives of the target cell: along axis a
         * between the face Gauss points k of its two faces normal to a */
        const ld g = 0.5L / std::sqrt(3.0L);
        for (int a = 0; a < 3; ++a)
            for (int k = 0; k < 4; ++k, ++r) {
                ld x1[3], x2[3];
                x1[a] = -0.5L;
                x2[a] = 0.5L;
                x1[(a + 1) % 3] = x2[(a + 1) % 3] = (k & 1) ? g : -g;
                x1[(a + 2) % 3] = x2[(a + 2) % 3] = (k & 2) ? g : -g;
                for (int i = 0; i < 34; ++i) B[r][i] = mono_at(x2, b.d[i]) - mono_at(x1, b.d[i]);
            }
    }

    /* row weights h_1, h_2, h_3 of Eq. compact-big-5 (relative to the cell
     * size that scales the derivative data): the paper states only their
     * purpose, a smaller condition number of the reconstruction matrix.
     * Reading: 1 for the face neighbours' gradients and the own gradient,
     * 0.1 for the edge neighbours' tangential derivatives, near the minimum
     * of the condition number of the weighted least-squares system on the
     * null space of the constraints (5.07 against 29.6 with unit weights). */
    ld wq[54];
    for (int q = 0; q < nB; ++q) wq[q] = (q >= 18 && q < 42) ? 0.1L : 1.0L;
    for (int q = 0; q < nB; ++q) {
        T.wq[q] = (double)wq[q];
        for (int i = 0; i < 34; ++i) T.B[q][i] = (double)B[q][i];
    }
    for (int q = 0; q < nB; ++q)
        for (int i = 0; i < 34; ++i) B[q][i] *= wq[q];
    const int n = 34 + 18, m = nd, w = n + m;
    std::vector<ld> A((size_t)n * w, 0);
    for (int i = 0; i < 34; ++i) {
        for (int j = 0; j < 34; ++j) {
            ld s = 0;
            for (int q = 0; q < nB; ++q) s += B[q][i] * B[q][j];
            A[i * w + j] = s;
        }
        for (int k = 0; k < 18; ++k) A[i * w + 34 + k] = C[k][i];
        /* right-hand side for the derivative data: (W B)^T W e_q */
        for (int q = 0; q < nB; ++q) A[i * w + n + 18 + q] = wq[q] * B[q][i];
    }
    for (int k = 0; k < 18; ++k) {
        for (int j = 0; j < 34; ++j) A[(34 + k) * w + j] = C[k][j];
        A[(34 + k) * w + n + k] = 1;  /* right-hand side for d_C */
    }
    if (gauss_jordan(n, m, A)) { T.ok = 0; return T; }
    for (int i = 0; i < 34; ++i)
        for (int c = 0; c < nd; ++c) T.R[i][c] = (double)A[i * w + n + c];
    T.nd = nd;
    T.nB = nB;

    for (int i = 0; i < 34; ++i) T.mean0[i] = (double)avg_mono(z, b.d[i]);
    T.ok = 1;
    return T;
}

const Recon5Tables &tables(int variant = 0) {
    static Recon5Tables T[2];
    static std::once_flag once[2];
    std::call_once(once[variant ? 1 : 0], [variant] { T[variant ? 1 : 0] = build_tables(variant); });
    return T[variant ? 1 : 0];
}

const Basis &basis() {
    static const Basis b = make_basis();
    return b;
}

/* value and normalised gradient of p_d at x */
void eval_basis(const double x[3], double p[34], double dp[3][34]) {
    const Basis &b = basis();
    const Recon5Tables &T = tables();
    for (int i = 0; i < 34; ++i) {
        const int *d = b.d[i];
        double v = 1.0;
        for (int j = 0; j < 3; ++j) v *= std::pow(x[j], d[j]) / (double)fact(d[j]);
        p[i] = v - T.mean0[i];
        for (int q = 0; q < 3; ++q) {
            if (d[q] == 0) { dp[q][i] = 0.0; continue; }
            double g = 1.0;
            for (int j = 0; j < 3; ++j) {
                const int e = d[j] - (j == q ? 1 : 0);
                g *= std::pow(x[j], e) / (double)fact(e);
            }
            dp[q][i] = g;
        }
    }
}

}  // namespace

/* GENO's switch chi (reading R5). The quartic P4 of Eq. compact-big-5
 * meets the 18 neighbour averages exactly and the 45 derivative data in
 * the weighted least-squares sense; what it cannot meet measures how far
 * the stencil's data are from one smooth function:
 *   sigma = |W (B a - d_B)|^2 / (|d_C|^2 + |W d_B|^2 + (kappa S)^2 + eps),
 * W the row weights of R3, d_C the 18 average differences, d_B the 45
 * derivative data. sigma = 0 for data sampled from any quartic, O(h^8) for
 * a smooth field (the least-squares residual is the quintic remainder,
 * O(h^4) relative to the data), O(1) across a discontinuity. S is the
 * cell's own magnitude (rho; rho E; sqrt(rho rho E) for a momentum
 * component) and kappa = 0.01: variations below about a percent of it are
 * not limited. chi = 1/(1 + s + s^2), s = sigma/sigma0, sigma0 = 5e-4:
 * 1 - chi = O(h^8) on smooth data and grows only linearly with a small
 * misfit (no sharp switch on smooth but under-resolved data, whose
 * rounding it would amplify), chi ~ s^-2 at a discontinuity (chi < 1e-3
 * where sigma > 0.016; a jump through the cell gives 0.02 to 0.1). */
double geno_misfit(const double *q0, const double *d, const double *a, int v, int variant) {
    const Recon5Tables &T = tables(variant);
    const double eps = 1e-15, kappa = 0.01;
    double res2 = 0.0, norm2 = 0.0;
    for (int k = 0; k < 18; ++k) norm2 += d[k] * d[k];
    for (int q = 0; q < T.nB; ++q) {
        double Ba = 0.0;
        for (int i = 0; i < 34; ++i) Ba += T.B[q][i] * a[i];
        const double r = T.wq[q] * (Ba - d[18 + q]);
        const double wd = T.wq[q] * d[18 + q];
        res2 += r * r;
        norm2 += wd * wd;
    }
    double S;
    if (v == 0) S = q0[0];
    else if (v == 4) S = q0[4];
    else S = std::sqrt(std::fabs(q0[0] * q0[4]));
    return res2 / (norm2 + kappa * kappa * S * S + eps);
}

double geno_chi(double sigma) {
    const double s = sigma / 5e-4;
    return 1.0 / (1.0 + s + s * s);
}

void recon5_cell(const double *q0, const double *dvec, double hx, double hy,
                 double hz, int nonlinear, double *out, double *chi5, int variant) {
    const Recon5Tables &T = tables(variant);
    const double h[3] = {hx, hy, hz};
    /* GENO constants of Eq. weno-new */
    const double eps = 1e-15, dm = 1.0 / 6.0;
    double val[5][24], grad[5][24][3];
    for (int v = 0; v < 5; ++v) {
        const double *d = dvec + T.nd * v;
        double a[34];
        for (int i = 0; i < 34; ++i) {
            double s = 0.0;
            for (int c = 0; c < T.nd; ++c) s += T.R[i][c] * d[c];
            a[i] = s;
        }
        /* the own averaged gradient (normalised): stored, or the mean of
         * the four line derivatives per axis (reading B) */
        double g0[3];
        for (int j = 0; j < 3; ++j)
            g0[j] = variant ? 0.25 * (d[60 + 4 * j] + d[61 + 4 * j] + d[62 + 4 * j] + d[63 + 4 * j])
                            : d[60 + j];
        double chi = 1.0, w[6] = {0, 0, 0, 0, 0, 0}, bm[6][3];
        if (nonlinear) {
            /* linear sub-stencil polynomials P1_m (reading R4) and their
             * ENO weights of Eq. weno-new */
            double wsum = 0.0;
            for (int m = 0; m < 6; ++m) {
                const int ax = m / 2;
                const double sg = (m % 2) ? 1.0 : -1.0;
                for (int j = 0; j < 3; ++j) bm[m][j] = g0[j];
                bm[m][ax] = sg * d[m];
                const double IS = bm[m][0] * bm[m][0] + bm[m][1] * bm[m][1] + bm[m][2] * bm[m][2];
                w[m] = dm / std::pow(IS + eps, 5);
                wsum += w[m];
            }
            for (int m = 0; m < 6; ++m) w[m] /= wsum;
            chi = geno_chi(geno_misfit(q0, d, a, v, variant));
        }
        if (chi5) chi5[v] = chi;
        for (int f = 0; f < 6; ++f)
            for (int k = 0; k < 4; ++k) {
                double x[3], p[34], dp[3][34];
                face_gauss_point(f, k, x);
                eval_basis(x, p, dp);
                double P4 = q0[v], dP4[3] = {0, 0, 0};
                for (int i = 0; i < 34; ++i) {
                    P4 += a[i] * p[i];
                    for (int j = 0; j < 3; ++j) dP4[j] += a[i] * dp[j][i];
                }
                double Q = P4, dQ[3] = {dP4[0], dP4[1], dP4[2]};
                if (nonlinear) {
                    double P1 = 0.0, dP1[3] = {0, 0, 0};
                    for (int m = 0; m < 6; ++m) {
                        P1 += w[m] * (q0[v] + bm[m][0] * x[0] + bm[m][1] * x[1] +
                                      bm[m][2] * x[2]);
                        for (int j = 0; j < 3; ++j) dP1[j] += w[m] * bm[m][j];
                    }
                    Q = chi * P4 + (1.0 - chi) * P1;
                    for (int j = 0; j < 3; ++j) dQ[j] = chi * dP4[j] + (1.0 - chi) * dP1[j];
                }
                val[v][f * 4 + k] = Q;
                for (int j = 0; j < 3; ++j) grad[v][f * 4 + k][j] = dQ[j] / h[j];
            }
    }
    /* face-frame output */
    for (int f = 0; f < 6; ++f) {
        const int d = f / 2;
        for (int k = 0; k < 4; ++k) {
            double *o = out + (f * 4 + k) * 20;
            const int g = f * 4 + k;
            for (int c = 0; c < 5; ++c) {
                /* component c of the face-frame conserved vector */
                const int v = (c >= 1 && c <= 3) ? 1 + frame_axis(d, c - 1) : c;
                o[c] = val[v][g];
                for (int j = 0; j < 3; ++j) o[5 + 5 * j + c] = grad[v][g][frame_axis(d, j)];
            }
        }
    }
}

void recon2_cell(const double *q7, double hx, double hy, double hz,
                 int nonlinear, double *out, double *phi5) {
    const double h[3] = {hx, hy, hz};
    /* Venkatakrishnan parameter (reading R9) */
    const double hv = std::cbrt(hx * hy * hz);
    const double eps2 = hv * hv * hv;
    double b[5][3], phi[5];
    for (int v = 0; v < 5; ++v) {
        const double Q0 = q7[v];
        /* least squares of Sec. 3.3: averages of P1 over the six face
         * neighbours, Q0 + b . offset = Q_m, solved by normal equations  */
        double A[6][3], r[6];
        for (int m = 0; m < 6; ++m) {
            for (int j = 0; j < 3; ++j) A[m][j] = kFace[m][j];
            r[m] = q7[5 * (m + 1) + v] - Q0;
        }
        double N[9], rhs[3];
        for (int i = 0; i < 3; ++i) {
            rhs[i] = 0.0;
            for (int m = 0; m < 6; ++m) rhs[i] += A[m][i] * r[m];
            for (int j = 0; j < 3; ++j) {
                double s = 0.0;
                for (int m = 0; m < 6; ++m) s += A[m][i] * A[m][j];
                N[3 * i + j] = s;
            }
        }
        solve_dense(3, N, rhs, b[v]);
        phi[v] = 1.0;
        if (nonlinear) {
            double qmax = Q0, qmin = Q0;
            for (int m = 0; m < 6; ++m) {
                const double q = q7[5 * (m + 1) + v];
                if (q > qmax) qmax = q;
                if (q < qmin) qmin = q;
            }
            for (int f = 0; f < 6; ++f) {
                double xf[3] = {0, 0, 0};
                xf[f / 2] = (f % 2) ? 0.5 : -0.5;
                const double d2 = b[v][0] * xf[0] + b[v][1] * xf[1] + b[v][2] * xf[2];
                double pf = 1.0;
                if (d2 != 0.0) {
                    const double dp = (d2 > 0.0) ? qmax - Q0 : qmin - Q0;
                    pf = (dp * dp + eps2 + 2.0 * d2 * dp) /
                         (dp * dp + 2.0 * d2 * d2 + d2 * dp + eps2);
                }
                if (pf < phi[v]) phi[v] = pf;
            }
        }
        if (phi5) phi5[v] = phi[v];
    }
    for (int f = 0; f < 6; ++f) {
        const int d = f / 2;
        double xf[3] = {0, 0, 0};
        xf[d] = (f % 2) ? 0.5 : -0.5;
        double *o = out + f * 20;
        for (int c = 0; c < 5; ++c) {
            const int v = (c >= 1 && c <= 3) ? 1 + frame_axis(d, c - 1) : c;
            o[c] = q7[v] + phi[v] * (b[v][0] * xf[0] + b[v][1] * xf[1] + b[v][2] * xf[2]);
            for (int j = 0; j < 3; ++j) {
                const int ax = frame_axis(d, j);
                o[5 + 5 * j + c] = phi[v] * b[v][ax] / h[ax];
            }
        }
    }
}

}  // namespace orc

extern "C" int orc_recon5_matrix(double *R) {
    const orc::Recon5Tables &T = orc::tables(0);
    if (!T.ok) return -1;
    for (int i = 0; i < 34; ++i)
        for (int c = 0; c < 63; ++c) R[i * 63 + c] = T.R[i][c];
    return 0;
}

extern "C" int orc_recon5b_matrix(double *R) {
    const orc::Recon5Tables &T = orc::tables(1);
    if (!T.ok) return -1;
    for (int i = 0; i < 34; ++i)
        for (int c = 0; c < 72; ++c) R[i * 72 + c] = T.R[i][c];
    return 0;
}

extern "C" int orc_geno_misfit(const double *q0, const double *dvec, double *sigma5) {
    if (!orc::tables().ok) return -1;
    for (int v = 0; v < 5; ++v) {
        const double *d = dvec + 63 * v;
        double a[34];
        for (int i = 0; i < 34; ++i) {
            double s = 0.0;
            for (int c = 0; c < 63; ++c) s += orc::tables().R[i][c] * d[c];
            a[i] = s;
        }
        sigma5[v] = orc::geno_misfit(q0, d, a, v, 0);
    }
    return 0;
}

extern "C" int orc_recon5_cell(const double *q0, const double *dvec, double hx,
                               double hy, double hz, int nonlinear,
                               double *out480, double *chi5) {
    if (!orc::tables().ok) return -1;
    orc::recon5_cell(q0, dvec, hx, hy, hz, nonlinear, out480, chi5, 0);
    return 0;
}

extern "C" int orc_recon5b_cell(const double *q0, const double *dvec, double hx,
                                double hy, double hz, int nonlinear,
                                double *out480, double *chi5) {
    if (!orc::tables(1).ok) return -1;
    orc::recon5_cell(q0, dvec, hx, hy, hz, nonlinear, out480, chi5, 1);
    return 0;
}

extern "C" int orc_recon2_cell(const double *q7, double hx, double hy,
                               double hz, int nonlinear, double *out120,
                               double *phi5) {
    orc::recon2_cell(q7, hx, hy, hz, nonlinear, out120, phi5);
    return 0;
}
