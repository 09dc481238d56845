/*
 * Oracle: CGKS-5th with reading B of the target cell's data (row N2,
 * reading R17; Sec. 3.1-3.2: S^0 = {Q_0, (d_l Q)_{0,G}}). Grids uniform or
 * stretched along each axis, each axis periodic or bounded by mirror ghosts
 * (reading R15: a symmetry plane or an outflow boundary; a ghost's average
 * is s Q and its lines' mean along the normal -s, along the boundary s
 * times the cell's; a boundary face pairs the cell's own face states with
 * their mirror image).
 * Test infrastructure only (see oracle.h).
 *
 * State: Q[v][k][j][i] and the line-averaged derivatives
 * L[v][4a + g][k][j][i]: for axis a and face Gauss point g (the tangential
 * position of face_gauss_point on the faces normal to a), the derivative
 * along a averaged over the line through the cell between the two face
 * points, (Q(x_a + h_a/2) - Q(x_a - h_a/2))/h_a (Sec. 3.1). A cell's
 * averaged gradient along a is the mean of its four lines (2 x 2 Gauss
 * quadrature of the face averages of Gauss's theorem).
 *
 * Data vector (72 per variable, recon.cpp): the neighbours' averages, the
 * face neighbours' averaged gradients, the edge neighbours' tangential
 * derivatives (both from their lines' means), and the target cell's 12
 * lines. Update (Sec. 3.1, 3.4): Q as in reading A; every line from the
 * time-accurate interface values at its two face Gauss points:
 *   stage 1: L* = (Q^l_hi(dt/2) - Q^r_lo(dt/2))/h_a, Q(dt/2) = Q + dt/2 dQ/dt,
 *            S1 = (Q^l_hi - Q^r_lo)/h_a;
 *   stage 2: L^{n+1} = S1 + dt (dQ^l/dt at hi - dQ^r/dt at lo)/h_a (stage-2
 *            interface values),
 * the same two-stage update as the cell gradients of reading A, point by
 * point instead of averaged over the face.
 */
#include "oracle_internal.h"

#include <cmath>
#include <cstring>
#include <vector>

namespace orc {
namespace {

const int kF[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
const int kE[12][3] = {{-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 1, 0},
                       {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1}, {1, 0, 1},
                       {0, -1, -1}, {0, 1, -1}, {0, -1, 1}, {0, 1, 1}};

struct GridB {
    int nx, ny, nz;
    long n;
    int bc[3];
    std::vector<double> hs[3];
    int len(int a) const { return a == 0 ? nx : (a == 1 ? ny : nz); }
    long cell(int i, int j, int k) const { return ((long)k * ny + j) * nx + i; }
    /* neighbour of (i, j, k) at offset o: its cell, coordinates and the axes
     * across whose boundary it was mirrored (bit a of flip) */
    long nbr(int i, int j, int k, int o0, int o1, int o2, int c3[3], int &flip) const {
        const int c0[3] = {i + o0, j + o1, k + o2};
        flip = 0;
        for (int a = 0; a < 3; ++a) {
            const int m = len(a);
            int x = c0[a];
            if (bc[a] == 0) {
                x = (x % m + m) % m;
            } else if (x < 0) {
                x = -1 - x;
                flip |= 1 << a;
            } else if (x >= m) {
                x = 2 * m - 1 - x;
                flip |= 1 << a;
            }
            c3[a] = x;
        }
        return cell(c3[0], c3[1], c3[2]);
    }
    long idx(int i, int j, int k) const {
        int c3[3], f;
        return nbr(i, j, k, 0, 0, 0, c3, f);
    }
    /* sign of variable v's average in a ghost mirrored across the axes of
     * flip (the normal momentum of a symmetry plane changes sign) */
    double sval(int v, int flip) const {
        double s = 1.0;
        for (int a = 0; a < 3; ++a)
            if ((flip >> a & 1) && bc[a] == 1 && v == 1 + a) s = -s;
        return s;
    }
    /* sign of its derivatives along axis q */
    double sder(int v, int q, int flip) const {
        return (flip >> q & 1) ? -sval(v, flip) : sval(v, flip);
    }
    long plane(int d, int i, int j, int k) const {
        return d == 0 ? (long)j + (long)ny * k : (d == 1 ? (long)i + (long)nx * k
                                                         : (long)i + (long)nx * j);
    }
    long nplane() const {
        long a = (long)ny * nz, b = (long)nx * nz, c = (long)nx * ny;
        return a > b ? (a > c ? a : c) : (b > c ? b : c);
    }
    void ijk(long c, int &i, int &j, int &k) const {
        i = (int)(c % nx);
        j = (int)((c / nx) % ny);
        k = (int)(c / ((long)nx * ny));
    }
};

GridB make_grid_b(const orc_params &P) {
    GridB g;
    g.nx = P.nx; g.ny = P.ny; g.nz = P.nz;
    g.n = (long)P.nx * P.ny * P.nz;
    const double Ls[3] = {P.Lx, P.Ly, P.Lz};
    const double *h[3] = {P.hx, P.hy, P.hz};
    for (int a = 0; a < 3; ++a) {
        g.bc[a] = P.bc[a];
        g.hs[a].resize(g.len(a));
        for (int i = 0; i < g.len(a); ++i) g.hs[a][i] = h[a] ? h[a][i] : Ls[a] / g.len(a);
    }
    return g;
}

/* averaged gradient component a of variable v in cell c: the mean of its
 * four lines along a */
double grad_of(const GridB &g, const double *L, int v, int a, long c) {
    const long n = g.n;
    double s = 0.0;
    for (int k = 0; k < 4; ++k) s += L[(v * 12 + 4 * a + k) * n + c];
    return 0.25 * s;
}

void cell_face_states_b(const orc_params &P, const GridB &g, const double *Q, const double *L,
                        long c, double *o, double *chi5) {
    const long n = g.n;
    int i, j, k;
    g.ijk(c, i, j, k);
    const double h0[3] = {g.hs[0][i], g.hs[1][j], g.hs[2][k]};
    double q0[5], d[5 * 72];
    for (int v = 0; v < 5; ++v) {
        q0[v] = Q[v * n + c];
        double *dv = d + 72 * v;
        /* a neighbour (or mirror ghost) at c3 with flips fl: its average
         * s Q, its gradient from its lines' means with the derivative signs
         * of the mirror, scaled by its own sizes */
        for (int m = 0; m < 6; ++m) {
            int c3[3], fl;
            const long nb = g.nbr(i, j, k, kF[m][0], kF[m][1], kF[m][2], c3, fl);
            dv[m] = g.sval(v, fl) * Q[v * n + nb] - q0[v];
            for (int a = 0; a < 3; ++a)
                dv[18 + 3 * m + a] = g.hs[a][c3[a]] * g.sder(v, a, fl) * grad_of(g, L, v, a, nb);
        }
        for (int e = 0; e < 12; ++e) {
            int c3[3], fl;
            const long nb = g.nbr(i, j, k, kE[e][0], kE[e][1], kE[e][2], c3, fl);
            dv[6 + e] = g.sval(v, fl) * Q[v * n + nb] - q0[v];
            const int *o3 = kE[e];
            int ax[2], na = 0, ez = 0;
            for (int a = 0; a < 3; ++a) {
                if (o3[a] != 0) ax[na++] = a; else ez = a;
            }
            double gd[3];
            for (int a = 0; a < 3; ++a) gd[a] = g.hs[a][c3[a]] * g.sder(v, a, fl) * grad_of(g, L, v, a, nb);
            dv[36 + 2 * e] = (o3[ax[0]] * gd[ax[0]] - o3[ax[1]] * gd[ax[1]]) / std::sqrt(2.0);
            dv[36 + 2 * e + 1] = gd[ez];
        }
        for (int a = 0; a < 3; ++a)
            for (int kk = 0; kk < 4; ++kk)
                dv[60 + 4 * a + kk] = h0[a] * L[(v * 12 + 4 * a + kk) * n + c];
    }
    recon5_cell(q0, d, h0[0], h0[1], h0[2], P.nonlinear, o, chi5, 1);
}

/* face records of reading B, per axis d and cell c (the face on c's low
 * side): [0..9] F^n, F_t^n averaged over the Gauss points, then for each
 * Gauss point p: Q^l, dQ^l/dt, Q^r, dQ^r/dt at 10 + 20 p, global frame;
 * rec_hi [3][90][np]: the same for the faces on the high boundary of a
 * non-periodic axis (plane position of the cell inside) */
constexpr int kRecB = 90;

/* mirror image of a cell's face states across its face of normal axis d
 * (face frame: [0..4] values, [5..9] d/dn, [10..19] d/dt1, d/dt2;
 * component 1 the normal momentum), the 4 Gauss points in place */
void mirror_face_b(const GridB &g, int d, const double *s, double *m) {
    const double sn = g.bc[d] == 1 ? -1.0 : 1.0;
    for (int p = 0; p < 4; ++p)
        for (int v = 0; v < 5; ++v) {
            const double sv = v == 1 ? sn : 1.0;
            m[20 * p + v] = sv * s[20 * p + v];
            m[20 * p + 5 + v] = -sv * s[20 * p + 5 + v];
            m[20 * p + 10 + v] = sv * s[20 * p + 10 + v];
            m[20 * p + 15 + v] = sv * s[20 * p + 15 + v];
        }
}

/* the 90 record values of one face from its left and right states */
int face_record_b(const orc_params &P, int d, const double *sl, const double *sr, double dt,
                  double *r90) {
    double acc[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    int rc = 0;
    for (int p = 0; p < 4; ++p) {
        double out[30];
        const int e = flux_gp(P, sl + 20 * p, sr + 20 * p, dt, out);
        if (e) rc = e;
        for (int q = 0; q < 10; ++q) acc[q] += 0.25 * out[q];
        for (int blk = 0; blk < 4; ++blk) {
            const double *a = out + 10 + 5 * blk;
            double *gl = r90 + 10 + 20 * p + 5 * blk;
            gl[0] = a[0];
            gl[4] = a[4];
            for (int jj = 0; jj < 3; ++jj) gl[1 + frame_axis(d, jj)] = a[1 + jj];
        }
    }
    for (int blk = 0; blk < 2; ++blk) {
        const double *a = acc + 5 * blk;
        double *gl = r90 + 5 * blk;
        gl[0] = a[0];
        gl[4] = a[4];
        for (int jj = 0; jj < 3; ++jj) gl[1 + frame_axis(d, jj)] = a[1 + jj];
    }
    return rc;
}

int face_fluxes_b(const orc_params &P, const GridB &g, const std::vector<double> &fs, double dt,
                  double *rec, double *rec_hi) {
    const long n = g.n, np = g.nplane();
    int err = 0;
    for (int d = 0; d < 3; ++d) {
#pragma omp parallel for num_threads(P.threads > 0 ? P.threads : 1) schedule(static)
        for (long c = 0; c < n; ++c) {
            int i, j, k;
            g.ijk(c, i, j, k);
            const int cd = d == 0 ? i : (d == 1 ? j : k);
            double r90[kRecB], ghost[80];
            const double *sr = &fs[((size_t)c * 6 + 2 * d) * 4 * 20];
            const double *sl;
            if (g.bc[d] != 0 && cd == 0) {
                mirror_face_b(g, d, sr, ghost);
                sl = ghost;
            } else {
                const long left = g.idx(i - (d == 0), j - (d == 1), k - (d == 2));
                sl = &fs[((size_t)left * 6 + 2 * d + 1) * 4 * 20];
            }
            int rc = face_record_b(P, d, sl, sr, dt, r90);
            for (int q = 0; q < kRecB; ++q) rec[((size_t)d * kRecB + q) * n + c] = r90[q];
            if (g.bc[d] != 0 && cd == g.len(d) - 1) {
                const double *sh = &fs[((size_t)c * 6 + 2 * d + 1) * 4 * 20];
                mirror_face_b(g, d, sh, ghost);
                const int rc2 = face_record_b(P, d, sh, ghost, dt, r90);
                if (rc2) rc = rc2;
                for (int q = 0; q < kRecB; ++q)
                    rec_hi[((size_t)d * kRecB + q) * np + g.plane(d, i, j, k)] = r90[q];
            }
            if (rc) {
#pragma omp atomic write
                err = rc;
            }
        }
    }
    return err;
}

/* record value q of the face on cell c's high side along d */
double high_rec_b(const GridB &g, const double *rec, const double *rec_hi, int d, int q, long c) {
    int i, j, k;
    g.ijk(c, i, j, k);
    const int cd = d == 0 ? i : (d == 1 ? j : k);
    if (g.bc[d] != 0 && cd == g.len(d) - 1)
        return rec_hi[((size_t)d * kRecB + q) * g.nplane() + g.plane(d, i, j, k)];
    const long hi = g.idx(i + (d == 0), j + (d == 1), k + (d == 2));
    return rec[((size_t)d * kRecB + q) * g.n + hi];
}

void face_states_b(const orc_params &P, const GridB &g, const double *Q, const double *L,
                   std::vector<double> &fs) {
    fs.assign((size_t)g.n * 6 * 4 * 20, 0.0);
#pragma omp parallel for num_threads(P.threads > 0 ? P.threads : 1) schedule(static)
    for (long c = 0; c < g.n; ++c) cell_face_states_b(P, g, Q, L, c, &fs[(size_t)c * 480], nullptr);
}

void operator_L_b(const GridB &g, const double *rec, const double *rec_hi, double *Lq, double *Lt) {
    const long n = g.n;
    for (long c = 0; c < n; ++c) {
        int i, j, k;
        g.ijk(c, i, j, k);
        const double h0[3] = {g.hs[0][i], g.hs[1][j], g.hs[2][k]};
        for (int v = 0; v < 5; ++v) {
            double s = 0.0, st = 0.0;
            for (int d = 0; d < 3; ++d) {
                s += (high_rec_b(g, rec, rec_hi, d, v, c) - rec[((size_t)d * kRecB + v) * n + c]) / h0[d];
                st += (high_rec_b(g, rec, rec_hi, d, 5 + v, c) -
                       rec[((size_t)d * kRecB + 5 + v) * n + c]) / h0[d];
            }
            Lq[v * n + c] = -s;
            Lt[v * n + c] = -st;
        }
    }
}

/* record value: Gauss point p's interface value block blk (0 Q^l, 1 dQ^l/dt,
 * 2 Q^r, 3 dQ^r/dt), variable v, of the face normal to d on cell c's low side */
inline double ivb(const double *rec, long n, int d, int p, int blk, int v, long c) {
    return rec[((size_t)d * kRecB + 10 + 20 * p + 5 * blk + v) * n + c];
}

double time_step_b(const orc_params &P, const GridB &g, const double *Q) {
    const long n = g.n;
    double rate = 0.0, numax = 0.0;
    for (long c = 0; c < n; ++c) {
        double W[5];
        for (int v = 0; v < 5; ++v) W[v] = Q[v * n + c];
        const Prim p = primitive(W, P.gamma);
        const double cs = std::sqrt(P.gamma * p.p / p.rho);
        const double vel[3] = {p.U, p.V, p.W};
        int i, j, k;
        g.ijk(c, i, j, k);
        const double h0[3] = {g.hs[0][i], g.hs[1][j], g.hs[2][k]};
        for (int d = 0; d < 3; ++d) {
            const double r = (std::fabs(vel[d]) + cs) / h0[d];
            if (r > rate) rate = r;
        }
        double mu = P.mu0;
        if (P.mu_law) {
            const double th = (p.p / p.rho) / P.T_ref;
            mu = P.mu0 * 1.4042 * th * std::sqrt(th) / (th + 0.4042);
        }
        const double nu = mu / p.rho;
        if (nu > numax) numax = nu;
    }
    double dt = P.cfl / rate;
    if (!P.inviscid && numax > 0.0) {
        double hmin = INFINITY;
        for (int a = 0; a < 3; ++a)
            for (int i = 0; i < g.len(a); ++i) hmin = std::fmin(hmin, g.hs[a][i]);
        const double dv = P.cfl * hmin * hmin / (3.0 * numax);
        if (dv < dt) dt = dv;
    }
    return dt;
}

}  // namespace
}  // namespace orc

using namespace orc;

extern "C" int orc_face_states_b(const orc_params *P, const double *Q, const double *L,
                                 double *fs_out) {
    if (!P->scheme) return -1;
    for (int a = 0; a < 3; ++a)
        if (P->bc[a] < 0 || P->bc[a] > 2) return -1;
    const GridB g = make_grid_b(*P);
    std::vector<double> fs;
    face_states_b(*P, g, Q, L, fs);
    for (long c = 0; c < g.n; ++c)
        for (int f = 0; f < 6; ++f)
            for (int k = 0; k < 4; ++k)
                for (int q = 0; q < 20; ++q)
                    fs_out[(((size_t)f * 4 + k) * 20 + q) * g.n + c] =
                        fs[(((size_t)c * 6 + f) * 4 + k) * 20 + q];
    return 0;
}

extern "C" int orc_run_b(const orc_params *P, double *Q, double *L, int nsteps, double t_stop,
                         double *t, double *dt_last) {
    if (!P->scheme) return -1;
    for (int a = 0; a < 3; ++a)
        if (P->bc[a] < 0 || P->bc[a] > 2) return -1;
    const GridB g = make_grid_b(*P);
    const long n = g.n;
    std::vector<double> fs, rec((size_t)3 * kRecB * n), rec_hi((size_t)3 * kRecB * g.nplane()),
        Lq1(5 * n), Lt1(5 * n), Lq(5 * n), Lt(5 * n), Qs(5 * n), Ls(60 * n), S1(60 * n);
    /* interface value of Gauss point p, block blk (0 Q^l, 1 dQ^l/dt, 2 Q^r,
     * 3 dQ^r/dt), variable v: on the face at c's high side along a (hi) or
     * at its low side */
    auto iv_hi = [&](int a, int p, int blk, int v, long c) {
        return high_rec_b(g, rec.data(), rec_hi.data(), a, 10 + 20 * p + 5 * blk + v, c);
    };
    for (int step = 0; step < nsteps; ++step) {
        double dt = time_step_b(*P, g, Q);
        if (*t + dt > t_stop) dt = t_stop - *t;
        if (!(dt > 0.0)) break;
        /* stage 1 */
        face_states_b(*P, g, Q, L, fs);
        int rc = face_fluxes_b(*P, g, fs, dt, rec.data(), rec_hi.data());
        if (rc) return rc;
        operator_L_b(g, rec.data(), rec_hi.data(), Lq1.data(), Lt1.data());
        for (long q = 0; q < 5 * n; ++q) Qs[q] = Q[q] + 0.5 * dt * Lq1[q] + 0.125 * dt * dt * Lt1[q];
        for (long c = 0; c < n; ++c) {
            int i, j, k;
            g.ijk(c, i, j, k);
            const double h0[3] = {g.hs[0][i], g.hs[1][j], g.hs[2][k]};
            for (int a = 0; a < 3; ++a) {
                for (int p = 0; p < 4; ++p)
                    for (int v = 0; v < 5; ++v) {
                        const double ql = iv_hi(a, p, 0, v, c);
                        const double qlt = iv_hi(a, p, 1, v, c);
                        const double qr = ivb(rec.data(), n, a, p, 2, v, c);
                        const double qrt = ivb(rec.data(), n, a, p, 3, v, c);
                        const size_t li = (size_t)(v * 12 + 4 * a + p) * n + c;
                        Ls[li] = ((ql + 0.5 * dt * qlt) - (qr + 0.5 * dt * qrt)) / h0[a];
                        S1[li] = (ql - qr) / h0[a];
                    }
            }
        }
        /* stage 2 */
        face_states_b(*P, g, Qs.data(), Ls.data(), fs);
        rc = face_fluxes_b(*P, g, fs, dt, rec.data(), rec_hi.data());
        if (rc) return rc;
        operator_L_b(g, rec.data(), rec_hi.data(), Lq.data(), Lt.data());
        for (long q = 0; q < 5 * n; ++q)
            Q[q] = Q[q] + dt * Lq1[q] + dt * dt / 6.0 * (Lt1[q] + 2.0 * Lt[q]);
        for (long c = 0; c < n; ++c) {
            int i, j, k;
            g.ijk(c, i, j, k);
            const double h0[3] = {g.hs[0][i], g.hs[1][j], g.hs[2][k]};
            for (int a = 0; a < 3; ++a) {
                for (int p = 0; p < 4; ++p)
                    for (int v = 0; v < 5; ++v) {
                        const double qlt = iv_hi(a, p, 1, v, c);
                        const double qrt = ivb(rec.data(), n, a, p, 3, v, c);
                        const size_t li = (size_t)(v * 12 + 4 * a + p) * n + c;
                        L[li] = S1[li] + dt * (qlt - qrt) / h0[a];
                    }
            }
        }
        *t += dt;
        if (dt_last) *dt_last = dt;
    }
    return 0;
}
