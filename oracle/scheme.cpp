/*
 * Oracle: finite-volume scheme on a Cartesian grid (Sec. 2 Eq. semi,
 * Sec. 3.1, Sec. 3.4, Sec. 4), periodic or with mirror boundaries, uniform
 * or stretched along each axis.
 * Test infrastructure only (see oracle.h).
 *
 * State layout: Q[v][k][j][i] (v = rho, rho U, rho V, rho W, rho E; x
 * fastest), G[v][axis][k][j][i] the cell-averaged gradients (CGKS-5th).
 * Face records (per axis d, per cell c, for the face on c's low-d side):
 * [F(5), F_t(5), Q^l(5), dQ^l/dt(5), Q^r(5), dQ^r/dt(5)], global frame,
 * each averaged over the face's Gauss points; on a non-periodic axis the
 * faces of the high boundary have records of their own (faces_hi).
 *
 * Boundaries (reading R15): a ghost cell beyond a non-periodic boundary is
 * the mirror image of the cell inside it. The mirrored field is
 * F_g(x) = s F(M x), M the reflection in the boundary plane and s = -1 for
 * the normal momentum of a symmetry plane (bc 1), +1 otherwise (bc 2,
 * outflow); so its average is s Q, its derivative along the normal -s dQ/dn
 * and along the plane s dQ/dt.
 * Stretched meshes (reading R16, Sec. 3.2 last paragraph): every cell is
 * mapped to one reference cell by x = x_0 + h_a delta_a per axis, and the
 * stencil is taken in the index coordinates of that map: neighbours are
 * unit cells there, their averages are used as they are and their
 * gradients as h_a dQ/dx_a with each neighbour's own h_a; the quartic is
 * the reference-cell quartic of the uniform grid and its derivatives are
 * mapped back with the target cell's 1/h_a.
 */
#include "oracle_internal.h"

#include <cmath>
#include <cstring>
#include <vector>

namespace orc {
namespace {

struct Grid {
    int nx, ny, nz;
    long n;
    int bc[3];
    bool uniform;             /* no spacing arrays: h = L/n on every axis */
    std::vector<double> hs[3];
    int len(int a) const { return a == 0 ? nx : (a == 1 ? ny : nz); }
    double h(int a, int i) const { return hs[a][i]; }
    long cell(int i, int j, int k) const { return ((long)k * ny + j) * nx + i; }
    /* neighbour of (i, j, k) at offset o: its cell, its coordinates and the
     * axes across whose boundary it was mirrored (bit a of flip) */
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
    void ijk(long c, int &i, int &j, int &k) const {
        i = (int)(c % nx);
        j = (int)((c / nx) % ny);
        k = (int)(c / ((long)nx * ny));
    }
    /* sign of variable v's average in a ghost mirrored across the axes of flip */
    double sval(int v, int flip) const {
        double s = 1.0;
        for (int a = 0; a < 3; ++a)
            if ((flip >> a & 1) && bc[a] == 1 && v == 1 + a) s = -s;
        return s;
    }
    /* sign of its derivative along axis q */
    double sder(int v, int q, int flip) const {
        return (flip >> q & 1) ? -sval(v, flip) : sval(v, flip);
    }
    /* position of a cell in the boundary plane normal to axis d */
    long plane(int d, int i, int j, int k) const {
        return d == 0 ? (long)j + (long)ny * k : (d == 1 ? (long)i + (long)nx * k
                                                         : (long)i + (long)nx * j);
    }
    long nplane() const {
        long a = (long)ny * nz, b = (long)nx * nz, c = (long)nx * ny;
        return a > b ? (a > c ? a : c) : (b > c ? b : c);
    }
};

Grid make_grid(const orc_params &P) {
    Grid g;
    g.nx = P.nx; g.ny = P.ny; g.nz = P.nz;
    g.n = (long)P.nx * P.ny * P.nz;
    const double L[3] = {P.Lx, P.Ly, P.Lz};
    const double *hs[3] = {P.hx, P.hy, P.hz};
    g.uniform = true;
    for (int a = 0; a < 3; ++a) {
        g.bc[a] = P.bc[a];
        const int m = g.len(a);
        g.hs[a].resize(m);
        for (int i = 0; i < m; ++i) g.hs[a][i] = hs[a] ? hs[a][i] : L[a] / m;
        if (hs[a]) g.uniform = false;
    }
    return g;
}

/* Ghost face states: the mirror image of a cell's own face states across
 * its face of normal axis d (face frame: [0..4] values, [5..9] d/dn,
 * [10..19] d/dt1, d/dt2; component 1 is the normal momentum). */
void mirror_face(const Grid &g, int d, const double *s, double *m, int ngp) {
    const double sn = g.bc[d] == 1 ? -1.0 : 1.0;
    for (int p = 0; p < ngp; ++p)
        for (int v = 0; v < 5; ++v) {
            const double sv = v == 1 ? sn : 1.0;
            m[20 * p + v] = sv * s[20 * p + v];
            m[20 * p + 5 + v] = -sv * s[20 * p + 5 + v];
            m[20 * p + 10 + v] = sv * s[20 * p + 10 + v];
            m[20 * p + 15 + v] = sv * s[20 * p + 15 + v];
        }
}

const int kFaceOff[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0},
                            {0, 1, 0},  {0, 0, -1}, {0, 0, 1}};
const int kEdgeOff[12][3] = {{-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 1, 0},
                             {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1}, {1, 0, 1},
                             {0, -1, -1}, {0, 1, -1}, {0, -1, 1}, {0, 1, 1}};

int nthreads(const orc_params &P) { return P.threads > 0 ? P.threads : 1; }

/* Face states of cell c (Sec. 3.2 / 3.3): o[6][ngp][20]. */
void cell_face_states(const orc_params &P, const Grid &g, const double *Q,
                      const double *G, long c, double *o, double *chi5 = nullptr) {
    const long n = g.n;
    int i, j, k;
    g.ijk(c, i, j, k);
    const double h0[3] = {g.h(0, i), g.h(1, j), g.h(2, k)};
    if (P.scheme) {
        double q0[5], d[5 * 63];
        for (int v = 0; v < 5; ++v) {
            q0[v] = Q[v * n + c];
            double *dv = d + 63 * v;
            for (int m = 0; m < 6; ++m) {
                int c3[3], fl;
                const long nb = g.nbr(i, j, k, kFaceOff[m][0], kFaceOff[m][1], kFaceOff[m][2], c3, fl);
                dv[m] = g.sval(v, fl) * Q[v * n + nb] - q0[v];
                for (int a = 0; a < 3; ++a)
                    dv[18 + 3 * m + a] = g.h(a, c3[a]) * g.sder(v, a, fl) * G[(v * 3 + a) * n + nb];
            }
            for (int e = 0; e < 12; ++e) {
                int c3[3], fl;
                const long nb = g.nbr(i, j, k, kEdgeOff[e][0], kEdgeOff[e][1], kEdgeOff[e][2], c3, fl);
                dv[6 + e] = g.sval(v, fl) * Q[v * n + nb] - q0[v];
                /* tangential derivatives of the edge neighbour (R2) */
                const int *o = kEdgeOff[e];
                int ax[2], na = 0, ez = 0;
                for (int a = 0; a < 3; ++a) {
                    if (o[a] != 0) ax[na++] = a; else ez = a;
                }
                const double da = g.h(ax[0], c3[ax[0]]) * g.sder(v, ax[0], fl) * G[(v * 3 + ax[0]) * n + nb];
                const double db = g.h(ax[1], c3[ax[1]]) * g.sder(v, ax[1], fl) * G[(v * 3 + ax[1]) * n + nb];
                dv[36 + 2 * e] = (o[ax[0]] * da - o[ax[1]] * db) / std::sqrt(2.0);
                dv[36 + 2 * e + 1] = g.h(ez, c3[ez]) * g.sder(v, ez, fl) * G[(v * 3 + ez) * n + nb];
            }
            for (int a = 0; a < 3; ++a) dv[60 + a] = h0[a] * G[(v * 3 + a) * n + c];
        }
        recon5_cell(q0, d, h0[0], h0[1], h0[2], P.nonlinear, o, chi5);
    } else {
        double q7[35];
        for (int v = 0; v < 5; ++v) q7[v] = Q[v * n + c];
        for (int m = 0; m < 6; ++m) {
            int c3[3], fl;
            const long nb = g.nbr(i, j, k, kFaceOff[m][0], kFaceOff[m][1], kFaceOff[m][2], c3, fl);
            for (int v = 0; v < 5; ++v) q7[5 * (m + 1) + v] = g.sval(v, fl) * Q[v * n + nb];
        }
        recon2_cell(q7, h0[0], h0[1], h0[2], P.nonlinear, o, nullptr);
    }
}

/* Reconstructed face states of every cell: fs[c][f][k][20]. */
void face_states(const orc_params &P, const Grid &g, const double *Q,
                 const double *G, std::vector<double> &fs) {
    const int ngp = P.scheme ? 4 : 1;
    fs.assign((size_t)g.n * 6 * ngp * 20, 0.0);
    const long n = g.n;
#pragma omp parallel for num_threads(nthreads(P)) schedule(static)
    for (long c = 0; c < n; ++c) cell_face_states(P, g, Q, G, c, &fs[(size_t)c * 6 * ngp * 20]);
}

/* Record of one face normal to axis d (Sec. 2, 3.4): the Gauss-point
 * fluxes of the left cell's high face sl[ngp][20] and the right cell's low
 * face sr[ngp][20] averaged over the face, in the global frame: rec30 =
 * (F^n, F_t^n, Q^l, dQ^l/dt, Q^r, dQ^r/dt). */
int face_record(const orc_params &P, int d, const double *sl_all, const double *sr_all,
                double dt, double rec30[30]) {
    const int ngp = P.scheme ? 4 : 1;
    const double wgt = 1.0 / ngp;
    int err = 0;
    double acc[30];
    for (int q = 0; q < 30; ++q) acc[q] = 0.0;
    for (int p = 0; p < ngp; ++p) {
        double out[30];
        const int rc = flux_gp(P, sl_all + 20 * p, sr_all + 20 * p, dt, out);
        if (rc) err = rc;
        for (int q = 0; q < 30; ++q) acc[q] += wgt * out[q];
    }
    /* back to the global frame */
    for (int blk = 0; blk < 6; ++blk) {
        const double *a = acc + 5 * blk;
        double *gl = rec30 + 5 * blk;
        gl[0] = a[0];
        gl[4] = a[4];
        for (int jj = 0; jj < 3; ++jj) gl[1 + frame_axis(d, jj)] = a[1 + jj];
    }
    return err;
}

/* Records of every face: rec [3][30][cells] for the faces on each cell's
 * low side, rec_hi [3][30][np] for the high boundary of a non-periodic
 * axis. A boundary face sees the cell inside and its mirror ghost. */
int face_fluxes(const orc_params &P, const Grid &g, const std::vector<double> &fs,
                double dt, double *rec, double *rec_hi) {
    const int ngp = P.scheme ? 4 : 1;
    const long n = g.n, np = g.nplane();
    int err = 0;
    for (int d = 0; d < 3; ++d) {
#pragma omp parallel for num_threads(nthreads(P)) schedule(static)
        for (long c = 0; c < n; ++c) {
            int i, j, k;
            g.ijk(c, i, j, k);
            const int cd = d == 0 ? i : (d == 1 ? j : k);
            double r30[30], ghost[4 * 20];
            const double *sr = &fs[((size_t)c * 6 + 2 * d) * ngp * 20];
            const double *sl;
            if (g.bc[d] != 0 && cd == 0) {
                mirror_face(g, d, sr, ghost, ngp);
                sl = ghost;
            } else {
                const long left = g.idx(i - (d == 0), j - (d == 1), k - (d == 2));
                sl = &fs[((size_t)left * 6 + 2 * d + 1) * ngp * 20];
            }
            int rc = face_record(P, d, sl, sr, dt, r30);
            for (int q = 0; q < 30; ++q) rec[((size_t)d * 30 + q) * n + c] = r30[q];
            if (g.bc[d] != 0 && cd == g.len(d) - 1) {
                const double *sh = &fs[((size_t)c * 6 + 2 * d + 1) * ngp * 20];
                mirror_face(g, d, sh, ghost, ngp);
                const int rc2 = face_record(P, d, sh, ghost, dt, r30);
                if (rc2) rc = rc2;
                for (int q = 0; q < 30; ++q)
                    rec_hi[((size_t)d * 30 + q) * np + g.plane(d, i, j, k)] = r30[q];
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
double high_rec(const Grid &g, const double *rec, const double *rec_hi, int d, int q, long c) {
    int i, j, k;
    g.ijk(c, i, j, k);
    const int cd = d == 0 ? i : (d == 1 ? j : k);
    if (g.bc[d] != 0 && cd == g.len(d) - 1)
        return rec_hi[((size_t)d * 30 + q) * g.nplane() + g.plane(d, i, j, k)];
    const long hi = g.idx(i + (d == 0), j + (d == 1), k + (d == 2));
    return rec[((size_t)d * 30 + q) * g.n + hi];
}

/* L = -(1/|Omega|) sum_faces F.n S (Eq. semi), and its time derivative. */
void operator_L(const Grid &g, const double *rec, const double *rec_hi, double *L, double *Lt) {
    const long n = g.n;
    for (long c = 0; c < n; ++c) {
        int i, j, k;
        g.ijk(c, i, j, k);
        const double h0[3] = {g.h(0, i), g.h(1, j), g.h(2, k)};
        for (int v = 0; v < 5; ++v) {
            double s = 0.0, st = 0.0;
            for (int d = 0; d < 3; ++d) {
                s += (high_rec(g, rec, rec_hi, d, v, c) - rec[((size_t)d * 30 + v) * n + c]) / h0[d];
                st += (high_rec(g, rec, rec_hi, d, 5 + v, c) - rec[((size_t)d * 30 + 5 + v) * n + c]) / h0[d];
            }
            L[v * n + c] = -s;
            Lt[v * n + c] = -st;
        }
    }
}

double viscosity(const orc_params &P, double rho, double p) {
    if (P.mu_law == 0) return P.mu0;
    const double th = (p / rho) / P.T_ref;
    return P.mu0 * 1.4042 * th * std::sqrt(th) / (th + 0.4042);
}

/* Sec. 4: convective CFL bound and the viscous bound CFL h^2/(3 nu).    */
double time_step(const orc_params &P, const Grid &g, const double *Q) {
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
        const double h0[3] = {g.h(0, i), g.h(1, j), g.h(2, k)};
        for (int d = 0; d < 3; ++d) {
            const double r = (std::fabs(vel[d]) + cs) / h0[d];
            if (r > rate) rate = r;
        }
        const double nu = viscosity(P, p.rho, p.p) / p.rho;
        if (nu > numax) numax = nu;
    }
    double dt = P.cfl / rate;
    if (!P.inviscid && numax > 0.0) {
        double hmin = INFINITY;  /* the smallest cell size of the grid */
        for (int a = 0; a < 3; ++a)
            for (int i = 0; i < g.len(a); ++i) hmin = std::fmin(hmin, g.h(a, i));
        const double dv = P.cfl * hmin * hmin / (3.0 * numax);
        if (dv < dt) dt = dv;
    }
    return dt;
}

}  // namespace
}  // namespace orc

using namespace orc;

extern "C" int orc_face_states(const orc_params *P, const double *Q,
                               const double *G, double *fs_out) {
    const Grid g = make_grid(*P);
    std::vector<double> fs;
    face_states(*P, g, Q, G, fs);
    const int ngp = P->scheme ? 4 : 1;
    /* reorder to [f][k][20][cells] */
    for (long c = 0; c < g.n; ++c)
        for (int f = 0; f < 6; ++f)
            for (int k = 0; k < ngp; ++k)
                for (int q = 0; q < 20; ++q)
                    fs_out[(((size_t)f * ngp + k) * 20 + q) * g.n + c] =
                        fs[(((size_t)c * 6 + f) * ngp + k) * 20 + q];
    return 0;
}

extern "C" int orc_chi_field(const orc_params *P, const double *Q, const double *G,
                             double *chi) {
    if (!P->scheme) return -1;
    const Grid g = make_grid(*P);
    const long n = g.n;
#pragma omp parallel for num_threads(nthreads(*P)) schedule(static)
    for (long c = 0; c < n; ++c) {
        double o[6 * 4 * 20], c5[5];
        cell_face_states(*P, g, Q, G, c, o, c5);
        for (int v = 0; v < 5; ++v) chi[(size_t)v * n + c] = c5[v];
    }
    return 0;
}

extern "C" int orc_face_states_at(const orc_params *P, const double *Q, const double *G,
                                  const long long *cells, long long m, double *out) {
    const Grid g = make_grid(*P);
    const int ngp = P->scheme ? 4 : 1;
    for (long long s = 0; s < m; ++s) {
        if (cells[s] < 0 || cells[s] >= g.n) return -1;
        cell_face_states(*P, g, Q, G, (long)cells[s], out + (size_t)s * 6 * ngp * 20);
    }
    return 0;
}

extern "C" int orc_face_record(const orc_params *P, int d, const double *sl, const double *sr,
                               double dt, double *rec30) {
    if (d < 0 || d > 2) return -1;
    return face_record(*P, d, sl, sr, dt, rec30);
}

extern "C" int orc_stage(const orc_params *P, const double *Q, const double *G,
                         double dt, double *L, double *Lt, double *faces, double *faces_hi) {
    const Grid g = make_grid(*P);
    std::vector<double> fs;
    face_states(*P, g, Q, G, fs);
    std::vector<double> rec((size_t)3 * 30 * g.n), rec_hi((size_t)3 * 30 * g.nplane(), 0.0);
    const int rc = face_fluxes(*P, g, fs, dt, rec.data(), rec_hi.data());
    operator_L(g, rec.data(), rec_hi.data(), L, Lt);
    if (faces) std::memcpy(faces, rec.data(), sizeof(double) * rec.size());
    if (faces_hi) std::memcpy(faces_hi, rec_hi.data(), sizeof(double) * rec_hi.size());
    return rc;
}

extern "C" int orc_dt(const orc_params *P, const double *Q, double *dt) {
    *dt = time_step(*P, make_grid(*P), Q);
    return 0;
}

extern "C" int orc_run(const orc_params *P, double *Q, double *G, int nsteps,
                       double t_stop, double *t, double *dt_last) {
    const Grid g = make_grid(*P);
    const long n = g.n;
    std::vector<double> fs, rec((size_t)3 * 30 * n), L(5 * n), Lt(5 * n);
    std::vector<double> rec_hi((size_t)3 * 30 * g.nplane(), 0.0);
    std::vector<double> Qs, Gs, L1, Lt1, S1;
    for (int step = 0; step < nsteps; ++step) {
        double dt = time_step(*P, g, Q);
        if (*t + dt > t_stop) dt = t_stop - *t;
        if (!(dt > 0.0)) break;
        if (P->scheme == 0) {
            /* GKS-2nd: Q^{n+1} = Q^n + dt L + dt^2/2 dL/dt (Sec. 3.4) */
            face_states(*P, g, Q, nullptr, fs);
            const int rc = face_fluxes(*P, g, fs, dt, rec.data(), rec_hi.data());
            if (rc) return rc;
            operator_L(g, rec.data(), rec_hi.data(), L.data(), Lt.data());
            for (long q = 0; q < 5 * n; ++q) Q[q] += dt * L[q] + 0.5 * dt * dt * Lt[q];
        } else {
            /* CGKS-5th: two-stage fourth-order update (Sec. 3.4) */
            face_states(*P, g, Q, G, fs);
            int rc = face_fluxes(*P, g, fs, dt, rec.data(), rec_hi.data());
            if (rc) return rc;
            L1.resize(5 * n);
            Lt1.resize(5 * n);
            operator_L(g, rec.data(), rec_hi.data(), L1.data(), Lt1.data());
            Qs.resize(5 * n);
            Gs.resize(15 * n);
            S1.resize(15 * n);
            for (long q = 0; q < 5 * n; ++q)
                Qs[q] = Q[q] + 0.5 * dt * L1[q] + 0.125 * dt * dt * Lt1[q];
            /* interface values: Q* = Q^n + dt/2 dQ^n/dt; the cell gradient by
             * Gauss's theorem from the face averages (Sec. 3.1)             */
            for (long c = 0; c < n; ++c) {
                int i, j, k;
                g.ijk(c, i, j, k);
                const double h0[3] = {g.h(0, i), g.h(1, j), g.h(2, k)};
                for (int d = 0; d < 3; ++d) {
                    for (int v = 0; v < 5; ++v) {
                        const double ql = high_rec(g, rec.data(), rec_hi.data(), d, 10 + v, c);
                        const double qlt = high_rec(g, rec.data(), rec_hi.data(), d, 15 + v, c);
                        const double qr = rec[((size_t)d * 30 + 20 + v) * n + c];
                        const double qrt = rec[((size_t)d * 30 + 25 + v) * n + c];
                        Gs[(v * 3 + d) * n + c] = ((ql + 0.5 * dt * qlt) - (qr + 0.5 * dt * qrt)) / h0[d];
                        S1[(v * 3 + d) * n + c] = (ql - qr) / h0[d];
                    }
                }
            }
            face_states(*P, g, Qs.data(), Gs.data(), fs);
            rc = face_fluxes(*P, g, fs, dt, rec.data(), rec_hi.data());
            if (rc) return rc;
            operator_L(g, rec.data(), rec_hi.data(), L.data(), Lt.data());
            for (long q = 0; q < 5 * n; ++q)
                Q[q] = Q[q] + dt * L1[q] + dt * dt / 6.0 * (Lt1[q] + 2.0 * Lt[q]);
            /* Q_G^{n+1} = Q_G^n + dt (dQ_G/dt at the second stage) */
            for (long c = 0; c < n; ++c) {
                int i, j, k;
                g.ijk(c, i, j, k);
                const double h0[3] = {g.h(0, i), g.h(1, j), g.h(2, k)};
                for (int d = 0; d < 3; ++d) {
                    for (int v = 0; v < 5; ++v) {
                        const double qlt = high_rec(g, rec.data(), rec_hi.data(), d, 15 + v, c);
                        const double qrt = rec[((size_t)d * 30 + 25 + v) * n + c];
                        G[(v * 3 + d) * n + c] = S1[(v * 3 + d) * n + c] + dt * (qlt - qrt) / h0[d];
                    }
                }
            }
        }
        *t += dt;
        if (dt_last) *dt_last = dt;
    }
    return 0;
}

extern "C" int orc_diagnostics(const orc_params *P, const double *Q,
                               const double *G, double *out) {
    const Grid g = make_grid(*P);
    const long n = g.n;
    /* the domain's volume: cells of one size (uniform grid), or the sum of
     * the cell volumes (stretched) */
    double Omega = g.h(0, 0) * g.h(1, 0) * g.h(2, 0) * n;
    if (!g.uniform) {
        Omega = 0.0;
        for (long c = 0; c < n; ++c) {
            int i, j, k;
            g.ijk(c, i, j, k);
            Omega += g.h(0, i) * g.h(1, j) * g.h(2, k);
        }
    }
    double ek = 0, es = 0, ed = 0, rmin = INFINITY, pmin = INFINITY, bad = 0, smax = 0;
    double sums[5] = {0, 0, 0, 0, 0};
    for (long c = 0; c < n; ++c) {
        int i, j, k;
        g.ijk(c, i, j, k);
        const double vol = g.h(0, i) * g.h(1, j) * g.h(2, k);
        double W[5];
        for (int v = 0; v < 5; ++v) {
            W[v] = Q[v * n + c];
            sums[v] += W[v] * vol;
        }
        const Prim p = primitive(W, P->gamma);
        bool ok = std::isfinite(p.rho) && std::isfinite(p.p) && p.rho > 0 && p.p > 0;
        for (int v = 0; v < 5; ++v) ok = ok && std::isfinite(W[v]);
        if (!ok) { bad += 1; continue; }
        rmin = std::fmin(rmin, p.rho);
        pmin = std::fmin(pmin, p.p);
        const double vel[3] = {p.U, p.V, p.W};
        const double cs = std::sqrt(P->gamma * p.p / p.rho);
        for (int d = 0; d < 3; ++d) smax = std::fmax(smax, std::fabs(vel[d]) + cs);
        ek += 0.5 * p.rho * (p.U * p.U + p.V * p.V + p.W * p.W) * vol;
        /* cell gradients of the conserved variables: stored (CGKS-5th) or
         * central differences of the cell averages (GKS-2nd)             */
        double dQ[5][3];
        for (int v = 0; v < 5; ++v)
            for (int d = 0; d < 3; ++d) {
                if (G) {
                    dQ[v][d] = G[(v * 3 + d) * n + c];
                } else {
                    /* centres of the two neighbours: h_c + (h_hi + h_lo)/2 apart */
                    int chi[3], clo[3], fhi, flo;
                    const long hi = g.nbr(i, j, k, d == 0, d == 1, d == 2, chi, fhi);
                    const long lo = g.nbr(i, j, k, -(d == 0), -(d == 1), -(d == 2), clo, flo);
                    const int cd = d == 0 ? i : (d == 1 ? j : k);
                    const double dist = g.uniform ? 2.0 * g.h(d, 0)
                                                  : g.h(d, cd) + 0.5 * (g.h(d, chi[d]) + g.h(d, clo[d]));
                    dQ[v][d] = (g.sval(v, fhi) * Q[v * n + hi] - g.sval(v, flo) * Q[v * n + lo]) / dist;
                }
            }
        double du[3][3];  /* du[a][d] = d U_a / dx_d */
        for (int a = 0; a < 3; ++a)
            for (int d = 0; d < 3; ++d) du[a][d] = (dQ[1 + a][d] - vel[a] * dQ[0][d]) / p.rho;
        const double wx = du[2][1] - du[1][2], wy = du[0][2] - du[2][0], wz = du[1][0] - du[0][1];
        const double div = du[0][0] + du[1][1] + du[2][2];
        const double mu = viscosity(*P, p.rho, p.p);
        es += mu * (wx * wx + wy * wy + wz * wz) * vol;
        ed += 4.0 / 3.0 * mu * div * div * vol;
    }
    out[0] = ek / Omega;
    out[1] = es / Omega;
    out[2] = ed / Omega;
    out[3] = rmin;
    out[4] = pmin;
    for (int v = 0; v < 5; ++v) out[5 + v] = sums[v];
    out[10] = bad;
    out[11] = smax;
    return 0;
}
