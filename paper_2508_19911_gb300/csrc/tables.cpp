// Host-side construction of the CGKS-5th reconstruction tables (Sec. 3.2).
//
// Eq. compact-big-5 asks for the quartic P4 = Q0 + sum_d a_d p_d that
// matches the 18 neighbour averages exactly and the 45 derivative data in
// the least-squares sense (unit weights in normalised coordinates, i.e.
// h1 = h2 = h3 = h). It is solved here by the null-space method:
//   C = [R_c^T 0] [Q1 Q2]^T   (Householder QR of C^T),
//   a = Q1 y + Q2 z,  R_c^T y = d_C,
//   z = argmin |B Q2 z - (d_B - B Q1 y)|   (Householder QR of B Q2).
// Applying this to the unit data vectors gives the 34 x 63 matrix R.
#include <cmath>
#include <memory>
#include <new>
#include <cstring>
#include <vector>

#include "basis.h"

namespace gks {
namespace {

double factorial(int n) {
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= i;
    return f;
}

// average of x^n over [o - 1/2, o + 1/2]
double avg1(int o, int n) {
    return (std::pow(o + 0.5, n + 1) - std::pow(o - 0.5, n + 1)) / (n + 1);
}

// average over the unit cell at offset o of x^e / e!
double cell_avg(const int o[3], const int e[3]) {
    double v = 1.0;
    for (int j = 0; j < 3; ++j) {
        if (e[j] < 0) return 0.0;
        v *= avg1(o[j], e[j]) / factorial(e[j]);
    }
    return v;
}

// average over offset o of d p_i / d x_q
double cell_avg_deriv(const int o[3], int i, int q) {
    int e[3] = {kExp[i][0], kExp[i][1], kExp[i][2]};
    if (e[q] == 0) return 0.0;
    e[q] -= 1;
    return cell_avg(o, e);
}

// Dense column-major helpers ------------------------------------------------
struct Mat {
    int r, c;
    std::vector<double> a;
    Mat(int rr, int cc) : r(rr), c(cc), a((size_t)rr * cc, 0.0) {}
    double &operator()(int i, int j) { return a[(size_t)j * r + i]; }
    double operator()(int i, int j) const { return a[(size_t)j * r + i]; }
};

// Householder QR: A (m x n, m >= n) -> explicit orthogonal Q (m x m) and the
// upper-triangular n x n factor Rt.
void householder_qr(const Mat &A, Mat &Q, Mat &Rt) {
    const int m = A.r, n = A.c;
    Mat W = A;
    Q = Mat(m, m);
    for (int i = 0; i < m; ++i) Q(i, i) = 1.0;
    std::vector<double> v(m);
    for (int k = 0; k < n; ++k) {
        double norm = 0.0;
        for (int i = k; i < m; ++i) norm += W(i, k) * W(i, k);
        norm = std::sqrt(norm);
        if (norm == 0.0) continue;
        const double alpha = W(k, k) > 0 ? -norm : norm;
        for (int i = 0; i < m; ++i) v[i] = (i < k) ? 0.0 : W(i, k);
        v[k] -= alpha;
        double vn = 0.0;
        for (int i = k; i < m; ++i) vn += v[i] * v[i];
        if (vn == 0.0) continue;
        // W <- (I - 2 v v^T / vn) W ; Q <- Q (I - 2 v v^T / vn)
        for (int j = 0; j < n; ++j) {
            double s = 0.0;
            for (int i = k; i < m; ++i) s += v[i] * W(i, j);
            s = 2.0 * s / vn;
            for (int i = k; i < m; ++i) W(i, j) -= s * v[i];
        }
        for (int i = 0; i < m; ++i) {
            double s = 0.0;
            for (int l = k; l < m; ++l) s += Q(i, l) * v[l];
            s = 2.0 * s / vn;
            for (int l = k; l < m; ++l) Q(i, l) -= s * v[l];
        }
    }
    Rt = Mat(n, n);
    for (int i = 0; i < n; ++i)
        for (int j = i; j < n; ++j) Rt(i, j) = W(i, j);
}

}  // namespace

int build_recon_tables(ReconTables *t) {
    std::memset(t, 0, sizeof(*t));
    constexpr int nb = kNumBasis, ne = 18, nl = 45;
    static const int zero[3] = {0, 0, 0};
    // constraint rows: neighbour cell averages of p_i (zero mean on Omega_0)
    Mat C(ne, nb);
    for (int k = 0; k < ne; ++k) {
        const int *o = (k < 6) ? kFaceOff[k] : kEdgeOff[k - 6];
        for (int i = 0; i < nb; ++i) {
            const int e[3] = {kExp[i][0], kExp[i][1], kExp[i][2]};
            C(k, i) = cell_avg(o, e) - cell_avg(zero, e);
        }
    }
    // least-squares rows in the order of the data columns 18..62
    Mat B(nl, nb);
    int r = 0;
    for (int m = 0; m < 6; ++m)
        for (int q = 0; q < 3; ++q, ++r)
            for (int i = 0; i < nb; ++i) B(r, i) = cell_avg_deriv(kFaceOff[m], i, q);
    const double rs2 = 1.0 / std::sqrt(2.0);
    for (int n = 0; n < 12; ++n) {
        const int *o = kEdgeOff[n];
        const int a = edge_axis_a(n), b = edge_axis_b(n), e = edge_axis_e(n);
        for (int i = 0; i < nb; ++i)
            B(r, i) = rs2 * (o[a] * cell_avg_deriv(o, i, a) - o[b] * cell_avg_deriv(o, i, b));
        ++r;
        for (int i = 0; i < nb; ++i) B(r, i) = cell_avg_deriv(o, i, e);
        ++r;
    }
    for (int q = 0; q < 3; ++q, ++r)
        for (int i = 0; i < nb; ++i) B(r, i) = cell_avg_deriv(zero, i, q);
    // row weights (the h_1, h_2, h_3 of Eq. compact-big-5, relative to the
    // cell size that already scales the derivative data): 1 for the face
    // neighbours' gradients and the own gradient, kEdgeWeight for the edge
    // neighbours' tangential derivatives -- near the minimum of the
    // condition number of the weighted least-squares system on the
    // constraints' null space (5.07; 29.6 with unit weights, which also
    // leaves the linear scheme with a growing grid-scale vortical mode)
    std::vector<double> wrow(nl, 1.0);
    for (int k = 0; k < nl; ++k) wrow[k] = col_weight(ne + k);
    for (int k = 0; k < nl; ++k)
        for (int i = 0; i < nb; ++i) B(k, i) *= wrow[k];

    // null-space method
    Mat Ct(nb, ne);
    for (int k = 0; k < ne; ++k)
        for (int i = 0; i < nb; ++i) Ct(i, k) = C(k, i);
    Mat Qc(1, 1), Rc(1, 1);
    householder_qr(Ct, Qc, Rc);
    const int nz = nb - ne;  // 16
    Mat BQ2(nl, nz), BQ1(nl, ne);
    for (int i = 0; i < nl; ++i) {
        for (int j = 0; j < nz; ++j) {
            double s = 0.0;
            for (int l = 0; l < nb; ++l) s += B(i, l) * Qc(l, ne + j);
            BQ2(i, j) = s;
        }
        for (int j = 0; j < ne; ++j) {
            double s = 0.0;
            for (int l = 0; l < nb; ++l) s += B(i, l) * Qc(l, j);
            BQ1(i, j) = s;
        }
    }
    Mat Qm(1, 1), Rm(1, 1);
    householder_qr(BQ2, Qm, Rm);
    for (int i = 0; i < ne; ++i)
        if (std::fabs(Rc(i, i)) < 1e-12) return -1;
    for (int i = 0; i < nz; ++i)
        if (std::fabs(Rm(i, i)) < 1e-12) return -1;

    std::vector<double> dC(ne), dB(nl), y(ne), res(nl), z(nz), rhs(nz);
    for (int col = 0; col < kNumData; ++col) {
        for (int k = 0; k < ne; ++k) dC[k] = (col == k) ? 1.0 : 0.0;
        for (int k = 0; k < nl; ++k) dB[k] = (col == ne + k) ? wrow[k] : 0.0;
        // R_c^T y = d_C (forward substitution)
        for (int i = 0; i < ne; ++i) {
            double s = dC[i];
            for (int j = 0; j < i; ++j) s -= Rc(j, i) * y[j];
            y[i] = s / Rc(i, i);
        }
        for (int i = 0; i < nl; ++i) {
            double s = dB[i];
            for (int j = 0; j < ne; ++j) s -= BQ1(i, j) * y[j];
            res[i] = s;
        }
        // z = Rm^{-1} (Qm^T res)[0..nz)
        for (int j = 0; j < nz; ++j) {
            double s = 0.0;
            for (int i = 0; i < nl; ++i) s += Qm(i, j) * res[i];
            rhs[j] = s;
        }
        for (int j = nz - 1; j >= 0; --j) {
            double s = rhs[j];
            for (int l = j + 1; l < nz; ++l) s -= Rm(j, l) * z[l];
            z[j] = s / Rm(j, j);
        }
        for (int i = 0; i < nb; ++i) {
            double s = 0.0;
            for (int j = 0; j < ne; ++j) s += Qc(i, j) * y[j];
            for (int j = 0; j < nz; ++j) s += Qc(i, ne + j) * z[j];
            t->R[i][col] = s;
        }
    }

    // R in the symmetrised data basis: column r of R T^{-1}, T^{-1} = T^T
    // diag(1/nm) (the rows of T are orthogonal); by the reflection symmetry
    // it maps a class-c combination to class-c monomials only, which is
    // checked here
    double rmax = 0.0;
    for (int i = 0; i < nb; ++i)
        for (int col = 0; col < kNumData; ++col) rmax = std::fmax(rmax, std::fabs(t->R[i][col]));
    for (int r = 0; r < kNumData; ++r) {
        const int c = kSym.cls[r];
        for (int i = 0; i < nb; ++i) {
            double s = 0.0;
            for (int q = 0; q < kSym.nm[r]; ++q) s += kSym.sgn[r][q] * t->R[i][kSym.mem[r][q]];
            s /= kSym.nm[r];
            if (parity_class(kExp[i][0], kExp[i][1], kExp[i][2]) == c)
                t->Rs[r][kClass.pos[i]] = s;
            else if (std::fabs(s) > 1e-12 * rmax)
                return -1;
        }
    }

    // GENO's misfit: the weighted derivative rows W B (B was weighted in
    // place above) in the symmetrised data basis, row r = sum_m T[r][m]
    // (W B)_m over the orbit's columns; by the reflection symmetry it has
    // entries on class(r) monomials only, which is checked here. Rows of
    // the average combinations stay zero (those data are met exactly).
    double bmax = 0.0;
    for (int k = 0; k < nl; ++k)
        for (int i = 0; i < nb; ++i) bmax = std::fmax(bmax, std::fabs(B(k, i)));
    for (int r = 0; r < kNumData; ++r) {
        if (kSym.mem[r][0] < kColFaceGrad) continue;
        const int c = kSym.cls[r];
        for (int i = 0; i < nb; ++i) {
            double s = 0.0;
            for (int q = 0; q < kSym.nm[r]; ++q)
                s += kSym.sgn[r][q] * B(kSym.mem[r][q] - ne, i);
            if (parity_class(kExp[i][0], kExp[i][1], kExp[i][2]) == c)
                t->Bs[r][kClass.pos[i]] = s;
            else if (std::fabs(s) > 1e-12 * bmax)
                return -1;
        }
    }

    // means of the monomials on the unit cell [-1/2, 1/2]^3
    auto mono_int = [](int n) { return (n % 2) ? 0.0 : std::pow(0.5, n) / (n + 1); };
    for (int i = 0; i < nb; ++i) {
        t->mean[i] = 1.0;
        for (int j = 0; j < 3; ++j) t->mean[i] *= mono_int(kExp[i][j]) / factorial(kExp[i][j]);
    }

    // magnitudes of x^e/e! and of its derivatives at the Gauss points of the
    // faces normal to axis d: |x_d| = 1/2, the two tangential |x| = g
    const double g = 0.5 / std::sqrt(3.0);
    for (int d = 0; d < 3; ++d) {
        double ax[3] = {g, g, g};
        ax[d] = 0.5;
        for (int i = 0; i < nb; ++i) {
            double v = 1.0;
            for (int j = 0; j < 3; ++j) v *= std::pow(ax[j], kExp[i][j]) / factorial(kExp[i][j]);
            t->mval[d][i] = v;
            for (int q = 0; q < 3; ++q) {
                if (kExp[i][q] == 0) { t->mder[d][q][i] = 0.0; continue; }
                double w = 1.0;
                for (int j = 0; j < 3; ++j) {
                    const int e = kExp[i][j] - (j == q ? 1 : 0);
                    w *= std::pow(ax[j], e) / factorial(e);
                }
                t->mder[d][q][i] = w;
            }
        }
    }
    return 0;
}

// Reading B of the target cell's data (line-averaged derivatives, the
// paper's S^0): the same constrained least squares with the 12 line rows
// (value of x^e/e! at the line's end on the high face minus at its end on
// the low face, tangential position of face Gauss point k) in place of the
// 3 own-gradient rows, weight 1; solved by the same null-space method.
int build_recon_tables_lines(ReconTablesLines *t) {
    std::memset(t, 0, sizeof(*t));
    constexpr int nb = kNumBasis, ne = 18, nl = 54, ncol = 72;
    static const int zero[3] = {0, 0, 0};
    Mat C(ne, nb);
    for (int k = 0; k < ne; ++k) {
        const int *o = (k < 6) ? kFaceOff[k] : kEdgeOff[k - 6];
        for (int i = 0; i < nb; ++i) {
            const int e[3] = {kExp[i][0], kExp[i][1], kExp[i][2]};
            C(k, i) = cell_avg(o, e) - cell_avg(zero, e);
        }
    }
    Mat B(nl, nb);
    int r = 0;
    for (int m = 0; m < 6; ++m)
        for (int q = 0; q < 3; ++q, ++r)
            for (int i = 0; i < nb; ++i) B(r, i) = cell_avg_deriv(kFaceOff[m], i, q);
    const double rs2 = 1.0 / std::sqrt(2.0);
    for (int n = 0; n < 12; ++n) {
        const int *o = kEdgeOff[n];
        const int a = edge_axis_a(n), b = edge_axis_b(n), e = edge_axis_e(n);
        for (int i = 0; i < nb; ++i)
            B(r, i) = rs2 * (o[a] * cell_avg_deriv(o, i, a) - o[b] * cell_avg_deriv(o, i, b));
        ++r;
        for (int i = 0; i < nb; ++i) B(r, i) = cell_avg_deriv(o, i, e);
        ++r;
    }
    const double g = 0.5 / std::sqrt(3.0);
    auto mono = [](const double x[3], int i) {
        double v = 1.0;
        for (int j = 0; j < 3; ++j) v *= std::pow(x[j], kExp[i][j]) / factorial(kExp[i][j]);
        return v;
    };
    for (int a = 0; a < 3; ++a)
        for (int k = 0; k < 4; ++k, ++r) {
            double x1[3], x2[3];
            x1[a] = -0.5;
            x2[a] = 0.5;
            x1[(a + 1) % 3] = x2[(a + 1) % 3] = (k & 1) ? g : -g;
            x1[(a + 2) % 3] = x2[(a + 2) % 3] = (k & 2) ? g : -g;
            for (int i = 0; i < nb; ++i) B(r, i) = mono(x2, i) - mono(x1, i);
        }
    std::vector<double> wrow(nl, 1.0);
    for (int k = 0; k < nl; ++k) wrow[k] = (k >= 18 && k < 42) ? kEdgeWeight : 1.0;
    for (int k = 0; k < nl; ++k) {
        t->w[k] = wrow[k];
        for (int i = 0; i < nb; ++i) {
            B(k, i) *= wrow[k];
            t->WB[k][i] = B(k, i);
        }
    }
    Mat Ct(nb, ne);
    for (int k = 0; k < ne; ++k)
        for (int i = 0; i < nb; ++i) Ct(i, k) = C(k, i);
    Mat Qc(1, 1), Rc(1, 1);
    householder_qr(Ct, Qc, Rc);
    const int nz = nb - ne;
    Mat BQ2(nl, nz), BQ1(nl, ne);
    for (int i = 0; i < nl; ++i) {
        for (int j = 0; j < nz; ++j) {
            double s = 0.0;
            for (int l = 0; l < nb; ++l) s += B(i, l) * Qc(l, ne + j);
            BQ2(i, j) = s;
        }
        for (int j = 0; j < ne; ++j) {
            double s = 0.0;
            for (int l = 0; l < nb; ++l) s += B(i, l) * Qc(l, j);
            BQ1(i, j) = s;
        }
    }
    Mat Qm(1, 1), Rm(1, 1);
    householder_qr(BQ2, Qm, Rm);
    for (int i = 0; i < ne; ++i)
        if (std::fabs(Rc(i, i)) < 1e-12) return -1;
    for (int i = 0; i < nz; ++i)
        if (std::fabs(Rm(i, i)) < 1e-12) return -1;
    std::vector<double> dC(ne), dB(nl), y(ne), res(nl), z(nz), rhs(nz);
    for (int col = 0; col < ncol; ++col) {
        for (int k = 0; k < ne; ++k) dC[k] = (col == k) ? 1.0 : 0.0;
        for (int k = 0; k < nl; ++k) dB[k] = (col == ne + k) ? wrow[k] : 0.0;
        for (int i = 0; i < ne; ++i) {
            double s = dC[i];
            for (int j = 0; j < i; ++j) s -= Rc(j, i) * y[j];
            y[i] = s / Rc(i, i);
        }
        for (int i = 0; i < nl; ++i) {
            double s = dB[i];
            for (int j = 0; j < ne; ++j) s -= BQ1(i, j) * y[j];
            res[i] = s;
        }
        for (int j = 0; j < nz; ++j) {
            double s = 0.0;
            for (int i = 0; i < nl; ++i) s += Qm(i, j) * res[i];
            rhs[j] = s;
        }
        for (int j = nz - 1; j >= 0; --j) {
            double s = rhs[j];
            for (int l = j + 1; l < nz; ++l) s -= Rm(j, l) * z[l];
            z[j] = s / Rm(j, j);
        }
        for (int i = 0; i < nb; ++i) {
            double s = 0.0;
            for (int j = 0; j < ne; ++j) s += Qc(i, j) * y[j];
            for (int j = 0; j < nz; ++j) s += Qc(i, ne + j) * z[j];
            t->R[i][col] = s;
        }
    }
    auto mono_int = [](int n) { return (n % 2) ? 0.0 : std::pow(0.5, n) / (n + 1); };
    for (int i = 0; i < nb; ++i) {
        t->mean[i] = 1.0;
        for (int j = 0; j < 3; ++j) t->mean[i] *= mono_int(kExp[i][j]) / factorial(kExp[i][j]);
    }
    // R and the weighted derivative rows in the symmetrised basis of the
    // line-form data vector (as for the averaged-gradient form; entries on
    // class(r) monomials only, checked)
    double rmax = 0.0, bmax = 0.0;
    for (int i = 0; i < nb; ++i)
        for (int k = 0; k < ncol; ++k) rmax = std::fmax(rmax, std::fabs(t->R[i][k]));
    for (int k = 0; k < nl; ++k)
        for (int i = 0; i < nb; ++i) bmax = std::fmax(bmax, std::fabs(t->WB[k][i]));
    for (int r = 0; r < kNumDataL; ++r) {
        const int c = kSymL.cls[r];
        for (int i = 0; i < nb; ++i) {
            double sr = 0.0, sb = 0.0;
            for (int q = 0; q < kSymL.nm[r]; ++q) {
                const int m = kSymL.mem[r][q];
                sr += kSymL.sgn[r][q] * t->R[i][m];
                if (m >= ne) sb += kSymL.sgn[r][q] * t->WB[m - ne][i];
            }
            sr /= kSymL.nm[r];
            if (parity_class(kExp[i][0], kExp[i][1], kExp[i][2]) == c) {
                t->Rs[r][kClass.pos[i]] = sr;
                t->Bs[r][kClass.pos[i]] = sb;
            } else if (std::fabs(sr) > 1e-12 * rmax || std::fabs(sb) > 1e-12 * bmax) {
                return -1;
            }
        }
    }
    // magnitudes of the monomials and their derivatives at the face Gauss
    // points: the same as for the averaged-gradient form
    std::unique_ptr<ReconTables> base(new (std::nothrow) ReconTables);
    if (!base || build_recon_tables(base.get())) return -1;
    std::memcpy(t->mval, base->mval, sizeof(t->mval));
    std::memcpy(t->mder, base->mder, sizeof(t->mder));
    return 0;
}

}  // namespace gks
