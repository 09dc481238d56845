// Compile-time description of the CGKS-5th reconstruction (Sec. 3.2):
// the 34 zero-mean monomials p_d of Eq. base (1 <= |d| <= 4) and the
// compact stencil S^cell-5th (face neighbours Omega_{1,m}, edge neighbours
// Omega_{2,n}). Shared by the host table builder and the device kernels so
// that the kernels can resolve every index at compile time.
#pragma once

#if defined(__CUDACC__)
#define GKS_HD __host__ __device__
#else
#define GKS_HD
#endif

namespace gks {

constexpr int kNumBasis = 34;
constexpr int kNumData = 63;  // S^data-5th entries per conserved variable

// exponents (d1, d2, d3) of p_d, ordered by degree
constexpr int kExp[kNumBasis][3] = {
    {1, 0, 0}, {0, 1, 0}, {0, 0, 1},
    {2, 0, 0}, {1, 1, 0}, {1, 0, 1}, {0, 2, 0}, {0, 1, 1}, {0, 0, 2},
    {3, 0, 0}, {2, 1, 0}, {2, 0, 1}, {1, 2, 0}, {1, 1, 1}, {1, 0, 2},
    {0, 3, 0}, {0, 2, 1}, {0, 1, 2}, {0, 0, 3},
    {4, 0, 0}, {3, 1, 0}, {3, 0, 1}, {2, 2, 0}, {2, 1, 1}, {2, 0, 2},
    {1, 3, 0}, {1, 2, 1}, {1, 1, 2}, {1, 0, 3}, {0, 4, 0}, {0, 3, 1},
    {0, 2, 2}, {0, 1, 3}, {0, 0, 4}};

// parity class of a multi-index: bit j set when the exponent along axis j
// is odd. Monomials of different classes are orthogonal on the symmetric
// unit cell, and at points (+-x, +-y, +-z) a class contributes with the
// sign prod_j s_j^{bit j}.
GKS_HD constexpr int parity_class(int a, int b, int c) {
    return (a & 1) | ((b & 1) << 1) | ((c & 1) << 2);
}
// exponent j of monomial i, computed (usable in device code): the same
// enumeration as kExp
GKS_HD constexpr int basis_exp(int i, int j) {
    int n = 0;
    for (int deg = 1; deg <= 4; ++deg)
        for (int a = deg; a >= 0; --a)
            for (int b = deg - a; b >= 0; --b) {
                if (n == i) return j == 0 ? a : (j == 1 ? b : deg - a - b);
                ++n;
            }
    return -1;
}
GKS_HD constexpr int basis_class(int i) {
    return parity_class(basis_exp(i, 0), basis_exp(i, 1), basis_exp(i, 2));
}
// class of the derivative of p_i along axis q (its exponent drops by one)
GKS_HD constexpr int deriv_class(int i, int q) { return basis_class(i) ^ (1 << q); }
GKS_HD constexpr bool has_deriv(int i, int q) { return basis_exp(i, q) > 0; }

// face neighbours: -x, +x, -y, +y, -z, +z
constexpr int kFaceOff[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0},
                                {0, 1, 0},  {0, 0, -1}, {0, 0, 1}};
// edge neighbours (two non-zero offsets)
constexpr int kEdgeOff[12][3] = {
    {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 1, 0}, {-1, 0, -1}, {1, 0, -1},
    {-1, 0, 1},  {1, 0, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}, {0, 1, 1}};

// the same offsets as functions (usable in device code)
GKS_HD constexpr int face_off(int m, int j) { return (m / 2 == j) ? ((m & 1) ? 1 : -1) : 0; }
// edge neighbours come in planes (x,y), (x,z), (y,z) of four; bit 0 of n is
// the sign along the plane's first axis, bit 1 along its second
GKS_HD constexpr int edge_axis_a(int n) { return n / 4 == 2 ? 1 : 0; }
GKS_HD constexpr int edge_axis_b(int n) { return n / 4 == 0 ? 1 : 2; }
GKS_HD constexpr int edge_axis_e(int n) { return 3 - edge_axis_a(n) - edge_axis_b(n); }
GKS_HD constexpr int edge_off(int n, int j) {
    return j == edge_axis_a(n) ? ((n & 1) ? 1 : -1)
                               : (j == edge_axis_b(n) ? ((n & 2) ? 1 : -1) : 0);
}

constexpr bool tables_agree() {
    for (int i = 0; i < kNumBasis; ++i)
        for (int j = 0; j < 3; ++j)
            if (basis_exp(i, j) != kExp[i][j]) return false;
    for (int m = 0; m < 6; ++m)
        for (int j = 0; j < 3; ++j)
            if (face_off(m, j) != kFaceOff[m][j]) return false;
    for (int n = 0; n < 12; ++n)
        for (int j = 0; j < 3; ++j)
            if (edge_off(n, j) != kEdgeOff[n][j]) return false;
    return true;
}
static_assert(tables_agree(), "basis/stencil tables disagree");

// Layout of the per-variable data vector d (the columns of the
// reconstruction matrix):
//   [m]         Q_{1,m} - Q_0                     m = 0..5
//   [6 + n]     Q_{2,n} - Q_0                     n = 0..11
//   [18 + 3m+j] h_j dQ/dx_j averaged over Omega_{1,m}
//   [36 + 2n]   h (o_a d_a - o_b d_b) Q / sqrt 2 over Omega_{2,n} (in-plane
//               direction orthogonal to the offset o)
//   [37 + 2n]   h d_e Q over Omega_{2,n} (edge direction)
//   [60 + j]    h_j dQ/dx_j averaged over Omega_0
// learned smoothness indicator: a 63 -> kMlpHidden (ReLU) -> 1 network on
// the data vector normalised by its max norm (+ kMlpDelta)
constexpr int kMlpHidden = 8;
constexpr int kMlpParams = kMlpHidden * kNumData + 2 * kMlpHidden + 1;
constexpr float kMlpDelta = 1e-30f;

constexpr int kColFace = 0, kColEdge = 6, kColFaceGrad = 18, kColEdgeGrad = 36,
              kColCentreGrad = 60;
// least-squares weight of data column k (the h_1, h_2, h_3 of Eq.
// compact-big-5 relative to the cell size that scales the derivative data):
// 1 for the averages, the face neighbours' gradients and the own gradient,
// kEdgeWeight for the edge neighbours' tangential derivatives
constexpr double kEdgeWeight = 0.1;
GKS_HD constexpr double col_weight(int k) {
    return (k >= kColEdgeGrad && k < kColCentreGrad) ? kEdgeWeight : 1.0;
}
// GENO's switch (reading of Eq. weno-new's chi): the misfit sigma of the
// quartic against the derivative data, relative to the data's norm plus
// (kGenoKappa S)^2 with S the cell's own magnitude; chi = 1/(1 + s + s^2),
// s = sigma / kGenoSigma0
constexpr double kGenoSigma0 = 5e-4;
constexpr double kGenoKappa = 0.01;

// ---- reflection structure of the data vector ---------------------------
// The stencil and the least-squares problem are invariant under the eight
// reflections x_j -> -x_j (s: bit j set when axis j is reflected). A
// reflection maps data column k to a column of the same kind at the
// mirrored site, times a sign: +1 for averages and for the in-plane edge
// combination, s_j for a derivative along axis j. Symmetrising each orbit
// of columns with the characters of the group gives 63 combinations
// d^s_r = sum_m T[r][m] d_m (T[r][m] in {-1, 0, 1}) of definite parity
// class; R then maps class-c combinations only to class-c monomials, so
// a = R d is 303 products instead of 34 x 63.
GKS_HD constexpr int data_kind(int k) {  // 0 average, 1 derivative, 2 edge in-plane
    return k < kColFaceGrad ? 0 : (k < kColEdgeGrad ? 1 : (k < kColCentreGrad ? ((k - kColEdgeGrad) % 2 ? 1 : 2) : 1));
}
// derivative axis of a kind-1 column
GKS_HD constexpr int data_axis(int k) {
    return k < kColEdgeGrad ? (k - kColFaceGrad) % 3
                            : (k < kColCentreGrad ? edge_axis_e((k - kColEdgeGrad) / 2) : k - kColCentreGrad);
}
GKS_HD constexpr int data_off(int k, int j) {
    return k < kColEdge ? face_off(k, j)
         : k < kColFaceGrad ? edge_off(k - kColEdge, j)
         : k < kColEdgeGrad ? face_off((k - kColFaceGrad) / 3, j)
         : k < kColCentreGrad ? edge_off((k - kColEdgeGrad) / 2, j) : 0;
}
GKS_HD constexpr int refl(int s, int j) { return (s >> j) & 1 ? -1 : 1; }
// column reached from k by reflection s
GKS_HD constexpr int data_reflect(int k, int s) {
    for (int m = 0; m < kNumData; ++m) {
        if (data_kind(m) != data_kind(k)) continue;
        if (data_kind(k) == 1 && data_axis(m) != data_axis(k)) continue;
        bool same = true;
        for (int j = 0; j < 3; ++j)
            if (data_off(m, j) != refl(s, j) * data_off(k, j)) same = false;
        if (same) return m;
    }
    return -1;
}
GKS_HD constexpr int data_reflect_sign(int k, int s) {
    return data_kind(k) == 1 ? refl(s, data_axis(k)) : 1;
}
struct SymTable {
    int cls[kNumData];     // parity class of combination r
    int nm[kNumData];      // its number of columns (1, 2 or 4)
    int mem[kNumData][8];  // the columns
    int sgn[kNumData][8];  // their signs T[r][m]
    int orbit[kNumData];   // first combination of r's orbit
};
constexpr SymTable make_sym_table() {
    SymTable t{};
    bool seen[kNumData] = {};
    int r = 0;
    for (int k = 0; k < kNumData; ++k) {
        if (seen[k]) continue;
        const int first = r;
        for (int s = 0; s < 8; ++s) seen[data_reflect(k, s)] = true;
        for (int c = 0; c < 8; ++c) {
            int coef[kNumData] = {};
            for (int s = 0; s < 8; ++s) {
                int chi = 1;
                for (int j = 0; j < 3; ++j)
                    if ((c >> j) & 1) chi *= refl(s, j);
                coef[data_reflect(k, s)] += chi * data_reflect_sign(k, s);
            }
            int n = 0;
            for (int m = 0; m < kNumData; ++m)
                if (coef[m] != 0) {
                    t.mem[r][n] = m;
                    t.sgn[r][n] = coef[m] > 0 ? 1 : -1;
                    ++n;
                }
            if (n == 0) continue;
            t.cls[r] = c;
            t.nm[r] = n;
            t.orbit[r] = first;
            ++r;
        }
    }
    return t;
}
constexpr SymTable kSym = make_sym_table();
// basis monomials of each parity class, in order: kClassMember[c][j]
constexpr int kMaxClass = 9;
struct ClassTable {
    int n[8];
    int member[8][kMaxClass];
    int pos[kNumBasis];  // position of monomial i within its class
};
constexpr ClassTable make_class_table() {
    ClassTable t{};
    for (int i = 0; i < kNumBasis; ++i) {
        const int c = parity_class(kExp[i][0], kExp[i][1], kExp[i][2]);
        t.pos[i] = t.n[c];
        t.member[c][t.n[c]++] = i;
    }
    return t;
}
constexpr ClassTable kClass = make_class_table();
constexpr bool sym_table_ok() {
    int covered[kNumData] = {};
    int per_class[8] = {};
    for (int r = 0; r < kNumData; ++r) {
        if (kSym.nm[r] < 1 || kSym.nm[r] > 8) return false;
        for (int q = 0; q < kSym.nm[r]; ++q) covered[kSym.mem[r][q]] += 1;
        per_class[kSym.cls[r]] += 1;
    }
    for (int m = 0; m < kNumData; ++m)
        if (covered[m] < 1) return false;
    for (int c = 0; c < 8; ++c)
        if (kClass.n[c] > kMaxClass) return false;
    // every combination of an orbit uses the orbit's columns, in one order
    for (int r = 0; r < kNumData; ++r) {
        const int f = kSym.orbit[r];
        if (kSym.nm[r] != kSym.nm[f]) return false;
        for (int q = 0; q < kSym.nm[r]; ++q)
            if (kSym.mem[r][q] != kSym.mem[f][q]) return false;
    }
    return true;
}
static_assert(sym_table_ok(), "reflection table of the data vector is incomplete");

// The data vector of the line form (reading B of the own data: the
// target cell's 12 line-averaged derivatives replace its averaged
// gradient): columns 0..59 as above, then line k of axis a at
// kColLines + 4a + k (k's bit 0: the side of axis (a+1)%3, bit 1: of
// (a+2)%3). A reflection s maps a line of axis a to the line with the
// tangential bits of the reflected axes flipped, times s_a (its end points
// swap when axis a is reflected).
constexpr int kNumDataL = 72, kColLines = 60;
GKS_HD constexpr int data_reflect_l(int k, int s) {
    if (k < kColLines) return data_reflect(k, s);
    const int a = (k - kColLines) / 4, kk = (k - kColLines) % 4;
    const int flip = ((s >> ((a + 1) % 3)) & 1) | (((s >> ((a + 2) % 3)) & 1) << 1);
    return kColLines + 4 * a + (kk ^ flip);
}
GKS_HD constexpr int data_reflect_sign_l(int k, int s) {
    return k < kColLines ? data_reflect_sign(k, s) : refl(s, (k - kColLines) / 4);
}
struct SymTableL {
    int cls[kNumDataL];
    int nm[kNumDataL];
    int mem[kNumDataL][8];
    int sgn[kNumDataL][8];
    int orbit[kNumDataL];
    int count;  // combinations found (kNumDataL when the basis is complete)
};
constexpr SymTableL make_sym_table_l() {
    SymTableL t{};
    bool seen[kNumDataL] = {};
    int r = 0;
    for (int k = 0; k < kNumDataL; ++k) {
        if (seen[k]) continue;
        const int first = r;
        for (int s = 0; s < 8; ++s) seen[data_reflect_l(k, s)] = true;
        for (int c = 0; c < 8; ++c) {
            int coef[kNumDataL] = {};
            for (int s = 0; s < 8; ++s) {
                int chi = 1;
                for (int j = 0; j < 3; ++j)
                    if ((c >> j) & 1) chi *= refl(s, j);
                coef[data_reflect_l(k, s)] += chi * data_reflect_sign_l(k, s);
            }
            int n = 0;
            for (int m = 0; m < kNumDataL; ++m)
                if (coef[m] != 0) {
                    t.mem[r][n] = m;
                    t.sgn[r][n] = coef[m] > 0 ? 1 : -1;
                    ++n;
                }
            if (n == 0) continue;
            if (r >= kNumDataL) return t;  // incomplete: caught below
            t.cls[r] = c;
            t.nm[r] = n;
            t.orbit[r] = first;
            ++r;
        }
    }
    t.count = r;
    return t;
}
constexpr SymTableL kSymL = make_sym_table_l();
constexpr bool sym_table_l_ok() {
    if (kSymL.count != kNumDataL) return false;
    int covered[kNumDataL] = {};
    for (int r = 0; r < kNumDataL; ++r) {
        if (kSymL.nm[r] < 1 || kSymL.nm[r] > 8) return false;
        for (int q = 0; q < kSymL.nm[r]; ++q) covered[kSymL.mem[r][q]] += 1;
        const int f = kSymL.orbit[r];
        if (kSymL.nm[r] != kSymL.nm[f]) return false;
        for (int q = 0; q < kSymL.nm[r]; ++q)
            if (kSymL.mem[r][q] != kSymL.mem[f][q]) return false;
    }
    for (int m = 0; m < kNumDataL; ++m)
        if (covered[m] < 1) return false;
    return true;
}
static_assert(sym_table_l_ok(), "reflection table of the line-form data vector is incomplete");

struct ReconTables {
    double R[kNumBasis][kNumData];      // coefficients a = R d
    double Rs[kNumData][kMaxClass];     // a_{class(r), j} += Rs[r][j] d^s_r
    double Bs[kNumData][kMaxClass];     // weighted derivative rows W B of the
                                        // least squares in the symmetrised
                                        // basis (zero for the average rows)
    double mean[kNumBasis];             // mean of delta^d/d! over Omega_0
    double mval[3][kNumBasis];          // |value| factors at the Gauss points
                                        // of the faces normal to axis d
    double mder[3][3][kNumBasis];       // |d/dx_q| factors, same points
};

// Builds the tables (host). Returns 0 on success.
int build_recon_tables(ReconTables *t);

// Reading B of the target cell's data (its 12 line-averaged derivatives
// instead of its averaged gradient; data vector of 72 entries: 60 as above,
// then the lines 60 + 4a + k): the dense least-squares matrix, the weighted
// derivative rows for GENO's misfit, the monomial means and the magnitudes
// of the monomials and their derivatives at the face Gauss points.
struct ReconTablesLines {
    double R[kNumBasis][72];
    double WB[54][kNumBasis];
    double w[54];
    double mean[kNumBasis];
    double mval[3][kNumBasis];      // as ReconTables::mval
    double mder[3][3][kNumBasis];   // as ReconTables::mder
    double Rs[kNumDataL][kMaxClass];  // R in the symmetrised basis (kSymL)
    double Bs[kNumDataL][kMaxClass];  // weighted derivative rows, same basis
};
int build_recon_tables_lines(ReconTablesLines *t);

}  // namespace gks
