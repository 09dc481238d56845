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

struct ReconTables {
    double R[kNumBasis][kNumData];      // coefficients a = R d
    double H[kNumBasis][kNumBasis];     // IS_H = a^T H a
    double mean[kNumBasis];             // mean of delta^d/d! over Omega_0
    double mval[3][kNumBasis];          // |value| factors at the Gauss points
                                        // of the faces normal to axis d
    double mder[3][3][kNumBasis];       // |d/dx_q| factors, same points
};

// Builds the tables (host). Returns 0 on success.
int build_recon_tables(ReconTables *t);

}  // namespace gks
