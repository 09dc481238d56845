// Device helpers shared by the FP64 (recon_fp64.cu) and the mixed-precision
// (recon.cu) reconstruction kernels.
#pragma once
#include <cmath>
#include <type_traits>
#include <utility>

#include "basis.h"
#include "common.cuh"

namespace gks {
namespace {

// Compile-time loop: f(std::integral_constant<int, I>) for I = 0..N-1, so
// that every table index below is a constant expression of the front end.
template <typename F, int... I>
__device__ __forceinline__ void static_for_impl(F &&f, std::integer_sequence<int, I...>) {
    (f(std::integral_constant<int, I>{}), ...);
}
template <int N, typename F>
__device__ __forceinline__ void static_for(F &&f) {
    static_for_impl(f, std::make_integer_sequence<int, N>{});
}

constexpr double kG = 0.28867513459481288225;     // 1/(2 sqrt 3)
constexpr double kRs2 = 0.70710678118654752440;   // 1/sqrt 2

// Stencil geometry of one cell on a general grid (non-periodic axes,
// stretched meshes): per face / edge neighbour, bits 0-2 the axes across
// which it is a mirror ghost and bit 3 whether variable v's average changes
// sign there; hm[a][o + 1] the cell size along axis a at offset o.
struct NbGeo {
    int fF[6], fE[12];
    double hm[3][3];
};

template <typename T>
__device__ __forceinline__ T neg_if(T x, bool neg) {
    return neg ? -x : x;
}

// sign of a ghost's derivative along axis q (bits of NbGeo::fF / fE)
__device__ __forceinline__ bool der_neg(int f, int q) {
    return (((f >> 3) ^ (f >> q)) & 1) != 0;
}

// neighbour indices (and, on a general grid, the geometry) of cell (i, j, k)
// for conserved variable v
template <bool GEN>
__device__ __forceinline__ void stencil(const GridDesc &g, int i, int j, int k, int v,
                                        long long nbF[6], long long nbE[12], NbGeo &geo) {
    if constexpr (!GEN) {
#pragma unroll
        for (int m = 0; m < 6; ++m)
            nbF[m] = cell_index(g, wrap(i + face_off(m, 0), g.nx), wrap(j + face_off(m, 1), g.ny),
                                wrap(k + face_off(m, 2), g.nz));
#pragma unroll
        for (int e = 0; e < 12; ++e)
            nbE[e] = cell_index(g, wrap(i + edge_off(e, 0), g.nx), wrap(j + edge_off(e, 1), g.ny),
                                wrap(k + edge_off(e, 2), g.nz));
    } else {
        const int c0[3] = {i, j, k};
        int cm[3][3], fl[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int o = 0; o < 3; ++o) {
                fl[a][o] = 0;
                cm[a][o] = nb_coord(g, a, c0[a] + o - 1, fl[a][o]);
                geo.hm[a][o] = cell_h(g, a, cm[a][o]);
            }
#pragma unroll
        for (int m = 0; m < 6; ++m) {
            const int ox = face_off(m, 0) + 1, oy = face_off(m, 1) + 1, oz = face_off(m, 2) + 1;
            const int f = fl[0][ox] | fl[1][oy] | fl[2][oz];
            nbF[m] = cell_index(g, cm[0][ox], cm[1][oy], cm[2][oz]);
            geo.fF[m] = f | (ghost_neg(g, v, f) ? 8 : 0);
        }
#pragma unroll
        for (int e = 0; e < 12; ++e) {
            const int ox = edge_off(e, 0) + 1, oy = edge_off(e, 1) + 1, oz = edge_off(e, 2) + 1;
            const int f = fl[0][ox] | fl[1][oy] | fl[2][oz];
            nbE[e] = cell_index(g, cm[0][ox], cm[1][oy], cm[2][oz]);
            geo.fE[e] = f | (ghost_neg(g, v, f) ? 8 : 0);
        }
    }
}

// face-frame component of conserved variable v on a face normal to axis d
__device__ __forceinline__ int frame_comp(int v, int d) {
    return (v == 0 || v == 4) ? v : 1 + (v - 1 - d + 3) % 3;
}

// In-place Walsh-Hadamard transform over the three axis bits: from class
// sums X[cls] to the values at the eight points (+-x, +-y, +-z); afterwards
// X[p] is the value where axis j has sign + if bit j of p is set, else -.
template <typename T>
__device__ __forceinline__ void class_to_points(T X[8]) {
#pragma unroll
    for (int b = 1; b < 8; b <<= 1)
#pragma unroll
        for (int p = 0; p < 8; ++p)
            if (!(p & b)) {
                const T lo = X[p], hi = X[p | b];
                X[p] = lo - hi;
                X[p | b] = lo + hi;
            }
}

}  // namespace
}  // namespace gks
