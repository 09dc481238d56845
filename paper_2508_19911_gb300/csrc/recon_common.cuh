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
