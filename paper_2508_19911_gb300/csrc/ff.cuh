// Float-float arithmetic: a value is the unevaluated sum hi + lo of two
// FP32 numbers with |lo| <= ulp(hi)/2, about 48 significant bits, computed
// with FP32 instructions only (GB300 runs FP32 at 64x its FP64 rate).
// Error-free transformations: Knuth's TwoSum, the FMA-based TwoProduct
// (exact product error), Dekker's Fast2Sum for renormalisation; the
// division is a Newton correction of the FP32 quotient. Every operation
// uses the __fadd_rn / __fmul_rn / __fmaf_rn intrinsics, which the compiler
// never contracts or reassociates (a product fused into a later sum would
// break the error-free steps). Relative error per operation about 2^-46.
#pragma once

namespace gks {

struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff ff_make(float hi, float lo) {
    ff r;
    r.hi = hi;
    r.lo = lo;
    return r;
}

// s + e = a + b exactly (no ordering assumption)
__device__ __forceinline__ ff two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return ff_make(s, e);
}

// s + e = a + b exactly when |a| >= |b| (or a = 0)
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return ff_make(s, __fsub_rn(b, __fsub_rn(s, a)));
}

// p + e = a * b exactly
__device__ __forceinline__ ff two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return ff_make(p, __fmaf_rn(a, b, -p));
}

__device__ __forceinline__ ff ff_from_double(double x) {
    const float h = __double2float_rn(x);
    return ff_make(h, __double2float_rn(x - (double)h));
}

__device__ __forceinline__ ff ff_from_float(float x) { return ff_make(x, 0.0f); }

// exact: hi + lo has at most 48 significant bits
__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ ff ff_neg(ff a) { return ff_make(-a.hi, -a.lo); }

__device__ __forceinline__ ff ff_add(ff a, ff b) {
    ff s = two_sum(a.hi, b.hi);
    const ff t = two_sum(a.lo, b.lo);
    s.lo = __fadd_rn(s.lo, t.hi);
    s = fast_two_sum(s.hi, s.lo);
    s.lo = __fadd_rn(s.lo, t.lo);
    return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }

__device__ __forceinline__ ff ff_add_f(ff a, float b) {
    ff s = two_sum(a.hi, b);
    s.lo = __fadd_rn(s.lo, a.lo);
    return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    ff p = two_prod(a.hi, b.hi);
    p.lo = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
    return fast_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ ff ff_mul_f(ff a, float b) {
    ff p = two_prod(a.hi, b);
    p.lo = __fmaf_rn(a.lo, b, p.lo);
    return fast_two_sum(p.hi, p.lo);
}

// a * b + c
__device__ __forceinline__ ff ff_fma(ff a, ff b, ff c) { return ff_add(ff_mul(a, b), c); }

// a / b: FP32 quotient, two Newton corrections with the exact residual
__device__ __forceinline__ ff ff_div(ff a, ff b) {
    const float rb = __frcp_rn(b.hi);
    const float q1 = __fmul_rn(a.hi, rb);
    ff r = ff_sub(a, ff_mul_f(b, q1));
    const float q2 = __fmul_rn(r.hi, rb);
    ff q = fast_two_sum(q1, q2);
    r = ff_sub(a, ff_mul(b, q));
    return ff_add_f(q, __fmul_rn(r.hi, rb));
}

// 1/b: the FP32 reciprocal r and one Newton step r + r (1 - b r), the
// residual 1 - b.hi r formed exactly by an FMA (quadratic convergence: the
// relative error ~2^-24 of r becomes ~2^-46)
__device__ __forceinline__ ff ff_recip(ff b) {
    const float r = __frcp_rn(b.hi);
    const float e = __fmaf_rn(-b.lo, r, __fmaf_rn(-b.hi, r, 1.0f));
    return fast_two_sum(r, __fmul_rn(r, e));
}

// a + b with the two lo parts added in FP32: about 2^-46 (|a| + |b|), not
// relative to |a + b| where the two cancel (for sums of like terms)
__device__ __forceinline__ ff ff_add_like(ff a, ff b) {
    ff s = two_sum(a.hi, b.hi);
    s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ ff ff_sub_like(ff a, ff b) { return ff_add_like(a, ff_neg(b)); }

// sqrt(a), a > 0: FP32 root, one Newton correction with the exact residual
__device__ __forceinline__ ff ff_sqrt(ff a) {
    const float h = __fsqrt_rn(a.hi);
    const ff r = ff_sub(a, two_prod(h, h));
    return fast_two_sum(h, __fmul_rn(r.hi, __fdividef(0.5f, h)));
}

// a double constant as a float-float pair, at compile time
struct ffc {
    float hi, lo;
};
__host__ __device__ constexpr ffc ff_const(double x) { return ffc{(float)x, (float)(x - (double)(float)x)}; }
__device__ __forceinline__ ff ff_of(ffc c) { return ff_make(c.hi, c.lo); }

}  // namespace gks
