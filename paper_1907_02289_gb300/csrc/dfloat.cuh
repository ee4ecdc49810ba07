// dfloat.cuh -- unevaluated sums of two FP32 numbers (hi + lo, |lo| <= ulp(hi)/2)
// and their arithmetic, built from the error-free transformations of
// Knuth (TwoSum: a + b = s + e exactly) and of the fused multiply-add
// (TwoProd: a * b = p + e exactly, e = fma(a, b, -p)); about 44 significant
// bits, on the FP32 pipe.  Used where an FP32 evaluation is too ill-conditioned
// for its result: the refinement of the FP32 force kernel.
#pragma once
#include <cuda_runtime.h>

namespace bh {

struct df {
    float hi, lo;
};

__device__ __forceinline__ df df_make(float a) { return {a, 0.f}; }

// s + e == a + b exactly, s = fl(a + b) (no condition on the magnitudes)
__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

// the same when |a| >= |b| (or a == 0)
__device__ __forceinline__ df fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

// p + e == a * b exactly
__device__ __forceinline__ df two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ df df_add(df a, df b) {
    df s = two_sum(a.hi, b.hi);
    const df t = two_sum(a.lo, b.lo);
    s.lo = __fadd_rn(s.lo, t.hi);
    s = fast_two_sum(s.hi, s.lo);
    s.lo = __fadd_rn(s.lo, t.lo);
    return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ df df_mul(df a, df b) {
    df p = two_prod(a.hi, b.hi);
    p.lo = __fmaf_rn(a.hi, b.lo, p.lo);
    p.lo = __fmaf_rn(a.lo, b.hi, p.lo);
    return fast_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ df df_mul_f(df a, float b) {
    df p = two_prod(a.hi, b);
    p.lo = __fmaf_rn(a.lo, b, p.lo);
    return fast_two_sum(p.hi, p.lo);
}

// (x_hi + x_lo) - (y_hi + y_lo) for two hi/lo splits of FP64 values
__device__ __forceinline__ df df_diff(float xh, float xl, float yh, float yl) {
    df d = two_sum(xh, -yh);
    d.lo = __fadd_rn(d.lo, __fsub_rn(xl, yl));
    return fast_two_sum(d.hi, d.lo);
}

__device__ __forceinline__ df df_dot3(df x, df y, df z) { return df_add(df_add(df_mul(x, x), df_mul(y, y)), df_mul(z, z)); }

// 1 / sqrt(s), s > 0: an FP32 estimate y0 and one Newton step carried out in
// df, y = y0 + y0 (1 - s y0^2) / 2 (the residual in df; the step squares the
// estimate's relative error).
__device__ __forceinline__ df df_rsqrt(df s) {
    const float y0 = rsqrtf(s.hi);
    const df y2 = two_prod(y0, y0);
    const df r = df_sub(df_make(1.f), df_mul(s, y2));
    return fast_two_sum(y0, __fmul_rn(__fmul_rn(y0, 0.5f), r.hi));
}

__device__ __forceinline__ bool df_gt(df a, df b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }

__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

}  // namespace bh
