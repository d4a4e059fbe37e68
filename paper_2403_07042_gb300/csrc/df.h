// Double-float arithmetic (an unevaluated sum of two FP32 words, about 48 significant
// bits) for the element-wise work of the split-precision step: GB300 runs FP64 at a small
// fraction of its FP32 rate, so the per-step element operations use FP32 error-free
// transformations instead.
#pragma once

#include <cuda_fp16.h>

namespace qed {

// Error-free transformations (Knuth's TwoSum, Dekker's FastTwoSum, FMA-based TwoProd).
struct df {
    float hi, lo;
};

__device__ __forceinline__ df two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ df fast_two_sum(float a, float b) {  // |a| >= |b|
    float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df df_add(df x, df y) {
    df s = two_sum(x.hi, y.hi);
    float e = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
    return fast_two_sum(s.hi, e);
}

__device__ __forceinline__ df df_add_f(df x, float y) {
    df s = two_sum(x.hi, y);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, x.lo));
}

__device__ __forceinline__ df df_mul(df x, df y) {
    float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    return fast_two_sum(p, e);
}

__device__ __forceinline__ df df_neg(df x) { return {-x.hi, -x.lo}; }

struct cdf {
    df re, im;
};

__device__ __forceinline__ cdf load_cdf(const float4 &v) { return {{v.x, v.y}, {v.z, v.w}}; }
__device__ __forceinline__ float4 store_cdf(const cdf &c) { return make_float4(c.re.hi, c.re.lo, c.im.hi, c.im.lo); }

__device__ __forceinline__ cdf cdf_mul(cdf a, cdf b) {
    return {df_add(df_mul(a.re, b.re), df_neg(df_mul(a.im, b.im))), df_add(df_mul(a.re, b.im), df_mul(a.im, b.re))};
}

__device__ __forceinline__ cdf cdf_mul_conj(cdf a, cdf b) {  // a * conj(b)
    return {df_add(df_mul(a.re, b.re), df_mul(a.im, b.im)), df_add(df_mul(a.im, b.re), df_neg(df_mul(a.re, b.im)))};
}

// FP16 hi/lo pieces of a scaled double-float value, in FP32 arithmetic: x = hi + lo.
__device__ __forceinline__ void df_to_half2(df x, float s, __half &h, __half &l) {
    const float xs = x.hi * s;  // power-of-two scaling is exact
    h = __float2half_rn(xs);
    l = __float2half_rn(__fadd_rn(__fsub_rn(xs, __half2float(h)), x.lo * s));
}


}  // namespace qed
