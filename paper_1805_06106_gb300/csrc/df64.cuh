// Double-float arithmetic: a value is the unevaluated sum h + l of two FP32 numbers with
// |l| <= ulp(h)/2, about 48 significant bits.  Built from error-free transformations:
//   two-sum (Knuth, TAOCP vol. 2, 4.2.2):      s = a + b, e = (a - (s - bb)) + (b - bb), bb = s - a
//   fast two-sum (Dekker 1971), |a| >= |b|:    s = a + b, e = b - (s - a)
//   two-product with a fused multiply-add:      p = a b,  e = fma(a, b, -p)   (exact for FP32 inputs)
// Sums use the "sloppy" form (two-sum of the leading parts, the trailing parts added in FP32, then
// renormalised), whose error is below 2^-44 (|a| + |b|): the error bound of a sum is relative to the
// summed magnitudes anyway.  Products are relative to 2^-45.  The range is FP32's, so callers keep
// their quantities scaled (box- or radius-relative) well inside it.
//
// Why: GB300 issues FP64 at about 1/70 of its FP32 rate, so kernels bound by FP64 operations run
// several times faster on FP32 pairs, at an accuracy far below every tolerance of the method.
// Every operation is an explicitly rounded intrinsic, so the compiler can neither contract nor
// reorder the transformations.
#pragma once

#include <cuda_runtime.h>

namespace qbx {

struct df {
    float h, l;
};

__device__ __forceinline__ df df_make(float h, float l) { return df{h, l}; }

// nearest double-float of a double (the leading part rounded to nearest, then the remainder)
__device__ __forceinline__ df df_from(double x)
{
    const float h = __double2float_rn(x);
    return df{h, __double2float_rn(x - (double)h)};
}

__device__ __forceinline__ double df_to(df a) { return (double)a.h + (double)a.l; }

__device__ __forceinline__ df df_fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return df{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df df_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return df{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

__device__ __forceinline__ df df_neg(df a) { return df{-a.h, -a.l}; }

__device__ __forceinline__ df df_add(df a, df b)
{
    const df s = df_two_sum(a.h, b.h);
    return df_fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}

__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

// a + b for a double-float and a float
__device__ __forceinline__ df df_add_f(df a, float b)
{
    const df s = df_two_sum(a.h, b);
    return df_fast_two_sum(s.h, __fadd_rn(s.l, a.l));
}

__device__ __forceinline__ df df_mul(df a, df b)
{
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    return df_fast_two_sum(p, e);
}

// a * b for a double-float and a float
__device__ __forceinline__ df df_mul_f(df a, float b)
{
    const float p = __fmul_rn(a.h, b);
    float e = __fmaf_rn(a.h, b, -p);
    e = __fmaf_rn(a.l, b, e);
    return df_fast_two_sum(p, e);
}

__device__ __forceinline__ df df_sqr(df a)
{
    const float p = __fmul_rn(a.h, a.h);
    float e = __fmaf_rn(a.h, a.h, -p);
    e = __fmaf_rn(__fmul_rn(2.0f, a.h), a.l, e);
    return df_fast_two_sum(p, e);
}

// a * b + c
__device__ __forceinline__ df df_fma(df a, df b, df c) { return df_add(df_mul(a, b), c); }

// 1 / sqrt(a), a > 0: the FP32 estimate y then one Newton step y + y (1 - a y^2) / 2 in double-float
// (the step squares the estimate's relative error, about 2^-23, to below 2^-45)
__device__ __forceinline__ df df_rsqrt(df a)
{
    const float y = rsqrtf(a.h);
    const df y2{__fmul_rn(y, y), __fmaf_rn(y, y, -__fmul_rn(y, y))};
    const df t = df_add_f(df_neg(df_mul(a, y2)), 1.0f);  // 1 - a y^2, small
    return df_add_f(df_mul_f(t, __fmul_rn(0.5f, y)), y);
}

// Compensated sum of products (the Dot2 scheme of Ogita, Rump and Oishi, 2005, with double-float
// factors): s carries the running FP32 sum, c the FP32 sum of every rounding error (two-product and
// two-sum remainders) and of the cross terms with the trailing parts.  The result equals the sum
// computed in about twice FP32's precision and then rounded, i.e. an error near 2^-44 of the summed
// magnitudes, at 12 FP32 operations per product (against 18 for a double-float multiply and add).
struct dacc {
    float s, c;
};

__device__ __forceinline__ void dacc_add_prod(dacc &a, df x, df y)
{
    const float p = __fmul_rn(x.h, y.h);
    const float pe = __fmaf_rn(x.h, y.h, -p);
    const df t = df_two_sum(a.s, p);
    a.s = t.h;
    float c = __fadd_rn(a.c, __fadd_rn(pe, t.l));
    c = __fmaf_rn(x.h, y.l, c);
    a.c = __fmaf_rn(x.l, y.h, c);
}

__device__ __forceinline__ void dacc_add(dacc &a, df x)
{
    const df t = df_two_sum(a.s, x.h);
    a.s = t.h;
    a.c = __fadd_rn(a.c, __fadd_rn(t.l, x.l));
}

__device__ __forceinline__ df dacc_get(dacc a) { return df_two_sum(a.s, a.c); }

}  // namespace qbx
