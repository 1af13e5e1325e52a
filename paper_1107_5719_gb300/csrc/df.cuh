// Double-float arithmetic: a value is the unevaluated sum hi + lo of two
// FP32 numbers with |lo| <= ulp(hi)/2, carrying about 48 significant bits.
// Built from the error-free transformations TwoSum (Knuth) and TwoProduct
// (one FMA), as in Dekker's double-length arithmetic.  On GB300 the FP32
// pipes issue 64x more operations per clock than the FP64 pipe, so a march
// written in double-float arithmetic reaches FP64-level accuracy (about
// 1e-14 relative per operation) at a fraction of the cost.
#pragma once

#include <cuda_runtime.h>

namespace rt3d {
namespace {

struct dfl {
    float h, l;
};

__device__ __forceinline__ dfl df_make(float h, float l) { return dfl{h, l}; }

// s + e = a + b exactly
__device__ __forceinline__ dfl two_sum(float a, float b)
{
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return dfl{s, e};
}

// s + e = a + b exactly when |a| >= |b| (or a == 0)
__device__ __forceinline__ dfl quick_two_sum(float a, float b)
{
    const float s = a + b;
    return dfl{s, b - (s - a)};
}

// p + e = a * b exactly
__device__ __forceinline__ dfl two_prod(float a, float b)
{
    const float p = a * b;
    return dfl{p, fmaf(a, b, -p)};
}

// a + b, both operands double-float; accurate also under cancellation.
__device__ __forceinline__ dfl df_add(dfl a, dfl b)
{
    dfl s = two_sum(a.h, b.h);
    const dfl t = two_sum(a.l, b.l);
    s.l += t.h;
    s = quick_two_sum(s.h, s.l);
    s.l += t.l;
    return quick_two_sum(s.h, s.l);
}

__device__ __forceinline__ dfl df_neg(dfl a) { return dfl{-a.h, -a.l}; }

__device__ __forceinline__ dfl df_sub(dfl a, dfl b) { return df_add(a, df_neg(b)); }

// a + b with the low parts added once (Dekker's add, 11 operations against
// 20): the error is bounded by ~2^-47 (|a| + |b|) instead of 2^-47 |a + b|.
// Used wherever that bound is already the rounding level of the operands
// (sums of like-signed terms, differences of quantities that each carry a
// 2^-48 representation error).
__device__ __forceinline__ dfl df_add_s(dfl a, dfl b)
{
    dfl s = two_sum(a.h, b.h);
    s.l += a.l + b.l;
    return quick_two_sum(s.h, s.l);
}

__device__ __forceinline__ dfl df_sub_s(dfl a, dfl b) { return df_add_s(a, df_neg(b)); }

// a + b with b a float
__device__ __forceinline__ dfl df_add_f(dfl a, float b)
{
    dfl s = two_sum(a.h, b);
    s.l += a.l;
    return quick_two_sum(s.h, s.l);
}

// a * b
__device__ __forceinline__ dfl df_mul(dfl a, dfl b)
{
    dfl p = two_prod(a.h, b.h);
    p.l = fmaf(a.h, b.l, p.l);
    p.l = fmaf(a.l, b.h, p.l);
    return quick_two_sum(p.h, p.l);
}

// a * b with b a float
__device__ __forceinline__ dfl df_mul_f(dfl a, float b)
{
    dfl p = two_prod(a.h, b);
    p.l = fmaf(a.l, b, p.l);
    return quick_two_sum(p.h, p.l);
}

// a * 2^k for a power-of-two float factor (exact)
__device__ __forceinline__ dfl df_scale(dfl a, float pow2) { return dfl{a.h * pow2, a.l * pow2}; }

// a / b: quotient estimate from the FP32 reciprocal, one correction with
// the exact residual a - q b.
__device__ __forceinline__ dfl df_div(dfl a, dfl b)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(b.h));
    const float q1 = a.h * r;
    const dfl res = df_sub(a, df_mul_f(b, q1));
    const float q2 = res.h * r;
    const dfl q = quick_two_sum(q1, q2);
    const dfl res2 = df_sub(a, df_mul(b, q));
    return df_add_f(q, res2.h * r);
}

// As df_div with the residuals formed by df_sub_s: each residual is
// a - b q with |a - b q| ~ 2^-23 |a|, formed to ~2^-48 |a|, so every
// correction still gains ~23 bits.
__device__ __forceinline__ dfl df_div_s(dfl a, dfl b)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(b.h));
    const float q1 = a.h * r;
    const dfl res = df_sub_s(a, df_mul_f(b, q1));
    const float q2 = res.h * r;
    const dfl q = quick_two_sum(q1, q2);
    const dfl res2 = df_sub_s(a, df_mul(b, q));
    return df_add_f(q, res2.h * r);
}

__device__ __forceinline__ double df_to_double(dfl a) { return (double)a.h + (double)a.l; }

__host__ __device__ __forceinline__ dfl df_from_double(double x)
{
    const float h = (float)x;
    return dfl{h, (float)(x - (double)h)};
}

}  // namespace
}  // namespace rt3d
