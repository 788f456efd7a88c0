// Float-float ("double-single") arithmetic on the FP32 pipe.
//
// A value is the unevaluated sum h + l of two floats with |l| <= ulp(h) / 2, which carries a
// 48-bit significand. The building blocks are the classical error-free transformations:
// Knuth's two-sum (the rounding error of a + b, exactly), Dekker's fast two-sum (the same when
// |a| >= |b|) and the exact product error fma(a, b, -a b). On this GPU the FP64 rate is 1/64
// of the FP32 rate, so a float-float operation (4 to 20 FP32 instructions) is several times
// cheaper than the FP64 instruction it replaces, at ~1e-14 relative accuracy.
//
// These helpers need IEEE FP32 semantics: no fast-math, no flush-to-zero assumptions on the
// error terms (the build uses neither). The exponent range is FP32's.
#pragma once

#include <cuda_runtime.h>

struct ff {
    float h, l;
};

__device__ __forceinline__ ff ff_two_sum(float a, float b)
{
    float s = a + b;
    float bb = s - a;
    float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}

__device__ __forceinline__ ff ff_fast_two_sum(float a, float b)
{
    float s = a + b;
    float e = b - (s - a);
    return {s, e};
}

__host__ __device__ __forceinline__ ff ff_from(double x)
{
    float h = (float)x;
    return {h, (float)(x - (double)h)};
}

__host__ __device__ __forceinline__ double ff_to(ff a) { return (double)a.h + (double)a.l; }

__device__ __forceinline__ ff ff_neg(ff a) { return {-a.h, -a.l}; }

// a + b, error ~2^-48 (|a| + |b|)
__device__ __forceinline__ ff ff_add(ff a, ff b)
{
    ff s = ff_two_sum(a.h, b.h);
    s.l += a.l + b.l;
    return ff_fast_two_sum(s.h, s.l);
}

__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }

__device__ __forceinline__ ff ff_add_f(ff a, float b)
{
    ff s = ff_two_sum(a.h, b);
    s.l += a.l;
    return ff_fast_two_sum(s.h, s.l);
}

// a b, relative error ~2^-46
__device__ __forceinline__ ff ff_mul(ff a, ff b)
{
    float p = a.h * b.h;
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    return ff_fast_two_sum(p, e);
}

__device__ __forceinline__ ff ff_mul_f(ff a, float b)
{
    float p = a.h * b;
    float e = fmaf(a.h, b, -p);
    e = fmaf(a.l, b, e);
    return ff_fast_two_sum(p, e);
}

__device__ __forceinline__ ff ff_sqr(ff a)
{
    float p = a.h * a.h;
    float e = fmaf(a.h, a.h, -p);
    e = fmaf(2.0f * a.h, a.l, e);
    return ff_fast_two_sum(p, e);
}

// a b + c
__device__ __forceinline__ ff ff_fma(ff a, ff b, ff c) { return ff_add(ff_mul(a, b), c); }

// 1 / sqrt(a) for a > 0: the FP32 estimate and one Newton step y + y (1 - a y^2) / 2, with
// the residual 1 - a y^2 formed in float-float (its leading bits cancel exactly).
__device__ __forceinline__ ff ff_rsqrt(ff a)
{
    float y = rsqrtf(a.h);
    float p = y * y;
    ff y2 = {p, fmaf(y, y, -p)};
    ff r = ff_add_f(ff_neg(ff_mul(a, y2)), 1.0f);
    return ff_fast_two_sum(y, 0.5f * y * r.h);
}
