// Packed FP32 pairs for sm_100-class GPUs: two FP32 values in one 64-bit register pair (the
// low half first), operated on by the PTX f32x2 instructions (add, sub, mul, fma with
// round-to-nearest, each half rounded exactly as the scalar instruction would round it). One
// instruction then carries two independent lanes of work, which halves the issue slots of
// FP32-bound loops whose iterations come in pairs.
#pragma once

typedef unsigned long long f2x;

__device__ __forceinline__ f2x x2_pack(float lo, float hi)
{
    f2x r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ f2x x2_dup(float v) { return x2_pack(v, v); }
__device__ __forceinline__ void x2_unpack(f2x v, float& lo, float& hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2x x2_add(f2x a, f2x b)
{
    f2x r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2x x2_sub(f2x a, f2x b)
{
    f2x r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2x x2_mul(f2x a, f2x b)
{
    f2x r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
// a * b + c, one rounding per half
__device__ __forceinline__ f2x x2_fma(f2x a, f2x b, f2x c)
{
    f2x r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
