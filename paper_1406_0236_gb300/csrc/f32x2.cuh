// Packed FP32 pairs for sm_100-class GPUs: one 64-bit register pair holds two
// floats and a single add/sub/mul/fma.f32x2 instruction operates on both, which
// halves the issue slots of FP32 arithmetic (the FMA pipe still does two lane
// operations).  lo = first element, hi = second.  Flush-to-zero, round to nearest.
#pragma once

#include <cuda_runtime.h>

namespace hzb {

typedef unsigned long long f2x;

__device__ __forceinline__ f2x f2_pack(float lo, float hi)
{
    f2x r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ f2x f2_splat(float v) { return f2_pack(v, v); }
__device__ __forceinline__ void f2_unpack(f2x v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2x f2_add(f2x a, f2x b)
{
    f2x d;
    asm("add.rn.ftz.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2x f2_sub(f2x a, f2x b)
{
    f2x d;
    asm("sub.rn.ftz.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2x f2_mul(f2x a, f2x b)
{
    f2x d;
    asm("mul.rn.ftz.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
// a * b + c
__device__ __forceinline__ f2x f2_fma(f2x a, f2x b, f2x c)
{
    f2x d;
    asm("fma.rn.ftz.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

}  // namespace hzb
