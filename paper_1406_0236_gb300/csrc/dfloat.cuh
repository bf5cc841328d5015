// Double-float arithmetic on the FP32 pipe: a value is hi + lo with two floats,
// |lo| <= ulp(hi)/2, about 48 significant bits (relative rounding ~3.6e-15).
// Built from the error-free transformations of Knuth (TwoSum) and Dekker
// (FastTwoSum, and TwoProduct written with a fused multiply-add).  The translation
// unit that includes this file is compiled with -fmad=false so that the compiler
// does not contract the separate operations these transformations rely on.
#pragma once

#include <cuda_runtime.h>

namespace hzb {

struct dfl {
    float hi, lo;
};

__device__ __forceinline__ dfl df_two_sum(float a, float b)
{
    float s = a + b;
    float bb = s - a;
    float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}

__device__ __forceinline__ dfl df_fast_two_sum(float a, float b)        // |a| >= |b|
{
    float s = a + b;
    float e = b - (s - a);
    return {s, e};
}

__device__ __forceinline__ dfl df_add(dfl x, dfl y)
{
    dfl s = df_two_sum(x.hi, y.hi);
    float e = s.lo + (x.lo + y.lo);
    return df_fast_two_sum(s.hi, e);
}

__device__ __forceinline__ dfl df_neg(dfl x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ dfl df_sub(dfl x, dfl y) { return df_add(x, df_neg(y)); }

__device__ __forceinline__ dfl df_mul(dfl x, dfl y)
{
    float p = x.hi * y.hi;
    float e = fmaf(x.hi, y.hi, -p);
    e = fmaf(x.hi, y.lo, e);
    e = fmaf(x.lo, y.hi, e);
    return df_fast_two_sum(p, e);
}

__device__ __forceinline__ dfl df_mulf(dfl x, float f)
{
    float p = x.hi * f;
    float e = fmaf(x.hi, f, -p);
    e = fmaf(x.lo, f, e);
    return df_fast_two_sum(p, e);
}

__device__ __forceinline__ dfl df_addf(dfl x, float f)
{
    dfl s = df_two_sum(x.hi, f);
    return df_fast_two_sum(s.hi, s.lo + x.lo);
}

__host__ __device__ inline dfl df_from_double(double v)
{
    float h = (float)v;
    return {h, (float)(v - (double)h)};
}

__device__ __forceinline__ double df_to_double(dfl x) { return (double)x.hi + (double)x.lo; }

}  // namespace hzb
