// Lean double-float arithmetic for kernels on the FP32 pipe: a value is hi + lo (two
// floats).  Products and sums are the error-free transformations of Dekker (the
// product's rounding error by a fused multiply-add) and Knuth (two_sum), with results
// left unnormalised (lo may reach a few ulps of hi instead of half an ulp), which
// saves the renormalising fast_two_sum of every operation; a caller renormalises an
// accumulator after a bounded number of additions.  Every operation is written with
// the round-to-nearest intrinsics, which the compiler never contracts into fused
// multiply-adds, so the transformations hold whatever the -fmad setting.
#pragma once

namespace hzb {
namespace lean {

struct dd {
    float h, l;
};

__device__ __forceinline__ dd two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

// the exact product of the high parts plus the cross terms (lo * lo dropped)
__device__ __forceinline__ dd mul(dd a, dd b)
{
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    return {p, e};
}

__device__ __forceinline__ dd add(dd a, dd b)
{
    const dd s = two_sum(a.h, b.h);
    return {s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l))};
}

__device__ __forceinline__ dd sub(dd a, dd b)
{
    const dd s = two_sum(a.h, -b.h);
    return {s.h, __fadd_rn(s.l, __fsub_rn(a.l, b.l))};
}

__device__ __forceinline__ dd neg(dd a) { return {-a.h, -a.l}; }

// renormalise (|lo| <= ulp(hi) / 2 again)
__device__ __forceinline__ dd norm(dd a)
{
    const float s = __fadd_rn(a.h, a.l);
    return {s, __fsub_rn(a.l, __fsub_rn(s, a.h))};
}

__device__ __forceinline__ dd split(double v)
{
    const float h = __double2float_rn(v);
    return {h, __double2float_rn(v - (double)h)};
}

__device__ __forceinline__ double value(dd a) { return (double)a.h + (double)a.l; }

// complex value in double-float: (re.h, re.l, im.h, im.l)
__device__ __forceinline__ float4 csplit(double2 v)
{
    const dd r = split(v.x), i = split(v.y);
    return make_float4(r.h, r.l, i.h, i.l);
}

// acc += a b for complex double-float a, b (four products, four sums)
__device__ __forceinline__ void cmac(dd &ar, dd &ai, float4 a, float4 b)
{
    const dd xr = {a.x, a.y}, xi = {a.z, a.w}, yr = {b.x, b.y}, yi = {b.z, b.w};
    ar = add(ar, sub(mul(xr, yr), mul(xi, yi)));
    ai = add(ai, add(mul(xr, yi), mul(xi, yr)));
}

}  // namespace lean
}  // namespace hzb
