// FP64 pieces of the inter-body pair kernel shared by the one-directional and the
// pair-symmetric FP64 kernels: 1/sqrt and e^{ix} with few FP64 instructions (GB300
// runs FP64 at 1/64 of the FP32 rate, so integer and FP32-unit work is nearly free).
#pragma once

#include <cuda_runtime.h>

namespace hzb {

static const int SC_N = 4096;           // entries of the FP64 cos/sin table (global memory, read through L1)

// FP64 1/sqrt(x), for normal x inside the FP32 exponent range (1e-37 < x < 1e38):
// the hardware FP32 estimate of x truncated to 20 mantissa bits (the float is built
// from the high word with integer operations) is refined by one Halley step
// y <- y (1 + e/2 + 3e^2/8), e = 1 - x y^2 (cubic convergence: |e| <= 1.2e-6 gives a
// truncation error below 1e-18, so the result is within about 1 ulp).  Five FP64
// operations; the rest runs on the integer and transcendental units.
__device__ __forceinline__ double rsqrt_fp64(double x)
{
    const int hi = __double2hiint(x);
    const float xf = __int_as_float((hi - (896 << 20)) << 3);       // rebias 1023 -> 127
    const int yb = __float_as_int(rsqrtf(xf));
    const double y = __hiloint2double((yb >> 3) + (896 << 20), yb << 29);
    const double e = fma(-x, y * y, 1.0);
    return fma(y * e, fma(e, 0.375, 0.5), y);
}

// FP64 (cos, sin)(2 pi t / SC_N) for 0 <= t < 2^51 (after Tang's table method):
// adding 1.5 * 2^52 rounds t to the integer j, whose low bits are then the low word of
// the sum (no conversion instruction); u = t - j in [-1/2, 1/2].  With
// delta = 2 pi u / SC_N (|delta| <= 7.7e-4), sin(delta) ~ delta - delta^3/6 and
// cos(delta) - 1 ~ -delta^2/2 + delta^4/24 (truncation below 2.3e-18), then angle
// addition with the tabulated (cos, sin)(2 pi j / SC_N).  Nine FP64 operations.
__device__ __forceinline__ void cis_turns(double t, const double2 *__restrict__ tab, double &c, double &s)
{
    constexpr double MAGIC = 6755399441055744.0;           // 1.5 * 2^52
    constexpr double D = 6.283185307179586476925286766559 / SC_N;
    constexpr double A1 = D, A3 = -D * D * D / 6.0;
    constexpr double B2 = -D * D / 2.0, B4 = D * D * D * D / 24.0;
    const double sh = t + MAGIC;
    const int j = __double2loint(sh);
    const double u = t - (sh - MAGIC);
    const double u2 = u * u;
    const double sd = u * fma(u2, A3, A1);                 // sin(delta)
    const double cm = u2 * fma(u2, B4, B2);                // cos(delta) - 1
    const double2 cs = __ldg(&tab[j & (SC_N - 1)]);
    c = fma(cs.x, cm, fma(-cs.y, sd, cs.x));
    s = fma(cs.y, cm, fma(cs.x, sd, cs.y));
}

}  // namespace hzb
