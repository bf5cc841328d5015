// Device arithmetic shared by the library's kernels: complex helpers and the
// combined-field kernel
//     K(x, y) = d phi/d n(y) - i eta phi,   phi = e^{ikR} / (4 pi R)
// (Sec. 2, Eq. (Gkappa) with the coupling -i eta), written as
//     K = e^{ikR} / (4 pi R) * [ (1 - ikR) n(y).(x - y) / R^2 - i eta ].
#pragma once

#include <cuda_runtime.h>
#include <math.h>

namespace hzb {

#define HZB_INV4PI 0.07957747154594767

__host__ __device__ inline double2 cmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ inline double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ inline double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ inline double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__host__ __device__ inline double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
// a += b * c
__host__ __device__ inline void cfma(double2 &a, double2 b, double2 c)
{
    a.x = fma(b.x, c.x, fma(-b.y, c.y, a.x));
    a.y = fma(b.x, c.y, fma(b.y, c.x, a.y));
}
__host__ __device__ inline float2 cmulf(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// K for a target at (r, 0, z) and a source on the ring of radius rs at azimuth psi,
// whose profile point is offset (dr, dz) from the target's, with profile normal
// (nrs, nzs).  1 - cos psi is formed as 2 sin^2(psi/2) for nearly touching rings.
__device__ inline double2 ring_kernel64(double r, double rs, double dr, double dz, double nrs,
                                        double nzs, double psi, double k, double eta)
{
    double sh = sin(0.5 * psi);
    double s2 = 2.0 * sh * sh;
    double R2 = fma(dr, dr, fma(dz, dz, 2.0 * r * rs * s2));
    double R = sqrt(R2);
    double iR = 1.0 / R;
    double ndx = -(nrs * (dr + r * s2) + nzs * dz);      // n(y).(x - y)
    double a = ndx * iR * iR;
    double kR = k * R;
    double b = -(kR * a + eta);                            // bracket = a + i b
    double s, c;
    sincos(kR, &s, &c);
    double f = iR * HZB_INV4PI;
    return make_double2((c * a - s * b) * f, (s * a + c * b) * f);
}

}  // namespace hzb
