// Generating-curve pieces, evaluable on host and device (Sec. 3.2: a body is a
// curve gamma(t) = (r(t), z(t)) swept about the body z axis).
//
// Piece types (parameters in Piece::p):
//   0  ellipse arc      (a sin t, c cos t),                 p = {a, c}
//   1  circular arc     R (sin phi, cos phi), phi = th0 + sg t, p = {R, th0, sg}
//   2  rim semicircle   C u + rho (cos s u + sin s e),      p = {u_r, u_z, e_r, e_z, C, rho}
//   3  cubic segment    r = a + b u + c u^2 + d u^3 (u = t - t_k), the same for z,
//                       p = {a_r, b_r, c_r, d_r, a_z, b_z, c_z, d_z, t_k}: one segment of the
//                       spline generating curve (HZB_CURVE_SPLINE)
// Each provides gamma, gamma' and an offset gamma(t + h) - gamma(t) written with
// difference identities (cos(a+h) - cos a = -2 sin(a + h/2) sin(h/2), ...), so the
// offset keeps full relative accuracy for tiny h: the singular quadrature on a
// target's own panel needs the distance from the target without cancellation.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

namespace hzb {

struct CurvePiece {
    int type;
    double p[10];
};

__host__ __device__ inline void curve_eval(const CurvePiece &pc, double t, double &r, double &z,
                                           double &dr, double &dz)
{
    if (pc.type == 0) {
        double s = sin(t), c = cos(t);
        r = pc.p[0] * s;
        z = pc.p[1] * c;
        dr = pc.p[0] * c;
        dz = -pc.p[1] * s;
    } else if (pc.type == 1) {
        double ph = pc.p[1] + pc.p[2] * t;
        double s = sin(ph), c = cos(ph);
        r = pc.p[0] * s;
        z = pc.p[0] * c;
        dr = pc.p[2] * pc.p[0] * c;
        dz = -pc.p[2] * pc.p[0] * s;
    } else if (pc.type == 3) {
        const double u = t - pc.p[8];
        r = pc.p[0] + u * (pc.p[1] + u * (pc.p[2] + u * pc.p[3]));
        z = pc.p[4] + u * (pc.p[5] + u * (pc.p[6] + u * pc.p[7]));
        dr = pc.p[1] + u * (2.0 * pc.p[2] + 3.0 * u * pc.p[3]);
        dz = pc.p[5] + u * (2.0 * pc.p[6] + 3.0 * u * pc.p[7]);
    } else {
        double s = sin(t), c = cos(t);
        double ur = pc.p[0], uz = pc.p[1], er = pc.p[2], ez = pc.p[3], C = pc.p[4], rho = pc.p[5];
        r = C * ur + rho * (c * ur + s * er);
        z = C * uz + rho * (c * uz + s * ez);
        dr = rho * (-s * ur + c * er);
        dz = rho * (-s * uz + c * ez);
    }
}

// gamma(t + h) - gamma(t)
__host__ __device__ inline void curve_offset(const CurvePiece &pc, double t, double h, double &ddr,
                                             double &ddz)
{
    if (pc.type == 0) {
        double q = 2.0 * sin(0.5 * h);
        ddr = pc.p[0] * cos(t + 0.5 * h) * q;
        ddz = -pc.p[1] * sin(t + 0.5 * h) * q;
    } else if (pc.type == 1) {
        double ph = pc.p[1] + pc.p[2] * t, dp = pc.p[2] * h;
        double q = 2.0 * sin(0.5 * dp);
        ddr = pc.p[0] * cos(ph + 0.5 * dp) * q;
        ddz = -pc.p[0] * sin(ph + 0.5 * dp) * q;
    } else if (pc.type == 3) {
        // p(u + h) - p(u) = h (b + c (2u + h) + d (3u^2 + 3uh + h^2)): no cancellation
        const double u = t - pc.p[8];
        const double e1 = 2.0 * u + h, e2 = 3.0 * u * u + 3.0 * u * h + h * h;
        ddr = h * (pc.p[1] + pc.p[2] * e1 + pc.p[3] * e2);
        ddz = h * (pc.p[5] + pc.p[6] * e1 + pc.p[7] * e2);
    } else {
        double q = 2.0 * sin(0.5 * h);
        double dc = -sin(t + 0.5 * h) * q;      // cos(t+h) - cos t
        double dsn = cos(t + 0.5 * h) * q;      // sin(t+h) - sin t
        double rho = pc.p[5];
        ddr = rho * (dc * pc.p[0] + dsn * pc.p[2]);
        ddz = rho * (dc * pc.p[1] + dsn * pc.p[3]);
    }
}

}  // namespace hzb
