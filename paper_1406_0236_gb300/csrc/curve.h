// Generating-curve pieces, evaluable on host and device (Sec. 3.2: a body is a
// curve gamma(t) = (r(t), z(t)) swept about the body z axis).
//
// Piece types (parameters in Piece::p):
//   0  ellipse arc      (a sin t, c cos t),                 p = {a, c}
//   1  circular arc     R (sin phi, cos phi), phi = th0 + sg t, p = {R, th0, sg}
//   2  rim semicircle   C u + rho (cos s u + sin s e),      p = {u_r, u_z, e_r, e_z, C, rho}
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
    double p[6];
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
