// Host-side discretisation of one body shape: Gauss-Legendre panels on the
// generating curve, ring nodes, arclength weights, outward profile normals and the
// near-panel sets used by the product integration (Sec. 3.1-3.2).
#include <algorithm>
#include <cmath>
#include <cstdio>

#include "curve.h"
#include "hzb_internal.h"

namespace hzb {

// n-point Gauss-Legendre rule on [-1, 1]: Newton iteration on P_n from the
// asymptotic guesses cos(pi (i - 1/4) / (n + 1/2)); P_n and P_n' by the three-term
// recurrence; weights 2 / ((1 - x^2) P_n'(x)^2).  Nodes ascending.
void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w)
{
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 1; i <= n; ++i) {
        double xi = std::cos(M_PI * (i - 0.25) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = xi;
            for (int j = 1; j < n; ++j) {
                double p2 = ((2.0 * j + 1.0) * xi * p1 - j * p0) / (j + 1.0);
                p0 = p1;
                p1 = p2;
            }
            // p1 = P_n(xi), p0 = P_{n-1}(xi)
            dp = n * (xi * p1 - p0) / (xi * xi - 1.0);
            double dx = p1 / dp;
            xi -= dx;
            if (std::fabs(dx) < 1e-16) break;
        }
        {
            double p0 = 1.0, p1 = xi;
            for (int j = 1; j < n; ++j) {
                double p2 = ((2.0 * j + 1.0) * xi * p1 - j * p0) / (j + 1.0);
                p0 = p1;
                p1 = p2;
            }
            dp = n * (xi * p1 - p0) / (xi * xi - 1.0);
        }
        x[n - i] = xi;   // the guesses run from the right end to the left
        w[n - i] = 2.0 / ((1.0 - xi * xi) * dp * dp);
    }
}

void piece_eval(const Piece &pc, double t, double &r, double &z, double &dr, double &dz)
{
    CurvePiece cp;
    cp.type = pc.type;
    for (int q = 0; q < 10; ++q) cp.p[q] = pc.p[q];
    curve_eval(cp, t, r, z, dr, dz);
}

static double dist2_to(const Piece &pc, double t, double r0, double z0)
{
    double r, z, dr, dz;
    piece_eval(pc, t, r, z, dr, dz);
    return (r - r0) * (r - r0) + (z - z0) * (z - z0);
}

// Parameter of the point of [ta, tb] nearest (r0, z0): best of 128 samples, then
// a ternary search on the bracketing sample interval.
static double nearest_parameter(const Piece &pc, double ta, double tb, double r0, double z0)
{
    const int S = 128;
    int best = 0;
    double bd = 1e300;
    for (int s = 0; s <= S; ++s) {
        double t = ta + (tb - ta) * s / S;
        double d = dist2_to(pc, t, r0, z0);
        if (d < bd) { bd = d; best = s; }
    }
    double lo = ta + (tb - ta) * std::max(best - 1, 0) / S;
    double hi = ta + (tb - ta) * std::min(best + 1, S) / S;
    for (int it = 0; it < 200 && hi - lo > 1e-15 * std::max(1.0, std::fabs(tb - ta)); ++it) {
        double m1 = lo + (hi - lo) / 3.0, m2 = hi - (hi - lo) / 3.0;
        if (dist2_to(pc, m1, r0, z0) < dist2_to(pc, m2, r0, z0)) hi = m2; else lo = m1;
    }
    double t = 0.5 * (lo + hi);
    return std::min(std::max(t, ta), tb);
}

// Near-panel radius in units of the panel's arclength (shared reading of the
// paper's "small distance" entries, Sec. 3.1): panel b is treated by product
// integration for target ring i when b is i's own panel or a neighbour along the
// curve, or when some node of b lies closer to i than NEAR_RHO * L_b.
static const double NEAR_RHO = 1.0;

// Cubic spline through (t_k, y_k), k = 0..n-1, as power-form segments
// y = a + b u + c u^2 + d u^3, u = t - t_k: second derivatives M_k from the tridiagonal
// continuity equations (Thomas algorithm); end conditions either y'' = 0 (natural) or
// y' = 0 (clamped) at both ends.
static void cubic_spline(const std::vector<double> &t, const std::vector<double> &y, bool clamped,
                         std::vector<double> &a, std::vector<double> &b, std::vector<double> &c,
                         std::vector<double> &d)
{
    const int n = (int)t.size();
    std::vector<double> h(n - 1), lo(n, 0.0), di(n, 0.0), up(n, 0.0), rhs(n, 0.0), M(n, 0.0);
    for (int k = 0; k + 1 < n; ++k) h[k] = t[k + 1] - t[k];
    for (int k = 1; k + 1 < n; ++k) {
        lo[k] = h[k - 1];
        di[k] = 2.0 * (h[k - 1] + h[k]);
        up[k] = h[k];
        rhs[k] = 6.0 * ((y[k + 1] - y[k]) / h[k] - (y[k] - y[k - 1]) / h[k - 1]);
    }
    if (clamped) {              // y'(t_0) = y'(t_{n-1}) = 0
        di[0] = 2.0 * h[0]; up[0] = h[0]; rhs[0] = 6.0 * (y[1] - y[0]) / h[0];
        lo[n - 1] = h[n - 2]; di[n - 1] = 2.0 * h[n - 2]; rhs[n - 1] = -6.0 * (y[n - 1] - y[n - 2]) / h[n - 2];
    } else {                    // y''(t_0) = y''(t_{n-1}) = 0
        di[0] = 1.0; up[0] = 0.0; rhs[0] = 0.0;
        lo[n - 1] = 0.0; di[n - 1] = 1.0; rhs[n - 1] = 0.0;
    }
    for (int k = 1; k < n; ++k) {       // forward elimination
        const double m = lo[k] / di[k - 1];
        di[k] -= m * up[k - 1];
        rhs[k] -= m * rhs[k - 1];
    }
    M[n - 1] = rhs[n - 1] / di[n - 1];
    for (int k = n - 2; k >= 0; --k) M[k] = (rhs[k] - up[k] * M[k + 1]) / di[k];
    a.resize(n - 1); b.resize(n - 1); c.resize(n - 1); d.resize(n - 1);
    for (int k = 0; k + 1 < n; ++k) {
        a[k] = y[k];
        b[k] = (y[k + 1] - y[k]) / h[k] - h[k] * (2.0 * M[k] + M[k + 1]) / 6.0;
        c[k] = 0.5 * M[k];
        d[k] = (M[k + 1] - M[k]) / (6.0 * h[k]);
    }
}

bool build_shape_geometry(const hzb_shape &spec, const std::vector<double> &curve_rz, ShapeGeom &g,
                          std::string &err)
{
    g.spec = spec;
    g.curve_rz = curve_rz;
    if (spec.n_modes < 3 || spec.n_modes > 1023 || spec.n_modes % 2 == 0) {
        err = "n_modes must be odd in [3, 1023]";
        return false;
    }
    if (spec.gl_order < 2 || spec.gl_order > 32 || spec.n_panels < 1 || spec.n_panels > 4096) {
        err = "gl_order must be in [2, 32] and n_panels in [1, 4096]";
        return false;
    }
    g.pieces.clear();
    std::vector<int> counts;
    if (spec.kind == HZB_SPHERE || spec.kind == HZB_SPHEROID) {
        double a = spec.p[0], c = (spec.kind == HZB_SPHERE) ? spec.p[0] : spec.p[1];
        if (!(a > 0) || !(c > 0)) { err = "semi-axes must be positive"; return false; }
        Piece pc{0, {a, c, 0, 0, 0, 0}, 0.0, M_PI};
        g.pieces.push_back(pc);
        counts.push_back(spec.n_panels);
    } else if (spec.kind == HZB_OPEN_SHELL) {
        double Ro = spec.p[0], Ri = spec.p[1], half = spec.p[2], rho = spec.p[3];
        if (!(Ro > Ri) || !(Ri > 0) || !(half > 0 && half < M_PI) ||
            std::fabs(2.0 * rho - (Ro - Ri)) > 1e-12) {
            err = "open shell needs R_out > R_in > 0, 0 < half-angle < pi, rim = (R_out-R_in)/2";
            return false;
        }
        double th = M_PI - half;
        double ur = std::sin(th), uz = std::cos(th), er = std::cos(th), ez = -std::sin(th);
        g.pieces.push_back(Piece{1, {Ro, 0.0, 1.0, 0, 0, 0}, 0.0, th});
        g.pieces.push_back(Piece{2, {ur, uz, er, ez, 0.5 * (Ro + Ri), rho}, 0.0, M_PI});
        g.pieces.push_back(Piece{1, {Ri, th, -1.0, 0, 0, 0}, 0.0, th});
        // panels proportional to arclength, at least two on the rim
        double Lo = Ro * th, Lr = M_PI * rho, Li = Ri * th, L = Lo + Lr + Li;
        int n = spec.n_panels;
        if (n < 4) { err = "open shell needs at least 4 panels"; return false; }
        int nr = std::max(2, (int)std::lround(n * Lr / L));
        int rest = n - nr;
        int no = (int)std::lround(rest * Lo / (Lo + Li));
        counts = {no, nr, rest - no};
    } else if (spec.kind == HZB_CURVE_SPLINE) {
        // points from the top pole to the bottom pole (both on the axis); chord-length
        // parameter; r natural, z clamped (z' = 0) at the poles; one panel per segment
        const int n = (int)curve_rz.size() / 2;
        if (n < 3 || (int)curve_rz.size() != 2 * n || n - 1 != spec.n_panels) {
            err = "curve needs >= 3 points (r, z) and n_panels = points - 1";
            return false;
        }
        if (curve_rz[0] != 0.0 || curve_rz[2 * (n - 1)] != 0.0) {
            err = "the curve must start and end on the axis (r = 0)";
            return false;
        }
        std::vector<double> t(n, 0.0), r(n), z(n);
        for (int k = 0; k < n; ++k) {
            r[k] = curve_rz[2 * k];
            z[k] = curve_rz[2 * k + 1];
            if (!std::isfinite(r[k]) || !std::isfinite(z[k]) || (k > 0 && k < n - 1 && !(r[k] > 0.0))) {
                err = "curve points must be finite with r > 0 between the poles";
                return false;
            }
            if (k > 0) {
                const double h = std::hypot(r[k] - r[k - 1], z[k] - z[k - 1]);
                if (!(h > 0.0)) { err = "consecutive curve points coincide"; return false; }
                t[k] = t[k - 1] + h;
            }
        }
        if (!(z[0] > z[n - 1])) { err = "the curve must run from the top pole down (outward normal)"; return false; }
        std::vector<double> ar, br, cr, dr, az, bz, cz, dz;
        cubic_spline(t, r, false, ar, br, cr, dr);
        cubic_spline(t, z, true, az, bz, cz, dz);
        for (int k = 0; k + 1 < n; ++k) {
            g.pieces.push_back(Piece{3, {ar[k], br[k], cr[k], dr[k], az[k], bz[k], cz[k], dz[k], t[k], 0.0}, t[k], t[k + 1]});
            counts.push_back(1);
        }
    } else {
        err = "unknown shape kind";
        return false;
    }

    g.panels.clear();
    for (size_t q = 0; q < g.pieces.size(); ++q) {
        const Piece &pc = g.pieces[q];
        for (int m = 0; m < counts[q]; ++m) {
            double ta = pc.t0 + (pc.t1 - pc.t0) * m / counts[q];
            double tb = pc.t0 + (pc.t1 - pc.t0) * (m + 1) / counts[q];
            g.panels.push_back(Panel{(int)q, ta, tb});
        }
    }

    std::vector<double> x, w;
    gauss_legendre(spec.gl_order, x, w);
    const int P = spec.gl_order;
    g.NG = (int)g.panels.size() * P;
    g.NF = spec.n_modes;
    g.M = (spec.n_modes - 1) / 2;
    g.t.resize(g.NG); g.r.resize(g.NG); g.z.resize(g.NG); g.nr.resize(g.NG); g.nz.resize(g.NG);
    g.ds.resize(g.NG); g.speed.resize(g.NG); g.piece_of.resize(g.NG); g.panel_of.resize(g.NG);
    g.panel_len.assign(g.panels.size(), 0.0);
    for (size_t b = 0; b < g.panels.size(); ++b) {
        const Panel &pn = g.panels[b];
        double h = 0.5 * (pn.tb - pn.ta), c = 0.5 * (pn.ta + pn.tb);
        for (int q = 0; q < P; ++q) {
            int i = (int)b * P + q;
            double t = c + h * x[q], r, z, dr, dz;
            piece_eval(g.pieces[pn.piece], t, r, z, dr, dz);
            double sp = std::sqrt(dr * dr + dz * dz);
            g.t[i] = t; g.r[i] = r; g.z[i] = z;
            g.nr[i] = -dz / sp; g.nz[i] = dr / sp;        // outward for this traversal
            g.speed[i] = sp; g.ds[i] = h * w[q] * sp;
            g.piece_of[i] = pn.piece; g.panel_of[i] = (int)b;
            g.panel_len[b] += g.ds[i];
        }
    }

    g.near_start.assign(1, 0);
    g.near_panel.clear();
    g.near_tstar.clear();
    const int NP = (int)g.panels.size();
    for (int i = 0; i < g.NG; ++i) {
        int bi = g.panel_of[i];
        for (int b = 0; b < NP; ++b) {
            bool nr = (b >= bi - 1 && b <= bi + 1);
            if (!nr) {
                double dmin = 1e300;
                for (int q = 0; q < P; ++q) {
                    int j = b * P + q;
                    double d = std::hypot(g.r[j] - g.r[i], g.z[j] - g.z[i]);
                    dmin = std::min(dmin, d);
                }
                nr = dmin < NEAR_RHO * g.panel_len[b];
            }
            if (!nr) continue;
            double ts = (b == bi) ? g.t[i]
                                  : nearest_parameter(g.pieces[g.panels[b].piece], g.panels[b].ta,
                                                      g.panels[b].tb, g.r[i], g.z[i]);
            g.near_panel.push_back(b);
            g.near_tstar.push_back(ts);
        }
        g.near_start.push_back((int)g.near_panel.size());
    }
    return true;
}

}  // namespace hzb
