/*
 * Oracle arithmetic in plain C, double precision throughout.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library includes, links or
 * calls this file; only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark load it (through oracle/_native.py).
 *
 * Kernel (Sec. 2, Eq. (Gkappa), with the coupling written as -i*eta for a signed
 * real eta; the paper's own choice is eta = -kappa):
 *     phi(x,y)  = exp(i k R) / (4 pi R),          R = |x - y|
 *     K(x,y)    = d phi(x,y) / d n(y)  -  i eta phi(x,y)
 * and d phi / d n(y) = n(y) . grad_y phi = phi * (i k - 1/R) * n(y).(y - x) / R.
 *
 * Modal kernel (Sec. 3.2, Eqs. (forSeries3), (seqBIE)): for a target on the
 * generating curve at (r, 0, z) and a source ring (r', psi, z') with profile normal
 * (nr', nz'),
 *     k_p = int_0^{2pi} K(x(r,0,z), y(r',psi,z')) exp(i p psi) dpsi .
 * K is even in psi, so k_p = 2 int_0^pi K(psi) cos(p psi) dpsi = k_{-p}.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>

typedef double complex cplx;

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* K(x, y) for world points x, y and unit normal n at y (the definition above). */
static cplx kernel_xyz(const double *x, const double *y, const double *n, double k, double eta)
{
    double d0 = y[0] - x[0], d1 = y[1] - x[1], d2 = y[2] - x[2];
    double R = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    cplx phi = cexp(I * k * R) / (4.0 * M_PI * R);
    double n_dot_ymx = n[0] * d0 + n[1] * d1 + n[2] * d2;
    cplx dphi_dn = phi * (I * k - 1.0 / R) * n_dot_ymx / R;
    return dphi_dn - I * eta * phi;
}

/* The same kernel for a target (r,0,z) and a source at azimuth psi on the ring of
 * radius rs whose profile point is offset by (dr, dz) = (rs - r, zs - z) from the
 * target's, with profile normal (nrs, nzs).  The offsets are passed in (callers
 * form them without cancellation for nearly coincident points) and 1 - cos(psi)
 * is formed as 2 sin^2(psi/2), so nearly coincident points keep their relative
 * accuracy. */
static cplx kernel_ring(double r, double rs, double dr, double dz, double nrs, double nzs,
                        double psi, double k, double eta)
{
    double sh = sin(0.5 * psi);
    double s2 = 2.0 * sh * sh;                       /* 1 - cos psi */
    double R2 = dr * dr + dz * dz + 2.0 * r * rs * s2;
    double R = sqrt(R2);
    /* n(y).(y - x) with y = (rs cos psi, rs sin psi, zs), x = (r, 0, z) */
    double n_dot_ymx = nrs * (dr + r * s2) + nzs * dz;
    cplx phi = cexp(I * k * R) / (4.0 * M_PI * R);
    cplx dphi_dn = phi * (I * k - 1.0 / R) * n_dot_ymx / R;
    return dphi_dn - I * eta * phi;
}

/*
 * Inter-body direct sum (Sec. 3.3, off-diagonal blocks by Eq. (nystromnaive)):
 *   out[t][r] = sum_{j : body[j] != body[tgt[t]]} W[j] K(x_tgt, x_j) sigma[j][r]
 * x, nrm: N x 3; W: N; body: N; sigma: N x R complex (interleaved re, im);
 * tgt: T target indices; out: T x R complex.
 */
void orc_direct_sum(int N, const double *x, const double *nrm, const double *W, const int *body,
                    int R, const double *sigma, double k, double eta,
                    int T, const int *tgt, double *out)
{
    #pragma omp parallel for schedule(dynamic, 16)
    for (int t = 0; t < T; ++t) {
        int i = tgt[t];
        cplx *acc = (cplx *)calloc((size_t)R, sizeof(cplx));
        for (int j = 0; j < N; ++j) {
            if (body[j] == body[i]) continue;
            cplx g = W[j] * kernel_xyz(x + 3 * i, x + 3 * j, nrm + 3 * j, k, eta);
            const cplx *s = (const cplx *)(sigma + 2 * (size_t)j * R);
            for (int q = 0; q < R; ++q) acc[q] += g * s[q];
        }
        cplx *o = (cplx *)(out + 2 * (size_t)t * R);
        for (int q = 0; q < R; ++q) o[q] = acc[q];
        free(acc);
    }
}

/*
 * Field of the density at arbitrary points off the surface (Eq. (intHelm1)
 * discretised with the smooth rule): out[t][r] = sum_j W[j] K(p_t, x_j) sigma[j][r].
 */
void orc_field(int N, const double *x, const double *nrm, const double *W,
               int R, const double *sigma, double k, double eta,
               int T, const double *pts, double *out)
{
    #pragma omp parallel for schedule(dynamic, 4)
    for (int t = 0; t < T; ++t) {
        cplx *acc = (cplx *)calloc((size_t)R, sizeof(cplx));
        for (int j = 0; j < N; ++j) {
            cplx g = W[j] * kernel_xyz(pts + 3 * t, x + 3 * j, nrm + 3 * j, k, eta);
            const cplx *s = (const cplx *)(sigma + 2 * (size_t)j * R);
            for (int q = 0; q < R; ++q) acc[q] += g * s[q];
        }
        cplx *o = (cplx *)(out + 2 * (size_t)t * R);
        for (int q = 0; q < R; ++q) o[q] = acc[q];
        free(acc);
    }
}

/*
 * Modal kernels k_p, p = 0..M, by the trapezoid rule in psi with L equispaced
 * samples, L doubled (starting from the smallest power of two >= max(64, 4(M+1)))
 * until every k_p changes by at most tol * max_p |k_p| (or, past 4096 samples,
 * the change stops halving: the rounding floor).  One call handles one
 * target ring against S source rings (rs, offsets drs, dzs, normals nrs, nzs).  out: S x (M+1) complex;
 * naz_used (may be NULL): the L finally used for each source.
 */
void orc_modes_trapezoid(double r, int S, const double *rs, const double *drs, const double *dzs,
                         const double *nrs, const double *nzs, double k, double eta,
                         int M, double tol, double *out, int *naz_used)
{
    #pragma omp parallel for schedule(dynamic, 8)
    for (int s = 0; s < S; ++s) {
        cplx *sum = (cplx *)calloc((size_t)(M + 1), sizeof(cplx));
        cplx *prev = (cplx *)calloc((size_t)(M + 1), sizeof(cplx));
        int L = 64;
        while (L < 4 * (M + 1)) L *= 2;
        /* initial pass: all L samples */
        for (int q = 0; q < L; ++q) {
            double psi = 2.0 * M_PI * q / L;
            cplx f = kernel_ring(r, rs[s], drs[s], dzs[s], nrs[s], nzs[s], psi, k, eta);
            cplx e = cexp(I * psi), ep = 1.0;
            for (int p = 0; p <= M; ++p) { sum[p] += f * ep; ep *= e; }
        }
        for (int p = 0; p <= M; ++p) prev[p] = sum[p] * (2.0 * M_PI / L);
        double dlast = INFINITY;
        for (;;) {
            /* add the L new midpoints: samples of the 2L-point rule */
            for (int q = 0; q < L; ++q) {
                double psi = 2.0 * M_PI * (q + 0.5) / L;
                cplx f = kernel_ring(r, rs[s], drs[s], dzs[s], nrs[s], nzs[s], psi, k, eta);
                cplx e = cexp(I * psi), ep = 1.0;
                for (int p = 0; p <= M; ++p) { sum[p] += f * ep; ep *= e; }
            }
            L *= 2;
            double dmax = 0.0, vmax = 0.0;
            for (int p = 0; p <= M; ++p) {
                cplx cur = sum[p] * (2.0 * M_PI / L);
                double dd = cabs(cur - prev[p]);
                if (dd > dmax) dmax = dd;
                if (cabs(cur) > vmax) vmax = cabs(cur);
                prev[p] = cur;
            }
            /* converged, or at the rounding floor (no longer halving), or at the cap */
            if (dmax <= tol * vmax || (L >= 4096 && dmax > 0.5 * dlast) || L >= (1 << 18)) break;
            dlast = dmax;
        }
        cplx *o = (cplx *)(out + 2 * (size_t)s * (M + 1));
        for (int p = 0; p <= M; ++p) o[p] = prev[p];
        if (naz_used) naz_used[s] = L;
        free(sum);
        free(prev);
    }
}

/*
 * Modal kernels k_p, p = 0..M, by composite Gauss-Legendre quadrature of
 * 2 int_0^pi K(psi) cos(p psi) dpsi on a mesh graded toward psi = 0, where the
 * integrand peaks when source and target rings nearly touch.  With profile
 * distance d and peak half-width w = d / sqrt(r rs), the first interval is
 * [0, min(w/2, hmax)]; each later interval is [a, a + min(a, hmax)] (so widths
 * double until they reach hmax) until pi.  hmax bounds the phase of cos(p psi)
 * per interval.  glx, glw: an ngl-point Gauss-Legendre rule on [-1, 1].
 */
void orc_modes_graded(double r, int S, const double *rs, const double *drs, const double *dzs,
                      const double *nrs, const double *nzs, double k, double eta,
                      int M, double hmax, int ngl, const double *glx, const double *glw,
                      double *out)
{
    #pragma omp parallel for schedule(dynamic, 8)
    for (int s = 0; s < S; ++s) {
        cplx *acc = (cplx *)calloc((size_t)(M + 1), sizeof(cplx));
        double d = sqrt(drs[s] * drs[s] + dzs[s] * dzs[s]);
        double rr = r * rs[s];
        double w = (rr > 0.0) ? d / sqrt(rr) : M_PI;
        double a = 0.0;
        double b = fmin(0.5 * w, hmax);
        if (b <= 0.0) b = 1e-300;
        while (a < M_PI) {
            if (b > M_PI) b = M_PI;
            double c = 0.5 * (a + b), h = 0.5 * (b - a);
            for (int q = 0; q < ngl; ++q) {
                double psi = c + h * glx[q];
                cplx f = kernel_ring(r, rs[s], drs[s], dzs[s], nrs[s], nzs[s], psi, k, eta) * (h * glw[q]);
                /* cos(p psi) by the three-term recurrence cos((p+1)x) = 2cos x cos(px) - cos((p-1)x) */
                double c1 = cos(psi), cm = 1.0, cp = c1;
                acc[0] += f;
                if (M >= 1) acc[1] += f * c1;
                for (int p = 2; p <= M; ++p) {
                    double cn = 2.0 * c1 * cp - cm;
                    acc[p] += f * cn;
                    cm = cp;
                    cp = cn;
                }
            }
            a = b;
            b = a + fmin(a, hmax);
        }
        cplx *o = (cplx *)(out + 2 * (size_t)s * (M + 1));
        for (int p = 0; p <= M; ++p) o[p] = 2.0 * acc[p];
        free(acc);
    }
}

/* One kernel value on a ring, exposed for pinning the modal sums against a
 * library adaptive quadrature: out = K(psi) (complex). */
void orc_kernel_ring(double r, double rs, double dr, double dz, double nrs, double nzs,
                     double psi, double k, double eta, double *out)
{
    cplx v = kernel_ring(r, rs, dr, dz, nrs, nzs, psi, k, eta);
    out[0] = creal(v);
    out[1] = cimag(v);
}

/* One kernel value for world points, exposed for the same purpose. */
void orc_kernel_xyz(const double *x, const double *y, const double *n, double k, double eta,
                    double *out)
{
    cplx v = kernel_xyz(x, y, n, k, eta);
    out[0] = creal(v);
    out[1] = cimag(v);
}
