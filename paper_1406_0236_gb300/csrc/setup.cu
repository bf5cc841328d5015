// Setup on the device, once per distinct shape (Sec. 3.2 and its Remark on the cost
// of precomputation), all in FP64:
//   * surface nodes, normals and weights of every body (tensor-product rule);
//   * far pairs: modal kernels k_p by the trapezoid rule in psi, p = 0..M;
//   * near panels: product integration of k_p against the panel's Lagrange basis;
//   * A~_p = 1/2 I + K_p and S_p = A~_p^{-1} by Gauss-Jordan with partial pivoting.
//
// Modal kernel (Eqs. (forSeries3), (seqBIE) with unnormalised Fourier factors):
//   k_p(y, y') = int_0^{2pi} K(x(y, 0), x(y', psi)) e^{i p psi} dpsi,
// and, K being even in psi, k_p = 2 int_0^pi K cos(p psi) dpsi.
// Per-mode matrix entries (Nystrom, Eq. (nystromnaive) per mode):
//   far panel:  K_p(i, j) = k_p(y_i, y_j) r_j ds_j,
//   near panel: K_p(i, j) = int_panel k_p(y_i, gamma(t)) L_j(t) r(t) |gamma'(t)| dt.
//
// Quadratures of this file (converged to ~1e-14; see the near-panel kernel for the
// singular case):
//   far pairs   trapezoid with L = 2^m >= M + 1 + 45 / alpha samples, alpha =
//               acosh(1 + d^2 / (2 r r')) the half-width of the strip of analyticity
//               of the periodic integrand (d: profile distance);
//   near panels t: composite 20-point Gauss-Legendre on intervals graded
//               geometrically (ratio 0.15, down to 1e-18 of the side) toward the
//               panel point t* nearest the target, on each side of t*;
//               psi: on [0, 1/4] a 64-point Gauss-Legendre rule after the sinh
//               substitution psi = w sinh(mu (x+1)/2), mu = asinh(1/(4w)), which
//               removes the peak of half-width w = d / sqrt(r r') at psi = 0; on
//               [1/4, pi] a fixed composite 12 x 16-point Gauss-Legendre rule.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <string>
#include <vector>

#include "curve.h"
#include "hzb_internal.h"
#include "kernel_math.cuh"

namespace hzb {

static const int LMAX = 4096;           // largest trapezoid rule for far pairs
static const double PSI_C = 0.25;       // end of the sinh-substituted psi interval
static const int NPSI_S = 64;           // nodes of the sinh-substituted rule
static const int NPSI_C = 192;          // nodes of the composite rule on [PSI_C, pi]
static const int NPSI = NPSI_S + NPSI_C;
static const int GL_T = 20;             // Gauss-Legendre order of the graded t-mesh
static const double T_RATIO = 0.15;
static const int T_LEVELS = 22;         // 0.15^22 < 1e-18
static const int NT_SIDE = GL_T * T_LEVELS;

// ------------------------------------------------------------------ nodes

struct Xform {
    double c[3];
    double R[9];
    double o[3];
};

__global__ void body_nodes_kernel(int NG, int NF, const double *__restrict__ ring, Xform xf, int body,
                                  long long off, double4 *pos64, double4 *nrm64, float4 *pos32,
                                  float4 *nrm32, int *body_of)
{
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)NG * NF) return;
    int i = (int)(idx / NF), l = (int)(idx % NF);
    double s, c;
    sincospi(2.0 * l / NF, &s, &c);
    const double *rg = ring + 8 * i;
    double r = rg[0], z = rg[1], nr = rg[2], nz = rg[3], ds = rg[4];
    double lx = r * c, ly = r * s, lz = z;
    double mx = nr * c, my = nr * s, mz = nz;
    double x = xf.c[0] + xf.R[0] * lx + xf.R[1] * ly + xf.R[2] * lz;
    double y = xf.c[1] + xf.R[3] * lx + xf.R[4] * ly + xf.R[5] * lz;
    double zz = xf.c[2] + xf.R[6] * lx + xf.R[7] * ly + xf.R[8] * lz;
    double nx = xf.R[0] * mx + xf.R[1] * my + xf.R[2] * mz;
    double ny = xf.R[3] * mx + xf.R[4] * my + xf.R[5] * mz;
    double nzw = xf.R[6] * mx + xf.R[7] * my + xf.R[8] * mz;
    double w = ds * r * (2.0 * M_PI / NF);
    long long g = off + idx;
    pos64[g] = make_double4(x, y, zz, w);
    nrm64[g] = make_double4(nx, ny, nzw, 0.0);
    pos32[g] = make_float4((float)(x - xf.o[0]), (float)(y - xf.o[1]), (float)(zz - xf.o[2]), (float)w);
    nrm32[g] = make_float4((float)nx, (float)ny, (float)nzw, 0.0f);
    body_of[g] = body;
}

// Validation of the generated surface rule: finite positions and normals, |n| = 1 to
// 1e-9, weights finite and > 0.  out[0] counts bad nodes, out[1] holds the smallest
// bad index (both start at 0 and INT_MAX).
__global__ void check_nodes_kernel(long long N, const double4 *__restrict__ pos, const double4 *__restrict__ nrm,
                                   int *out)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double4 p = pos[i], n = nrm[i];
    const double nn = n.x * n.x + n.y * n.y + n.z * n.z;
    const bool ok = isfinite(p.x) && isfinite(p.y) && isfinite(p.z) && isfinite(p.w) && p.w > 0.0 &&
                    isfinite(nn) && fabs(nn - 1.0) < 1e-9;
    if (!ok) {
        atomicAdd(out, 1);
        atomicMin(out + 1, (int)i);
    }
}

// The closed profile of a shape in its (r, z) half-plane: the curve's first end, the ring
// nodes in order, its last end (both ends lie on the axis), closed along the axis.
static void shape_profile(const ShapeGeom &g, std::vector<double> &pr, std::vector<double> &pz)
{
    double r, z, dr, dz;
    pr.clear();
    pz.clear();
    piece_eval(g.pieces.front(), g.pieces.front().t0, r, z, dr, dz);
    pr.push_back(std::fabs(r)); pz.push_back(z);
    for (int i = 0; i < g.NG; ++i) { pr.push_back(g.r[i]); pz.push_back(g.z[i]); }
    piece_eval(g.pieces.back(), g.pieces.back().t1, r, z, dr, dz);
    pr.push_back(std::fabs(r)); pz.push_back(z);
}

// even-odd crossing test of (r, z) against the closed polygon (pr, pz)
static bool inside_profile(const std::vector<double> &pr, const std::vector<double> &pz, double r, double z)
{
    bool in = false;
    const size_t n = pr.size();
    for (size_t a = 0, b = n - 1; a < n; b = a++) {
        if ((pz[a] > z) != (pz[b] > z)) {
            const double rc = pr[a] + (z - pz[a]) * (pr[b] - pr[a]) / (pz[b] - pz[a]);
            if (r < rc) in = !in;
        }
    }
    return in;
}

// Bodies must not intersect: for every pair whose bounding spheres meet, the ring nodes of
// each (at up to 32 azimuths) are tested against the other's solid (its profile rotated
// about its axis).  Returns false with p, q set for the first overlapping pair.
static bool bodies_disjoint(const hzb_ctx *c, int &p_out, int &q_out)
{
    const size_t nb = c->bodies.size(), ns = c->shapes.size();
    std::vector<std::vector<double>> PR(ns), PZ(ns);
    std::vector<double> bound(ns, 0.0);
    for (size_t s = 0; s < ns; ++s) {
        shape_profile(c->shapes[s]->geom, PR[s], PZ[s]);
        for (size_t a = 0; a < PR[s].size(); ++a) bound[s] = std::max(bound[s], std::hypot(PR[s][a], PZ[s][a]));
        bound[s] *= 1.001;
    }
    for (size_t p = 0; p < nb; ++p)
        for (size_t q = 0; q < nb; ++q) {
            if (p == q) continue;
            const BodyRec &A = c->bodies[p], &B = c->bodies[q];
            const double dc = std::sqrt((A.c[0] - B.c[0]) * (A.c[0] - B.c[0]) + (A.c[1] - B.c[1]) * (A.c[1] - B.c[1]) +
                                        (A.c[2] - B.c[2]) * (A.c[2] - B.c[2]));
            if (dc > bound[A.shape] + bound[B.shape]) continue;
            const ShapeGeom &ga = c->shapes[A.shape]->geom;
            const int step = std::max(1, ga.NF / 32);
            for (int i = 0; i < ga.NG; ++i)
                for (int l = 0; l < ga.NF; l += step) {
                    const double th = 2.0 * M_PI * l / ga.NF;
                    const double lx = ga.r[i] * std::cos(th), ly = ga.r[i] * std::sin(th), lz = ga.z[i];
                    double x[3], y[3];
                    for (int e = 0; e < 3; ++e)
                        x[e] = A.c[e] + A.rot[3 * e] * lx + A.rot[3 * e + 1] * ly + A.rot[3 * e + 2] * lz - B.c[e];
                    for (int e = 0; e < 3; ++e)          // into B's frame: rot^T (x - c_B)
                        y[e] = B.rot[e] * x[0] + B.rot[3 + e] * x[1] + B.rot[6 + e] * x[2];
                    if (y[0] * y[0] + y[1] * y[1] + y[2] * y[2] > bound[B.shape] * bound[B.shape]) continue;
                    if (inside_profile(PR[B.shape], PZ[B.shape], std::hypot(y[0], y[1]), y[2])) {
                        p_out = (int)p;
                        q_out = (int)q;
                        return false;
                    }
                }
        }
    return true;
}

hzb_status make_nodes(hzb_ctx *c)
{
    if (c->nodes_ready) return HZB_OK;
    size_t N = (size_t)c->N;
    {
        int bp = -1, bq = -1;
        if (!bodies_disjoint(c, bp, bq))
            return fail(c, HZB_EINVAL, "bodies " + std::to_string(bp) + " and " + std::to_string(bq) +
                                           " overlap (a node of body " + std::to_string(bp) +
                                           " lies inside body " + std::to_string(bq) + ")");
    }
    if (check_cuda(c, c->pos64.ensure(N), "alloc nodes") || check_cuda(c, c->nrm64.ensure(N), "alloc") ||
        check_cuda(c, c->pos32.ensure(N), "alloc") || check_cuda(c, c->nrm32.ensure(N), "alloc") ||
        check_cuda(c, c->body_of.ensure(N), "alloc"))
        return HZB_ENOMEM;
    // origin of the FP32 coordinates: mean of the body centres
    double o[3] = {0, 0, 0};
    for (auto &b : c->bodies)
        for (int q = 0; q < 3; ++q) o[q] += b.c[q] / c->bodies.size();
    for (int q = 0; q < 3; ++q) c->center[q] = o[q];
    for (size_t s = 0; s < c->shapes.size(); ++s) {
        ShapeDev &sd = *c->shapes[s];
        const ShapeGeom &g = sd.geom;
        std::vector<double> ring(8 * g.NG, 0.0);
        for (int i = 0; i < g.NG; ++i) {
            ring[8 * i + 0] = g.r[i];
            ring[8 * i + 1] = g.z[i];
            ring[8 * i + 2] = g.nr[i];
            ring[8 * i + 3] = g.nz[i];
            ring[8 * i + 4] = g.ds[i];
            ring[8 * i + 5] = g.t[i];
        }
        if (check_cuda(c, sd.ring.ensure(ring.size()), "alloc ring")) return HZB_ENOMEM;
        std::vector<long long> offs;
        for (int b : sd.bodies) offs.push_back(c->bodies[b].offset);
        if (check_cuda(c, sd.body_offs.ensure(offs.size()), "alloc offsets")) return HZB_ENOMEM;
        if (check_cuda(c, cudaMemcpyAsync(sd.body_offs.ptr, offs.data(), offs.size() * sizeof(long long),
                                          cudaMemcpyHostToDevice, c->stream), "copy offsets"))
            return HZB_ECUDA;
        if (check_cuda(c, cudaMemcpyAsync(sd.ring.ptr, ring.data(), ring.size() * sizeof(double),
                                          cudaMemcpyHostToDevice, c->stream), "copy ring"))
            return HZB_ECUDA;
    }
    for (size_t bi = 0; bi < c->bodies.size(); ++bi) {
        const BodyRec &b = c->bodies[bi];
        ShapeDev &sd = *c->shapes[b.shape];
        Xform xf;
        for (int q = 0; q < 3; ++q) { xf.c[q] = b.c[q]; xf.o[q] = o[q]; }
        for (int q = 0; q < 9; ++q) xf.R[q] = b.rot[q];
        long long n = (long long)sd.geom.NG * sd.geom.NF;
        int th = 256;
        int bl = (int)((n + th - 1) / th);
        body_nodes_kernel<<<bl, th, 0, c->stream>>>(sd.geom.NG, sd.geom.NF, sd.ring.ptr, xf, (int)bi,
                                                    b.offset, c->pos64.ptr, c->nrm64.ptr, c->pos32.ptr,
                                                    c->nrm32.ptr, c->body_of.ptr);
        if (check_cuda(c, cudaGetLastError(), "body_nodes_kernel")) return HZB_ECUDA;
    }
    // target blocks of the inter-body sum: contiguous ranges inside one body
    const int TB = 512;
    std::vector<TargetBlock> blocks;
    c->body_block0.clear();
    for (const BodyRec &b : c->bodies) {
        c->body_block0.push_back((int)blocks.size());
        for (int s = 0; s < b.n_nodes; s += TB) {
            TargetBlock t;
            t.start = (int)(b.offset + s);
            t.count = std::min(TB, b.n_nodes - s);
            t.excl_lo = (int)b.offset;
            t.excl_hi = (int)(b.offset + b.n_nodes);
            blocks.push_back(t);
        }
    }
    c->n_tblocks = (int)blocks.size();
    c->body_block0.push_back(c->n_tblocks);
    if (check_cuda(c, c->tblocks.ensure(blocks.size()), "alloc blocks")) return HZB_ENOMEM;
    if (check_cuda(c, cudaMemcpyAsync(c->tblocks.ptr, blocks.data(), blocks.size() * sizeof(TargetBlock),
                                      cudaMemcpyHostToDevice, c->stream), "copy blocks"))
        return HZB_ECUDA;
    if (check_cuda(c, c->nodecheck.ensure(2), "alloc node check")) return HZB_ENOMEM;
    if ((c->fault & FAULT_GEOM) && !(c->fault_spent & FAULT_GEOM)) {      // injected: a NaN weight
        c->fault_spent |= FAULT_GEOM;
        static const double qnan = std::nan("");
        if (check_cuda(c, cudaMemcpyAsync(&c->pos64.ptr[N / 2].w, &qnan, sizeof(double), cudaMemcpyHostToDevice,
                                          c->stream), "inject geometry fault"))
            return HZB_ECUDA;
    }
    int hchk[2] = {0, 0x7fffffff};
    if (check_cuda(c, cudaMemcpyAsync(c->nodecheck.ptr, hchk, sizeof(hchk), cudaMemcpyHostToDevice, c->stream),
                   "node check"))
        return HZB_ECUDA;
    check_nodes_kernel<<<(unsigned)((N + 255) / 256), 256, 0, c->stream>>>((long long)N, c->pos64.ptr, c->nrm64.ptr,
                                                                           c->nodecheck.ptr);
    if (check_cuda(c, cudaGetLastError(), "check_nodes_kernel") ||
        check_cuda(c, cudaMemcpyAsync(hchk, c->nodecheck.ptr, sizeof(hchk), cudaMemcpyDeviceToHost, c->stream),
                   "node check") ||
        check_cuda(c, cudaStreamSynchronize(c->stream), "nodes"))
        return HZB_ECUDA;
    if (hchk[0] > 0)
        return fail(c, HZB_EINVAL, std::to_string(hchk[0]) + " surface nodes are invalid (first: node " +
                                       std::to_string(hchk[1]) +
                                       "): non-finite position or normal, |n| != 1 or weight <= 0");
    c->nodes_ready = true;
    return HZB_OK;
}

// ------------------------------------------------------------------ far pairs

__global__ void far_modes_kernel(int NG, int M, const double *__restrict__ ring,
                                 const int *__restrict__ panel_of, const int *__restrict__ near_start,
                                 const int *__restrict__ near_panel, double k, double eta, double2 *A)
{
    extern __shared__ double sm[];
    double *costab = sm;                               // LMAX: cos(2 pi m / LMAX)
    double2 *f = (double2 *)(sm + LMAX);               // LMAX / 2 + 1 samples
    __shared__ int nlist[64];
    __shared__ int nn;
    const int i = blockIdx.x;
    const int tid = threadIdx.x;
    for (int m = tid; m < LMAX; m += blockDim.x) costab[m] = cospi(2.0 * m / LMAX);
    if (tid == 0) {
        int a = near_start[i], b = near_start[i + 1];
        nn = min(b - a, 64);
        for (int q = 0; q < nn; ++q) nlist[q] = near_panel[a + q];
    }
    __syncthreads();
    const double ri = ring[8 * i], zi = ring[8 * i + 1];
    for (int j = 0; j < NG; ++j) {
        int pj = panel_of[j];
        bool near = false;
        for (int q = 0; q < nn; ++q) near |= (nlist[q] == pj);
        if (near) continue;                                     // uniform over the block
        const double rs = ring[8 * j], zs = ring[8 * j + 1], nrs = ring[8 * j + 2], nzs = ring[8 * j + 3],
                     ds = ring[8 * j + 4];
        const double dr = rs - ri, dz = zs - zi;
        const double alpha = acosh(1.0 + (dr * dr + dz * dz) / (2.0 * ri * rs));
        const double need = M + 1 + 45.0 / alpha;
        int L = 64;
        while (L < need && L < LMAX) L *= 2;
        const int half = L / 2;
        for (int q = tid; q <= half; q += blockDim.x)
            f[q] = ring_kernel64(ri, rs, dr, dz, nrs, nzs, 2.0 * M_PI * q / L, k, eta);
        __syncthreads();
        const int stride = LMAX / L;
        const double scale = 2.0 * M_PI / L * rs * ds;
        for (int p = tid; p <= M; p += blockDim.x) {
            double2 acc = f[0];
            double sg = (p & 1) ? -1.0 : 1.0;
            acc.x += sg * f[half].x;
            acc.y += sg * f[half].y;
            double ax = 0.0, ay = 0.0;
            int idx = 0;
            for (int q = 1; q < half; ++q) {
                idx += p;
                if (idx >= L) idx -= L;
                double cq = costab[idx * stride];
                ax = fma(f[q].x, cq, ax);
                ay = fma(f[q].y, cq, ay);
            }
            acc.x += 2.0 * ax;
            acc.y += 2.0 * ay;
            A[((size_t)p * NG + i) * NG + j] = make_double2(acc.x * scale, acc.y * scale);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ near panels

struct NearItem {
    int i;        // target ring
    int b;        // panel
    int self;     // target lies on this panel
    int pad;
    double tstar;
};

struct NearArgs {
    int NG, M, P;
    const double *ring;          // NG x 8
    const CurvePiece *pieces;
    const int *panel_piece;
    const double *panel_ta, *panel_tb;
    const NearItem *items;
    const double *glt_x, *glt_w;       // GL_T
    const double *gls_x, *gls_w;       // NPSI_S
    const double *psic, *psic_w;       // NPSI_C composite nodes on [PSI_C, pi]
    const double *Cc;                  // NPSI_C x (M+1): cos(p psi)
    double k, eta;
    double2 *A;
};

// Per t-node scratch in shared memory.
struct TNode {
    double r, offr, offz, nr, nz, wJ, t, w;
};

__global__ void near_panel_kernel(NearArgs a, int TB, int SPT)
{
    extern __shared__ double sm[];
    const int M1 = a.M + 1, P = a.P;
    TNode *geo = (TNode *)sm;                                   // TB
    double *coef = (double *)(geo + TB);                        // TB x P (padded to even)
    double *psi0 = coef + ((TB * P + 1) & ~1);                  // TB x NPSI_S
    double *wps0 = psi0 + TB * NPSI_S;                          // TB x NPSI_S
    double2 *F = (double2 *)(wps0 + TB * NPSI_S);               // TB x NPSI
    double *Cw = (double *)(F + TB * NPSI);                     // TB x M1 x NPSI_S
    double2 *mom = (double2 *)(Cw + (size_t)TB * M1 * NPSI_S);  // TB x M1

    const NearItem it = a.items[blockIdx.x];
    const int tid = threadIdx.x, nth = blockDim.x;
    const double ri = a.ring[8 * it.i], zi = a.ring[8 * it.i + 1];
    const CurvePiece pc = a.pieces[a.panel_piece[it.b]];
    const double ta = a.panel_ta[it.b], tb = a.panel_tb[it.b];
    const double ts = it.tstar;
    const int col0 = it.b * P;

    double2 acc[8];
    for (int s = 0; s < 8; ++s) acc[s] = make_double2(0.0, 0.0);

    const int NT = 2 * NT_SIDE;
    for (int base = 0; base < NT; base += TB) {
        // A: geometry of the TB t-nodes
        if (tid < TB) {
            int n = base + tid;
            TNode g;
            g.wJ = 0.0; g.w = 1.0; g.r = ri; g.offr = 1.0; g.offz = 0.0; g.nr = 0.0; g.nz = 1.0; g.t = ts;
            if (n < NT) {
                int side = n / NT_SIDE, rem = n % NT_SIDE;
                int lev = rem / GL_T, q = rem % GL_T;
                double H = side ? (tb - ts) : (ta - ts);
                if (H != 0.0) {
                    double hi = pow(T_RATIO, (double)lev), lo = hi * T_RATIO;
                    double x0 = lo * H, x1 = hi * H;
                    double h = 0.5 * (x0 + x1) + 0.5 * (x1 - x0) * a.glt_x[q];
                    double wt = 0.5 * fabs(x1 - x0) * a.glt_w[q];
                    double t = ts + h, r, z, dr, dz;
                    curve_eval(pc, t, r, z, dr, dz);
                    double sp = sqrt(dr * dr + dz * dz);
                    double offr, offz;
                    if (it.self) curve_offset(pc, ts, h, offr, offz);
                    else { offr = r - ri; offz = z - zi; }
                    g.r = r; g.offr = offr; g.offz = offz; g.nr = -dz / sp; g.nz = dr / sp;
                    g.wJ = wt * r * sp; g.t = t;
                    g.w = sqrt(offr * offr + offz * offz) / sqrt(ri * r);
                }
            }
            geo[tid] = g;
        }
        __syncthreads();
        // B: Lagrange coefficients and the t-node dependent psi nodes
        for (int e = tid; e < TB * P; e += nth) {
            int q = e / P, j = e % P;
            double t = geo[q].t, tj = a.ring[8 * (col0 + j) + 5], L = 1.0;
            for (int m = 0; m < P; ++m)
                if (m != j) {
                    double tm = a.ring[8 * (col0 + m) + 5];
                    L *= (t - tm) / (tj - tm);
                }
            coef[e] = geo[q].wJ * L;
        }
        for (int e = tid; e < TB * NPSI_S; e += nth) {
            int q = e / NPSI_S, m = e % NPSI_S;
            double w = geo[q].w, x = a.gls_x[m], ps, wp;
            if (w < PSI_C) {
                double mu = asinh(PSI_C / w), s = 0.5 * mu * (x + 1.0);
                ps = w * sinh(s);
                wp = a.gls_w[m] * w * 0.5 * mu * cosh(s);
            } else {
                ps = 0.5 * PSI_C * (x + 1.0);
                wp = 0.5 * PSI_C * a.gls_w[m];
            }
            psi0[e] = ps;
            wps0[e] = wp;
        }
        __syncthreads();
        // C: weighted kernel samples and cos(p psi) of the t-node dependent nodes
        for (int e = tid; e < TB * NPSI; e += nth) {
            int q = e / NPSI, m = e % NPSI;
            const TNode &g = geo[q];
            double ps, wp;
            if (m < NPSI_S) { ps = psi0[q * NPSI_S + m]; wp = wps0[q * NPSI_S + m]; }
            else { ps = a.psic[m - NPSI_S]; wp = a.psic_w[m - NPSI_S]; }
            double2 v = ring_kernel64(ri, g.r, g.offr, g.offz, g.nr, g.nz, ps, a.k, a.eta);
            F[e] = make_double2(v.x * wp, v.y * wp);
        }
        for (int e = tid; e < TB * NPSI_S; e += nth) {
            int q = e / NPSI_S, m = e % NPSI_S;
            double c1 = cos(psi0[e]), cm = 1.0, cp = c1;
            double *col = Cw + (size_t)q * M1 * NPSI_S;
            col[m] = 1.0;
            if (M1 > 1) col[NPSI_S + m] = c1;
            for (int p = 2; p < M1; ++p) {          // cos((p)x) = 2 cos x cos((p-1)x) - cos((p-2)x)
                double cn = 2.0 * c1 * cp - cm;
                col[(size_t)p * NPSI_S + m] = cn;
                cm = cp;
                cp = cn;
            }
        }
        __syncthreads();
        // D: modal moments 2 sum_q F cos(p psi_q)
        for (int e = tid; e < TB * M1; e += nth) {
            int q = e / M1, p = e % M1;
            const double2 *Fq = F + q * NPSI;
            const double *cw = Cw + ((size_t)q * M1 + p) * NPSI_S;
            double sx = 0.0, sy = 0.0;
            for (int m = 0; m < NPSI_S; ++m) {
                sx = fma(Fq[m].x, cw[m], sx);
                sy = fma(Fq[m].y, cw[m], sy);
            }
            for (int m = 0; m < NPSI_C; ++m) {
                double cc = a.Cc[(size_t)m * M1 + p];
                sx = fma(Fq[NPSI_S + m].x, cc, sx);
                sy = fma(Fq[NPSI_S + m].y, cc, sy);
            }
            mom[e] = make_double2(2.0 * sx, 2.0 * sy);
        }
        __syncthreads();
        // E: accumulate into the owned (p, j) entries
        for (int s = 0; s < SPT; ++s) {
            int e = tid + s * nth;
            if (e < M1 * P) {
                int p = e / P, j = e % P;
                for (int q = 0; q < TB; ++q) {
                    double cj = coef[q * P + j];
                    acc[s].x = fma(cj, mom[q * M1 + p].x, acc[s].x);
                    acc[s].y = fma(cj, mom[q * M1 + p].y, acc[s].y);
                }
            }
        }
        __syncthreads();
    }
    for (int s = 0; s < SPT; ++s) {
        int e = tid + s * nth;
        if (e < M1 * P) {
            int p = e / P, j = e % P;
            int col = col0 + j;
            double2 v = acc[s];
            if (col == it.i) v.x += 0.5;          // A~_p = 1/2 I + K_p
            a.A[((size_t)p * a.NG + it.i) * a.NG + col] = v;
        }
    }
}

// ------------------------------------------------------------------ Gauss-Jordan inverse

// Pivot step k of in-place Gauss-Jordan inversion, one block per matrix: choose the
// largest |A[i][k]|, i >= k, swap it into row k, scale row k by 1/pivot (with
// A[k][k] := 1/pivot) and save the column-k multipliers of the other rows.
__global__ void gj_pivot_kernel(int n, int k, double2 *A, double2 *colk, int *perm, int *singular)
{
    const int mat = blockIdx.x;
    double2 *Am = A + (size_t)mat * n * n;
    double2 *ck = colk + (size_t)mat * n;
    __shared__ double bestv[256];
    __shared__ int besti[256];
    const int tid = threadIdx.x;
    double bv = -1.0;
    int bi = k;
    for (int i = k + tid; i < n; i += blockDim.x) {
        double2 v = Am[(size_t)i * n + k];
        double m = v.x * v.x + v.y * v.y;
        if (m > bv) { bv = m; bi = i; }
    }
    bestv[tid] = bv;
    besti[tid] = bi;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (tid < s) {
            double o = bestv[tid + s];
            int oi = besti[tid + s];
            if (o > bestv[tid] || (o == bestv[tid] && oi < besti[tid])) { bestv[tid] = o; besti[tid] = oi; }
        }
        __syncthreads();
    }
    const int r = besti[0];
    if (tid == 0) {
        perm[(size_t)mat * n + k] = r;
        if (!(bestv[0] > 0.0)) singular[mat] = 1;
    }
    if (r != k)
        for (int j = tid; j < n; j += blockDim.x) {
            double2 t = Am[(size_t)k * n + j];
            Am[(size_t)k * n + j] = Am[(size_t)r * n + j];
            Am[(size_t)r * n + j] = t;
        }
    __syncthreads();
    double2 pv = Am[(size_t)k * n + k];
    double den = pv.x * pv.x + pv.y * pv.y;
    double2 inv = (den > 0.0) ? make_double2(pv.x / den, -pv.y / den) : make_double2(0.0, 0.0);
    for (int i = tid; i < n; i += blockDim.x) ck[i] = (i == k) ? make_double2(0.0, 0.0) : Am[(size_t)i * n + k];
    __syncthreads();
    for (int j = tid; j < n; j += blockDim.x) {
        if (j == k) Am[(size_t)k * n + k] = inv;
        else Am[(size_t)k * n + j] = cmul(Am[(size_t)k * n + j], inv);
    }
}

// Elimination of step k: A[i][j] -= f_i A[k][j] (i != k, j != k); A[i][k] = -f_i A[k][k].
__global__ void gj_elim_kernel(int n, int k, double2 *A, const double2 *colk)
{
    const int mat = blockIdx.y;
    double2 *Am = A + (size_t)mat * n * n;
    const double2 *ck = colk + (size_t)mat * n;
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)n * n) return;
    int i = (int)(e / n), j = (int)(e % n);
    if (i == k) return;
    double2 f = ck[i];
    double2 akj = Am[(size_t)k * n + j];
    if (j == k) {
        double2 v = cmul(f, akj);
        Am[(size_t)i * n + k] = make_double2(-v.x, -v.y);
    } else {
        double2 v = Am[(size_t)i * n + j];
        cfma(v, make_double2(-f.x, -f.y), akj);
        Am[(size_t)i * n + j] = v;
    }
}

// Undo the row interchanges as column interchanges, last pivot first.
__global__ void gj_colswap_kernel(int n, double2 *A, const int *perm)
{
    const int mat = blockIdx.x;
    double2 *Am = A + (size_t)mat * n * n;
    for (int k = n - 1; k >= 0; --k) {
        int r = perm[(size_t)mat * n + k];
        if (r != k)
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                double2 t = Am[(size_t)i * n + k];
                Am[(size_t)i * n + k] = Am[(size_t)i * n + r];
                Am[(size_t)i * n + r] = t;
            }
        __syncthreads();
    }
}

__global__ void to_fp32_kernel(size_t n, const double2 *a, float2 *b)
{
    size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) b[e] = make_float2((float)a[e].x, (float)a[e].y);
}

// ------------------------------------------------------------------ host driver

template <typename T>
static hzb_status upload(hzb_ctx *c, DevBuf<T> &buf, const std::vector<T> &v)
{
    if (check_cuda(c, buf.ensure(v.size() ? v.size() : 1), "setup alloc")) return HZB_ENOMEM;
    if (!v.empty() &&
        check_cuda(c, cudaMemcpyAsync(buf.ptr, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice,
                                      c->stream), "setup upload"))
        return HZB_ECUDA;
    return HZB_OK;
}

hzb_status build_shape_matrices(hzb_ctx *c, ShapeDev &sd)
{
    const ShapeGeom &g = sd.geom;
    const int NG = g.NG, M = g.M, M1 = M + 1, P = g.spec.gl_order;
    if ((size_t)M1 * P > 8 * 256) return fail(c, HZB_EINVAL, "(M+1) * gl_order too large for the setup kernel");
    const size_t nmat = (size_t)M1 * NG * NG;
    if (check_cuda(c, sd.A64.ensure(nmat), "alloc A") || check_cuda(c, sd.S64.ensure(nmat), "alloc S") ||
        check_cuda(c, sd.S32.ensure(nmat), "alloc S32"))
        return HZB_ENOMEM;

    DevBuf<int> d_panel_of, d_near_start, d_near_panel, d_panel_piece, d_perm, d_sing;
    DevBuf<double> d_ta, d_tb, d_glt_x, d_glt_w, d_gls_x, d_gls_w, d_psic, d_psic_w, d_Cc;
    DevBuf<CurvePiece> d_pieces;
    DevBuf<NearItem> d_items;
    DevBuf<double2> d_colk;
    hzb_status st = HZB_OK;
    auto cleanup = [&]() {
        d_panel_of.release(); d_near_start.release(); d_near_panel.release(); d_panel_piece.release();
        d_perm.release(); d_sing.release(); d_ta.release(); d_tb.release(); d_glt_x.release();
        d_glt_w.release(); d_gls_x.release(); d_gls_w.release(); d_psic.release(); d_psic_w.release();
        d_Cc.release(); d_pieces.release(); d_items.release(); d_colk.release();
    };

    std::vector<CurvePiece> pieces;
    for (const Piece &p : g.pieces) {
        CurvePiece cp;
        cp.type = p.type;
        for (int q = 0; q < 10; ++q) cp.p[q] = p.p[q];
        pieces.push_back(cp);
    }
    std::vector<int> panel_piece;
    std::vector<double> ta, tb;
    for (const Panel &pn : g.panels) { panel_piece.push_back(pn.piece); ta.push_back(pn.ta); tb.push_back(pn.tb); }
    std::vector<double> gx, gw, sx, sw, cx, cw;
    gauss_legendre(GL_T, gx, gw);
    gauss_legendre(NPSI_S, sx, sw);
    gauss_legendre(16, cx, cw);
    std::vector<double> psic, psicw;
    const int NCI = NPSI_C / 16;
    for (int q = 0; q < NCI; ++q) {
        double a0 = PSI_C + (M_PI - PSI_C) * q / NCI, a1 = PSI_C + (M_PI - PSI_C) * (q + 1) / NCI;
        for (int m = 0; m < 16; ++m) {
            psic.push_back(0.5 * (a0 + a1) + 0.5 * (a1 - a0) * cx[m]);
            psicw.push_back(0.5 * (a1 - a0) * cw[m]);
        }
    }
    std::vector<double> Cc((size_t)NPSI_C * M1);
    for (int m = 0; m < NPSI_C; ++m)
        for (int p = 0; p < M1; ++p) Cc[(size_t)m * M1 + p] = std::cos(p * psic[m]);
    std::vector<NearItem> items;
    for (int i = 0; i < NG; ++i)
        for (int e = g.near_start[i]; e < g.near_start[i + 1]; ++e) {
            NearItem it;
            it.i = i;
            it.b = g.near_panel[e];
            it.self = (g.panel_of[i] == it.b);
            it.pad = 0;
            it.tstar = g.near_tstar[e];
            items.push_back(it);
        }

    if ((st = upload(c, d_panel_of, g.panel_of)) || (st = upload(c, d_near_start, g.near_start)) ||
        (st = upload(c, d_near_panel, g.near_panel)) || (st = upload(c, d_panel_piece, panel_piece)) ||
        (st = upload(c, d_ta, ta)) || (st = upload(c, d_tb, tb)) || (st = upload(c, d_glt_x, gx)) ||
        (st = upload(c, d_glt_w, gw)) || (st = upload(c, d_gls_x, sx)) || (st = upload(c, d_gls_w, sw)) ||
        (st = upload(c, d_psic, psic)) || (st = upload(c, d_psic_w, psicw)) || (st = upload(c, d_Cc, Cc)) ||
        (st = upload(c, d_pieces, pieces)) || (st = upload(c, d_items, items))) {
        cleanup();
        return st;
    }

    // far pairs
    {
        size_t smem = (LMAX + 2 * (LMAX / 2 + 1)) * sizeof(double);
        cudaFuncSetAttribute(far_modes_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        far_modes_kernel<<<NG, 128, smem, c->stream>>>(NG, M, sd.ring.ptr, d_panel_of.ptr, d_near_start.ptr,
                                                        d_near_panel.ptr, c->k, c->eta, sd.A64.ptr);
        if (check_cuda(c, cudaGetLastError(), "far_modes_kernel")) { cleanup(); return HZB_ECUDA; }
    }
    // near panels
    {
        NearArgs a;
        a.NG = NG; a.M = M; a.P = P; a.ring = sd.ring.ptr; a.pieces = d_pieces.ptr;
        a.panel_piece = d_panel_piece.ptr; a.panel_ta = d_ta.ptr; a.panel_tb = d_tb.ptr; a.items = d_items.ptr;
        a.glt_x = d_glt_x.ptr; a.glt_w = d_glt_w.ptr; a.gls_x = d_gls_x.ptr; a.gls_w = d_gls_w.ptr;
        a.psic = d_psic.ptr; a.psic_w = d_psic_w.ptr; a.Cc = d_Cc.ptr; a.k = c->k; a.eta = c->eta;
        a.A = sd.A64.ptr;
        const int nth = 256;
        const int SPT = (M1 * P + nth - 1) / nth;
        int TB = 2;
        auto smem_of = [&](int tb) {
            return sizeof(TNode) * tb + sizeof(double) * ((size_t)((tb * P + 1) & ~1) + (size_t)tb * 2 * NPSI_S) +
                   sizeof(double2) * (size_t)tb * NPSI + sizeof(double) * (size_t)tb * M1 * NPSI_S +
                   sizeof(double2) * (size_t)tb * M1;
        };
        while (TB > 1 && smem_of(TB) > 200 * 1024) --TB;
        size_t smem = smem_of(TB);
        if (smem > 220 * 1024) { cleanup(); return fail(c, HZB_EINVAL, "n_modes too large for the setup kernel"); }
        cudaFuncSetAttribute(near_panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        near_panel_kernel<<<(unsigned)items.size(), nth, smem, c->stream>>>(a, TB, SPT);
        if (check_cuda(c, cudaGetLastError(), "near_panel_kernel")) { cleanup(); return HZB_ECUDA; }
    }
    // S_p = A~_p^{-1}
    if (check_cuda(c, cudaMemcpyAsync(sd.S64.ptr, sd.A64.ptr, nmat * sizeof(double2), cudaMemcpyDeviceToDevice,
                                      c->stream), "copy A")) { cleanup(); return HZB_ECUDA; }
    if (check_cuda(c, d_colk.ensure((size_t)M1 * NG), "alloc") || check_cuda(c, d_perm.ensure((size_t)M1 * NG), "alloc") ||
        check_cuda(c, d_sing.ensure(M1), "alloc")) { cleanup(); return HZB_ENOMEM; }
    cudaMemsetAsync(d_sing.ptr, 0, M1 * sizeof(int), c->stream);
    for (int kk = 0; kk < NG; ++kk) {
        gj_pivot_kernel<<<M1, 256, 0, c->stream>>>(NG, kk, sd.S64.ptr, d_colk.ptr, d_perm.ptr, d_sing.ptr);
        dim3 grid((unsigned)(((size_t)NG * NG + 255) / 256), M1);
        gj_elim_kernel<<<grid, 256, 0, c->stream>>>(NG, kk, sd.S64.ptr, d_colk.ptr);
    }
    gj_colswap_kernel<<<M1, 256, 0, c->stream>>>(NG, sd.S64.ptr, d_perm.ptr);
    to_fp32_kernel<<<(unsigned)((nmat + 255) / 256), 256, 0, c->stream>>>(nmat, sd.S64.ptr, sd.S32.ptr);
    sd.Sdd_ready = false;
    if (check_cuda(c, cudaGetLastError(), "gauss-jordan")) { cleanup(); return HZB_ECUDA; }
    std::vector<int> sing(M1, 0);
    if (check_cuda(c, cudaMemcpyAsync(sing.data(), d_sing.ptr, M1 * sizeof(int), cudaMemcpyDeviceToHost, c->stream),
                   "copy") ||
        check_cuda(c, cudaStreamSynchronize(c->stream), "setup")) { cleanup(); return HZB_ECUDA; }
    cleanup();
    for (int p = 0; p < M1; ++p)
        if (sing[p]) return fail(c, HZB_EINVAL, "a per-mode matrix is singular");
    return HZB_OK;
}

}  // namespace hzb
