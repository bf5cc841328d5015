// Accelerated scheme (Sec. 5, Eqs. (ip0)-(ip6)): per shape, an interpolative
// decomposition of the body's interactions with everything outside a proxy sphere gives
// one skeleton index set J (k nodes) and T (k x n, T(:, J) = I) with V_p^* = T and
// U_p = T^T, so that A_pq ~ U_p A_pq(J_p, J_q) V_q^*; GMRES then runs on
//     sig~ + S B~ sig~ = -v~,   S_p = T A_pp^{-1} T^T,   v~_p = T A_pp^{-1} v_p,
// and the density on all nodes follows from Eq. (ip1):  sig = D^{-1} (-v - U B~ sig~).
//
// Construction of the ID on the GPU, in the body frame of each shape:
//  1. Proxy matrix M: rows = points z of a sphere of radius rho (n_theta Gauss-Legendre
//     rings in cos(theta) times the body's N_F azimuths), columns = nodes; blocks
//     [K(z, y_j) w_j ; G(x_i, z) ; dG/dn_z(x_i, z)], each scaled to unit Frobenius norm
//     (outgoing fields, and the single- and double-layer sources that fix any incoming
//     field inside the sphere).  Body and proxy share the azimuthal grid and every entry
//     depends on the cosine of the azimuth difference only, so each block is
//     block-circulant: M = (1/N_F) F^* diag(M^_p) F with M^_p = M^_{-p};
//     proxy_modes_kernel forms M^_p for p = 0..M.
//  2. Column-pivoted QR of every M^_p, stopped once all trailing columns are below
//     0.3 eps |M|_col: R_p with |M^_p u| ~ |R_p P_p^T u|.  The matrix Z with
//     rows (p, s),  Z[(p,s), (i,l)] = R_p[s, i] e^{-2 pi i p l / N_F} / sqrt(N_F),  has
//     |Z x| ~ |M x| for all x (Parseval), so a column ID of Z is a column ID of M with
//     about as many rows as the rank instead of 3 n_theta N_F.
//  3. Column-pivoted QR of Z, stopped at |R_jj| <= eps |R_11|; T = [I, R11^{-1} R12] P^T
//     by a blocked triangular solve.
//  4. S_p = T (A_pp^{-1} T^T): the modal apply on the columns of T^T, then an FP64 GEMM.
// The reduced system runs as a context of its own over the skeleton nodes: the inter-body
// kernels unchanged (B~ = B(J, J) is the direct sum over skeleton nodes) and, as local
// operator, the dense S_p of each body (reduced_local).
#include <algorithm>
#include <cmath>
#include <numeric>
#include <type_traits>
#include <vector>

#include "hzb_internal.h"

namespace hzb {

static const double CP_PI = 3.14159265358979323846;

// ------------------------------------------------------------------ block reductions

__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// sum over the block (blockDim.x a multiple of 32, <= 1024), fixed order; every thread gets it
__device__ double block_sum(double v, double *sh)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    for (int q = 0; q < nw; ++q) t += sh[q];
    return t;
}

// ------------------------------------------------------------------ 1. proxy modal matrices

// One block per (proxy ring r, body ring i): samples f_b(m) at the azimuth
// 2 pi (m + t / Q) / N_F for the three blocks, t = r / nth_base the ring's offset class
// (Q = 1: the body's own azimuths; Q = 3: offsets 0, +1/3 and +2/3 of the azimuthal step,
// a set closed under reflection, so M^_{-p} and M^_p have the same Gram matrix and one
// pivoted QR per |p| still serves both), then M^_p(b nth + r, i) = sum_m f_b(m)
// e^{-2 pi i p m / N_F} (for Q = 1, f_b is even in m and the sum is the cosine sum).
// Mh: (M+1) matrices of 3 nth rows x N_G columns, column-major (nth = Q nth_base rings:
// class-major, cth repeated per class); fsq: per (i, r) the three sums of |f_b|^2.
__global__ void proxy_modes_kernel(int NG, int NF, int nth, int nth_base, int Q, const double *__restrict__ ring,
                                   const double *__restrict__ cth, double rho, double k, double eta,
                                   double2 *__restrict__ Mh, double *__restrict__ fsq)
{
    extern __shared__ double2 psm[];
    double2 *f = psm;                                 // 3 x NF samples
    double *cs = (double *)(psm + 3 * NF);            // cos(2 pi m / NF)
    double *sn = cs + NF;                             // sin(2 pi m / NF)
    __shared__ double red[32];
    const int r = blockIdx.x, i = blockIdx.y;
    const int M = (NF - 1) / 2, rows = 3 * nth;
    const double frac = (double)(r / nth_base) / Q;   // the ring's azimuth offset, in steps
    const double ri = ring[8 * i], zi = ring[8 * i + 1], nri = ring[8 * i + 2], nzi = ring[8 * i + 3];
    const double wi = ring[8 * i + 4] * ri * 2.0 * CP_PI / NF;
    const double ct = cth[r], st = sqrt(fmax(0.0, 1.0 - ct * ct));
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int m = threadIdx.x; m < NF; m += blockDim.x) {
        double sd, cd;
        sincospi(2.0 * m / NF, &sd, &cd);
        cs[m] = cd;
        sn[m] = sd;
        if (Q > 1) sincospi(2.0 * (m + frac) / NF, &sd, &cd);
        const double ux = st * cd, uy = st * sd, uz = ct;                    // n_z
        const double dx = rho * ux - ri, dy = rho * uy, dz = rho * uz - zi;  // z - y
        const double R = sqrt(dx * dx + dy * dy + dz * dz), iR = 1.0 / R;
        double sk, ck;
        sincos(k * R, &sk, &ck);
        const double gr = ck * iR * (0.25 / CP_PI), gi = sk * iR * (0.25 / CP_PI);   // G
        const double ar = -iR * iR, ai = k * iR;                                      // (ik - 1/R) / R
        const double dgr = gr * ar - gi * ai, dgi = gr * ai + gi * ar;                // G'(R) / R
        const double ndy = -(nri * dx + nzi * dz);                                    // n_y . (y - z)
        const double ndz = ux * dx + uy * dy + uz * dz;                               // n_z . (z - x)
        const double2 o = make_double2((dgr * ndy + eta * gi) * wi, (dgi * ndy - eta * gr) * wi);
        const double2 d2 = make_double2(dgr * ndz, dgi * ndz);
        f[m] = o;
        f[NF + m] = make_double2(gr, gi);
        f[2 * NF + m] = d2;
        s0 += o.x * o.x + o.y * o.y;
        s1 += gr * gr + gi * gi;
        s2 += d2.x * d2.x + d2.y * d2.y;
    }
    s0 = block_sum(s0, red);
    s1 = block_sum(s1, red);
    s2 = block_sum(s2, red);
    if (threadIdx.x == 0) {
        double *o = fsq + ((size_t)i * nth + r) * 3;
        o[0] = s0;
        o[1] = s1;
        o[2] = s2;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 3 * (M + 1); e += blockDim.x) {
        const int p = e / 3, b = e % 3;
        const double2 *fb = f + b * NF;
        double ax = 0.0, ay = 0.0;
        int idx = 0;
        for (int m = 0; m < NF; ++m) {
            const double cv = cs[idx];
            ax = fma(fb[m].x, cv, ax);
            ay = fma(fb[m].y, cv, ay);
            if (Q > 1) {                              // f (cos - i sin)
                const double sv = sn[idx];
                ax = fma(fb[m].y, sv, ax);
                ay = fma(-fb[m].x, sv, ay);
            }
            idx += p;
            if (idx >= NF) idx -= NF;
        }
        Mh[(size_t)p * rows * NG + (size_t)i * rows + b * nth + r] = make_double2(ax, ay);
    }
}

// scale[b] = 1 / |M_b|_F with |M_b|_F^2 = N_F sum_{i,r} fsq (one block)
__global__ void block_scale_kernel(int n_ir, int NF, const double *__restrict__ fsq, double *__restrict__ scale)
{
    __shared__ double red[32];
    for (int b = 0; b < 3; ++b) {
        double s = 0.0;
        for (int e = threadIdx.x; e < n_ir; e += blockDim.x) s += fsq[(size_t)e * 3 + b];
        s = block_sum(s, red);
        if (threadIdx.x == 0) scale[b] = s > 0.0 ? 1.0 / sqrt(s * NF) : 0.0;
        __syncthreads();
    }
}

__global__ void scale_rows_kernel(size_t total, int nth, const double *__restrict__ scale, double2 *__restrict__ Mh)
{
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    const int row = (int)(e % (size_t)(3 * nth));
    const double s = scale[row / nth];
    double2 v = Mh[e];
    v.x *= s;
    v.y *= s;
    Mh[e] = v;
}

// ------------------------------------------------------------------ column-pivoted QR

// nrm2[b][c] = |A_b(:, c)|^2, perm[b][c] = c.  Grid (n, batch), one block per column.
__global__ void cpqr_init_kernel(int m, int n, const double2 *__restrict__ A, size_t sA, double *__restrict__ nrm2,
                                 int *__restrict__ perm)
{
    __shared__ double red[32];
    const int c = blockIdx.x, b = blockIdx.y;
    const double2 *col = A + b * sA + (size_t)c * m;
    double s = 0.0;
    for (int r = threadIdx.x; r < m; r += blockDim.x) s += col[r].x * col[r].x + col[r].y * col[r].y;
    s = block_sum(s, red);
    if (threadIdx.x == 0) {
        nrm2[(size_t)b * n + c] = s;
        perm[(size_t)b * n + c] = c;
    }
}

// Per-mode stopping thresholds: |M|_col^2 = max_i (1/N_F) (n_0(i) + 2 sum_{p>=1} n_p(i)),
// thr2[p] = (0.3 eps |M|_col)^2 for every mode (one block): the rows dropped from each
// mode change |Z x| by about the largest trailing column norm, below the ID tolerance.
__global__ void mode_threshold_kernel(int NG, int modes, int NF, double eps, const double *__restrict__ nrm2,
                                      double *__restrict__ thr2, int *__restrict__ rank)
{
    __shared__ double red[32];
    double mx = 0.0;
    for (int i = threadIdx.x; i < NG; i += blockDim.x) {
        double s = nrm2[i];
        for (int p = 1; p < modes; ++p) s += 2.0 * nrm2[(size_t)p * NG + i];
        mx = fmax(mx, s / NF);
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t = fmax(t, red[q]);
        const double th = 0.3 * eps * sqrt(t);
        for (int p = 0; p < modes; ++p) {
            thr2[p] = th * th;
            rank[p] = -1;
        }
    }
}

// thr2[0] = (eps max_c |A(:, c)|)^2 for one matrix (one block)
__global__ void max_threshold_kernel(int n, double eps, const double *__restrict__ nrm2, double *__restrict__ thr2,
                                     int *__restrict__ rank)
{
    __shared__ double red[32];
    double mx = 0.0;
    for (int c = threadIdx.x; c < n; c += blockDim.x) mx = fmax(mx, nrm2[c]);
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t = fmax(t, red[q]);
        thr2[0] = eps * eps * t;
        rank[0] = -1;
    }
}

// Step j, one block (1024 threads) per matrix: pivot = the trailing column of largest
// norm (ties: lowest index); stop (rank = j) when it is <= the threshold; else swap it
// into position j and form the Householder reflector H = I - beta u u^H with
// H x = alpha e_1, alpha = -e^{i arg x_0} |x| (x = A(j:m, j)); A(j, j) = alpha, below 0.
__global__ void __launch_bounds__(1024) cpqr_pivot_kernel(int j, int m, int n, double2 *__restrict__ A, size_t sA,
                                                          double *__restrict__ nrm2, int *__restrict__ perm,
                                                          int *__restrict__ rank, const double *__restrict__ thr2,
                                                          double2 *__restrict__ u, double *__restrict__ beta)
{
    __shared__ double bv[32];
    __shared__ int bi[32];
    __shared__ double red[32];
    __shared__ int piv;
    __shared__ bool stop;
    const int b = blockIdx.x;
    if (rank[b] >= 0) return;
    double2 *Ab = A + b * sA;
    double *nb = nrm2 + (size_t)b * n;
    double best = -1.0;
    int bidx = n;
    for (int c = j + threadIdx.x; c < n; c += blockDim.x) {
        const double v = nb[c];
        if (v > best) { best = v; bidx = c; }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
        if (ov > best || (ov == best && oi < bidx)) { best = ov; bidx = oi; }
    }
    if ((threadIdx.x & 31) == 0) {
        bv[threadIdx.x >> 5] = best;
        bi[threadIdx.x >> 5] = bidx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = -1.0;
        int ix = n;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q)
            if (bv[q] > v || (bv[q] == v && bi[q] < ix)) { v = bv[q]; ix = bi[q]; }
        stop = (j >= m) || ix >= n || !(v > thr2[b]);
        piv = ix;
        if (stop) rank[b] = j;
    }
    __syncthreads();
    if (stop) return;
    const int pc = piv;
    if (pc != j) {
        double2 *cj = Ab + (size_t)j * m, *cp = Ab + (size_t)pc * m;
        for (int r = threadIdx.x; r < m; r += blockDim.x) {
            const double2 t = cj[r];
            cj[r] = cp[r];
            cp[r] = t;
        }
        if (threadIdx.x == 0) {
            const double t = nb[j];
            nb[j] = nb[pc];
            nb[pc] = t;
            int *pb = perm + (size_t)b * n;
            const int q = pb[j];
            pb[j] = pb[pc];
            pb[pc] = q;
        }
        __syncthreads();
    }
    double2 *x = Ab + (size_t)j * m;
    double s = 0.0;
    for (int r = j + threadIdx.x; r < m; r += blockDim.x) s += x[r].x * x[r].x + x[r].y * x[r].y;
    const double xn2 = block_sum(s, red);
    const double xn = sqrt(xn2);
    const double2 x0 = x[j];
    const double ax0 = hypot(x0.x, x0.y);
    const double phx = ax0 > 0.0 ? x0.x / ax0 : 1.0, phy = ax0 > 0.0 ? x0.y / ax0 : 0.0;
    const double alx = -phx * xn, aly = -phy * xn;
    const double uu = 2.0 * xn2 + 2.0 * ax0 * xn;
    double2 *ub = u + (size_t)b * m;
    __syncthreads();
    for (int r = j + threadIdx.x; r < m; r += blockDim.x) {
        if (r == j) {
            ub[r] = make_double2(x0.x - alx, x0.y - aly);
            x[r] = make_double2(alx, aly);
        } else {
            ub[r] = x[r];
            x[r] = make_double2(0.0, 0.0);
        }
    }
    if (threadIdx.x == 0) beta[b] = uu > 0.0 ? 2.0 / uu : 0.0;
}

// Step j: apply the reflector to every trailing column c > j and store the exact norm of
// its rows j+1..m-1 as the column's new trailing norm.  One warp per column, eight per
// block, no block-wide synchronisation: the column part j..m-1 is held in registers, W
// values per lane, when it fits; W = 0 makes two passes over memory (spreading longer
// columns over several warps with shared-memory sums measured slower).
// Grid (ceil((n-j-1)/8), batch).
template <int W>
__global__ void __launch_bounds__(256) cpqr_update_kernel(int j, int m, int n, double2 *__restrict__ A, size_t sA,
                                                          double *__restrict__ nrm2, const int *__restrict__ rank,
                                                          const double2 *__restrict__ u,
                                                          const double *__restrict__ beta)
{
    const int b = blockIdx.y;
    if (rank[b] >= 0) return;
    const int lane = threadIdx.x & 31;
    const int c = j + 1 + blockIdx.x * 8 + (threadIdx.x >> 5);
    if (c >= n) return;
    double2 *col = A + b * sA + (size_t)c * m;
    const double2 *ub = u + (size_t)b * m;
    const double bt = beta[b];
    double sr = 0.0, si = 0.0, nn = 0.0;
    if (W > 0) {
        double2 v[W > 0 ? W : 1];
#pragma unroll
        for (int q = 0; q < (W > 0 ? W : 1); ++q) {
            const int r = j + lane + 32 * q;
            if (r < m) {
                v[q] = col[r];
                const double2 w = ub[r];
                sr += w.x * v[q].x + w.y * v[q].y;      // conj(u) a
                si += w.x * v[q].y - w.y * v[q].x;
            }
        }
        sr = warp_sum(sr);
        si = warp_sum(si);
        const double fr = bt * sr, fi = bt * si;
#pragma unroll
        for (int q = 0; q < (W > 0 ? W : 1); ++q) {
            const int r = j + lane + 32 * q;
            if (r < m) {
                const double2 w = ub[r];
                double2 a = v[q];
                a.x -= fr * w.x - fi * w.y;
                a.y -= fr * w.y + fi * w.x;
                col[r] = a;
                if (r > j) nn += a.x * a.x + a.y * a.y;
            }
        }
    } else {
        for (int r = j + lane; r < m; r += 32) {
            const double2 a = col[r], w = ub[r];
            sr += w.x * a.x + w.y * a.y;
            si += w.x * a.y - w.y * a.x;
        }
        sr = warp_sum(sr);
        si = warp_sum(si);
        const double fr = bt * sr, fi = bt * si;
        for (int r = j + lane; r < m; r += 32) {
            const double2 w = ub[r];
            double2 a = col[r];
            a.x -= fr * w.x - fi * w.y;
            a.y -= fr * w.y + fi * w.x;
            col[r] = a;
            if (r > j) nn += a.x * a.x + a.y * a.y;
        }
    }
    nn = warp_sum(nn);
    if (lane == 0) nrm2[(size_t)b * n + c] = nn;
}

// Column-pivoted QR of `batch` m x n column-major matrices (stride sA), in place, each
// stopped at its threshold (thr2, rank[] = -1 on entry).  On return rank[b] holds k_b,
// perm[b][0..n) the column order, and the matrix R (upper part) in pivoted order.
static hzb_status cpqr_run(hzb_ctx *c, int m, int n, int batch, double2 *A, size_t sA, double *nrm2, int *perm,
                           int *rank, const double *thr2, double2 *u, double *beta, std::vector<int> &ranks)
{
    const int steps = std::min(m, n);
    auto update = [&](int j, int batch_) {
        const int len = m - j, nc = n - j - 1;
        const dim3 g8((unsigned)((nc + 7) / 8), batch_);
        if (len <= 4 * 32)
            cpqr_update_kernel<4><<<g8, 256, 0, c->stream>>>(j, m, n, A, sA, nrm2, rank, u, beta);
        else if (len <= 16 * 32)
            cpqr_update_kernel<16><<<g8, 256, 0, c->stream>>>(j, m, n, A, sA, nrm2, rank, u, beta);
        else if (len <= 32 * 32)
            cpqr_update_kernel<32><<<g8, 256, 0, c->stream>>>(j, m, n, A, sA, nrm2, rank, u, beta);
        else
            cpqr_update_kernel<0><<<g8, 256, 0, c->stream>>>(j, m, n, A, sA, nrm2, rank, u, beta);
    };
    ranks.assign(batch, -1);
    for (int j = 0; j < steps; ++j) {
        cpqr_pivot_kernel<<<batch, 1024, 0, c->stream>>>(j, m, n, A, sA, nrm2, perm, rank, thr2, u, beta);
        if (n - j - 1 > 0) update(j, batch);
        c->launches += 2;
        if ((j & 31) == 31 || j == steps - 1) {
            if (check_cuda(c, cudaGetLastError(), "cpqr")) return HZB_ECUDA;
            if (check_cuda(c, cudaMemcpyAsync(ranks.data(), rank, batch * sizeof(int), cudaMemcpyDeviceToHost,
                                              c->stream), "cpqr rank") ||
                check_cuda(c, cudaStreamSynchronize(c->stream), "cpqr"))
                return HZB_ECUDA;
            if (std::all_of(ranks.begin(), ranks.end(), [](int r) { return r >= 0; })) break;
        }
    }
    for (int &r : ranks)
        if (r < 0) r = steps;
    return HZB_OK;
}

// ------------------------------------------------------------------ 2. the matrix Z

__global__ void inverse_perm_kernel(int n, int batch, const int *__restrict__ perm, int *__restrict__ pos)
{
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)n * batch) return;
    const size_t b = e / n;
    pos[b * n + perm[e]] = (int)(e % n);
}

// Z[(row), (i, l)] = R_p[s, pos_p(i)] e^{-+2 pi i p l / N_F} / sqrt(N_F) for the row's
// (p, sign, s) = rdesc[row] (sign 0: +p, 1: -p), column-major with leading dimension lz.
__global__ void assemble_z_kernel(int lz, int NG, int NF, int mrows, const int4 *__restrict__ rdesc,
                                  const double2 *__restrict__ Mh, const int *__restrict__ pos,
                                  double2 *__restrict__ Z)
{
    const size_t total = (size_t)lz * NG * NF;
    const double sc = 1.0 / sqrt((double)NF);
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int row = (int)(e % lz);
        const size_t col = e / lz;
        const int i = (int)(col / NF), l = (int)(col % NF);
        const int4 d = rdesc[row];
        const int p = d.x, s = d.z;
        const int q = pos[(size_t)p * NG + i];
        const double2 rv = Mh[(size_t)p * mrows * NG + (size_t)q * mrows + s];
        double sn, cn;
        const int pl = (int)(((long long)p * l) % NF);
        sincospi((d.y ? 2.0 : -2.0) * pl / NF, &sn, &cn);
        Z[e] = make_double2(sc * (rv.x * cn - rv.y * sn), sc * (rv.x * sn + rv.y * cn));
    }
}

// ------------------------------------------------------------------ dense FP64 kernels

// C = alpha A B + beta C for complex FP64 matrices given by element strides:
// A(i, p) = A[i ars + p acs], B(p, j) = B[p brs + j bcs], C(i, j) = C[i crs + j ccs].
// 64 x 64 tiles, 16-deep slices, 256 threads with 4 x 4 outputs each.
__global__ void __launch_bounds__(256) zgemm_kernel(int m, int n, int kk, const double2 *__restrict__ A, long long ars,
                                                    long long acs, const double2 *__restrict__ B, long long brs,
                                                    long long bcs, double2 *__restrict__ C, long long crs,
                                                    long long ccs, double alpha, double beta)
{
    __shared__ double2 As[16][65];
    __shared__ double2 Bs[16][65];
    const bool cm = crs == 1;
    const int ti = cm ? (threadIdx.x & 15) : (threadIdx.x >> 4);
    const int tj = cm ? (threadIdx.x >> 4) : (threadIdx.x & 15);
    const int i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
    double ar[4][4], ai[4][4];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int r = 0; r < 4; ++r) ar[q][r] = ai[q][r] = 0.0;
    for (int p0 = 0; p0 < kk; p0 += 16) {
        for (int e = threadIdx.x; e < 1024; e += 256) {
            int ii, pp;
            if (acs == 1) { pp = e & 15; ii = e >> 4; } else { ii = e & 63; pp = e >> 6; }
            const int gi = i0 + ii, gp = p0 + pp;
            As[pp][ii] = (gi < m && gp < kk) ? A[gi * ars + gp * acs] : make_double2(0.0, 0.0);
            int jj, pq;
            if (bcs == 1) { jj = e & 63; pq = e >> 6; } else { pq = e & 15; jj = e >> 4; }
            const int gj = j0 + jj, gq = p0 + pq;
            Bs[pq][jj] = (gj < n && gq < kk) ? B[gq * brs + gj * bcs] : make_double2(0.0, 0.0);
        }
        __syncthreads();
#pragma unroll 4
        for (int pp = 0; pp < 16; ++pp) {
            double2 a[4], bb[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                a[q] = As[pp][ti + 16 * q];
                bb[q] = Bs[pp][tj + 16 * q];
            }
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    ar[q][r] = fma(a[q].x, bb[r].x, fma(-a[q].y, bb[r].y, ar[q][r]));
                    ai[q][r] = fma(a[q].x, bb[r].y, fma(a[q].y, bb[r].x, ai[q][r]));
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int gi = i0 + ti + 16 * q, gj = j0 + tj + 16 * r;
            if (gi < m && gj < n) {
                double2 *cp = C + gi * crs + gj * ccs;
                double2 v = make_double2(alpha * ar[q][r], alpha * ai[q][r]);
                if (beta != 0.0) {
                    const double2 o = *cp;
                    v.x += beta * o.x;
                    v.y += beta * o.y;
                }
                *cp = v;
            }
        }
}

static void zgemm(hzb_ctx *c, int m, int n, int kk, const double2 *A, long long ars, long long acs, const double2 *B,
                  long long brs, long long bcs, double2 *C, long long crs, long long ccs, double alpha, double beta)
{
    if (m <= 0 || n <= 0) return;
    zgemm_kernel<<<dim3((n + 63) / 64, (m + 63) / 64), 256, 0, c->stream>>>(m, n, kk, A, ars, acs, B, brs, bcs, C, crs,
                                                                          ccs, alpha, beta);
    c->launches++;
}

static const int TRSM_NB = 32;

// X(r0:r1, c) = R(r0:r1, r0:r1)^{-1} X(r0:r1, c) for the columns c in [c0, n) of the
// column-major matrix A (ld m): R upper triangular.  One thread per column.
__global__ void __launch_bounds__(128) trsm_diag_kernel(int r0, int r1, int c0, int n, int m,
                                                        double2 *__restrict__ A)
{
    __shared__ double2 Rb[TRSM_NB][TRSM_NB + 1];
    __shared__ double2 Rinv[TRSM_NB];
    const int nb = r1 - r0;
    for (int e = threadIdx.x; e < TRSM_NB * TRSM_NB; e += blockDim.x) {
        const int a = e % TRSM_NB, bq = e / TRSM_NB;      // row a, column bq of the block
        Rb[a][bq] = (a < nb && bq < nb) ? A[(size_t)(r0 + bq) * m + r0 + a] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    if (threadIdx.x < nb) {
        const double2 d = Rb[threadIdx.x][threadIdx.x];
        const double den = d.x * d.x + d.y * d.y;
        Rinv[threadIdx.x] = make_double2(d.x / den, -d.y / den);
    }
    __syncthreads();
    const int col = c0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= n) return;
    double2 *x = A + (size_t)col * m + r0;
    double2 v[TRSM_NB];
#pragma unroll
    for (int a = 0; a < TRSM_NB; ++a) v[a] = a < nb ? x[a] : make_double2(0.0, 0.0);
#pragma unroll
    for (int a = TRSM_NB - 1; a >= 0; --a) {
        if (a < nb) {
            double sx = v[a].x, sy = v[a].y;
#pragma unroll
            for (int q = a + 1; q < TRSM_NB; ++q) {
                const double2 rr = Rb[a][q];
                sx -= rr.x * v[q].x - rr.y * v[q].y;
                sy -= rr.x * v[q].y + rr.y * v[q].x;
            }
            const double2 ri = Rinv[a];
            v[a] = make_double2(sx * ri.x - sy * ri.y, sx * ri.y + sy * ri.x);
        }
    }
#pragma unroll
    for (int a = 0; a < TRSM_NB; ++a)
        if (a < nb) x[a] = v[a];
}

// X(0:k, k:n) = R11^{-1} R12 in place (A column-major, ld m), blocked from the bottom:
// solve the diagonal block, then subtract its contribution from the rows above.
static hzb_status trsm_upper(hzb_ctx *c, int m, int n, int k, double2 *A)
{
    if (k <= 0 || k >= n) return HZB_OK;
    const int ncol = n - k;
    for (int r0 = ((k - 1) / TRSM_NB) * TRSM_NB; r0 >= 0; r0 -= TRSM_NB) {
        const int r1 = std::min(k, r0 + TRSM_NB);
        trsm_diag_kernel<<<(ncol + 127) / 128, 128, 0, c->stream>>>(r0, r1, k, n, m, A);
        c->launches++;
        if (r0 > 0)
            zgemm(c, r0, ncol, r1 - r0, A + (size_t)r0 * m, 1, m, A + (size_t)k * m + r0, 1, m, A + (size_t)k * m, 1, m,
                  -1.0, 1.0);
    }
    return check_cuda(c, cudaGetLastError(), "trsm");
}

// T[s, i] (k x n row-major, rows in the order of the sorted skeleton) from the pivoted
// factorisation: q = qrow[s] is the pivot position of row s, j = pos[i] that of column i;
// T = delta_{jq} for j < k, else X(q, j) = A[j m + q].
__global__ void build_t_kernel(int k, int n, int m, const int *__restrict__ qrow, const int *__restrict__ pos,
                               const double2 *__restrict__ A, double2 *__restrict__ T)
{
    const size_t total = (size_t)k * n;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int s = (int)(e / n), i = (int)(e % n);
        const int q = qrow[s], j = pos[i];
        double2 v;
        if (j < k) v = make_double2(j == q ? 1.0 : 0.0, 0.0);
        else v = A[(size_t)j * m + q];
        T[e] = v;
    }
}

// ------------------------------------------------------------------ S_p = T A^{-1} T^T

// X[i R + r] = T[(s0 + r) n + i], r < R
__global__ void t_columns_kernel(int n, int R, int s0, const double2 *__restrict__ T, double2 *__restrict__ X)
{
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)n * R) return;
    const int i = (int)(e / R), r = (int)(e % R);
    X[e] = T[(size_t)(s0 + r) * n + i];
}

// W[i k + s0 + r] = Y[i R + r]
__global__ void w_columns_kernel(int n, int R, int k, int s0, const double2 *__restrict__ Y, double2 *__restrict__ W)
{
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)n * R) return;
    const int i = (int)(e / R), r = (int)(e % R);
    W[(size_t)i * k + s0 + r] = Y[e];
}

__global__ void to_f32_kernel(size_t n, const double2 *__restrict__ a, float2 *__restrict__ b)
{
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) b[e] = make_float2((float)a[e].x, (float)a[e].y);
}

static unsigned grid_for(size_t n, int th = 256)
{
    return (unsigned)std::min<size_t>((n + th - 1) / th, (size_t)152 * 64);
}

// S_p = T (A_pp^{-1} T^T) for a shape whose T64 is set; also its FP32 copy.
static hzb_status reduced_blocks(hzb_ctx *c, ShapeDev &sd)
{
    const int k = sd.skel_k, n = sd.geom.NG * sd.geom.NF, NF = sd.geom.NF;
    DevBuf<double2> W, X, Y;
    const int rmax = std::max(1, std::min(64, (int)(200 * 1024 / (16 * NF)) - 1));
    auto done = [&](hzb_status s) {
        W.release();
        X.release();
        Y.release();
        return s;
    };
    if (check_cuda(c, W.ensure((size_t)n * k), "alloc W") || check_cuda(c, X.ensure((size_t)n * rmax), "alloc") ||
        check_cuda(c, Y.ensure((size_t)n * rmax), "alloc") || check_cuda(c, sd.St64.ensure((size_t)k * k), "alloc S") ||
        check_cuda(c, sd.St32.ensure((size_t)k * k), "alloc S"))
        return done(HZB_ENOMEM);
    hzb_status st;
    for (int s0 = 0; s0 < k; s0 += rmax) {
        const int R = std::min(rmax, k - s0);
        const size_t ne = (size_t)n * R;
        t_columns_kernel<<<(unsigned)((ne + 255) / 256), 256, 0, c->stream>>>(n, R, s0, sd.T64.ptr, X.ptr);
        if ((st = shape_inverse64(c, sd, R, X.ptr, Y.ptr))) return done(st);
        w_columns_kernel<<<(unsigned)((ne + 255) / 256), 256, 0, c->stream>>>(n, R, k, s0, Y.ptr, W.ptr);
        c->launches += 2;
    }
    zgemm(c, k, k, n, sd.T64.ptr, n, 1, W.ptr, k, 1, sd.St64.ptr, k, 1, 1.0, 0.0);
    to_f32_kernel<<<(unsigned)(((size_t)k * k + 255) / 256), 256, 0, c->stream>>>((size_t)k * k, sd.St64.ptr,
                                                                                  sd.St32.ptr);
    c->launches++;
    if (check_cuda(c, cudaGetLastError(), "reduced blocks") || check_cuda(c, cudaStreamSynchronize(c->stream), "S"))
        return done(HZB_ECUDA);
    return done(HZB_OK);
}

// ------------------------------------------------------------------ the ID of one shape

// Column ID of the column-major rows x cols matrix Z (device, overwritten) at tolerance
// eps: J in pivot order, T (k x cols, row-major, rows in J order) on the device.
static hzb_status column_id(hzb_ctx *c, int rows, int cols, double2 *Z, double eps, std::vector<int> &J,
                            DevBuf<double2> &T)
{
    DevBuf<double> nrm2, thr2, beta;
    DevBuf<int> perm, rank, pos, qrow;
    DevBuf<double2> u;
    auto done = [&](hzb_status s) {
        nrm2.release(); thr2.release(); beta.release(); perm.release(); rank.release(); pos.release();
        qrow.release(); u.release();
        return s;
    };
    if (check_cuda(c, nrm2.ensure(cols), "alloc") || check_cuda(c, thr2.ensure(1), "alloc") ||
        check_cuda(c, beta.ensure(1), "alloc") || check_cuda(c, perm.ensure(cols), "alloc") ||
        check_cuda(c, rank.ensure(1), "alloc") || check_cuda(c, pos.ensure(cols), "alloc") ||
        check_cuda(c, u.ensure(rows), "alloc"))
        return done(HZB_ENOMEM);
    cpqr_init_kernel<<<dim3(cols, 1), 128, 0, c->stream>>>(rows, cols, Z, 0, nrm2.ptr, perm.ptr);
    max_threshold_kernel<<<1, 1024, 0, c->stream>>>(cols, eps, nrm2.ptr, thr2.ptr, rank.ptr);
    c->launches += 2;
    std::vector<int> ranks;
    hzb_status st = cpqr_run(c, rows, cols, 1, Z, 0, nrm2.ptr, perm.ptr, rank.ptr, thr2.ptr, u.ptr, beta.ptr, ranks);
    if (st) return done(st);
    const int k = ranks[0];
    if (k <= 0) return done(fail(c, HZB_EINVAL, "interpolative decomposition of a zero matrix"));
    if ((st = trsm_upper(c, rows, cols, k, Z))) return done(st);
    std::vector<int> hperm(cols);
    if (check_cuda(c, cudaMemcpyAsync(hperm.data(), perm.ptr, cols * sizeof(int), cudaMemcpyDeviceToHost, c->stream),
                   "perm") ||
        check_cuda(c, cudaStreamSynchronize(c->stream), "perm"))
        return done(HZB_ECUDA);
    J.assign(hperm.begin(), hperm.begin() + k);
    std::vector<int> hq(k);
    std::iota(hq.begin(), hq.end(), 0);
    if (check_cuda(c, qrow.ensure(k), "alloc") || check_cuda(c, T.ensure((size_t)k * cols), "alloc T"))
        return done(HZB_ENOMEM);
    if (check_cuda(c, cudaMemcpyAsync(qrow.ptr, hq.data(), k * sizeof(int), cudaMemcpyHostToDevice, c->stream), "q"))
        return done(HZB_ECUDA);
    inverse_perm_kernel<<<(cols + 255) / 256, 256, 0, c->stream>>>(cols, 1, perm.ptr, pos.ptr);
    build_t_kernel<<<grid_for((size_t)k * cols), 256, 0, c->stream>>>(k, cols, rows, qrow.ptr, pos.ptr, Z, T.ptr);
    c->launches += 2;
    if (check_cuda(c, cudaGetLastError(), "build T") || check_cuda(c, cudaStreamSynchronize(c->stream), "T"))
        return done(HZB_ECUDA);
    return done(HZB_OK);
}

// Rows of T (k x n, row-major) reordered so that J is ascending.
__global__ void permute_rows_kernel(int k, int n, const int *__restrict__ src_row, const double2 *__restrict__ Tin,
                                    double2 *__restrict__ Tout)
{
    const size_t total = (size_t)k * n;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int s = (int)(e / n), i = (int)(e % n);
        Tout[e] = Tin[(size_t)src_row[s] * n + i];
    }
}

// Ut = T^T (n x k row-major) from T (k x n row-major)
__global__ void transpose_kernel(int k, int n, const double2 *__restrict__ T, double2 *__restrict__ Ut)
{
    __shared__ double2 tile[32][33];
    const int s0 = blockIdx.y * 32, i0 = blockIdx.x * 32;
    for (int q = threadIdx.y; q < 32; q += blockDim.y) {
        const int s = s0 + q, i = i0 + threadIdx.x;
        if (s < k && i < n) tile[q][threadIdx.x] = T[(size_t)s * n + i];
    }
    __syncthreads();
    for (int q = threadIdx.y; q < 32; q += blockDim.y) {
        const int i = i0 + q, s = s0 + threadIdx.x;
        if (s < k && i < n) Ut[(size_t)i * k + s] = tile[threadIdx.x][q];
    }
}

__global__ void split_df_kernel(size_t n, const double2 *__restrict__ a, float4 *__restrict__ out);

// Install J (any order, distinct) and T (device, k x n rows in J's order) as the shape's
// skeleton with J ascending, and form its reduced blocks.
hzb_status install_skeleton(hzb_ctx *c, ShapeDev &sd, const std::vector<int> &J, DevBuf<double2> &T,
                            const double2 *S_host)
{
    const int k = (int)J.size(), n = sd.geom.NG * sd.geom.NF;
    std::vector<int> order(k);
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](int a, int b) { return J[a] < J[b]; });
    DevBuf<int> src;
    if (check_cuda(c, src.ensure(k), "alloc") || check_cuda(c, sd.T64.ensure((size_t)k * n), "alloc T")) {
        src.release();
        return HZB_ENOMEM;
    }
    if (check_cuda(c, cudaMemcpyAsync(src.ptr, order.data(), k * sizeof(int), cudaMemcpyHostToDevice, c->stream), "J")) {
        src.release();
        return HZB_ECUDA;
    }
    permute_rows_kernel<<<grid_for((size_t)k * n), 256, 0, c->stream>>>(k, n, src.ptr, T.ptr, sd.T64.ptr);
    c->launches++;
    if (check_cuda(c, sd.U64.ensure((size_t)k * n), "alloc U")) {
        src.release();
        return HZB_ENOMEM;
    }
    transpose_kernel<<<dim3((n + 31) / 32, (k + 31) / 32), dim3(32, 8), 0, c->stream>>>(k, n, sd.T64.ptr, sd.U64.ptr);
    c->launches++;
    if (check_cuda(c, sd.Tdf.ensure((size_t)k * n), "alloc T") || check_cuda(c, sd.Udf.ensure((size_t)k * n), "alloc U")) {
        src.release();
        return HZB_ENOMEM;
    }
    split_df_kernel<<<(unsigned)(((size_t)k * n + 255) / 256), 256, 0, c->stream>>>((size_t)k * n, sd.T64.ptr, sd.Tdf.ptr);
    split_df_kernel<<<(unsigned)(((size_t)k * n + 255) / 256), 256, 0, c->stream>>>((size_t)k * n, sd.U64.ptr, sd.Udf.ptr);
    c->launches += 2;
    hzb_status st = check_cuda(c, cudaStreamSynchronize(c->stream), "skeleton");
    src.release();
    if (st) return st;
    sd.skel_J.resize(k);
    for (int s = 0; s < k; ++s) sd.skel_J[s] = J[order[s]];
    sd.skel_k = k;
    if (!S_host) return reduced_blocks(c, sd);
    const size_t kk = (size_t)k * k;
    if (check_cuda(c, sd.St64.ensure(kk), "alloc S") || check_cuda(c, sd.St32.ensure(kk), "alloc S"))
        return HZB_ENOMEM;
    if (check_cuda(c, cudaMemcpyAsync(sd.St64.ptr, S_host, kk * sizeof(double2), cudaMemcpyHostToDevice, c->stream),
                   "upload S"))
        return HZB_ECUDA;
    to_f32_kernel<<<(unsigned)((kk + 255) / 256), 256, 0, c->stream>>>(kk, sd.St64.ptr, sd.St32.ptr);
    c->launches++;
    return check_cuda(c, cudaStreamSynchronize(c->stream), "reduced blocks");
}

// Smallest distance from a body of the shape to another body's bounding sphere, and the
// shape's bounding radius (largest node distance from the body centre).
static void proxy_geometry(const hzb_ctx *c, int shape, double &rb, double &gap)
{
    const ShapeDev &sd = *c->shapes[shape];
    rb = 0.0;
    for (int i = 0; i < sd.geom.NG; ++i) rb = std::max(rb, std::hypot(sd.geom.r[i], sd.geom.z[i]));
    gap = INFINITY;
    for (size_t p = 0; p < c->bodies.size(); ++p) {
        if (c->bodies[p].shape != shape) continue;
        for (size_t q = 0; q < c->bodies.size(); ++q) {
            if (q == p) continue;
            const ShapeDev &sq = *c->shapes[c->bodies[q].shape];
            double rq = 0.0;
            for (int i = 0; i < sq.geom.NG; ++i) rq = std::max(rq, std::hypot(sq.geom.r[i], sq.geom.z[i]));
            const double *a = c->bodies[p].c, *b = c->bodies[q].c;
            const double d = std::sqrt((a[0] - b[0]) * (a[0] - b[0]) + (a[1] - b[1]) * (a[1] - b[1]) +
                                       (a[2] - b[2]) * (a[2] - b[2]));
            gap = std::min(gap, d - rq);
        }
    }
}

bool proxy_fits(const hzb_ctx *c, int shape, double rho)
{
    double rb, gap;
    proxy_geometry(c, shape, rb, gap);
    return rho > rb && rho < gap;
}

static hzb_status compress_shape(hzb_ctx *c, int shape, double eps, int n_theta, double rho)
{
    ShapeDev &sd = *c->shapes[shape];
    const int NG = sd.geom.NG, NF = sd.geom.NF, M = sd.geom.M, n = NG * NF, modes = M + 1;
    // proxy azimuths: the body's own N_F, or (open shells, whose cavity sits inside the proxy
    // sphere with the body) 3 N_F in three offset classes, which removes the ~1e-6 error
    // floor of the off-diagonal blocks of Eq. (ip0) at small N_F
    const int Q = sd.geom.spec.kind == HZB_OPEN_SHELL ? 3 : 1;
    const int nth = Q * n_theta, mrows = 3 * nth;
    std::vector<double> cthv, wts;
    gauss_legendre(n_theta, cthv, wts);
    for (int t = 1; t < Q; ++t)
        for (int r = 0; r < n_theta; ++r) cthv.push_back(cthv[r]);
    DevBuf<double> cth, fsq, scale, nrm2, thr2, beta;
    DevBuf<double2> Mh, u, Z;
    DevBuf<int> perm, rank, pos;
    DevBuf<int4> rdesc;
    auto done = [&](hzb_status s) {
        cth.release(); fsq.release(); scale.release(); nrm2.release(); thr2.release(); beta.release();
        Mh.release(); u.release(); Z.release(); perm.release(); rank.release(); pos.release(); rdesc.release();
        return s;
    };
    const size_t mhn = (size_t)modes * mrows * NG;
    if (check_cuda(c, cth.ensure(nth), "alloc") || check_cuda(c, fsq.ensure((size_t)NG * nth * 3), "alloc") ||
        check_cuda(c, scale.ensure(3), "alloc") || check_cuda(c, Mh.ensure(mhn), "alloc proxy modes") ||
        check_cuda(c, nrm2.ensure((size_t)modes * NG), "alloc") || check_cuda(c, thr2.ensure(modes), "alloc") ||
        check_cuda(c, beta.ensure(modes), "alloc") || check_cuda(c, perm.ensure((size_t)modes * NG), "alloc") ||
        check_cuda(c, rank.ensure(modes), "alloc") || check_cuda(c, pos.ensure((size_t)modes * NG), "alloc") ||
        check_cuda(c, u.ensure((size_t)modes * mrows), "alloc"))
        return done(HZB_ENOMEM);
    if (check_cuda(c, cudaMemcpyAsync(cth.ptr, cthv.data(), nth * sizeof(double), cudaMemcpyHostToDevice, c->stream),
                   "proxy"))
        return done(HZB_ECUDA);
    const size_t smem = (size_t)NF * (3 * sizeof(double2) + 2 * sizeof(double));
    if (smem > 200 * 1024) return done(fail(c, HZB_EINVAL, "n_modes too large for the proxy modes"));
    cudaFuncSetAttribute(proxy_modes_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    proxy_modes_kernel<<<dim3(nth, NG), 128, smem, c->stream>>>(NG, NF, nth, n_theta, Q, sd.ring.ptr, cth.ptr, rho,
                                                                c->k, c->eta, Mh.ptr, fsq.ptr);
    block_scale_kernel<<<1, 1024, 0, c->stream>>>(NG * nth, NF, fsq.ptr, scale.ptr);
    scale_rows_kernel<<<(unsigned)((mhn + 255) / 256), 256, 0, c->stream>>>(mhn, nth, scale.ptr, Mh.ptr);
    // row compression: column-pivoted QR of every mode
    cpqr_init_kernel<<<dim3(NG, modes), 128, 0, c->stream>>>(mrows, NG, Mh.ptr, (size_t)mrows * NG, nrm2.ptr, perm.ptr);
    mode_threshold_kernel<<<1, 1024, 0, c->stream>>>(NG, modes, NF, eps, nrm2.ptr, thr2.ptr, rank.ptr);
    c->launches += 5;
    if (check_cuda(c, cudaGetLastError(), "proxy modes")) return done(HZB_ECUDA);
    std::vector<int> rk;
    hzb_status st = cpqr_run(c, mrows, NG, modes, Mh.ptr, (size_t)mrows * NG, nrm2.ptr, perm.ptr, rank.ptr, thr2.ptr,
                             u.ptr, beta.ptr, rk);
    if (st) return done(st);
    inverse_perm_kernel<<<(unsigned)(((size_t)modes * NG + 255) / 256), 256, 0, c->stream>>>(NG, modes, perm.ptr,
                                                                                             pos.ptr);
    c->launches++;
    // rows of Z: mode 0, then +p and -p for p = 1..M
    std::vector<int4> rd;
    for (int p = 0; p <= M; ++p)
        for (int sg = 0; sg < (p ? 2 : 1); ++sg)
            for (int s = 0; s < rk[p]; ++s) rd.push_back(make_int4(p, sg, s, 0));
    const int lz = (int)rd.size();
    if (lz == 0) return done(fail(c, HZB_EINVAL, "proxy matrix is zero"));
    if (check_cuda(c, rdesc.ensure(lz), "alloc") || check_cuda(c, Z.ensure((size_t)lz * n), "alloc Z"))
        return done(HZB_ENOMEM);
    if (check_cuda(c, cudaMemcpyAsync(rdesc.ptr, rd.data(), lz * sizeof(int4), cudaMemcpyHostToDevice, c->stream), "rd"))
        return done(HZB_ECUDA);
    assemble_z_kernel<<<grid_for((size_t)lz * n), 256, 0, c->stream>>>(lz, NG, NF, mrows, rdesc.ptr, Mh.ptr, pos.ptr,
                                                                        Z.ptr);
    c->launches++;
    if (check_cuda(c, cudaGetLastError(), "assemble Z") || check_cuda(c, cudaStreamSynchronize(c->stream), "Z"))
        return done(HZB_ECUDA);
    Mh.release();
    std::vector<int> J;
    DevBuf<double2> T;
    if ((st = column_id(c, lz, n, Z.ptr, eps, J, T))) {
        T.release();
        return done(st);
    }
    Z.release();
    st = install_skeleton(c, sd, J, T);
    T.release();
    if (!st) {
        sd.skel_rho = rho;
        sd.skel_eps = eps;
    }
    return done(st);
}

// ------------------------------------------------------------------ the reduced system

__global__ void gather_nodes_kernel(long long nr, const long long *__restrict__ gidx, const double4 *__restrict__ p64,
                                    const double4 *__restrict__ n64, const float4 *__restrict__ p32,
                                    const float4 *__restrict__ n32, const int *__restrict__ body,
                                    double4 *__restrict__ q64, double4 *__restrict__ m64, float4 *__restrict__ q32,
                                    float4 *__restrict__ m32, int *__restrict__ qbody)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nr) return;
    const long long g = gidx[e];
    q64[e] = p64[g];
    m64[e] = n64[g];
    q32[e] = p32[g];
    m32[e] = n32[g];
    qbody[e] = body[g];
}

static void free_ctx_buffers(hzb_ctx *r)
{
    r->pos64.release(); r->nrm64.release(); r->pos32.release(); r->nrm32.release(); r->body_of.release();
    r->tblocks.release(); r->w_a.release(); r->w_b.release(); r->w_c.release(); r->w_d.release();
    r->f_a.release(); r->f_b.release(); r->s_b.release(); r->s_r.release(); r->s_d.release(); r->io_in.release();
    r->io_out.release(); r->tiny.release(); r->sol.release(); r->red.release(); r->krylov.release();
    r->small.release(); r->sctab.release(); r->nb_part64.release(); r->nb_part32.release(); r->sig32.release();
    r->blockpairs.release(); r->kerr.release(); r->dfa.release(); r->dfb.release(); r->dfc.release();
    r->dftab.release(); r->rb.release(); r->rx.release(); r->zero_off.release(); r->yhat64.release();
    r->that64.release(); r->yhat32.release(); r->that32.release(); r->Ximg.release(); r->io_small.release();
    if (r->host_pinned) cudaFreeHost(r->host_pinned);
    r->host_pinned = nullptr;
    release_graphs(r);
    for (cudaEvent_t e : r->evpool) cudaEventDestroy(e);
    r->evpool.clear();
}

void release_compression(hzb_ctx *c)
{
    if (c->rctx) {
        hzb_ctx *r = c->rctx;
        free_ctx_buffers(r);
        if (r->ev0) cudaEventDestroy(r->ev0);
        if (r->ev1) cudaEventDestroy(r->ev1);
        delete r;
        c->rctx = nullptr;
    }
    for (ShapeDev *s : c->shapes) {
        s->T64.release(); s->U64.release(); s->Tdf.release(); s->Udf.release(); s->St64.release();
        s->St32.release(); s->red_offs.release();
        s->skel_k = 0;
        s->skel_rho = 0.0;
        s->skel_eps = 0.0;
        s->skel_J.clear();
    }
    c->rb.release();
    c->rx.release();
    c->ysplit.release();
    c->accel = false;
}

// The reduced context over the skeleton nodes of every body (all shapes must have one).
hzb_status build_reduced(hzb_ctx *c)
{
    if (c->rctx) {
        hzb_ctx *r = c->rctx;
        free_ctx_buffers(r);
        if (r->ev0) cudaEventDestroy(r->ev0);
        if (r->ev1) cudaEventDestroy(r->ev1);
        delete r;
        c->rctx = nullptr;
    }
    hzb_ctx *r = new (std::nothrow) hzb_ctx();
    if (!r) return HZB_ENOMEM;
    r->opt = c->opt;
    r->stream = c->stream;
    r->k = c->k;
    r->eta = c->eta;
    r->reduced = true;
    r->state = 3;
    for (int q = 0; q < 3; ++q) r->center[q] = c->center[q];
    if (cudaEventCreate(&r->ev0) != cudaSuccess || cudaEventCreate(&r->ev1) != cudaSuccess) {
        delete r;
        return check_cuda(c, cudaErrorUnknown, "events");
    }
    c->rctx = r;
    // skeleton nodes body by body; per shape the reduced offsets of its bodies
    std::vector<long long> gidx;
    std::vector<std::vector<long long>> offs(c->shapes.size());
    std::vector<TargetBlock> blocks;
    for (size_t b = 0; b < c->bodies.size(); ++b) {
        const BodyRec &br = c->bodies[b];
        const ShapeDev &sd = *c->shapes[br.shape];
        const long long o = (long long)gidx.size();
        offs[br.shape].push_back(o);
        for (int s : sd.skel_J) gidx.push_back(br.offset + s);
        const int k = sd.skel_k;
        for (int s = 0; s < k; s += 512) {
            TargetBlock t;
            t.start = (int)(o + s);
            t.count = std::min(512, k - s);
            t.excl_lo = (int)o;
            t.excl_hi = (int)(o + k);
            blocks.push_back(t);
        }
    }
    const long long nr = (long long)gidx.size();
    r->N = nr;
    DevBuf<long long> g;
    if (check_cuda(c, g.ensure(nr), "alloc") || check_cuda(c, r->pos64.ensure(nr), "alloc") ||
        check_cuda(c, r->nrm64.ensure(nr), "alloc") || check_cuda(c, r->pos32.ensure(nr), "alloc") ||
        check_cuda(c, r->nrm32.ensure(nr), "alloc") || check_cuda(c, r->body_of.ensure(nr), "alloc") ||
        check_cuda(c, r->tblocks.ensure(blocks.size()), "alloc")) {
        g.release();
        return HZB_ENOMEM;
    }
    hzb_status st = HZB_OK;
    if (check_cuda(c, cudaMemcpyAsync(g.ptr, gidx.data(), nr * sizeof(long long), cudaMemcpyHostToDevice, c->stream),
                   "gather") ||
        check_cuda(c, cudaMemcpyAsync(r->tblocks.ptr, blocks.data(), blocks.size() * sizeof(TargetBlock),
                                      cudaMemcpyHostToDevice, c->stream), "blocks"))
        st = HZB_ECUDA;
    if (!st) {
        gather_nodes_kernel<<<(unsigned)((nr + 255) / 256), 256, 0, c->stream>>>(
            nr, g.ptr, c->pos64.ptr, c->nrm64.ptr, c->pos32.ptr, c->nrm32.ptr, c->body_of.ptr, r->pos64.ptr,
            r->nrm64.ptr, r->pos32.ptr, r->nrm32.ptr, r->body_of.ptr);
        c->launches++;
        r->n_tblocks = (int)blocks.size();
        r->nodes_ready = true;
        for (size_t s = 0; s < c->shapes.size() && !st; ++s) {
            ShapeDev &sd = *c->shapes[s];
            if (check_cuda(c, sd.red_offs.ensure(offs[s].size()), "alloc")) { st = HZB_ENOMEM; break; }
            if (check_cuda(c, cudaMemcpyAsync(sd.red_offs.ptr, offs[s].data(), offs[s].size() * sizeof(long long),
                                              cudaMemcpyHostToDevice, c->stream), "offsets"))
                st = HZB_ECUDA;
            hzb_ctx::RShape rs;
            rs.k = sd.skel_k;
            rs.ms = (int)offs[s].size();
            rs.S64 = sd.St64.ptr;
            rs.S32 = sd.St32.ptr;
            rs.offs = sd.red_offs.ptr;
            r->rshapes.push_back(rs);
        }
    }
    if (!st && check_cuda(c, cudaStreamSynchronize(c->stream), "reduced nodes")) st = HZB_ECUDA;
    g.release();
    return st;
}

// out[ooff_b + i][r] = alpha sig[ooff_b + i][r] + beta sum_j A[i][j] y[yoff_b + j][r] for the
// ms bodies b of a shape and i < rows; A rows x cols row-major.  One warp per row, eight
// rows per block; the right-hand-side columns (body, r) go in groups of 8, and each
// 256-wide slice of their y values is staged once in shared memory for the block's
// eight rows.  F32: A in FP32 and FP32 accumulation (the reduced system's FP32
// operator), else FP64.  The restriction T w (A = T), the extension T^T y (A = T^T)
// and the reduced local operator S y (A = S) all take this form.
static const int GEMV_ROWS = 8;
template <bool F32>
__global__ void __launch_bounds__(256) body_gemv_kernel(int rows, int cols, int ms, int R,
                                                        const long long *__restrict__ yoff,
                                                        const long long *__restrict__ ooff, const void *__restrict__ Av,
                                                        const double2 *__restrict__ y, const double2 *__restrict__ sig,
                                                        double alpha, double beta, double2 *__restrict__ out)
{
    typedef typename std::conditional<F32, float, double>::type acc_t;
    __shared__ acc_t ys[8][256][2];
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * GEMV_ROWS + (threadIdx.x >> 5);
    const int ncol = ms * R;
    for (int c0 = 0; c0 < ncol; c0 += 8) {
        const int nc = min(8, ncol - c0);
        acc_t sx[8], sy[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) sx[q] = sy[q] = (acc_t)0;
        for (int jc = 0; jc < cols; jc += 256) {
            __syncthreads();
            {
                const int j = jc + threadIdx.x;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    if (q < nc) {
                        const int cc = c0 + q;
                        double2 v = make_double2(0.0, 0.0);
                        if (j < cols) v = y[(yoff[cc / R] + j) * R + cc % R];
                        ys[q][threadIdx.x][0] = (acc_t)v.x;
                        ys[q][threadIdx.x][1] = (acc_t)v.y;
                    }
                }
            }
            __syncthreads();
            if (i < rows) {
                const int jn = min(256, cols - jc);
#pragma unroll 4
                for (int jj = lane; jj < jn; jj += 32) {
                    acc_t ax, ay;
                    if (F32) {
                        const float2 av = ((const float2 *)Av)[(size_t)i * cols + jc + jj];
                        ax = av.x;
                        ay = av.y;
                    } else {
                        const double2 av = ((const double2 *)Av)[(size_t)i * cols + jc + jj];
                        ax = (acc_t)av.x;
                        ay = (acc_t)av.y;
                    }
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        if (q < nc) {
                            const acc_t vx = ys[q][jj][0], vy = ys[q][jj][1];
                            sx[q] = fma(ax, vx, fma(-ay, vy, sx[q]));
                            sy[q] = fma(ax, vy, fma(ay, vx, sy[q]));
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int q = 0; q < 8; ++q)
            for (int o = 16; o > 0; o >>= 1) {
                sx[q] += __shfl_xor_sync(0xffffffffu, sx[q], o);
                sy[q] += __shfl_xor_sync(0xffffffffu, sy[q], o);
            }
        if (i < rows && lane < nc) {
            double vx = 0.0, vy = 0.0;
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (q == lane) {
                    vx = (double)sx[q];
                    vy = (double)sy[q];
                }
            const int cc = c0 + lane;
            const size_t o = (size_t)(ooff[cc / R] + i) * R + cc % R;
            double2 res = make_double2(beta * vx, beta * vy);
            if (alpha != 0.0) {
                res.x += alpha * sig[o].x;
                res.y += alpha * sig[o].y;
            }
            out[o] = res;
        }
    }
}

static unsigned gemv_blocks(int rows) { return (unsigned)((rows + GEMV_ROWS - 1) / GEMV_ROWS); }

// x -> (hi, lo) in FP32 with hi = fl(x), lo = fl(x - hi): x = hi + lo to about 2^-48 |x|
__global__ void split_df_kernel(size_t n, const double2 *__restrict__ a, float4 *__restrict__ out)
{
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const double2 v = a[e];
    const float hx = (float)v.x, hy = (float)v.y;
    out[e] = make_float4(hx, hy, (float)(v.x - (double)hx), (float)(v.y - (double)hy));
}

// a + b exactly as (s, err) (Knuth's two-sum), FP32; the _rn intrinsics keep the
// compiler from fusing these operations with a neighbouring multiply
__device__ __forceinline__ void two_sum_f(float a, float b, float &s, float &err)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (uh + ul)(vh + vl) ~ p + e with p = fl(uh vh) and e its rounding error plus the
// cross terms (the ul vl term, ~2^-48 of the product, is dropped)
__device__ __forceinline__ void prod_df(float uh, float ul, float vh, float vl, float &p, float &e)
{
    p = __fmul_rn(uh, vh);
    e = fmaf(uh, vh, -p);
    e = fmaf(uh, vl, e);
    e = fmaf(ul, vh, e);
}

__device__ __forceinline__ void acc_df(float &sh, float &sl, float p, float e)
{
    float s, err;
    two_sum_f(sh, p, s, err);
    sh = s;
    sl += err + e;
}

// The GEMV of body_gemv_kernel in double-float on the FP32 pipe: A and y split into FP32
// hi/lo pairs (split_df_kernel), each real product formed with its rounding error and
// added by two-sum into a (hi, lo) accumulator; about 48 FP32 operations per complex
// multiply-add instead of 4 FP64 ones (FP64 runs at 1/64 of the FP32 rate), relative
// error about 1e-14 per term.  Used by the mixed path's restriction and recovery.
__global__ void __launch_bounds__(256) body_gemv_df_kernel(int rows, int cols, int ms, int R,
                                                           const long long *__restrict__ yoff,
                                                           const long long *__restrict__ ooff,
                                                           const float4 *__restrict__ A, const float4 *__restrict__ y,
                                                           const double2 *__restrict__ sig, double alpha, double beta,
                                                           double2 *__restrict__ out)
{
    __shared__ float4 ys[8][256];
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * GEMV_ROWS + (threadIdx.x >> 5);
    const int ncol = ms * R;
    for (int c0 = 0; c0 < ncol; c0 += 8) {
        const int nc = min(8, ncol - c0);
        float rh[8], rl[8], ih[8], il[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) rh[q] = rl[q] = ih[q] = il[q] = 0.f;
        for (int jc = 0; jc < cols; jc += 256) {
            __syncthreads();
            {
                const int j = jc + threadIdx.x;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    if (q < nc) {
                        const int cc = c0 + q;
                        ys[q][threadIdx.x] =
                            j < cols ? y[(yoff[cc / R] + j) * R + cc % R] : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                }
            }
            __syncthreads();
            if (i < rows) {
                const int jn = min(256, cols - jc);
#pragma unroll 2
                for (int jj = lane; jj < jn; jj += 32) {
                    const float4 a = A[(size_t)i * cols + jc + jj];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        if (q < nc) {
                            const float4 v = ys[q][jj];
                            float p, e;
                            prod_df(a.x, a.z, v.x, v.z, p, e);          // ar yr
                            acc_df(rh[q], rl[q], p, e);
                            prod_df(-a.y, -a.w, v.y, v.w, p, e);        // - ai yi
                            acc_df(rh[q], rl[q], p, e);
                            prod_df(a.x, a.z, v.y, v.w, p, e);          // ar yi
                            acc_df(ih[q], il[q], p, e);
                            prod_df(a.y, a.w, v.x, v.z, p, e);          // ai yr
                            acc_df(ih[q], il[q], p, e);
                        }
                    }
                }
            }
        }
        double sx[8], sy[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            sx[q] = (double)rh[q] + (double)rl[q];
            sy[q] = (double)ih[q] + (double)il[q];
            for (int o = 16; o > 0; o >>= 1) {
                sx[q] += __shfl_xor_sync(0xffffffffu, sx[q], o);
                sy[q] += __shfl_xor_sync(0xffffffffu, sy[q], o);
            }
        }
        if (i < rows && lane < nc) {
            double vx = 0.0, vy = 0.0;
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (q == lane) {
                    vx = sx[q];
                    vy = sy[q];
                }
            const int cc = c0 + lane;
            const size_t o = (size_t)(ooff[cc / R] + i) * R + cc % R;
            double2 res = make_double2(beta * vx, beta * vy);
            if (alpha != 0.0) {
                res.x += alpha * sig[o].x;
                res.y += alpha * sig[o].y;
            }
            out[o] = res;
        }
    }
}

hzb_status reduced_local(hzb_ctx *c, int R, const double2 *y, const double2 *sigma, double alpha, double beta,
                         double2 *tau, bool fp32)
{
    for (const hzb_ctx::RShape &rs : c->rshapes) {
        if (fp32)
            body_gemv_kernel<true><<<gemv_blocks(rs.k), 256, 0, c->stream>>>(rs.k, rs.k, rs.ms, R, rs.offs, rs.offs, rs.S32, y,
                                                                sigma, alpha, beta, tau);
        else
            body_gemv_kernel<false><<<gemv_blocks(rs.k), 256, 0, c->stream>>>(rs.k, rs.k, rs.ms, R, rs.offs, rs.offs, rs.S64, y,
                                                                 sigma, alpha, beta, tau);
        c->launches++;
    }
    return check_cuda(c, cudaGetLastError(), "reduced local operator");
}

// sig~ = s T w per body (restriction V_p^* of node vectors), out in reduced numbering;
// df: in double-float on the FP32 pipe (mixed path), else FP64
static hzb_status restrict_all(hzb_ctx *c, int R, const double2 *w, double s, double2 *out, bool df)
{
    if (df) {
        const size_t nw = (size_t)c->N * R;
        if (check_cuda(c, c->ysplit.ensure(nw), "alloc")) return HZB_ENOMEM;
        split_df_kernel<<<(unsigned)((nw + 255) / 256), 256, 0, c->stream>>>(nw, w, c->ysplit.ptr);
        c->launches++;
    }
    for (ShapeDev *sp : c->shapes) {
        ShapeDev &sd = *sp;
        const int n = sd.geom.NG * sd.geom.NF;
        if (df)
            body_gemv_df_kernel<<<gemv_blocks(sd.skel_k), 256, 0, c->stream>>>(
                sd.skel_k, n, (int)sd.bodies.size(), R, sd.body_offs.ptr, sd.red_offs.ptr, sd.Tdf.ptr, c->ysplit.ptr,
                nullptr, 0.0, s, out);
        else
            body_gemv_kernel<false><<<gemv_blocks(sd.skel_k), 256, 0, c->stream>>>(
                sd.skel_k, n, (int)sd.bodies.size(), R, sd.body_offs.ptr, sd.red_offs.ptr, sd.T64.ptr, w, nullptr,
                0.0, s, out);
        c->launches++;
    }
    return check_cuda(c, cudaGetLastError(), "restrict");
}

static void sync_settings(hzb_ctx *c, hzb_ctx *r)
{
    r->opt = c->opt;
    r->stream = c->stream;
    r->nbody_engine = c->nbody_engine;
    r->nbody64_engine = c->nbody64_engine;
    r->check_every = c->check_every;
    r->use_graphs = c->use_graphs;
}

hzb_status solve_reduced(hzb_ctx *c, int R, const double2 *v, const double2 *x0, hzb_stats *stats)
{
    hzb_ctx *r = c->rctx;
    sync_settings(c, r);
    const size_t NR = (size_t)c->N * R, RR = (size_t)r->N * R;
    if (check_cuda(c, c->sol.ensure(NR), "alloc") || check_cuda(c, c->w_a.ensure(NR), "alloc") ||
        check_cuda(c, c->w_b.ensure(NR), "alloc") || check_cuda(c, c->rb.ensure(RR), "alloc") ||
        check_cuda(c, c->rx.ensure(RR), "alloc"))
        return HZB_ENOMEM;
    cudaEventRecord(c->ev0, c->stream);
    const long long l0 = c->launches, rl0 = r->launches;
    hzb_status st;
    // v~ = T A^{-1} v per body; right-hand side -v~.  The two direct D^{-1} applies run in
    // double-float when the refinement residual does (mixed path), else in FP64.
    const bool df = c->opt.precision != HZB_PREC_FP64;
    auto dinv = (df && c->opt.residual == HZB_PREC_DOUBLE_FLOAT) ? local_inverse_dfl : local_inverse64;
    if ((st = dinv(c, R, v, nullptr, 0.0, 1.0, c->w_a.ptr))) return st;
    if ((st = restrict_all(c, R, c->w_a.ptr, -1.0, c->rb.ptr, df))) return st;
    if (x0 && (st = restrict_all(c, R, x0, 1.0, c->rx.ptr, df))) return st;
    hzb_stats rs{};
    hzb_status solve_st = solve_driver(r, R, nullptr, x0 ? c->rx.ptr : nullptr, &rs, c->rb.ptr);
    if (solve_st && solve_st != HZB_ENOCONV) return fail(c, solve_st, r->err);
    // sig = D^{-1} (-v - U B~ sig~)
    const double2 *sig_t = r->sol.ptr;
    if (check_cuda(c, r->s_r.ensure(RR), "alloc")) return HZB_ENOMEM;
    // FP64 path: FP64; mixed path: double-float (about 1e-13 per term, far below its tolerance)
    st = c->opt.precision == HZB_PREC_FP64 ? interbody64(r, R, sig_t, r->s_r.ptr) : interbody_df(r, R, sig_t, r->s_r.ptr);
    if (st) return fail(c, st, r->err);
    if (df) {
        if (check_cuda(c, c->ysplit.ensure(std::max(RR, NR)), "alloc")) return HZB_ENOMEM;
        split_df_kernel<<<(unsigned)((RR + 255) / 256), 256, 0, c->stream>>>(RR, r->s_r.ptr, c->ysplit.ptr);
        c->launches++;
    }
    for (ShapeDev *sp : c->shapes) {
        ShapeDev &sd = *sp;
        const int n = sd.geom.NG * sd.geom.NF;
        if (df)
            body_gemv_df_kernel<<<gemv_blocks(n), 256, 0, c->stream>>>(n, sd.skel_k, (int)sd.bodies.size(), R,
                                                                      sd.red_offs.ptr, sd.body_offs.ptr, sd.Udf.ptr,
                                                                      c->ysplit.ptr, v, -1.0, -1.0, c->w_b.ptr);
        else
            body_gemv_kernel<false><<<gemv_blocks(n), 256, 0, c->stream>>>(n, sd.skel_k, (int)sd.bodies.size(), R,
                                                                          sd.red_offs.ptr, sd.body_offs.ptr, sd.U64.ptr,
                                                                          r->s_r.ptr, v, -1.0, -1.0, c->w_b.ptr);
        c->launches++;
    }
    if (check_cuda(c, cudaGetLastError(), "extend")) return HZB_ECUDA;
    if ((st = dinv(c, R, c->w_b.ptr, nullptr, 0.0, 1.0, c->sol.ptr))) return st;
    c->sol_R = R;
    cudaEventRecord(c->ev1, c->stream);
    if (check_cuda(c, cudaEventSynchronize(c->ev1), "reduced solve")) return HZB_ECUDA;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    c->launches += r->launches - rl0;
    if (stats) {
        *stats = rs;
        stats->t_solve_ms = ms;
        stats->t_setup_ms = c->t_setup_ms;
        stats->interbody_applies = rs.interbody_applies + 1;
        stats->kernel_launches = c->launches - l0;
    }
    if (solve_st == HZB_ENOCONV) return fail(c, HZB_ENOCONV, "GMRES did not reach the tolerance (reduced system)");
    return HZB_OK;
}

}  // namespace hzb

using namespace hzb;

#define CP_GUARD(c) HZB_GUARD(c)

extern "C" hzb_status hzb_compress(hzb_ctx *c, double eps, int n_theta, double proxy_radius)
{
    CP_GUARD(c);
    if (c->state != 3) return fail(c, HZB_ESTATE, "hzb_compress needs the scattering matrices");
    if (!(eps >= 0.0 && eps < 1.0) || n_theta < 0 || n_theta > 4096 || !(proxy_radius >= 0.0))
        return fail(c, HZB_EINVAL, "eps must be in [0, 1), n_theta in [0, 4096], proxy_radius >= 0");
    release_compression(c);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, c->stream);
    hzb_status st = HZB_OK;
    for (size_t s = 0; s < c->shapes.size() && !st; ++s) {
        double rb, gap;
        proxy_geometry(c, (int)s, rb, gap);
        double rho = proxy_radius;
        if (rho == 0.0) {
            if (!std::isfinite(gap)) rho = 1.5 * rb;
            else if (gap <= 1.02 * rb) st = fail(c, HZB_EINVAL, "bodies too close for a proxy sphere");
            else rho = 0.5 * (rb + gap);
        } else if (rho <= rb || rho >= gap) {
            st = fail(c, HZB_EINVAL, "proxy sphere must enclose its body and exclude every other body");
        }
        if (st) break;
        const int nt = n_theta > 0 ? n_theta : std::max(16, (int)std::ceil(1.2 * c->shapes[s]->geom.NG));
        st = compress_shape(c, (int)s, eps, nt, rho);
    }
    if (!st) st = build_reduced(c);
    cudaEventRecord(e1, c->stream);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st) {
        release_compression(c);
        return st;
    }
    c->t_compress_ms = ms;
    c->accel = true;
    return HZB_OK;
}

extern "C" hzb_status hzb_set_skeleton(hzb_ctx *c, int body, int k, const int *J, const double *T)
{
    CP_GUARD(c);
    if (c->state != 3) return fail(c, HZB_ESTATE, "hzb_set_skeleton needs the scattering matrices");
    if (body < 0 || body >= (int)c->bodies.size() || !J || !T) return fail(c, HZB_EINVAL, "bad body or pointer");
    ShapeDev &sd = *c->shapes[c->bodies[body].shape];
    const int n = sd.geom.NG * sd.geom.NF;
    if (k <= 0 || k > n) return fail(c, HZB_EINVAL, "skeleton size out of range");
    std::vector<int> Jv(J, J + k), chk(Jv);
    std::sort(chk.begin(), chk.end());
    if (chk.front() < 0 || chk.back() >= n || std::adjacent_find(chk.begin(), chk.end()) != chk.end())
        return fail(c, HZB_EINVAL, "skeleton indices must be distinct and in [0, n)");
    DevBuf<double2> Td;
    if (check_cuda(c, Td.ensure((size_t)k * n), "alloc T")) return HZB_ENOMEM;
    hzb_status st = check_cuda(c, cudaMemcpyAsync(Td.ptr, T, (size_t)k * n * sizeof(double2), cudaMemcpyHostToDevice,
                                                  c->stream), "upload T");
    if (!st) st = install_skeleton(c, sd, Jv, Td);
    Td.release();
    if (st) return st;
    sd.skel_rho = 0.0;
    sd.skel_eps = 0.0;
    bool all = true;
    for (ShapeDev *s : c->shapes) all = all && s->skel_k > 0;
    if (all) {
        if ((st = build_reduced(c))) return st;
        c->accel = true;
    }
    return HZB_OK;
}

extern "C" hzb_status hzb_get_skeleton(hzb_ctx *c, int body, int *k, int *J, double *T)
{
    CP_GUARD(c);
    if (body < 0 || body >= (int)c->bodies.size() || !k) return fail(c, HZB_EINVAL, "bad body or pointer");
    ShapeDev &sd = *c->shapes[c->bodies[body].shape];
    *k = sd.skel_k;
    if (sd.skel_k == 0) return HZB_OK;
    if (J) std::copy(sd.skel_J.begin(), sd.skel_J.end(), J);
    if (T) {
        const size_t ne = (size_t)sd.skel_k * sd.geom.NG * sd.geom.NF;
        if (check_cuda(c, cudaMemcpyAsync(T, sd.T64.ptr, ne * sizeof(double2), cudaMemcpyDeviceToHost, c->stream),
                       "copy T") ||
            check_cuda(c, cudaStreamSynchronize(c->stream), "copy T"))
            return HZB_ECUDA;
    }
    return HZB_OK;
}

extern "C" hzb_status hzb_get_skeleton_info(hzb_ctx *c, int body, int *k, double *eps, double *rho)
{
    CP_GUARD(c);
    if (body < 0 || body >= (int)c->bodies.size()) return fail(c, HZB_EINVAL, "bad body");
    const ShapeDev &sd = *c->shapes[c->bodies[body].shape];
    if (k) *k = sd.skel_k;
    if (eps) *eps = sd.skel_eps;
    if (rho) *rho = sd.skel_rho;
    return HZB_OK;
}

extern "C" hzb_status hzb_set_acceleration(hzb_ctx *c, int on)
{
    CP_GUARD(c);
    if (on && !c->rctx) return fail(c, HZB_ESTATE, "no skeletons: call hzb_compress first");
    c->accel = on != 0;
    return HZB_OK;
}

extern "C" hzb_status hzb_reduced_size(const hzb_ctx *c, long long *n)
{
    if (!c || !n) return HZB_EINVAL;
    *n = c->rctx ? c->rctx->N : 0;
    return HZB_OK;
}

extern "C" hzb_status hzb_apply_reduced(hzb_ctx *c, int R, const double *sig, double *out, int precision)
{
    CP_GUARD(c);
    if (!c->rctx) return fail(c, HZB_ESTATE, "no reduced system");
    if (R <= 0 || !sig || !out || (precision != HZB_PREC_FP64 && precision != HZB_PREC_MIXED_FP32 &&
                                   precision != HZB_PREC_DOUBLE_FLOAT))
        return fail(c, HZB_EINVAL, "bad R, pointer or precision");
    hzb_ctx *r = c->rctx;
    sync_settings(c, r);
    const size_t RR = (size_t)r->N * R;
    if (check_cuda(c, c->rb.ensure(RR), "alloc") || check_cuda(c, c->rx.ensure(RR), "alloc")) return HZB_ENOMEM;
    if (check_cuda(c, cudaMemcpyAsync(c->rb.ptr, sig, RR * sizeof(double2), cudaMemcpyHostToDevice, c->stream), "in"))
        return HZB_ECUDA;
    const long long rl0 = r->launches;
    hzb_status st = apply_op(r, R, c->rb.ptr, c->rx.ptr, precision);
    c->launches += r->launches - rl0;
    if (st) return fail(c, st, r->err);
    if (check_cuda(c, cudaMemcpyAsync(out, c->rx.ptr, RR * sizeof(double2), cudaMemcpyDeviceToHost, c->stream), "out") ||
        check_cuda(c, cudaStreamSynchronize(c->stream), "apply reduced"))
        return HZB_ECUDA;
    return HZB_OK;
}

extern "C" hzb_status hzb_interp_decomp(hzb_ctx *c, int rows, int cols, const double *Z, double eps, int *k, int *J,
                                        double *T)
{
    CP_GUARD(c);
    if (rows <= 0 || cols <= 0 || !Z || !k || !J || !T || !(eps >= 0.0 && eps < 1.0))
        return fail(c, HZB_EINVAL, "bad size, pointer or tolerance");
    DevBuf<double2> Zd, Td;
    const size_t ne = (size_t)rows * cols;
    if (check_cuda(c, Zd.ensure(ne), "alloc")) return HZB_ENOMEM;
    hzb_status st = check_cuda(c, cudaMemcpyAsync(Zd.ptr, Z, ne * sizeof(double2), cudaMemcpyHostToDevice, c->stream),
                               "upload");
    std::vector<int> Jv;
    if (!st) st = column_id(c, rows, cols, Zd.ptr, eps, Jv, Td);
    if (!st) {
        *k = (int)Jv.size();
        std::copy(Jv.begin(), Jv.end(), J);
        if (check_cuda(c, cudaMemcpyAsync(T, Td.ptr, Jv.size() * cols * sizeof(double2), cudaMemcpyDeviceToHost,
                                          c->stream), "download") ||
            check_cuda(c, cudaStreamSynchronize(c->stream), "download"))
            st = HZB_ECUDA;
    }
    Zd.release();
    Td.release();
    return st;
}
