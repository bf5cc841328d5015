// Inter-body sum y = B sigma (Sec. 3.3, Eq. (nystromnaive)) in double-float
// arithmetic on the FP32 pipe, for the refinement residual of the mixed-precision
// solve.  GB300's FP64 rate is 1/64 of its FP32 rate; a pair interaction in
// double-float (hi + lo floats, ~48-bit significand, error-free transformations of
// dfloat.cuh) costs ~400 FP32 instructions against ~60 FP64 ones, so it runs several
// times faster than the FP64 kernel at ~1e-13 relative accuracy per term.
//
// Per pair (d = x_i - x_j, r = |d|, sigma' = w_j sigma_j / (4 pi)):
//     K w_j sigma_j = e^{ikr} [ A - i B ] sigma',  A = n_j.d / r^3,  B = k n_j.d / r^2 + eta / r,
// with 1/r from the hardware reciprocal square root refined by one Newton step in
// double-float, and e^{ikr} by reduction of kr/(2pi) to a fraction of a turn, a
// 128-entry table of (cos, sin)(2 pi m / 128) and Taylor series of the remainder
// |delta| <= pi/128 (leading terms in double-float, the tail in FP32).
// Work decomposition as in nbody.cu: one CTA per (TargetBlock, RHS chunk, source
// chunk); source tiles of 128 staged in shared memory.
#include <algorithm>
#include <cmath>
#include <vector>

#include "dfloat.cuh"
#include "hzb_internal.h"

namespace hzb {

static const int DF_TBLOCK = 512;
static const int DF_TILE = 128;
static const int DF_TAB = 128;

struct DfConst {
    dfl k, eta, inv2pi, twopi, inv6;
};

// Split positions and normals (relative to the FP32 origin) into double-float.
__global__ void df_nodes_kernel(long long N, const double4 *__restrict__ pos, const double4 *__restrict__ nrm,
                                double ox, double oy, double oz, float4 *a, float4 *b, float4 *cn)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double4 p = pos[i], n = nrm[i];
    dfl x = df_from_double(p.x - ox), y = df_from_double(p.y - oy), z = df_from_double(p.z - oz);
    dfl nx = df_from_double(n.x), ny = df_from_double(n.y), nz = df_from_double(n.z);
    a[i] = make_float4(x.hi, y.hi, z.hi, nx.hi);
    b[i] = make_float4(x.lo, y.lo, z.lo, nx.lo);
    cn[i] = make_float4(ny.hi, nz.hi, ny.lo, nz.lo);
}

// Geometry of a pair in double-float: d = x_i - x_j, r^2, 1/r (hardware estimate and one
// Newton step) and r.
struct DfGeom {
    dfl dx, dy, dz, ir, r;
};

__device__ __forceinline__ DfGeom df_geom(dfl tx, dfl ty, dfl tz, float4 A4, float4 B4)
{
    DfGeom G;
    const dfl sx = df_two_sum(tx.hi, -A4.x), sy = df_two_sum(ty.hi, -A4.y), sz = df_two_sum(tz.hi, -A4.z);
    G.dx = df_fast_two_sum(sx.hi, sx.lo + (tx.lo - B4.x));
    G.dy = df_fast_two_sum(sy.hi, sy.lo + (ty.lo - B4.y));
    G.dz = df_fast_two_sum(sz.hi, sz.lo + (tz.lo - B4.z));
    // r^2 (three positive squares)
    const float px = G.dx.hi * G.dx.hi, py = G.dy.hi * G.dy.hi, pz = G.dz.hi * G.dz.hi;
    const float ex = fmaf(2.f * G.dx.hi, G.dx.lo, fmaf(G.dx.hi, G.dx.hi, -px));
    const float ey = fmaf(2.f * G.dy.hi, G.dy.lo, fmaf(G.dy.hi, G.dy.hi, -py));
    const float ez = fmaf(2.f * G.dz.hi, G.dz.lo, fmaf(G.dz.hi, G.dz.hi, -pz));
    const dfl s1 = df_two_sum(px, py), s2 = df_two_sum(s1.hi, pz);
    const dfl r2 = df_fast_two_sum(s2.hi, s2.lo + s1.lo + ((ex + ey) + ez));
    // 1/r: hardware estimate, one Newton step in double-float
    const float y0 = rsqrtf(r2.hi);
    const dfl y0sq = df_fast_two_sum(y0 * y0, fmaf(y0, y0, -(y0 * y0)));
    const dfl u = df_mul(r2, y0sq);
    const float e = (1.f - u.hi) - u.lo;
    G.ir = df_fast_two_sum(y0, 0.5f * y0 * e);
    G.r = df_mul(r2, G.ir);
    return G;
}

// e^{ikr} in double-float: kr/(2 pi) reduced to [-1/2, 1/2] turns, then to the nearest
// of DF_TAB table angles, Taylor series of the remainder (leading terms in
// double-float, the tail in FP32) and angle addition with the table entry.
__device__ __forceinline__ void df_cis(const DfConst &K, dfl r, const float4 *__restrict__ s_tab, dfl &cs, dfl &sn)
{
    const dfl turns = df_mul(df_mul(K.k, r), K.inv2pi);
    const float n0 = rintf(turns.hi);
    const dfl f = df_fast_two_sum(turns.hi - n0, turns.lo);            // [-1/2, 1/2] turns
    const float mm = rintf(f.hi * (float)DF_TAB);
    const dfl g = df_fast_two_sum(f.hi - mm * (1.f / DF_TAB), f.lo);    // |g| <= 1/256
    const dfl dl = df_mul(g, K.twopi);                                  // |dl| <= pi/128
    const dfl d2 = df_mul(dl, dl);
    const dfl d3 = df_mul(d2, dl);
    const float d2f = d2.hi;
    dfl sd = df_sub(dl, df_mul(d3, K.inv6));
    sd = df_addf(sd, dl.hi * d2f * d2f * fmaf(-d2f, 1.f / 5040.f, 1.f / 120.f));
    dfl cd = df_add({1.f, 0.f}, {-0.5f * d2.hi, -0.5f * d2.lo});
    cd = df_addf(cd, d2f * d2f * fmaf(-d2f, 1.f / 720.f, 1.f / 24.f));
    const float4 T = s_tab[((int)mm) & (DF_TAB - 1)];
    const dfl Ct = {T.x, T.y}, St = {T.z, T.w};
    cs = df_sub(df_mul(Ct, cd), df_mul(St, sd));
    sn = df_add(df_mul(St, cd), df_mul(Ct, sd));
}

template <int RC, int TPT>
__global__ void __launch_bounds__(DF_TBLOCK / TPT)
nbody_df_kernel(const TargetBlock *__restrict__ blocks, int N, int R, int chunk, const float4 *__restrict__ pa,
                const float4 *__restrict__ pb, const float4 *__restrict__ pc, const double4 *__restrict__ pos64,
                const double2 *__restrict__ sigma, const float4 *__restrict__ tab, DfConst K,
                double2 *__restrict__ y, size_t split_stride)
{
    constexpr int NT = DF_TBLOCK / TPT;
    __shared__ float4 s_a[DF_TILE], s_b[DF_TILE], s_c[DF_TILE];
    __shared__ float4 s_sig[DF_TILE * RC];          // re.hi, re.lo, im.hi, im.lo of w sigma / (4 pi)
    __shared__ float4 s_tab[DF_TAB];                // cos.hi, cos.lo, sin.hi, sin.lo
    const TargetBlock tb = blocks[blockIdx.x];
    const int r0 = blockIdx.y * RC;
    const int tid = threadIdx.x;
    for (int q = tid; q < DF_TAB; q += NT) s_tab[q] = tab[q];
    dfl tx[TPT], ty[TPT], tz[TPT];
    dfl ar[TPT][RC], ai[TPT][RC];
#pragma unroll
    for (int m = 0; m < TPT; ++m) {
        int t = tid + m * NT;
        int g = tb.start + min(t, tb.count - 1);
        float4 a = pa[g], b = pb[g];
        tx[m] = {a.x, b.x}; ty[m] = {a.y, b.y}; tz[m] = {a.z, b.z};
#pragma unroll
        for (int c = 0; c < RC; ++c) { ar[m][c] = {0.f, 0.f}; ai[m][c] = {0.f, 0.f}; }
    }
    const int c0 = blockIdx.z * chunk, c1 = min(N, c0 + chunk);
    for (int range = 0; range < 2; ++range) {
        const int lo = range ? max(c0, tb.excl_hi) : c0;
        const int hi = range ? c1 : min(c1, tb.excl_lo);
        for (int j0 = lo; j0 < hi; j0 += DF_TILE) {
            const int cnt = min(DF_TILE, hi - j0);
            __syncthreads();
            for (int q = tid; q < cnt; q += NT) {
                s_a[q] = pa[j0 + q];
                s_b[q] = pb[j0 + q];
                s_c[q] = pc[j0 + q];
                const double wq = pos64[j0 + q].w * 0.07957747154594767;
#pragma unroll
                for (int c = 0; c < RC; ++c) {
                    double2 s = (r0 + c < R) ? sigma[(size_t)(j0 + q) * R + r0 + c] : make_double2(0.0, 0.0);
                    dfl re = df_from_double(s.x * wq), im = df_from_double(s.y * wq);
                    s_sig[q * RC + c] = make_float4(re.hi, re.lo, im.hi, im.lo);
                }
            }
            __syncthreads();
            for (int jj = 0; jj < cnt; ++jj) {
                const float4 A4 = s_a[jj], B4 = s_b[jj], C4 = s_c[jj];
                const dfl nx = {A4.w, B4.w}, ny = {C4.x, C4.z}, nz = {C4.y, C4.w};
#pragma unroll
                for (int m = 0; m < TPT; ++m) {
                    const DfGeom G = df_geom(tx[m], ty[m], tz[m], A4, B4);
                    const dfl dx = G.dx, dy = G.dy, dz = G.dz, ir = G.ir;
                    // n.d, A = n.d / r^3, B = k n.d / r^2 + eta / r
                    const dfl nd = df_add(df_add(df_mul(nx, dx), df_mul(ny, dy)), df_mul(nz, dz));
                    const dfl ir2 = df_mul(ir, ir);
                    const dfl ndir2 = df_mul(nd, ir2);
                    const dfl A = df_mul(ndir2, ir);
                    const dfl B = df_add(df_mul(K.k, ndir2), df_mul(K.eta, ir));
                    dfl cs, sn;
                    df_cis(K, G.r, s_tab, cs, sn);
                    const dfl gre = df_add(df_mul(cs, A), df_mul(sn, B));
                    const dfl gim = df_sub(df_mul(sn, A), df_mul(cs, B));
#pragma unroll
                    for (int q = 0; q < RC; ++q) {
                        const float4 S = s_sig[jj * RC + q];
                        const dfl sr = {S.x, S.y}, si = {S.z, S.w};
                        ar[m][q] = df_add(ar[m][q], df_sub(df_mul(gre, sr), df_mul(gim, si)));
                        ai[m][q] = df_add(ai[m][q], df_add(df_mul(gre, si), df_mul(gim, sr)));
                    }
                }
            }
        }
    }
    double2 *yo = y + blockIdx.z * split_stride;
#pragma unroll
    for (int m = 0; m < TPT; ++m) {
        int t = tid + m * NT;
        if (t < tb.count)
#pragma unroll
            for (int c = 0; c < RC; ++c)
                if (r0 + c < R)
                    yo[(size_t)(tb.start + t) * R + r0 + c] = make_double2(df_to_double(ar[m][c]), df_to_double(ai[m][c]));
    }
}

// Pair-symmetric version (as nbody64_sym_kernel, nbody_sym.cu): one CTA per unordered
// pair of TargetBlocks on different bodies; d, 1/r and e^{ikr} of a node pair serve
// both directions; a warp meets a 32-source tile in 32 rotation steps, the source-side
// sums travel one lane down per step; FP64 atomic adds into y (zeroed first).
static const int DFS_T = 512, DFS_S = 32;

template <int RC>
__global__ void __launch_bounds__(DFS_T, 1)
nbody_df_sym_kernel(const int2 *__restrict__ pairs, const TargetBlock *__restrict__ blocks, int R,
                    const float4 *__restrict__ pa, const float4 *__restrict__ pb, const float4 *__restrict__ pc,
                    const double4 *__restrict__ pos64, const double2 *__restrict__ sigma,
                    const float4 *__restrict__ tab, DfConst K, double2 *__restrict__ y)
{
    __shared__ float4 s_a[DFS_S], s_b[DFS_S], s_c[DFS_S];
    __shared__ float4 s_sig[DFS_S][RC];              // re.hi, re.lo, im.hi, im.lo of w sigma / (4 pi)
    __shared__ float4 s_tab[DF_TAB];
    __shared__ float4 s_red[DFS_T / 32][RC][DFS_S];
    const int2 pr = pairs[blockIdx.x];
    const TargetBlock bi = blocks[pr.x], bj = blocks[pr.y];
    const int r0 = blockIdx.y * RC;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int q = tid; q < DF_TAB; q += DFS_T) s_tab[q] = tab[q];
    const bool live = tid < bi.count;
    dfl tx = {1e5f + tid, 0.f}, ty = {1e5f, 0.f}, tz = {1e5f, 0.f};
    dfl mx = {0.f, 0.f}, my = {0.f, 0.f}, mz = {0.f, 0.f};
    dfl wr[RC], wi[RC], atr[RC], ati[RC];
#pragma unroll
    for (int c = 0; c < RC; ++c) { wr[c] = wi[c] = atr[c] = ati[c] = {0.f, 0.f}; }
    if (live) {
        const int g = bi.start + tid;
        const float4 A = pa[g], B = pb[g], C = pc[g];
        tx = {A.x, B.x}; ty = {A.y, B.y}; tz = {A.z, B.z};
        mx = {A.w, B.w}; my = {C.x, C.z}; mz = {C.y, C.w};
        const double wq = pos64[g].w * 0.07957747154594767;
#pragma unroll
        for (int c = 0; c < RC; ++c)
            if (r0 + c < R) {
                const double2 v = sigma[(size_t)g * R + r0 + c];
                wr[c] = df_from_double(v.x * wq);
                wi[c] = df_from_double(v.y * wq);
            }
    }
    const bool warp_live = warp * 32 < bi.count;
    for (int j0 = 0; j0 < bj.count; j0 += DFS_S) {
        const int cnt = min(DFS_S, bj.count - j0);
        __syncthreads();
        if (tid < DFS_S) {
            if (tid < cnt) {
                const int g = bj.start + j0 + tid;
                s_a[tid] = pa[g];
                s_b[tid] = pb[g];
                s_c[tid] = pc[g];
                const double wq = pos64[g].w * 0.07957747154594767;
#pragma unroll
                for (int c = 0; c < RC; ++c) {
                    const double2 v = (r0 + c < R) ? sigma[(size_t)g * R + r0 + c] : make_double2(0.0, 0.0);
                    const dfl re = df_from_double(v.x * wq), im = df_from_double(v.y * wq);
                    s_sig[tid][c] = make_float4(re.hi, re.lo, im.hi, im.lo);
                }
            } else {                                   // far, zero density: contributes 0 both ways
                s_a[tid] = make_float4(-1e5f - tid, -1e5f, -1e5f, 0.f);
                s_b[tid] = make_float4(0.f, 0.f, 0.f, 0.f);
                s_c[tid] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int c = 0; c < RC; ++c) s_sig[tid][c] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        __syncthreads();
        dfl asr[RC], asi[RC];
#pragma unroll
        for (int c = 0; c < RC; ++c) asr[c] = asi[c] = {0.f, 0.f};
        if (warp_live) {
            for (int s = 0; s < DFS_S; ++s) {
                const int q = (lane + s) & (DFS_S - 1);
                const float4 A4 = s_a[q], B4 = s_b[q], C4 = s_c[q];
                const DfGeom G = df_geom(tx, ty, tz, A4, B4);
                const dfl ir2 = df_mul(G.ir, G.ir), eir = df_mul(K.eta, G.ir);
                dfl cs, sn;
                df_cis(K, G.r, s_tab, cs, sn);
                // i <- j: normal of source j
                const dfl nx = {A4.w, B4.w}, ny = {C4.x, C4.z}, nz = {C4.y, C4.w};
                const dfl X1 = df_mul(df_add(df_add(df_mul(nx, G.dx), df_mul(ny, G.dy)), df_mul(nz, G.dz)), ir2);
                const dfl A1 = df_mul(X1, G.ir), B1 = df_add(df_mul(K.k, X1), eir);
                const dfl g1r = df_add(df_mul(cs, A1), df_mul(sn, B1));
                const dfl g1i = df_sub(df_mul(sn, A1), df_mul(cs, B1));
                // j <- i: normal of target i, d reversed
                const dfl X2p = df_mul(df_add(df_add(df_mul(mx, G.dx), df_mul(my, G.dy)), df_mul(mz, G.dz)), ir2);
                const dfl A2n = df_mul(X2p, G.ir), B2 = df_sub(eir, df_mul(K.k, X2p));
                const dfl g2r = df_sub(df_mul(sn, B2), df_mul(cs, A2n));
                const dfl h = df_add(df_mul(sn, A2n), df_mul(cs, B2));
#pragma unroll
                for (int c = 0; c < RC; ++c) {
                    const float4 S = s_sig[q][c];
                    const dfl sr = {S.x, S.y}, si = {S.z, S.w};
                    atr[c] = df_add(atr[c], df_sub(df_mul(g1r, sr), df_mul(g1i, si)));
                    ati[c] = df_add(ati[c], df_add(df_mul(g1r, si), df_mul(g1i, sr)));
                    asr[c] = df_add(asr[c], df_add(df_mul(g2r, wr[c]), df_mul(h, wi[c])));
                    asi[c] = df_add(asi[c], df_sub(df_mul(g2r, wi[c]), df_mul(h, wr[c])));
                }
#pragma unroll
                for (int c = 0; c < RC; ++c) {
                    const int from = (lane + 1) & 31;
                    asr[c].hi = __shfl_sync(0xffffffffu, asr[c].hi, from);
                    asr[c].lo = __shfl_sync(0xffffffffu, asr[c].lo, from);
                    asi[c].hi = __shfl_sync(0xffffffffu, asi[c].hi, from);
                    asi[c].lo = __shfl_sync(0xffffffffu, asi[c].lo, from);
                }
            }
        }
#pragma unroll
        for (int c = 0; c < RC; ++c) s_red[warp][c][lane] = make_float4(asr[c].hi, asr[c].lo, asi[c].hi, asi[c].lo);
        __syncthreads();
        if (tid < DFS_S * RC) {
            const int src = tid & (DFS_S - 1), c = tid / DFS_S;
            if (src < cnt && r0 + c < R) {
                dfl sr = {0.f, 0.f}, si = {0.f, 0.f};
                for (int w = 0; w < DFS_T / 32; ++w) {
                    const float4 v = s_red[w][c][src];
                    sr = df_add(sr, {v.x, v.y});
                    si = df_add(si, {v.z, v.w});
                }
                double2 *o = y + (size_t)(bj.start + j0 + src) * R + r0 + c;
                atomicAdd(&o->x, df_to_double(sr));
                atomicAdd(&o->y, df_to_double(si));
            }
        }
    }
    if (live) {
#pragma unroll
        for (int c = 0; c < RC; ++c)
            if (r0 + c < R) {
                double2 *o = y + (size_t)(bi.start + tid) * R + r0 + c;
                atomicAdd(&o->x, df_to_double(atr[c]));
                atomicAdd(&o->y, df_to_double(ati[c]));
            }
    }
}

__global__ void df_split_reduce_kernel(size_t n, int nsplit, const double2 *__restrict__ part, double2 *__restrict__ y)
{
    size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    double sx = 0.0, sy = 0.0;
    for (int s = 0; s < nsplit; ++s) {
        double2 v = part[s * n + e];
        sx += v.x;
        sy += v.y;
    }
    y[e] = make_double2(sx, sy);
}

static hzb_status ensure_df(hzb_ctx *c)
{
    if (c->df_ready) return HZB_OK;
    const size_t N = (size_t)c->N;
    if (check_cuda(c, c->dfa.ensure(N), "alloc") || check_cuda(c, c->dfb.ensure(N), "alloc") ||
        check_cuda(c, c->dfc.ensure(N), "alloc") || check_cuda(c, c->dftab.ensure(DF_TAB), "alloc"))
        return HZB_ENOMEM;
    df_nodes_kernel<<<(unsigned)((N + 255) / 256), 256, 0, c->stream>>>((long long)N, c->pos64.ptr, c->nrm64.ptr,
                                                                        c->center[0], c->center[1], c->center[2],
                                                                        c->dfa.ptr, c->dfb.ptr, c->dfc.ptr);
    std::vector<float4> tab(DF_TAB);
    for (int q = 0; q < DF_TAB; ++q) {
        dfl cc = df_from_double(std::cos(2.0 * M_PI * q / DF_TAB)), ss = df_from_double(std::sin(2.0 * M_PI * q / DF_TAB));
        tab[q] = make_float4(cc.hi, cc.lo, ss.hi, ss.lo);
    }
    if (check_cuda(c, cudaMemcpyAsync(c->dftab.ptr, tab.data(), DF_TAB * sizeof(float4), cudaMemcpyHostToDevice,
                                      c->stream), "copy table") ||
        check_cuda(c, cudaStreamSynchronize(c->stream), "df nodes"))
        return HZB_ECUDA;
    c->df_ready = true;
    return HZB_OK;
}

template <int RC, int TPT>
static void launch_df(hzb_ctx *c, dim3 g, int N, int R, int chunk, const double2 *s, double2 *o, size_t st, DfConst K)
{
    nbody_df_kernel<RC, TPT><<<g, DF_TBLOCK / TPT, 0, c->stream>>>(c->tblocks.ptr, N, R, chunk, c->dfa.ptr,
                                                                   c->dfb.ptr, c->dfc.ptr, c->pos64.ptr, s,
                                                                   c->dftab.ptr, K, o, st);
}

static DfConst df_constants(const hzb_ctx *c)
{
    DfConst K;
    K.k = df_from_double(c->k);
    K.eta = df_from_double(c->eta);
    K.inv2pi = df_from_double(1.0 / (2.0 * M_PI));
    K.twopi = df_from_double(2.0 * M_PI);
    K.inv6 = df_from_double(1.0 / 6.0);
    return K;
}

static hzb_status interbody_df_sym(hzb_ctx *c, int R, const double2 *sigma, double2 *y)
{
    if (c->capturing && c->n_blockpairs == 0) return fail(c, HZB_ESTATE, "block pairs not built before capture");
    hzb_status st = ensure_block_pairs(c);
    if (st) return st;
    const size_t n = (size_t)c->N * R;
    if (check_cuda(c, cudaMemsetAsync(y, 0, n * sizeof(double2), c->stream), "zero y")) return HZB_ECUDA;
    c->interbody_calls++;
    if (c->n_blockpairs < 0) return HZB_OK;
    if (c->n_blockpairs > 0x7fffffffLL) return fail(c, HZB_EINVAL, "too many block pairs for one launch");
    c->launches += 1;
    const DfConst K = df_constants(c);
    const int slot = prof_begin(c, 2);
    const int rc = (R == 1) ? 1 : 2;
    dim3 g((unsigned)c->n_blockpairs, (R + rc - 1) / rc, 1);
    if (rc == 1)
        nbody_df_sym_kernel<1><<<g, DFS_T, 0, c->stream>>>(c->blockpairs.ptr, c->tblocks.ptr, R, c->dfa.ptr, c->dfb.ptr,
                                                           c->dfc.ptr, c->pos64.ptr, sigma, c->dftab.ptr, K, y);
    else
        nbody_df_sym_kernel<2><<<g, DFS_T, 0, c->stream>>>(c->blockpairs.ptr, c->tblocks.ptr, R, c->dfa.ptr, c->dfb.ptr,
                                                           c->dfc.ptr, c->pos64.ptr, sigma, c->dftab.ptr, K, y);
    cudaError_t e = cudaGetLastError();
    prof_end(c, slot);
    return check_cuda(c, e, "nbody_df_sym_kernel");
}

hzb_status interbody_df(hzb_ctx *c, int R, const double2 *sigma, double2 *y)
{
    if (!c->nodes_ready) return fail(c, HZB_ESTATE, "nodes not built");
    hzb_status st = ensure_df(c);
    if (st) return st;
    if (c->nbody64_engine == 2 && R <= 4) return interbody_df_sym(c, R, sigma, y);
    if (c->nbody64_engine == 1 || (c->nbody64_engine < 0 && R <= 4)) return interbody_dfl_sym(c, R, sigma, y);
    if (c->nbody64_engine != 2) {
        const int ns = c->tunedf_split > 0 ? c->tunedf_split : dfl_default_nsplit(c, R);
        return interbody_dfl(c, R, sigma, y, ns);
    }
    const int N = (int)c->N;
    const int rc = R == 1 ? 1 : (R <= 4 ? 4 : 8);
    const int tpt = c->tunedf_tpt > 0 ? c->tunedf_tpt : 1;
    int nsplit = c->tunedf_split > 0 ? c->tunedf_split : default_nsplit(c, R, tpt == 1 ? 1 : 2);
    int chunk = (N + nsplit - 1) / nsplit;
    chunk = ((chunk + DF_TILE - 1) / DF_TILE) * DF_TILE;
    nsplit = (N + chunk - 1) / chunk;
    const size_t n = (size_t)N * R;
    double2 *out = y;
    if (nsplit > 1) {
        if (check_cuda(c, c->nb_part64.ensure(n * nsplit), "alloc partial sums")) return HZB_ENOMEM;
        out = c->nb_part64.ptr;
    }
    const DfConst K = df_constants(c);
    c->interbody_calls++;
    c->launches += (nsplit > 1) ? 2 : 1;
    const int slot = prof_begin(c, 2);
    const int nb = (c->tune_limit_blocks > 0) ? std::min(c->tune_limit_blocks, c->n_tblocks) : c->n_tblocks;
    dim3 g(nb, (R + rc - 1) / rc, nsplit);
    if (rc == 1) { if (tpt == 1) launch_df<1, 1>(c, g, N, R, chunk, sigma, out, n, K); else launch_df<1, 2>(c, g, N, R, chunk, sigma, out, n, K); }
    else if (rc == 4) { if (tpt == 1) launch_df<4, 1>(c, g, N, R, chunk, sigma, out, n, K); else launch_df<4, 2>(c, g, N, R, chunk, sigma, out, n, K); }
    else { if (tpt == 1) launch_df<8, 1>(c, g, N, R, chunk, sigma, out, n, K); else launch_df<8, 2>(c, g, N, R, chunk, sigma, out, n, K); }
    if (nsplit > 1) df_split_reduce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(n, nsplit, out, y);
    cudaError_t e = cudaGetLastError();
    prof_end(c, slot);
    return check_cuda(c, e, "nbody_df_kernel");
}

}  // namespace hzb
