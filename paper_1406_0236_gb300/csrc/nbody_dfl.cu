// Inter-body sum y = B sigma (Sec. 3.3, Eq. (nystromnaive)) in lean double-float
// arithmetic on the FP32 pipe: the refinement residual's sum of the mixed-precision
// solve at about the accuracy of FP64 (measured max-norm error against the oracle
// ~1e-13 of max |y|), without the FP64 pipe (1/64 of the FP32 rate on GB300).
//
// Each unordered pair of nodes on different bodies is evaluated once for both
// directions (the block-pair scheme of nbody_sym.cu: one CTA per pair of TargetBlocks,
// 32-source tiles met in 32 rotation steps, source-side sums moving one lane per step,
// FP64 atomic adds into y).  With d = x_i - x_j, r = |d|, E = e^{ikr}/r:
//     w_j K(x_i, x_j) sigma_j / (4 pi) ... = E [X_1 - i (k r X_1 + eta)] sigma'_j,  X_1 =  n_j.d / r^2,
//     w_i K(x_j, x_i) sigma_i / (4 pi) ... = E [X_2 - i (k r X_2 + eta)] sigma'_i,  X_2 = -n_i.d / r^2,
// sigma' = w sigma / (4 pi); E, r and k r are shared by the two directions.
//
// Arithmetic: lean double-float (lean_df.cuh): error-free products and sums left
// unnormalised, accumulators renormalised once per tile.  1/r: the hardware estimate of
// 1/sqrt(r^2) and one Halley step (cubic convergence, so the estimate's 2^-23 error falls
// below 2^-60).
// e^{i k r}: k r / (2 pi) in turns is reduced to [-1/2, 1/2] and then to the nearest of
// 1024 table angles (cos, sin in double-float, shared memory); the remainder
// |delta| <= pi / 1024 enters through cos(delta) - 1 = -delta^2/2 + delta^4/24 and
// sin(delta) = delta - delta^3/6 + delta^5/120 (truncation below 1e-17) and angle addition.
// The translation unit is compiled with -fmad=false so that the compiler never fuses
// the separately rounded operations these transformations depend on.
#include <algorithm>
#include <cmath>
#include <vector>

#include "hzb_internal.h"
#include "lean_df.cuh"

namespace hzb {

using namespace lean;

static const int DFL_T = 512;          // targets per CTA (= TargetBlock size)
static const int DFL_S = 32;           // sources per tile (one per lane)
static const int DFL_TAB = 1024;       // table angles 2 pi m / 1024

struct DflConst {
    dd k, kt, twopi, eta;              // k, k / (2 pi), 2 pi, eta
};

// e^{2 pi i theta} for theta (turns) with |theta| < 2^21, in double-float
__device__ __forceinline__ void dfl_cis(dd theta, const float4 *__restrict__ tab, const DflConst &K, dd &cs, dd &sn)
{
    const float MAGIC = 12582912.0f;                      // 1.5 * 2^23: adding it rounds to an integer
    const float n0 = (theta.h + MAGIC) - MAGIC;
    const float f = theta.h - n0;                         // exact, |f| <= 1/2
    const float tm = f * (float)DFL_TAB + MAGIC;          // f * 1024 is exact
    const float mf = tm - MAGIC;                          // nearest table index, as a float
    const int idx = __float_as_int(tm) & (DFL_TAB - 1);   // its low bits are the integer
    const float g = fmaf(mf, -1.0f / DFL_TAB, f);         // exact: |g| <= 1/2048 turns
    const dd del = mul(two_sum(g, theta.l), K.twopi);     // remainder in radians, |delta| <= pi/1024
    const float q = del.h * del.h;
    const float qe = fmaf(del.h + del.h, del.l, fmaf(del.h, del.h, -q));   // delta^2 = q + qe
    const dd cm = {-0.5f * q, fmaf(q, q * (1.0f / 24.0f), -0.5f * qe)};     // cos(delta) - 1
    const dd sd = {del.h, fmaf(del.h * q, fmaf(q, 1.0f / 120.0f, -1.0f / 6.0f), del.l)};   // sin(delta)
    const float4 T = tab[idx];
    const dd C = {T.x, T.y}, S = {T.z, T.w};
    cs = add(C, sub(mul(C, cm), mul(S, sd)));
    sn = add(S, add(mul(S, cm), mul(C, sd)));
}

// Source j of a tile, staged in shared memory: position and normal (hi, lo split as
// in the double-float node arrays) and sigma'_j for RC right-hand sides.
template <int RC>
struct DflTile {
    float4 a[DFL_S], b[DFL_S], c[DFL_S];
    float4 sig[DFL_S][RC];                                // re.hi, re.lo, im.hi, im.lo of sigma'
};

template <int RC>
__global__ void __launch_bounds__(DFL_T, 1)
nbody_dfl_sym_kernel(const int2 *__restrict__ pairs, const TargetBlock *__restrict__ blocks, int R,
                     const float4 *__restrict__ pa, const float4 *__restrict__ pb, const float4 *__restrict__ pc,
                     const double4 *__restrict__ pos64, const double2 *__restrict__ sigma,
                     const float4 *__restrict__ tab, DflConst K, double2 *__restrict__ y)
{
    __shared__ DflTile<RC> s_tile[2];                     // double-buffered source tiles
    __shared__ float4 s_tab[DFL_TAB];
    const int2 pr = pairs[blockIdx.x];
    const TargetBlock bi = blocks[pr.x], bj = blocks[pr.y];
    const int r0 = blockIdx.y * RC;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int q = tid; q < DFL_TAB; q += DFL_T) s_tab[q] = tab[q];
    const bool live = tid < bi.count;
    dd tx = {1e5f + tid, 0.f}, ty = {1e5f, 0.f}, tz = {1e5f, 0.f};
    dd mx = {0.f, 0.f}, my = {0.f, 0.f}, mz = {0.f, 0.f};
    dd wr[RC], wi[RC], atr[RC], ati[RC];
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
                const double vr = v.x * wq, vi = v.y * wq;
                wr[c] = {(float)vr, (float)(vr - (double)(float)vr)};
                wi[c] = {(float)vi, (float)(vi - (double)(float)vi)};
            }
    }
    // the first warp loads the next tile's sources into registers while the tile runs
    float4 na, nb, nc, ns[RC];
    auto fetch = [&](int j0) {
        const int cnt = min(DFL_S, bj.count - j0);
        if (lane < cnt) {
            const int g = bj.start + j0 + lane;
            na = pa[g]; nb = pb[g]; nc = pc[g];
            const double wq = pos64[g].w * 0.07957747154594767;
#pragma unroll
            for (int c = 0; c < RC; ++c) {
                const double2 v = (r0 + c < R) ? sigma[(size_t)g * R + r0 + c] : make_double2(0.0, 0.0);
                const double vr = v.x * wq, vi = v.y * wq;
                const float hr = (float)vr, hi = (float)vi;
                ns[c] = make_float4(hr, (float)(vr - (double)hr), hi, (float)(vi - (double)hi));
            }
        } else {                                           // far, zero density: contributes 0 both ways
            na = make_float4(-1e5f - lane, -1e5f, -1e5f, 0.f);
            nb = nc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int c = 0; c < RC; ++c) ns[c] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };
    auto stage = [&](DflTile<RC> &T) {
        T.a[lane] = na; T.b[lane] = nb; T.c[lane] = nc;
#pragma unroll
        for (int c = 0; c < RC; ++c) T.sig[lane][c] = ns[c];
    };
    if (warp == 0) {
        fetch(0);
        stage(s_tile[0]);
        if (DFL_S < bj.count) fetch(DFL_S);
    }
    const bool warp_live = warp * 32 < bi.count;
    int buf = 0;
    for (int j0 = 0; j0 < bj.count; j0 += DFL_S, buf ^= 1) {
        const int cnt = min(DFL_S, bj.count - j0);
        __syncthreads();                                   // tile j0 staged; the other buffer is free
        if (warp == 0 && j0 + DFL_S < bj.count) {
            stage(s_tile[buf ^ 1]);
            if (j0 + 2 * DFL_S < bj.count) fetch(j0 + 2 * DFL_S);
        }
        if (!warp_live) continue;
        const DflTile<RC> &T = s_tile[buf];
        dd asr[RC], asi[RC];
#pragma unroll
        for (int c = 0; c < RC; ++c) asr[c] = asi[c] = {0.f, 0.f};
        for (int s = 0; s < DFL_S; ++s) {
            const int q = (lane + s) & (DFL_S - 1);
            const float4 A4 = T.a[q], B4 = T.b[q], C4 = T.c[q];
            // d = x_i - x_j
            const dd dx = sub(tx, {A4.x, B4.x}), dy = sub(ty, {A4.y, B4.y}), dz = sub(tz, {A4.z, B4.z});
            // r^2 from exact squares; the sums of the positive squares in fast_two_sum order
            const float px = dx.h * dx.h, py = dy.h * dy.h, pz = dz.h * dz.h;
            const float ex = fmaf(dx.h + dx.h, dx.l, fmaf(dx.h, dx.h, -px));
            const float ey = fmaf(dy.h + dy.h, dy.l, fmaf(dy.h, dy.h, -py));
            const float ez = fmaf(dz.h + dz.h, dz.l, fmaf(dz.h, dz.h, -pz));
            const float m1 = fmaxf(px, py), l1 = fminf(px, py);
            const float s1 = m1 + l1, e1 = l1 - (s1 - m1);
            const float m2 = fmaxf(s1, pz), l2 = fminf(s1, pz);
            const float s2 = m2 + l2, e2 = l2 - (s2 - m2);
            const dd r2 = {s2, (e1 + e2) + ((ex + ey) + ez)};
            // 1/r: hardware estimate y0, Halley step y0 (1 + e/2 + 3 e^2/8), e = 1 - r^2 y0^2
            const float y0 = rsqrtf(r2.h);
            const float q0 = y0 * y0, q0e = fmaf(y0, y0, -q0);
            const float u = r2.h * q0;
            const float ue = fmaf(r2.l, q0, fmaf(r2.h, q0e, fmaf(r2.h, q0, -u)));
            const float e = (1.0f - u) - ue;
            const dd ir = {y0, y0 * e * fmaf(e, 0.375f, 0.5f)};
            const dd r = mul(r2, ir);
            const dd ir2 = mul(ir, ir);
            const dd kr = mul(K.k, r);
            dd cs, sn;
            dfl_cis(mul(K.kt, r), s_tab, K, cs, sn);
            // E = e^{ikr} / r; G = E [X - i (k r X + eta)] = X P + Q with
            // P = E (1 - i k r), Q = -i eta E, shared by both directions
            const dd Er = mul(cs, ir), Ei = mul(sn, ir);
            const dd Pr = add(Er, mul(Ei, kr)), Pi = sub(Ei, mul(Er, kr));
            const dd Qr = mul(K.eta, Ei), Qi = neg(mul(K.eta, Er));
            // i <- j: normal of source j
            const dd nx = {A4.w, B4.w}, ny = {C4.x, C4.z}, nz = {C4.y, C4.w};
            const dd X1 = mul(add(add(mul(nx, dx), mul(ny, dy)), mul(nz, dz)), ir2);
            const dd g1r = add(mul(X1, Pr), Qr), g1i = add(mul(X1, Pi), Qi);
            // j <- i: normal of target i, d reversed
            const dd X2 = neg(mul(add(add(mul(mx, dx), mul(my, dy)), mul(mz, dz)), ir2));
            const dd g2r = add(mul(X2, Pr), Qr), g2i = add(mul(X2, Pi), Qi);
#pragma unroll
            for (int c = 0; c < RC; ++c) {
                const float4 S = T.sig[q][c];
                const dd sr = {S.x, S.y}, si = {S.z, S.w};
                atr[c] = add(atr[c], sub(mul(g1r, sr), mul(g1i, si)));
                ati[c] = add(ati[c], add(mul(g1r, si), mul(g1i, sr)));
                asr[c] = add(asr[c], sub(mul(g2r, wr[c]), mul(g2i, wi[c])));
                asi[c] = add(asi[c], add(mul(g2r, wi[c]), mul(g2i, wr[c])));
            }
#pragma unroll
            for (int c = 0; c < RC; ++c) {
                const int from = (lane + 1) & 31;
                asr[c].h = __shfl_sync(0xffffffffu, asr[c].h, from);
                asr[c].l = __shfl_sync(0xffffffffu, asr[c].l, from);
                asi[c].h = __shfl_sync(0xffffffffu, asi[c].h, from);
                asi[c].l = __shfl_sync(0xffffffffu, asi[c].l, from);
            }
        }
#pragma unroll
        for (int c = 0; c < RC; ++c) { atr[c] = norm(atr[c]); ati[c] = norm(ati[c]); }
        // after 32 steps lane l holds this warp's sum for source l: straight into y
        if (lane < cnt) {
#pragma unroll
            for (int c = 0; c < RC; ++c)
                if (r0 + c < R) {
                    double2 *o = y + (size_t)(bj.start + j0 + lane) * R + r0 + c;
                    atomicAdd(&o->x, (double)asr[c].h + (double)asr[c].l);
                    atomicAdd(&o->y, (double)asi[c].h + (double)asi[c].l);
                }
        }
    }
    if (live) {
#pragma unroll
        for (int c = 0; c < RC; ++c)
            if (r0 + c < R) {
                double2 *o = y + (size_t)(bi.start + tid) * R + r0 + c;
                atomicAdd(&o->x, (double)atr[c].h + (double)atr[c].l);
                atomicAdd(&o->y, (double)ati[c].h + (double)ati[c].l);
            }
    }
}

// One-directional form for several right-hand sides (the refinement residual of a
// batched solve): one CTA per (TargetBlock part, chunk of RC right-hand sides, source
// chunk); a CTA of NT threads owns NT targets of a 512-target block (512 / NT CTAs per
// block), one per thread; sources in tiles of DFL_OT staged in shared memory.  Per
// ordered pair the geometry, e^{ikr} and the kernel value
//     G = E [X - i (k r X + eta)],  E = e^{ikr} / r,  X = n_j.d / r^2
// are formed once and serve the RC right-hand sides (a double-float complex
// multiply-add each, ~48 FP32 operations against ~240 for the pair), so wide chunks
// (RC = 16 with 512 threads, RC = 32 with 256 threads and up to 255 registers) repeat
// the pair work least.  Source chunks write partial sums that a second kernel adds in a
// fixed order, so the result is bit-reproducible.
static const int DFL_OT = 64;

template <int RC, int NT>
__global__ void __launch_bounds__(NT, 1)
nbody_dfl_kernel(const TargetBlock *__restrict__ blocks, int N, int R, int chunk, const float4 *__restrict__ pa,
                 const float4 *__restrict__ pb, const float4 *__restrict__ pc, const double4 *__restrict__ pos64,
                 const double2 *__restrict__ sigma, const float4 *__restrict__ tab, DflConst K,
                 double2 *__restrict__ y, size_t split_stride)
{
    constexpr int PARTS = DFL_T / NT;
    constexpr int OT = RC >= 32 ? DFL_OT / 2 : DFL_OT;   // source tile: static shared memory under 48 KB
    __shared__ float4 s_a[OT], s_b[OT], s_c[OT];
    __shared__ float4 s_sig[OT][RC];
    __shared__ float4 s_tab[DFL_TAB];
    const TargetBlock tb = blocks[blockIdx.x / PARTS];
    const int t0 = (blockIdx.x % PARTS) * NT;
    const int r0 = blockIdx.y * RC;
    const int tid = threadIdx.x;
    for (int q = tid; q < DFL_TAB; q += NT) s_tab[q] = tab[q];
    const int g0 = tb.start + min(t0 + tid, tb.count - 1);
    const float4 TA = pa[g0], TB = pb[g0];
    const dd tx = {TA.x, TB.x}, ty = {TA.y, TB.y}, tz = {TA.z, TB.z};
    dd ar[RC], ai[RC];
#pragma unroll
    for (int c = 0; c < RC; ++c) ar[c] = ai[c] = {0.f, 0.f};
    const int c0 = blockIdx.z * chunk, c1 = min(N, c0 + chunk);
    for (int range = 0; range < 2; ++range) {
        const int lo = range ? max(c0, tb.excl_hi) : c0;
        const int hi = range ? c1 : min(c1, tb.excl_lo);
        for (int j0 = lo; j0 < hi; j0 += OT) {
            const int cnt = min(OT, hi - j0);
            __syncthreads();
            for (int q = tid; q < cnt; q += NT) {
                const int g = j0 + q;
                s_a[q] = pa[g];
                s_b[q] = pb[g];
                s_c[q] = pc[g];
                const double wq = pos64[g].w * 0.07957747154594767;
#pragma unroll
                for (int c = 0; c < RC; ++c) {
                    const double2 v = (r0 + c < R) ? sigma[(size_t)g * R + r0 + c] : make_double2(0.0, 0.0);
                    const double vr = v.x * wq, vi = v.y * wq;
                    const float hr = (float)vr, hi2 = (float)vi;
                    s_sig[q][c] = make_float4(hr, (float)(vr - (double)hr), hi2, (float)(vi - (double)hi2));
                }
            }
            __syncthreads();
            for (int jj = 0; jj < cnt; ++jj) {
                const float4 A4 = s_a[jj], B4 = s_b[jj], C4 = s_c[jj];
                const dd dx = sub(tx, {A4.x, B4.x}), dy = sub(ty, {A4.y, B4.y}), dz = sub(tz, {A4.z, B4.z});
                const float px = dx.h * dx.h, py = dy.h * dy.h, pz = dz.h * dz.h;
                const float ex = fmaf(dx.h + dx.h, dx.l, fmaf(dx.h, dx.h, -px));
                const float ey = fmaf(dy.h + dy.h, dy.l, fmaf(dy.h, dy.h, -py));
                const float ez = fmaf(dz.h + dz.h, dz.l, fmaf(dz.h, dz.h, -pz));
                const float m1 = fmaxf(px, py), l1 = fminf(px, py);
                const float s1 = m1 + l1, e1 = l1 - (s1 - m1);
                const float m2 = fmaxf(s1, pz), l2 = fminf(s1, pz);
                const float s2 = m2 + l2, e2 = l2 - (s2 - m2);
                const dd r2 = {s2, (e1 + e2) + ((ex + ey) + ez)};
                const float y0 = rsqrtf(r2.h);
                const float q0 = y0 * y0, q0e = fmaf(y0, y0, -q0);
                const float u = r2.h * q0;
                const float ue = fmaf(r2.l, q0, fmaf(r2.h, q0e, fmaf(r2.h, q0, -u)));
                const float e = (1.0f - u) - ue;
                const dd ir = {y0, y0 * e * fmaf(e, 0.375f, 0.5f)};
                const dd r = mul(r2, ir);
                const dd kr = mul(K.k, r);
                dd cs, sn;
                dfl_cis(mul(K.kt, r), s_tab, K, cs, sn);
                const dd Er = mul(cs, ir), Ei = mul(sn, ir);
                const dd nx = {A4.w, B4.w}, ny = {C4.x, C4.z}, nz = {C4.y, C4.w};
                const dd X = mul(add(add(mul(nx, dx), mul(ny, dy)), mul(nz, dz)), mul(ir, ir));
                const dd Bv = add(mul(kr, X), K.eta);
                const dd gr = add(mul(Er, X), mul(Ei, Bv)), gi = sub(mul(Ei, X), mul(Er, Bv));
#pragma unroll
                for (int c = 0; c < RC; ++c) {
                    const float4 S = s_sig[jj][c];
                    const dd sr = {S.x, S.y}, si = {S.z, S.w};
                    ar[c] = add(ar[c], sub(mul(gr, sr), mul(gi, si)));
                    ai[c] = add(ai[c], add(mul(gr, si), mul(gi, sr)));
                }
            }
#pragma unroll
            for (int c = 0; c < RC; ++c) { ar[c] = norm(ar[c]); ai[c] = norm(ai[c]); }
        }
    }
    if (t0 + tid < tb.count) {
        double2 *yo = y + blockIdx.z * split_stride;
#pragma unroll
        for (int c = 0; c < RC; ++c)
            if (r0 + c < R)
                yo[(size_t)(tb.start + t0 + tid) * R + r0 + c] =
                    make_double2((double)ar[c].h + (double)ar[c].l, (double)ai[c].h + (double)ai[c].l);
    }
}

__global__ void dfl_split_reduce_kernel(size_t n, int nsplit, const double2 *__restrict__ part,
                                        double2 *__restrict__ y)
{
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    double sx = 0.0, sy = 0.0;
    for (int s = 0; s < nsplit; ++s) {
        const double2 v = part[s * n + e];
        sx += v.x;
        sy += v.y;
    }
    y[e] = make_double2(sx, sy);
}

// cos/sin(2 pi m / 1024) split into double-float, built once per context
static hzb_status ensure_dfl_table(hzb_ctx *c)
{
    if (c->dfltab_ready) return HZB_OK;
    if (check_cuda(c, c->dfltab.ensure(DFL_TAB), "alloc table")) return HZB_ENOMEM;
    std::vector<float4> tab(DFL_TAB);
    for (int q = 0; q < DFL_TAB; ++q) {
        const long double a = 2.0L * 3.14159265358979323846264338327950288L * q / DFL_TAB;
        const double cv = (double)cosl(a), sv = (double)sinl(a);
        const float ch = (float)cv, sh = (float)sv;
        tab[q] = make_float4(ch, (float)(cv - (double)ch), sh, (float)(sv - (double)sh));
    }
    if (check_cuda(c, cudaMemcpyAsync(c->dfltab.ptr, tab.data(), DFL_TAB * sizeof(float4), cudaMemcpyHostToDevice,
                                      c->stream), "copy table") ||
        check_cuda(c, cudaStreamSynchronize(c->stream), "table"))
        return HZB_ECUDA;
    c->dfltab_ready = true;
    return HZB_OK;
}

static dd dd_of(double v)
{
    const float h = (float)v;
    return {h, (float)(v - (double)h)};
}

static DflConst dfl_constants(const hzb_ctx *c)
{
    DflConst K;
    K.k = dd_of(c->k);
    K.kt = dd_of(c->k / (2.0 * M_PI));
    K.twopi = dd_of(2.0 * M_PI);
    K.eta = dd_of(c->eta);
    return K;
}

// right-hand sides per CTA of the one-directional kernel
int dfl_rc(int R) { return R == 1 ? 1 : (R <= 4 ? 4 : (R <= 8 ? 8 : (R <= 16 ? 16 : 32))); }

// source chunks of the one-directional kernel: about four CTAs per SM in all (one is
// resident at a time: 512 threads at <= 128 registers, or 256 at <= 255)
int dfl_default_nsplit(hzb_ctx *c, int R)
{
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->opt.device);
    const int rc = dfl_rc(R), nt = rc == 32 ? 256 : 512;
    const long long ctas = std::max<long long>(1, (long long)c->n_tblocks * (DFL_T / nt) * ((R + rc - 1) / rc));
    const long long ns = (4LL * sms + ctas - 1) / ctas;
    return (int)std::min<long long>(64, std::max<long long>(1, ns));
}

// one-directional lean double-float sum (R right-hand sides in chunks of 1, 4, 8, 16 or
// 32, source chunks for occupancy, added in a fixed order); node arrays as for the
// symmetric form
hzb_status interbody_dfl(hzb_ctx *c, int R, const double2 *sigma, double2 *y, int nsplit)
{
    hzb_status st = ensure_dfl_table(c);
    if (st) return st;
    const int N = (int)c->N;
    const int rc = dfl_rc(R);
    int chunk = (N + nsplit - 1) / nsplit;
    chunk = ((chunk + DFL_OT - 1) / DFL_OT) * DFL_OT;
    nsplit = (N + chunk - 1) / chunk;
    const size_t n = (size_t)N * R;
    double2 *out = y;
    if (nsplit > 1) {
        if (check_cuda(c, c->nb_part64.ensure(n * nsplit), "alloc partial sums")) return HZB_ENOMEM;
        out = c->nb_part64.ptr;
    }
    const DflConst K = dfl_constants(c);
    c->interbody_calls++;
    c->launches += (nsplit > 1) ? 2 : 1;
    const int slot = prof_begin(c, 2);
    const int nb = (c->tune_limit_blocks > 0) ? std::min(c->tune_limit_blocks, c->n_tblocks - c->tblock_off)
                                              : c->n_tblocks - c->tblock_off;
    const TargetBlock *tb = c->tblocks.ptr + c->tblock_off;
    auto launch = [&](auto kern, int nt) {
        dim3 g((unsigned)(nb * (DFL_T / nt)), (R + rc - 1) / rc, nsplit);
        kern<<<g, nt, 0, c->stream>>>(tb, N, R, chunk, c->dfa.ptr, c->dfb.ptr, c->dfc.ptr, c->pos64.ptr, sigma,
                                      c->dfltab.ptr, K, out, n);
    };
    switch (rc) {
    case 1: launch(nbody_dfl_kernel<1, 512>, 512); break;
    case 4: launch(nbody_dfl_kernel<4, 512>, 512); break;
    case 8: launch(nbody_dfl_kernel<8, 512>, 512); break;
    case 16: launch(nbody_dfl_kernel<16, 512>, 512); break;
    default: launch(nbody_dfl_kernel<32, 256>, 256); break;
    }
    if (nsplit > 1) dfl_split_reduce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(n, nsplit, out, y);
    cudaError_t e = cudaGetLastError();
    prof_end(c, slot);
    return check_cuda(c, e, "nbody_dfl_kernel");
}

// pair-symmetric lean double-float sum; the split node arrays (dfa, dfb, dfc) come from
// the double-float set-up of nbody_df.cu (ensure_df), which the caller has run
hzb_status interbody_dfl_sym(hzb_ctx *c, int R, const double2 *sigma, double2 *y)
{
    if (c->capturing && (c->n_blockpairs == 0 || !c->dfltab_ready))
        return fail(c, HZB_ESTATE, "block pairs or table not built before capture");
    hzb_status st = ensure_block_pairs(c);
    if (st) return st;
    if ((st = ensure_dfl_table(c))) return st;
    const size_t n = (size_t)c->N * R;
    if (check_cuda(c, cudaMemsetAsync(y, 0, n * sizeof(double2), c->stream), "zero y")) return HZB_ECUDA;
    c->interbody_calls++;
    if (c->n_blockpairs < 0) return HZB_OK;
    if (c->n_blockpairs > 0x7fffffffLL) return fail(c, HZB_EINVAL, "too many block pairs for one launch");
    c->launches += 1;
    const DflConst K = dfl_constants(c);
    const int slot = prof_begin(c, 2);
    const int rc = (R == 1) ? 1 : 2;
    dim3 g((unsigned)c->n_blockpairs, (R + rc - 1) / rc, 1);
    if (rc == 1)
        nbody_dfl_sym_kernel<1><<<g, DFL_T, 0, c->stream>>>(c->blockpairs.ptr, c->tblocks.ptr, R, c->dfa.ptr,
                                                            c->dfb.ptr, c->dfc.ptr, c->pos64.ptr, sigma,
                                                            c->dfltab.ptr, K, y);
    else
        nbody_dfl_sym_kernel<2><<<g, DFL_T, 0, c->stream>>>(c->blockpairs.ptr, c->tblocks.ptr, R, c->dfa.ptr,
                                                            c->dfb.ptr, c->dfc.ptr, c->pos64.ptr, sigma,
                                                            c->dfltab.ptr, K, y);
    cudaError_t e = cudaGetLastError();
    prof_end(c, slot);
    return check_cuda(c, e, "nbody_dfl_sym_kernel");
}

}  // namespace hzb
