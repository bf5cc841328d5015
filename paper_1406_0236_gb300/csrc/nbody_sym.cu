// FP64 inter-body sum y = B sigma (Sec. 3.3, Eq. (nystromnaive)) with each unordered
// pair of nodes on different bodies evaluated once for both directions.
//
// For nodes i, j with d = x_i - x_j, r = |d|:
//     w_j K(x_i, x_j) = w_j / (4 pi) e^{ikr} [ n_j.d / r^3 - i (k n_j.d / r^2 + eta / r) ]
//     w_i K(x_j, x_i) = w_i / (4 pi) e^{ikr} [-n_i.d / r^3 - i (-k n_i.d / r^2 + eta / r) ]
// share d, r, 1/r and e^{ikr}, which are two thirds of the FP64 work of a pair; the
// two directions differ only in the normal projection.  About 27.5 FP64 operations
// per ordered pair instead of 41 for the one-directional kernel (nbody64_kernel).
//
// Work: one CTA per unordered pair of TargetBlocks (I, J), I < J, on different
// bodies (grid y: chunks of RC right-hand sides).  Thread t owns target i = I.start + t;
// sources of J come in tiles of 32.  Inside a warp the 32 x 32 pairs of a tile run in
// 32 steps: at step s lane l takes source (l + s) mod 32, adds the i <- j term to its
// own sum and the j <- i term to a rotating sum that then moves to lane l - 1, so each
// source's partial sum visits every lane once and no two lanes touch the same source
// at a step.  The warps' partial sums of a tile are added in a fixed order in shared
// memory.  Both directions reach y through FP64 atomic adds (y is zeroed first), so
// the order of the additions into one y entry varies between runs: the result is
// reproducible to rounding, not bit for bit.
#include <algorithm>
#include <vector>

#include "f32x2.cuh"
#include "fp64_pair.cuh"
#include "hzb_internal.h"
#include "kernel_math.cuh"

namespace hzb {

static const int SYM_T = 512;        // targets per CTA = TargetBlock size
static const int SYM_S = 32;         // sources per tile (one per lane)

template <int RC>
__global__ void __launch_bounds__(SYM_T, 1)
nbody64_sym_kernel(const int2 *__restrict__ pairs, const TargetBlock *__restrict__ blocks, int R,
                   const double4 *__restrict__ pos, const double4 *__restrict__ nrm,
                   const double2 *__restrict__ sigma, const double2 *__restrict__ sctab, double k, double eta,
                   double kt, double2 *__restrict__ y)
{
    __shared__ double4 s_p[SYM_S];               // x, y, z, w
    __shared__ double4 s_n[SYM_S];               // nx, ny, nz
    __shared__ double2 s_w[SYM_S][RC];           // w_j sigma_j / (4 pi)
    __shared__ double2 s_red[SYM_T / 32][RC][SYM_S];
    const int2 pr = pairs[blockIdx.x];
    const TargetBlock bi = blocks[pr.x], bj = blocks[pr.y];
    const int r0 = blockIdx.y * RC;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool live = tid < bi.count;
    // own target: position, normal, weighted densities (zero for padding threads)
    double tx = 1e6 + tid, ty = 1e6, tz = 1e6, mx = 0.0, my = 0.0, mz = 0.0;
    double2 wi[RC], acc_t[RC];
    if (live) {
        const double4 p = pos[bi.start + tid], n = nrm[bi.start + tid];
        tx = p.x; ty = p.y; tz = p.z; mx = n.x; my = n.y; mz = n.z;
        const double wq = p.w * HZB_INV4PI;
#pragma unroll
        for (int c = 0; c < RC; ++c) {
            const double2 v = (r0 + c < R) ? sigma[(size_t)(bi.start + tid) * R + r0 + c] : make_double2(0.0, 0.0);
            wi[c] = make_double2(v.x * wq, v.y * wq);
        }
    } else {
#pragma unroll
        for (int c = 0; c < RC; ++c) wi[c] = make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int c = 0; c < RC; ++c) acc_t[c] = make_double2(0.0, 0.0);
    const bool warp_live = warp * 32 < bi.count;
    const double eta_ = eta;
    for (int j0 = 0; j0 < bj.count; j0 += SYM_S) {
        const int cnt = min(SYM_S, bj.count - j0);
        __syncthreads();
        if (tid < SYM_S) {
            if (tid < cnt) {
                const double4 p = pos[bj.start + j0 + tid];
                s_p[tid] = p;
                s_n[tid] = nrm[bj.start + j0 + tid];
                const double wq = p.w * HZB_INV4PI;
#pragma unroll
                for (int c = 0; c < RC; ++c) {
                    const double2 v =
                        (r0 + c < R) ? sigma[(size_t)(bj.start + j0 + tid) * R + r0 + c] : make_double2(0.0, 0.0);
                    s_w[tid][c] = make_double2(v.x * wq, v.y * wq);
                }
            } else {                                   // far, zero density: contributes 0 both ways
                s_p[tid] = make_double4(-1e6 - tid, -1e6, -1e6, 0.0);
                s_n[tid] = make_double4(0.0, 0.0, 0.0, 0.0);
#pragma unroll
                for (int c = 0; c < RC; ++c) s_w[tid][c] = make_double2(0.0, 0.0);
            }
        }
        __syncthreads();
        double2 acc_s[RC];
#pragma unroll
        for (int c = 0; c < RC; ++c) acc_s[c] = make_double2(0.0, 0.0);
        if (warp_live) {
#pragma unroll 2
            for (int s = 0; s < SYM_S; ++s) {
                const int q = (lane + s) & (SYM_S - 1);
                const double4 p = s_p[q];
                const double4 n = s_n[q];
                const double dx = tx - p.x, dy = ty - p.y, dz = tz - p.z;
                const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
                const double ir = rsqrt_fp64(r2);
                const double ir2 = ir * ir, eir = eta_ * ir;
                double sn, cs;
                cis_turns((r2 * ir) * kt, sctab, cs, sn);
                // i <- j: normal of source j
                const double X1 = fma(n.x, dx, fma(n.y, dy, n.z * dz)) * ir2;
                const double A1 = X1 * ir, B1 = fma(k, X1, eir);
                const double g1r = fma(cs, A1, sn * B1), g1i = fma(sn, A1, -cs * B1);
                // j <- i: normal of target i, d reversed (X2 = -X2p)
                const double X2p = fma(mx, dx, fma(my, dy, mz * dz)) * ir2;
                const double A2n = X2p * ir, B2 = fma(-k, X2p, eir);
                const double g2r = fma(-cs, A2n, sn * B2);            // Re K(x_j, x_i) w
                const double h = fma(sn, A2n, cs * B2);                 // -Im K(x_j, x_i) w
#pragma unroll
                for (int c = 0; c < RC; ++c) {
                    const double2 wj = s_w[q][c];
                    acc_t[c].x = fma(g1r, wj.x, fma(-g1i, wj.y, acc_t[c].x));
                    acc_t[c].y = fma(g1r, wj.y, fma(g1i, wj.x, acc_t[c].y));
                    acc_s[c].x = fma(g2r, wi[c].x, fma(h, wi[c].y, acc_s[c].x));
                    acc_s[c].y = fma(g2r, wi[c].y, fma(-h, wi[c].x, acc_s[c].y));
                }
                // the rotating sum of source (l + s + 1) mod 32 comes from lane l + 1
#pragma unroll
                for (int c = 0; c < RC; ++c) {
                    acc_s[c].x = __shfl_sync(0xffffffffu, acc_s[c].x, (lane + 1) & 31);
                    acc_s[c].y = __shfl_sync(0xffffffffu, acc_s[c].y, (lane + 1) & 31);
                }
            }
        }
        // after 32 steps lane l holds the partial sum of source l
#pragma unroll
        for (int c = 0; c < RC; ++c) s_red[warp][c][lane] = acc_s[c];
        __syncthreads();
        if (tid < SYM_S * RC) {
            const int src = tid & (SYM_S - 1), c = tid / SYM_S;
            if (src < cnt && r0 + c < R) {
                double sx = 0.0, sy = 0.0;
                for (int w = 0; w < SYM_T / 32; ++w) {
                    sx += s_red[w][c][src].x;
                    sy += s_red[w][c][src].y;
                }
                double2 *o = y + (size_t)(bj.start + j0 + src) * R + r0 + c;
                atomicAdd(&o->x, sx);
                atomicAdd(&o->y, sy);
            }
        }
    }
    if (live) {
#pragma unroll
        for (int c = 0; c < RC; ++c)
            if (r0 + c < R) {
                double2 *o = y + (size_t)(bi.start + tid) * R + r0 + c;
                atomicAdd(&o->x, acc_t[c].x);
                atomicAdd(&o->y, acc_t[c].y);
            }
    }
}

// FP32 version for the inner solve, with packed f32x2 pairs (f32x2.cuh): thread t
// owns TP pairs of targets (t + 2p NT, t + (2p + 1) NT), packed in the two halves of
// each register pair, and meets one source per step as above, so one f32x2
// instruction serves two unordered node pairs.  The rotating source sums keep the
// two halves apart and add them at the end of the tile.  Densities come pre-weighted
// in FP32 (weighted_sigma32).  With E = e^{ikr}/r, both directions' kernels are
// G = X P + Q, P = E (1 - ikr), Q = -i eta E (X = n.d / r^2 with the source-side normal),
// so that P and Q, computed once per node pair, leave two FMAs per direction;
// e^{ikr} comes straight from the transcendental unit (its own argument scaling).
// One right-hand side with two packed target pairs per thread is held to 80 registers (a
// few bytes of spills): six 128-thread CTAs per SM (24 warps) hide more of the FMA and
// transcendental-unit latency than five at 96 registers, four at 120 or seven at 72 with
// more spills (36.8 / 37.5 / 38.6 / 39.3 ms on 258,560 unknowns).
static constexpr int SYM32_MIN_BLOCKS = 6;
template <int RC, int TP>
__global__ void __launch_bounds__(SYM_T / (2 * TP), (RC == 1 && TP == 2) ? SYM32_MIN_BLOCKS : 1)
nbody32_sym_kernel(const int2 *__restrict__ pairs, const TargetBlock *__restrict__ blocks, int R,
                   const float4 *__restrict__ pos, const float4 *__restrict__ nrm, const float2 *__restrict__ sw,
                   float k, float eta, float kt, double2 *__restrict__ y)
{
    constexpr int NT = SYM_T / (2 * TP);
    constexpr int NW = NT / 32;
    __shared__ float4 s_g0[SYM_S];               // x, y, z, nx
    __shared__ float2 s_g1[SYM_S];               // ny, nz
    __shared__ float2 s_w[SYM_S][RC];
    __shared__ float2 s_red[NW][RC][SYM_S];
    const int2 pr = pairs[blockIdx.x];
    const TargetBlock bi = blocks[pr.x], bj = blocks[pr.y];
    const int r0 = blockIdx.y * RC;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    f2x tx[TP], ty[TP], tz[TP], mx[TP], my[TP], mz[TP];      // target positions, negated normals
    f2x wr[TP][RC], wi[TP][RC], nwi[TP][RC], atx[TP][RC], aty[TP][RC];
#pragma unroll
    for (int p = 0; p < TP; ++p) {
        float4 P[2], Q[2];
        float2 V[2][RC];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int t = tid + (2 * p + h) * NT;
            const bool live = t < bi.count;
            P[h] = live ? pos[bi.start + t] : make_float4(1e5f + t, 1e5f, 1e5f, 0.f);
            Q[h] = live ? nrm[bi.start + t] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int c = 0; c < RC; ++c)
                V[h][c] = (live && r0 + c < R) ? sw[(size_t)(bi.start + t) * R + r0 + c] : make_float2(0.f, 0.f);
        }
        tx[p] = f2_pack(P[0].x, P[1].x); ty[p] = f2_pack(P[0].y, P[1].y); tz[p] = f2_pack(P[0].z, P[1].z);
        mx[p] = f2_pack(-Q[0].x, -Q[1].x); my[p] = f2_pack(-Q[0].y, -Q[1].y); mz[p] = f2_pack(-Q[0].z, -Q[1].z);
#pragma unroll
        for (int c = 0; c < RC; ++c) {
            wr[p][c] = f2_pack(V[0][c].x, V[1][c].x);
            wi[p][c] = f2_pack(V[0][c].y, V[1][c].y);
            nwi[p][c] = f2_pack(-V[0][c].y, -V[1][c].y);
            atx[p][c] = aty[p][c] = 0ull;
        }
    }
    const bool warp_live = warp * 32 < bi.count;
    const f2x k2 = f2_splat(k), nk2 = f2_splat(-k), eta2 = f2_splat(eta), neta2 = f2_splat(-eta);
    for (int j0 = 0; j0 < bj.count; j0 += SYM_S) {
        const int cnt = min(SYM_S, bj.count - j0);
        __syncthreads();
        if (tid < SYM_S) {
            if (tid < cnt) {
                const float4 p = pos[bj.start + j0 + tid], n = nrm[bj.start + j0 + tid];
                s_g0[tid] = make_float4(p.x, p.y, p.z, n.x);
                s_g1[tid] = make_float2(n.y, n.z);
#pragma unroll
                for (int c = 0; c < RC; ++c)
                    s_w[tid][c] = (r0 + c < R) ? sw[(size_t)(bj.start + j0 + tid) * R + r0 + c] : make_float2(0.f, 0.f);
            } else {                                   // far, zero density: contributes 0 both ways
                s_g0[tid] = make_float4(-1e5f - tid, -1e5f, -1e5f, 0.f);
                s_g1[tid] = make_float2(0.f, 0.f);
#pragma unroll
                for (int c = 0; c < RC; ++c) s_w[tid][c] = make_float2(0.f, 0.f);
            }
        }
        __syncthreads();
        f2x asx[RC], asy[RC];
#pragma unroll
        for (int c = 0; c < RC; ++c) asx[c] = asy[c] = 0ull;
        if (warp_live) {
#pragma unroll 2
            for (int s = 0; s < SYM_S; ++s) {
                const int q = (lane + s) & (SYM_S - 1);
                const float4 g0 = s_g0[q];
                const float2 g1 = s_g1[q];
                const f2x sx = f2_splat(g0.x), sy = f2_splat(g0.y), sz = f2_splat(g0.z);
                const f2x snx = f2_splat(g0.w), sny = f2_splat(g1.x), snz = f2_splat(g1.y);
                f2x swr[RC], swi[RC], nswi[RC];
#pragma unroll
                for (int c = 0; c < RC; ++c) {
                    const float2 v = s_w[q][c];
                    swr[c] = f2_splat(v.x); swi[c] = f2_splat(v.y); nswi[c] = f2_splat(-v.y);
                }
#pragma unroll
                for (int p = 0; p < TP; ++p) {
                    const f2x dx = f2_sub(tx[p], sx), dy = f2_sub(ty[p], sy), dz = f2_sub(tz[p], sz);
                    const f2x r2 = f2_fma(dx, dx, f2_fma(dy, dy, f2_mul(dz, dz)));
                    float r2a, r2b;
                    f2_unpack(r2, r2a, r2b);
                    const f2x ir = f2_pack(rsqrtf(r2a), rsqrtf(r2b));
                    const f2x ir2 = f2_mul(ir, ir);
                    const f2x r = f2_mul(r2, ir);
                    const f2x kr = f2_mul(r, k2), nkr = f2_mul(r, nk2);
                    // e^{ikr}: the transcendental unit reduces the argument itself (its
                    // scaling to turns rounds like an explicit reduction would)
                    float kra, krb, sa, ca, sb, cb;
                    f2_unpack(kr, kra, krb);
                    __sincosf(kra, &sa, &ca);
                    __sincosf(krb, &sb, &cb);
                    // E = e^{ikr} / r;  G = E [X - i (k r X + eta)] = X P + Q,
                    // P = E (1 - i k r), Q = -i eta E: shared by both directions
                    const f2x Er = f2_mul(f2_pack(ca, cb), ir), Ei = f2_mul(f2_pack(sa, sb), ir);
                    const f2x Pr = f2_fma(Ei, kr, Er), Pi = f2_fma(Er, nkr, Ei);
                    const f2x Qr = f2_mul(eta2, Ei), Qi = f2_mul(neta2, Er);
                    // target <- source q: X1 = n_q.d / r^2
                    const f2x X1 = f2_mul(f2_fma(snx, dx, f2_fma(sny, dy, f2_mul(snz, dz))), ir2);
                    const f2x g1r = f2_fma(X1, Pr, Qr), g1i = f2_fma(X1, Pi, Qi);
                    // source q <- target (d reversed): X2 = -m.d / r^2 (the target normals are stored negated)
                    const f2x X2 = f2_mul(f2_fma(mx[p], dx, f2_fma(my[p], dy, f2_mul(mz[p], dz))), ir2);
                    const f2x g2r = f2_fma(X2, Pr, Qr), g2i = f2_fma(X2, Pi, Qi);
#pragma unroll
                    for (int c = 0; c < RC; ++c) {
                        atx[p][c] = f2_fma(g1r, swr[c], f2_fma(g1i, nswi[c], atx[p][c]));
                        aty[p][c] = f2_fma(g1r, swi[c], f2_fma(g1i, swr[c], aty[p][c]));
                        asx[c] = f2_fma(g2r, wr[p][c], f2_fma(g2i, nwi[p][c], asx[c]));
                        asy[c] = f2_fma(g2r, wi[p][c], f2_fma(g2i, wr[p][c], asy[c]));
                    }
                }
#pragma unroll
                for (int c = 0; c < RC; ++c) {
                    asx[c] = __shfl_sync(0xffffffffu, asx[c], (lane + 1) & 31);
                    asy[c] = __shfl_sync(0xffffffffu, asy[c], (lane + 1) & 31);
                }
            }
        }
#pragma unroll
        for (int c = 0; c < RC; ++c) {
            float xa, xb, ya, yb;
            f2_unpack(asx[c], xa, xb);
            f2_unpack(asy[c], ya, yb);
            s_red[warp][c][lane] = make_float2(xa + xb, ya + yb);
        }
        __syncthreads();
        if (tid < SYM_S * RC) {
            const int src = tid & (SYM_S - 1), c = tid / SYM_S;
            if (src < cnt && r0 + c < R) {
                float sx = 0.f, sy = 0.f;
                for (int w = 0; w < NW; ++w) {
                    sx += s_red[w][c][src].x;
                    sy += s_red[w][c][src].y;
                }
                double2 *o = y + (size_t)(bj.start + j0 + src) * R + r0 + c;
                atomicAdd(&o->x, (double)sx);
                atomicAdd(&o->y, (double)sy);
            }
        }
    }
#pragma unroll
    for (int p = 0; p < TP; ++p)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int t = tid + (2 * p + h) * NT;
            if (t >= bi.count) continue;
#pragma unroll
            for (int c = 0; c < RC; ++c)
                if (r0 + c < R) {
                    float xa, xb, ya, yb;
                    f2_unpack(atx[p][c], xa, xb);
                    f2_unpack(aty[p][c], ya, yb);
                    double2 *o = y + (size_t)(bi.start + t) * R + r0 + c;
                    atomicAdd(&o->x, (double)(h ? xb : xa));
                    atomicAdd(&o->y, (double)(h ? yb : ya));
                }
        }
}

// Unordered pairs of target blocks on different bodies, built once per geometry.
hzb_status ensure_block_pairs(hzb_ctx *c)
{
    if (c->n_blockpairs > 0) return HZB_OK;
    std::vector<TargetBlock> tb(c->n_tblocks);
    if (check_cuda(c, cudaMemcpyAsync(tb.data(), c->tblocks.ptr, tb.size() * sizeof(TargetBlock),
                                      cudaMemcpyDeviceToHost, c->stream), "copy blocks") ||
        check_cuda(c, cudaStreamSynchronize(c->stream), "copy blocks"))
        return HZB_ECUDA;
    // the CTA's threads own the targets of pair.x and step through the sources of pair.y:
    // the larger block goes first, so a body's short last block is always the source side
    // (a short CTA) and never leaves most of a CTA's threads idle for a full pass
    std::vector<int2> pr;
    for (int i = 0; i < (int)tb.size(); ++i)
        for (int j = i + 1; j < (int)tb.size(); ++j)
            if (tb[i].excl_lo != tb[j].excl_lo)
                pr.push_back(tb[j].count > tb[i].count ? make_int2(j, i) : make_int2(i, j));
    if (pr.empty()) {
        c->n_blockpairs = -1;                   // one body: B = 0
        return HZB_OK;
    }
    if (check_cuda(c, c->blockpairs.ensure(pr.size()), "alloc block pairs")) return HZB_ENOMEM;
    if (check_cuda(c, cudaMemcpyAsync(c->blockpairs.ptr, pr.data(), pr.size() * sizeof(int2),
                                      cudaMemcpyHostToDevice, c->stream), "copy block pairs") ||
        check_cuda(c, cudaStreamSynchronize(c->stream), "copy block pairs"))
        return HZB_ECUDA;
    c->n_blockpairs = (long long)pr.size();
    return HZB_OK;
}

hzb_status interbody64_sym(hzb_ctx *c, int R, const double2 *sigma, double2 *y)
{
    if (!c->nodes_ready) return fail(c, HZB_ESTATE, "nodes not built");
    if (c->capturing && c->n_blockpairs == 0) return fail(c, HZB_ESTATE, "block pairs not built before capture");
    hzb_status st = ensure_sctab(c);
    if (st || (st = ensure_block_pairs(c))) return st;
    const size_t n = (size_t)c->N * R;
    if (check_cuda(c, cudaMemsetAsync(y, 0, n * sizeof(double2), c->stream), "zero y")) return HZB_ECUDA;
    c->interbody_calls++;
    if (c->n_blockpairs < 0) return HZB_OK;
    if (c->n_blockpairs > 0x7fffffffLL) return fail(c, HZB_EINVAL, "too many block pairs for one launch");
    c->launches += 1;
    const int slot = prof_begin(c, 0);
    const int rc = (R == 1) ? 1 : (R == 2 ? 2 : 4);
    dim3 g((unsigned)c->n_blockpairs, (R + rc - 1) / rc, 1);
    const double kt = c->k * (SC_N / (2.0 * M_PI));
    if (rc == 1)
        nbody64_sym_kernel<1><<<g, SYM_T, 0, c->stream>>>(c->blockpairs.ptr, c->tblocks.ptr, R, c->pos64.ptr,
                                                          c->nrm64.ptr, sigma, c->sctab.ptr, c->k, c->eta, kt, y);
    else if (rc == 2)
        nbody64_sym_kernel<2><<<g, SYM_T, 0, c->stream>>>(c->blockpairs.ptr, c->tblocks.ptr, R, c->pos64.ptr,
                                                          c->nrm64.ptr, sigma, c->sctab.ptr, c->k, c->eta, kt, y);
    else
        nbody64_sym_kernel<4><<<g, SYM_T, 0, c->stream>>>(c->blockpairs.ptr, c->tblocks.ptr, R, c->pos64.ptr,
                                                          c->nrm64.ptr, sigma, c->sctab.ptr, c->k, c->eta, kt, y);
    cudaError_t e = cudaGetLastError();
    prof_end(c, slot);
    return check_cuda(c, e, "nbody64_sym_kernel");
}

template <int RC, int TP>
static void launch_sym32(hzb_ctx *c, dim3 g, int R, const float2 *sw, double2 *y)
{
    nbody32_sym_kernel<RC, TP><<<g, SYM_T / (2 * TP), 0, c->stream>>>(
        c->blockpairs.ptr, c->tblocks.ptr, R, c->pos32.ptr, c->nrm32.ptr, sw, (float)c->k, (float)c->eta,
        (float)(c->k / (2.0 * M_PI)), y);
}

hzb_status interbody32_sym(hzb_ctx *c, int R, const double2 *sigma, double2 *y, int tp)
{
    if (!c->nodes_ready) return fail(c, HZB_ESTATE, "nodes not built");
    if (c->capturing && c->n_blockpairs == 0) return fail(c, HZB_ESTATE, "block pairs not built before capture");
    hzb_status st = ensure_block_pairs(c);
    if (st) return st;
    const size_t n = (size_t)c->N * R;
    if (check_cuda(c, cudaMemsetAsync(y, 0, n * sizeof(double2), c->stream), "zero y")) return HZB_ECUDA;
    c->interbody_calls++;
    if (c->n_blockpairs < 0) return HZB_OK;
    if (c->n_blockpairs > 0x7fffffffLL) return fail(c, HZB_EINVAL, "too many block pairs for one launch");
    const int slot = prof_begin(c, 1);
    const float2 *sw = weighted_sigma32(c, R, sigma);
    if (!sw) return HZB_ENOMEM;
    c->launches += 1;
    const int rc = (R == 1) ? 1 : (R == 2 ? 2 : 4);
    dim3 g((unsigned)c->n_blockpairs, (R + rc - 1) / rc, 1);
    if (tp == 2) {
        if (rc == 1) launch_sym32<1, 2>(c, g, R, sw, y);
        else if (rc == 2) launch_sym32<2, 2>(c, g, R, sw, y);
        else launch_sym32<4, 2>(c, g, R, sw, y);
    } else {
        if (rc == 1) launch_sym32<1, 1>(c, g, R, sw, y);
        else if (rc == 2) launch_sym32<2, 1>(c, g, R, sw, y);
        else launch_sym32<4, 1>(c, g, R, sw, y);
    }
    cudaError_t e = cudaGetLastError();
    prof_end(c, slot);
    return check_cuda(c, e, "nbody32_sym_kernel");
}

}  // namespace hzb
