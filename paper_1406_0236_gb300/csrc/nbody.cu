// Inter-body combined-field sum (Sec. 3.3: off-diagonal blocks by the plain Nystrom
// formula, Eq. (nystromnaive); the paper applies B with an FMM, here it is a tiled
// direct sum):
//     y_i = sum_{j not on body(i)} w_j K(x_i, x_j) sigma_j,
//     w_j K(x_i, x_j) = w_j / (4 pi) * e^{ikr} [ n_j.d / r^3 - i (k n_j.d / r^2 + eta / r) ],
// d = x_i - x_j, r = |d|.  Also: the field at off-surface points and the far field.
//
// Work decomposition: a CTA takes one TargetBlock (a run of <= 512 targets inside
// one body, so the sources of the target's own body are one contiguous range that
// the whole CTA skips without a per-pair test) and one of `nsplit` contiguous source
// chunks (grid z); each of its 512/TPT threads owns TPT targets; source tiles of
// blockDim sources are staged in shared memory with the density pre-multiplied by
// w_j / (4 pi).  With nsplit > 1 each chunk writes a partial sum and a second kernel
// adds the chunks in a fixed order (deterministic).  TPT and nsplit are picked per
// workload by the autotuner (hzb_autotune) or a default from the SM count.
#include <algorithm>
#include <cmath>
#include <vector>

#include "hzb_internal.h"
#include "f32x2.cuh"
#include "fp64_pair.cuh"
#include "kernel_math.cuh"

namespace hzb {

static const int TBLOCK = 512;          // targets per TargetBlock (make_nodes)
// ------------------------------------------------------------------ FP64

template <int RC, int TPT>
__global__ void __launch_bounds__(TBLOCK / TPT)
nbody64_kernel(const TargetBlock *__restrict__ blocks, int N, int R, int chunk, const double4 *__restrict__ pos,
               const double4 *__restrict__ nrm, const double2 *__restrict__ sigma, const double2 *__restrict__ sctab,
               double k, double eta, double kt, double2 *__restrict__ y, size_t split_stride)
{
    constexpr int NT = TBLOCK / TPT;
    __shared__ double4 s_pos[NT];
    __shared__ double4 s_nrm[NT];
    __shared__ double2 s_sig[NT * RC];
    const TargetBlock tb = blocks[blockIdx.x];
    const int r0 = blockIdx.y * RC;
    const int tid = threadIdx.x;
    double tx[TPT], ty[TPT], tz[TPT];
    double2 acc[TPT][RC];
#pragma unroll
    for (int m = 0; m < TPT; ++m) {
        int t = tid + m * NT;
        double4 p = (t < tb.count) ? pos[tb.start + t] : make_double4(1e6, 1e6, 1e6, 0.0);   // padding: far, finite
        tx[m] = p.x; ty[m] = p.y; tz[m] = p.z;
#pragma unroll
        for (int c = 0; c < RC; ++c) acc[m][c] = make_double2(0.0, 0.0);
    }
    const int c0 = blockIdx.z * chunk, c1 = min(N, c0 + chunk);
    for (int range = 0; range < 2; ++range) {
        const int lo = range ? max(c0, tb.excl_hi) : c0;
        const int hi = range ? c1 : min(c1, tb.excl_lo);
        for (int j0 = lo; j0 < hi; j0 += NT) {
            const int cnt = min(NT, hi - j0);
            __syncthreads();
            if (tid < cnt) {
                double4 p = pos[j0 + tid];
                s_pos[tid] = p;
                s_nrm[tid] = nrm[j0 + tid];
                const double wq = p.w * HZB_INV4PI;
#pragma unroll
                for (int c = 0; c < RC; ++c) {
                    double2 s = (r0 + c < R) ? sigma[(size_t)(j0 + tid) * R + r0 + c] : make_double2(0.0, 0.0);
                    s_sig[tid * RC + c] = make_double2(s.x * wq, s.y * wq);
                }
            }
            __syncthreads();
            for (int jj = 0; jj < cnt; ++jj) {
                const double4 p = s_pos[jj];
                const double4 n = s_nrm[jj];
#pragma unroll
                for (int m = 0; m < TPT; ++m) {
                    const double dx = tx[m] - p.x, dy = ty[m] - p.y, dz = tz[m] - p.z;
                    const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
                    const double ir = rsqrt_fp64(r2);
                    const double nd = fma(n.x, dx, fma(n.y, dy, n.z * dz));
                    const double ndir2 = nd * (ir * ir);
                    const double A = ndir2 * ir;
                    const double B = fma(k, ndir2, eta * ir);
                    double s, c;
                    cis_turns((r2 * ir) * kt, sctab, c, s);              // e^{ikr}, kr in units of 2 pi / SC_N
                    const double gre = fma(c, A, s * B);
                    const double gim = fma(s, A, -c * B);
#pragma unroll
                    for (int q = 0; q < RC; ++q) {
                        const double2 sg = s_sig[jj * RC + q];
                        acc[m][q].x = fma(gre, sg.x, fma(-gim, sg.y, acc[m][q].x));
                        acc[m][q].y = fma(gre, sg.y, fma(gim, sg.x, acc[m][q].y));
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
                if (r0 + c < R) yo[(size_t)(tb.start + t) * R + r0 + c] = acc[m][c];
    }
}

// ------------------------------------------------------------------ FP32

// Phase of e^{ikr}: r k / (2 pi) is reduced to [-1/2, 1/2] turns before the
// hardware sine and cosine, whose error grows with the argument.
template <int RC, int TPT>
__global__ void __launch_bounds__(TBLOCK / TPT)
nbody32_kernel(const TargetBlock *__restrict__ blocks, int N, int R, int chunk, const float4 *__restrict__ pos,
               const float4 *__restrict__ nrm, const float2 *__restrict__ sw, float k, float eta,
               float k_turns, float2 *__restrict__ ypart, double2 *__restrict__ y, size_t split_stride)
{
    constexpr int NT = TBLOCK / TPT;
    __shared__ float4 s_a[NT];           // x, y, z, nx
    __shared__ float2 s_b[NT];           // ny, nz
    __shared__ float2 s_sig[NT * RC];
    const TargetBlock tb = blocks[blockIdx.x];
    const int r0 = blockIdx.y * RC;
    const int tid = threadIdx.x;
    float tx[TPT], ty[TPT], tz[TPT];
    float2 acc[TPT][RC];
#pragma unroll
    for (int m = 0; m < TPT; ++m) {
        int t = tid + m * NT;
        float4 p = (t < tb.count) ? pos[tb.start + t] : make_float4(1e18f, 1e18f, 1e18f, 0.f);
        tx[m] = p.x; ty[m] = p.y; tz[m] = p.z;
#pragma unroll
        for (int c = 0; c < RC; ++c) acc[m][c] = make_float2(0.f, 0.f);
    }
    const int c0 = blockIdx.z * chunk, c1 = min(N, c0 + chunk);
    for (int range = 0; range < 2; ++range) {
        const int lo = range ? max(c0, tb.excl_hi) : c0;
        const int hi = range ? c1 : min(c1, tb.excl_lo);
        for (int j0 = lo; j0 < hi; j0 += NT) {
            const int cnt = min(NT, hi - j0);
            __syncthreads();
            if (tid < cnt) {
                const float4 p = pos[j0 + tid];
                const float4 n = nrm[j0 + tid];
                s_a[tid] = make_float4(p.x, p.y, p.z, n.x);
                s_b[tid] = make_float2(n.y, n.z);
#pragma unroll
                for (int c = 0; c < RC; ++c)
                    s_sig[tid * RC + c] = (r0 + c < R) ? sw[(size_t)(j0 + tid) * R + r0 + c] : make_float2(0.f, 0.f);
            }
            __syncthreads();
#pragma unroll 2
            for (int jj = 0; jj < cnt; ++jj) {
                const float4 a = s_a[jj];
                const float2 b = s_b[jj];
#pragma unroll
                for (int m = 0; m < TPT; ++m) {
                    const float dx = tx[m] - a.x, dy = ty[m] - a.y, dz = tz[m] - a.z;
                    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    const float ir = rsqrtf(r2);
                    const float nd = fmaf(a.w, dx, fmaf(b.x, dy, b.y * dz));
                    const float ndir2 = nd * (ir * ir);
                    const float A = ndir2 * ir;
                    const float B = fmaf(k, ndir2, eta * ir);
                    float turns = (r2 * ir) * k_turns;
                    turns -= rintf(turns);
                    float s, c;
                    __sincosf(turns * 6.283185307179586f, &s, &c);
                    const float gre = fmaf(c, A, s * B);
                    const float gim = fmaf(s, A, -c * B);
#pragma unroll
                    for (int q = 0; q < RC; ++q) {
                        const float2 sg = s_sig[jj * RC + q];
                        acc[m][q].x = fmaf(gre, sg.x, fmaf(-gim, sg.y, acc[m][q].x));
                        acc[m][q].y = fmaf(gre, sg.y, fmaf(gim, sg.x, acc[m][q].y));
                    }
                }
            }
        }
    }
#pragma unroll
    for (int m = 0; m < TPT; ++m) {
        int t = tid + m * NT;
        if (t < tb.count)
#pragma unroll
            for (int c = 0; c < RC; ++c)
                if (r0 + c < R) {
                    size_t e = (size_t)(tb.start + t) * R + r0 + c;
                    if (ypart) ypart[blockIdx.z * split_stride + e] = acc[m][c];
                    else y[e] = make_double2((double)acc[m][c].x, (double)acc[m][c].y);
                }
    }
}

// The same sum with packed FP32 pairs (f32x2.cuh): each thread takes two sources
// (an even and an odd one of the tile) per step, so every add/mul/fma of the pair
// kernel is one instruction for two pairs; the two accumulators of a target (even
// and odd sources) are added at the end.  Source tiles of 128 are stored as packed
// (even, odd) pairs; an odd tile end is padded with a far source of zero density.
// The phase is reduced with the 1.5 * 2^23 rounding constant (valid while
// k r / (2 pi) < 2^22 turns); rsqrt, sin and cos run per element on the
// transcendental unit.
static const int TS2 = 128;           // sources per tile of the packed kernel

template <int RC, int TPT>
__global__ void __launch_bounds__(TBLOCK / TPT)
nbody32x2_kernel(const TargetBlock *__restrict__ blocks, int N, int R, int chunk, const float4 *__restrict__ pos,
                 const float4 *__restrict__ nrm, const float2 *__restrict__ sw, float k, float eta,
                 float k_turns, float2 *__restrict__ ypart, double2 *__restrict__ y, size_t split_stride)
{
    constexpr int NT = TBLOCK / TPT;
    constexpr int NP = TS2 / 2;                  // source pairs per tile
    __shared__ ulonglong2 s_g[3][NP];            // {x, y}, {z, nx}, {ny, nz} of (even, odd) sources
    __shared__ ulonglong2 s_sg[NP][RC];          // {sr, si}
    __shared__ f2x s_ns[NP][RC];                 // -si
    const TargetBlock tb = blocks[blockIdx.x];
    const int r0 = blockIdx.y * RC;
    const int tid = threadIdx.x;
    f2x tx[TPT], ty[TPT], tz[TPT];
    f2x ax[TPT][RC], ay[TPT][RC];
#pragma unroll
    for (int m = 0; m < TPT; ++m) {
        int t = tid + m * NT;
        float4 p = (t < tb.count) ? pos[tb.start + t] : make_float4(1e18f, 1e18f, 1e18f, 0.f);
        tx[m] = f2_splat(p.x); ty[m] = f2_splat(p.y); tz[m] = f2_splat(p.z);
#pragma unroll
        for (int c = 0; c < RC; ++c) ax[m][c] = ay[m][c] = 0ull;
    }
    const f2x k2 = f2_splat(k), eta2 = f2_splat(eta);
    const int c0 = blockIdx.z * chunk, c1 = min(N, c0 + chunk);
    for (int range = 0; range < 2; ++range) {
        const int lo = range ? max(c0, tb.excl_hi) : c0;
        const int hi = range ? c1 : min(c1, tb.excl_lo);
        for (int j0 = lo; j0 < hi; j0 += TS2) {
            const int cnt = min(TS2, hi - j0);
            __syncthreads();
            if (tid < TS2) {
                const int pp = tid >> 1, h = tid & 1;
                float4 p = make_float4(-1e18f, -1e18f, -1e18f, 0.f), n = make_float4(0.f, 0.f, 0.f, 0.f);
                if (tid < cnt) { p = pos[j0 + tid]; n = nrm[j0 + tid]; }
                float *g0 = reinterpret_cast<float *>(&s_g[0][pp]);
                float *g1 = reinterpret_cast<float *>(&s_g[1][pp]);
                float *g2 = reinterpret_cast<float *>(&s_g[2][pp]);
                g0[h] = p.x; g0[2 + h] = p.y;
                g1[h] = p.z; g1[2 + h] = n.x;
                g2[h] = n.y; g2[2 + h] = n.z;
#pragma unroll
                for (int c = 0; c < RC; ++c) {
                    const float2 sv = (tid < cnt && r0 + c < R) ? sw[(size_t)(j0 + tid) * R + r0 + c]
                                                                : make_float2(0.f, 0.f);
                    float *sg = reinterpret_cast<float *>(&s_sg[pp][c]);
                    sg[h] = sv.x; sg[2 + h] = sv.y;
                    reinterpret_cast<float *>(&s_ns[pp][c])[h] = -sv.y;
                }
            }
            __syncthreads();
            const int npair = (cnt + 1) >> 1;
#pragma unroll 2
            for (int jp = 0; jp < npair; ++jp) {
                const ulonglong2 g0 = s_g[0][jp], g1 = s_g[1][jp], g2 = s_g[2][jp];
#pragma unroll
                for (int m = 0; m < TPT; ++m) {
                    const f2x dx = f2_sub(tx[m], g0.x), dy = f2_sub(ty[m], g0.y), dz = f2_sub(tz[m], g1.x);
                    const f2x r2 = f2_fma(dx, dx, f2_fma(dy, dy, f2_mul(dz, dz)));
                    float r2a, r2b;
                    f2_unpack(r2, r2a, r2b);
                    const f2x ir = f2_pack(rsqrtf(r2a), rsqrtf(r2b));
                    const f2x nd = f2_fma(g1.y, dx, f2_fma(g2.x, dy, f2_mul(g2.y, dz)));
                    const f2x X = f2_mul(nd, f2_mul(ir, ir));
                    const f2x A = f2_mul(X, ir);
                    const f2x B = f2_fma(k2, X, f2_mul(eta2, ir));
                    // e^{ikr} straight from the transcendental unit, which scales its argument
                    // to turns itself (the rounding an explicit reduction would make)
                    const f2x kr = f2_mul(f2_mul(r2, ir), k2);
                    float tha, thb, sa, ca, sb, cb;
                    f2_unpack(kr, tha, thb);
                    __sincosf(tha, &sa, &ca);
                    __sincosf(thb, &sb, &cb);
                    const f2x s2 = f2_pack(sa, sb), c2 = f2_pack(ca, cb);
                    const f2x gre = f2_fma(c2, A, f2_mul(s2, B));
                    const f2x gim = f2_sub(f2_mul(s2, A), f2_mul(c2, B));
#pragma unroll
                    for (int q = 0; q < RC; ++q) {
                        const ulonglong2 sg = s_sg[jp][q];
                        const f2x ns = s_ns[jp][q];
                        ax[m][q] = f2_fma(gre, sg.x, f2_fma(gim, ns, ax[m][q]));
                        ay[m][q] = f2_fma(gre, sg.y, f2_fma(gim, sg.x, ay[m][q]));
                    }
                }
            }
        }
    }
#pragma unroll
    for (int m = 0; m < TPT; ++m) {
        int t = tid + m * NT;
        if (t < tb.count)
#pragma unroll
            for (int c = 0; c < RC; ++c)
                if (r0 + c < R) {
                    float xa, xb, ya, yb;
                    f2_unpack(ax[m][c], xa, xb);
                    f2_unpack(ay[m][c], ya, yb);
                    const float2 v = make_float2(xa + xb, ya + yb);
                    size_t e = (size_t)(tb.start + t) * R + r0 + c;
                    if (ypart) ypart[blockIdx.z * split_stride + e] = v;
                    else y[e] = make_double2((double)v.x, (double)v.y);
                }
    }
}

// sigma'_{j,r} = w_j sigma_{j,r} / (4 pi), formed in FP64 and rounded once to FP32:
// the FP32 kernels stage it without per-tile FP64 work.
__global__ void weight_sigma32_kernel(size_t n, int R, const double4 *__restrict__ pos64,
                                      const double2 *__restrict__ sigma, float2 *__restrict__ out)
{
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const double wq = pos64[e / R].w * HZB_INV4PI;
    const double2 v = sigma[e];
    out[e] = make_float2((float)(v.x * wq), (float)(v.y * wq));
}

const float2 *weighted_sigma32(hzb_ctx *c, int R, const double2 *sigma)
{
    const size_t n = (size_t)c->N * R;
    if (check_cuda(c, c->sig32.ensure(n), "alloc weighted densities")) return nullptr;
    weight_sigma32_kernel<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(n, R, c->pos64.ptr, sigma, c->sig32.ptr);
    c->launches++;
    return c->sig32.ptr;
}

// y = sum over the nsplit partial sums (fixed order)
template <typename P>
__global__ void split_reduce_kernel(size_t n, int nsplit, const P *__restrict__ part, double2 *__restrict__ y)
{
    size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    double sx = 0.0, sy = 0.0;
    for (int s = 0; s < nsplit; ++s) {
        P v = part[s * n + e];
        sx += (double)v.x;
        sy += (double)v.y;
    }
    y[e] = make_double2(sx, sy);
}

void split_reduce_f2(hzb_ctx *c, size_t n, int nsplit, const float2 *part, double2 *y)
{
    split_reduce_kernel<float2><<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(n, nsplit, part, y);
}

// Launch shape of the inter-body kernels.
static int rc_of(int R) { return R == 1 ? 1 : (R <= 4 ? 4 : 8); }

int default_nsplit(hzb_ctx *c, int R, int tpt)
{
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->opt.device);
    const int rc = rc_of(R);
    const long long ctas = (long long)c->n_tblocks * ((R + rc - 1) / rc);
    const long long want = (long long)sms * (tpt == 1 ? 4 : (tpt == 2 ? 8 : 12));
    int ns = (int)std::max<long long>(1, (want + ctas - 1) / ctas);
    return std::min(ns, 64);
}

hzb_status ensure_sctab(hzb_ctx *c)
{
    if (c->sctab.ptr) return HZB_OK;
    std::vector<double2> tab(SC_N);
    // angles in long double so each entry is the correctly rounded value to within an ulp
    for (int q = 0; q < SC_N; ++q) {
        const long double a = 6.283185307179586476925286766559L * q / SC_N;
        tab[q] = make_double2((double)std::cos(a), (double)std::sin(a));
    }
    if (check_cuda(c, c->sctab.ensure(SC_N), "alloc table")) return HZB_ENOMEM;
    return check_cuda(c, cudaMemcpyAsync(c->sctab.ptr, tab.data(), SC_N * sizeof(double2), cudaMemcpyHostToDevice,
                                         c->stream), "copy table");
}

template <int RC, int TPT>
static void launch64(hzb_ctx *c, dim3 g, int N, int R, int chunk, const double2 *sigma, double2 *out, size_t stride)
{
    nbody64_kernel<RC, TPT><<<g, TBLOCK / TPT, 0, c->stream>>>(c->tblocks.ptr + c->tblock_off, N, R, chunk, c->pos64.ptr,
                                                               c->nrm64.ptr, sigma, c->sctab.ptr, c->k, c->eta,
                                                               c->k * (SC_N / (2.0 * M_PI)), out, stride);
}

template <int RC, int TPT>
static void launch32(hzb_ctx *c, dim3 g, int N, int R, int chunk, const float2 *sigma, float2 *part, double2 *y,
                     size_t stride)
{
    nbody32_kernel<RC, TPT><<<g, TBLOCK / TPT, 0, c->stream>>>(
        c->tblocks.ptr + c->tblock_off, N, R, chunk, c->pos32.ptr, c->nrm32.ptr, sigma, (float)c->k, (float)c->eta,
        (float)(c->k / (2.0 * M_PI)), part, y, stride);
}

template <int RC>
static void dispatch64(hzb_ctx *c, int tpt, dim3 g, int N, int R, int chunk, const double2 *s, double2 *o, size_t st)
{
    if (tpt == 1) launch64<RC, 1>(c, g, N, R, chunk, s, o, st);
    else if (tpt == 2) launch64<RC, 2>(c, g, N, R, chunk, s, o, st);
    else launch64<RC, 4>(c, g, N, R, chunk, s, o, st);
}

template <int RC, int TPT>
static void launch32x2(hzb_ctx *c, dim3 g, int N, int R, int chunk, const float2 *sigma, float2 *part, double2 *y,
                       size_t stride)
{
    nbody32x2_kernel<RC, TPT><<<g, TBLOCK / TPT, 0, c->stream>>>(
        c->tblocks.ptr + c->tblock_off, N, R, chunk, c->pos32.ptr, c->nrm32.ptr, sigma, (float)c->k, (float)c->eta,
        (float)(c->k / (2.0 * M_PI)), part, y, stride);
}

template <int RC>
static void dispatch32(hzb_ctx *c, int tpt, bool x2, dim3 g, int N, int R, int chunk, const float2 *s, float2 *p,
                       double2 *y, size_t st)
{
    if (x2) {
        if (tpt == 1) launch32x2<RC, 1>(c, g, N, R, chunk, s, p, y, st);
        else if (tpt == 2) launch32x2<RC, 2>(c, g, N, R, chunk, s, p, y, st);
        else launch32x2<RC, 4>(c, g, N, R, chunk, s, p, y, st);
        return;
    }
    if (tpt == 1) launch32<RC, 1>(c, g, N, R, chunk, s, p, y, st);
    else if (tpt == 2) launch32<RC, 2>(c, g, N, R, chunk, s, p, y, st);
    else launch32<RC, 4>(c, g, N, R, chunk, s, p, y, st);
}

static int chunk_of(int N, int nsplit, int tpt)
{
    const int nt = TBLOCK / tpt;
    int ch = (N + nsplit - 1) / nsplit;
    return ((ch + nt - 1) / nt) * nt;
}

hzb_status interbody64_cfg(hzb_ctx *c, int R, const double2 *sigma, double2 *y, int tpt, int nsplit)
{
    if (!c->nodes_ready) return fail(c, HZB_ESTATE, "nodes not built");
    hzb_status st = ensure_sctab(c);
    if (st) return st;
    const int N = (int)c->N;
    const int rc = rc_of(R);
    const int chunk = chunk_of(N, nsplit, tpt);
    nsplit = (N + chunk - 1) / chunk;
    const size_t n = (size_t)N * R;
    double2 *out = y;
    if (nsplit > 1) {
        if (check_cuda(c, c->nb_part64.ensure(n * nsplit), "alloc partial sums")) return HZB_ENOMEM;
        out = c->nb_part64.ptr;
    }
    c->interbody_calls++;
    c->launches += (nsplit > 1) ? 2 : 1;
    const int slot = prof_begin(c, 0);
    const int nb = (c->tune_limit_blocks > 0) ? std::min(c->tune_limit_blocks, c->n_tblocks - c->tblock_off)
                                              : c->n_tblocks - c->tblock_off;
    dim3 g(nb, (R + rc - 1) / rc, nsplit);
    if (rc == 1) dispatch64<1>(c, tpt, g, N, R, chunk, sigma, out, n);
    else if (rc == 4) dispatch64<4>(c, tpt, g, N, R, chunk, sigma, out, n);
    else dispatch64<8>(c, tpt, g, N, R, chunk, sigma, out, n);
    if (nsplit > 1)
        split_reduce_kernel<double2><<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(n, nsplit, out, y);
    cudaError_t e = cudaGetLastError();
    prof_end(c, slot);
    return check_cuda(c, e, "nbody64_kernel");
}

hzb_status interbody32_cfg(hzb_ctx *c, int R, const double2 *sigma, double2 *y, int tpt, int nsplit, bool x2)
{
    if (!c->nodes_ready) return fail(c, HZB_ESTATE, "nodes not built");
    const int N = (int)c->N;
    const int rc = rc_of(R);
    const int chunk = chunk_of(N, nsplit, tpt);
    nsplit = (N + chunk - 1) / chunk;
    const size_t n = (size_t)N * R;
    float2 *part = nullptr;
    if (nsplit > 1) {
        if (check_cuda(c, c->nb_part32.ensure(n * nsplit), "alloc partial sums")) return HZB_ENOMEM;
        part = c->nb_part32.ptr;
    }
    c->interbody_calls++;
    c->launches += (nsplit > 1) ? 2 : 1;
    const int slot = prof_begin(c, 1);
    const float2 *sw = weighted_sigma32(c, R, sigma);
    if (!sw) return HZB_ENOMEM;
    const int nb = (c->tune_limit_blocks > 0) ? std::min(c->tune_limit_blocks, c->n_tblocks - c->tblock_off)
                                              : c->n_tblocks - c->tblock_off;
    dim3 g(nb, (R + rc - 1) / rc, nsplit);
    if (rc == 1) dispatch32<1>(c, tpt, x2, g, N, R, chunk, sw, part, y, n);
    else if (rc == 4) dispatch32<4>(c, tpt, x2, g, N, R, chunk, sw, part, y, n);
    else dispatch32<8>(c, tpt, x2, g, N, R, chunk, sw, part, y, n);
    if (nsplit > 1)
        split_reduce_kernel<float2><<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(n, nsplit, part, y);
    cudaError_t e = cudaGetLastError();
    prof_end(c, slot);
    return check_cuda(c, e, "nbody32_kernel");
}

// Source split of the tensor-core kernel: about four CTAs per SM in all.
static int default_nsplit_tc(hzb_ctx *c, int R)
{
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->opt.device);
    const long long ctas = (long long)c->n_tblocks * 4 * ((R + 15) / 16);
    return (int)std::min<long long>(64, std::max<long long>(1, (4LL * sms + ctas - 1) / ctas));
}

// Source split of the tcgen05 kernel: about two resident CTAs per SM in all.
static int default_nsplit_tc5(hzb_ctx *c, int R)
{
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->opt.device);
    const int rc = (R <= 16) ? 16 : 32;
    const long long ctas = (long long)c->n_tblocks * 4 * ((R + rc - 1) / rc);
    return (int)std::min<long long>(64, std::max<long long>(1, (2LL * sms + ctas - 1) / ctas));
}

hzb_status interbody64(hzb_ctx *c, int R, const double2 *sigma, double2 *y)
{
    if (c->nbody64_engine >= 1 || (c->nbody64_engine < 0 && R <= 4)) return interbody64_sym(c, R, sigma, y);
    int tpt = c->tune64_tpt > 0 ? c->tune64_tpt : 2;
    int ns = c->tune64_split > 0 ? c->tune64_split : default_nsplit(c, R, tpt);
    return interbody64_cfg(c, R, sigma, y, tpt, ns);
}

hzb_status interbody32(hzb_ctx *c, int R, const double2 *sigma, double2 *y)
{
    // many right-hand sides: contraction on the tensor cores, tcgen05 (nbody_tc5.cu) or
    // mma.sync (nbody_tc.cu); engine choice 0 CUDA cores, 1 mma.sync, 2 tcgen05, 3 tcgen05
    // warp-specialised, 4 tcgen05 with single-term TF32 products (opt-in only)
    int e = -1;
    if (c->nbody_engine == 1) e = 1;
    else if (c->nbody_engine == 5) e = 2;
    else if (c->nbody_engine == 6) e = 3;
    else if (c->nbody_engine == 7) e = 4;
    else if (c->nbody_engine < 0) e = (c->tune32_tc >= 0 && c->tune32_tc_R == R) ? c->tune32_tc : (R >= 16 ? 2 : 0);
    if (e >= 2 && e <= 4)
        return interbody_tc5(c, R, sigma, y, default_nsplit_tc5(c, R),
                             e == 2 ? T5_SPLIT3 : (e == 3 ? T5_WS : T5_SINGLE));
    if (e == 1) {
        int ns = c->tunetc_split > 0 ? c->tunetc_split : default_nsplit_tc(c, R);
        return interbody_tc(c, R, sigma, y, ns);
    }
    // CUDA cores: variant 0 scalar, 1 packed pairs, 2 pair-symmetric packed
    int v = (c->tune32_x2 >= 0 && c->tune32_R == R) ? c->tune32_x2 : (R <= 2 ? 2 : 1);
    if (c->nbody_engine >= 2 && c->nbody_engine <= 4) v = c->nbody_engine - 2;
    if (v == 2) return interbody32_sym(c, R, sigma, y, (c->tune32_x2 == 2 && c->tune32_tpt == 1) ? 1 : 2);
    const bool x2 = v == 1;
    int tpt = c->tune32_tpt > 0 ? c->tune32_tpt : 4;
    int ns = c->tune32_split > 0 ? c->tune32_split : default_nsplit(c, R, tpt);
    return interbody32_cfg(c, R, sigma, y, tpt, ns, x2);
}

// ------------------------------------------------------------------ fields at points

static const int FP_CHUNK = 2048;     // sources per block of the point-field kernels

// Partial sums of u(p_t) = sum_j w_j K(p_t, x_j) sigma_j over one source chunk:
// grid (chunks, T); block reduce; partial[(t * nchunk + chunk) * R + r].
__global__ void field_partial_kernel(int N, int R, const double4 *__restrict__ pos,
                                     const double4 *__restrict__ nrm, const double2 *__restrict__ sigma,
                                     const double *__restrict__ pts, double k, double eta, double2 *partial)
{
    __shared__ double2 red[256];
    const int chunk = blockIdx.x, t = blockIdx.y, nchunk = gridDim.x;
    const double px = pts[3 * t], py = pts[3 * t + 1], pz = pts[3 * t + 2];
    const int j0 = chunk * FP_CHUNK, j1 = min(N, j0 + FP_CHUNK);
    for (int r = 0; r < R; ++r) {
        double2 acc = make_double2(0.0, 0.0);
        for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
            double4 p = pos[j], n = nrm[j];
            double dx = px - p.x, dy = py - p.y, dz = pz - p.z;
            double r2 = dx * dx + dy * dy + dz * dz, ir = rsqrt(r2), rr = r2 * ir;
            double nd = n.x * dx + n.y * dy + n.z * dz;
            double A = nd * ir * ir * ir, B = k * nd * ir * ir + eta * ir;
            double s, c;
            sincos(k * rr, &s, &c);
            double2 g = make_double2((c * A + s * B) * p.w * HZB_INV4PI, (s * A - c * B) * p.w * HZB_INV4PI);
            cfma(acc, g, sigma[(size_t)j * R + r]);
        }
        red[threadIdx.x] = acc;
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) red[threadIdx.x] = cadd(red[threadIdx.x], red[threadIdx.x + s]);
            __syncthreads();
        }
        if (threadIdx.x == 0) partial[((size_t)t * nchunk + chunk) * R + r] = red[0];
        __syncthreads();
    }
}

// Far-field partial sums: (1/4pi) sum_j w_j e^{-ik xh.x_j} (-ik xh.n_j - i eta) sigma_j.
__global__ void farfield_partial_kernel(int N, int R, const double4 *__restrict__ pos,
                                        const double4 *__restrict__ nrm, const double2 *__restrict__ sigma,
                                        const double *__restrict__ xh, double k, double eta, double2 *partial)
{
    __shared__ double2 red[256];
    const int chunk = blockIdx.x, t = blockIdx.y, nchunk = gridDim.x;
    const double hx = xh[3 * t], hy = xh[3 * t + 1], hz = xh[3 * t + 2];
    const int j0 = chunk * FP_CHUNK, j1 = min(N, j0 + FP_CHUNK);
    for (int r = 0; r < R; ++r) {
        double2 acc = make_double2(0.0, 0.0);
        for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
            double4 p = pos[j], n = nrm[j];
            double s, c;
            sincos(k * (hx * p.x + hy * p.y + hz * p.z), &s, &c);
            double2 ph = make_double2(c, -s);
            double2 fac = make_double2(0.0, -(k * (hx * n.x + hy * n.y + hz * n.z) + eta));
            double2 g = cscale(cmul(ph, fac), p.w * HZB_INV4PI);
            cfma(acc, g, sigma[(size_t)j * R + r]);
        }
        red[threadIdx.x] = acc;
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) red[threadIdx.x] = cadd(red[threadIdx.x], red[threadIdx.x + s]);
            __syncthreads();
        }
        if (threadIdx.x == 0) partial[((size_t)t * nchunk + chunk) * R + r] = red[0];
        __syncthreads();
    }
}

__global__ void chunk_reduce_kernel(int T, int nchunk, int R, const double2 *partial, double2 *out)
{
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= T * R) return;
    int t = e / R, r = e % R;
    double2 s = make_double2(0.0, 0.0);
    for (int q = 0; q < nchunk; ++q) s = cadd(s, partial[((size_t)t * nchunk + q) * R + r]);
    out[(size_t)t * R + r] = s;
}

static hzb_status point_sum(hzb_ctx *c, int R, const double2 *sigma, int T, const double *pts, double2 *out,
                            bool far)
{
    int N = (int)c->N;
    int nchunk = (N + FP_CHUNK - 1) / FP_CHUNK;
    size_t need = (size_t)T * nchunk * R;
    if (check_cuda(c, c->w_d.ensure(need), "alloc field partials")) return HZB_ENOMEM;
    dim3 grid(nchunk, T);
    if (far)
        farfield_partial_kernel<<<grid, 256, 0, c->stream>>>(N, R, c->pos64.ptr, c->nrm64.ptr, sigma, pts, c->k,
                                                             c->eta, c->w_d.ptr);
    else
        field_partial_kernel<<<grid, 256, 0, c->stream>>>(N, R, c->pos64.ptr, c->nrm64.ptr, sigma, pts, c->k,
                                                          c->eta, c->w_d.ptr);
    chunk_reduce_kernel<<<(T * R + 255) / 256, 256, 0, c->stream>>>(T, nchunk, R, c->w_d.ptr, out);
    c->launches += 2;
    return check_cuda(c, cudaGetLastError(), "point fields");
}

hzb_status field_points64(hzb_ctx *c, int R, const double2 *sigma, int T, const double *pts, double2 *out)
{
    return point_sum(c, R, sigma, T, pts, out, false);
}

hzb_status far_field64(hzb_ctx *c, int R, const double2 *sigma, int n, const double *xhat, double2 *out)
{
    return point_sum(c, R, sigma, n, xhat, out, true);
}

// v(x_i) = exp(i k d_r . x_i), N x R
__global__ void plane_wave_kernel(long long N, int R, const double4 *__restrict__ pos, const double *dirs,
                                  double k, double2 *v)
{
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N * R) return;
    long long i = e / R;
    int r = (int)(e % R);
    double4 p = pos[i];
    double s, c;
    sincos(k * (dirs[3 * r] * p.x + dirs[3 * r + 1] * p.y + dirs[3 * r + 2] * p.z), &s, &c);
    v[e] = make_double2(c, s);
}

hzb_status plane_waves(hzb_ctx *c, int R, const double *dirs_dev, double2 *v)
{
    long long n = c->N * R;
    plane_wave_kernel<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(c->N, R, c->pos64.ptr, dirs_dev, c->k, v);
    c->launches++;
    return check_cuda(c, cudaGetLastError(), "plane_wave_kernel");
}

}  // namespace hzb

namespace hzb {

// Time one inter-body configuration: one warm-up launch, then the mean of `reps`
// launches between CUDA events on the context's stream.
static hzb_status run_cfg(hzb_ctx *c, int prec, int R, int tpt, int ns, int xv, const double2 *x, double2 *y)
{
    if (!prec) return interbody64_cfg(c, R, x, y, tpt, ns);
    if (xv == 2) return interbody32_sym(c, R, x, y, tpt);
    return interbody32_cfg(c, R, x, y, tpt, ns, xv == 1);
}

static float time_cfg(hzb_ctx *c, int prec, int R, int tpt, int ns, int xv, const double2 *x, double2 *y, int reps)
{
    hzb_status st = run_cfg(c, prec, R, tpt, ns, xv, x, y);
    if (st) return -1.f;
    cudaEventRecord(c->ev0, c->stream);
    for (int q = 0; q < reps; ++q) {
        st = run_cfg(c, prec, R, tpt, ns, xv, x, y);
        if (st) return -1.f;
    }
    cudaEventRecord(c->ev1, c->stream);
    if (cudaEventSynchronize(c->ev1) != cudaSuccess) return -1.f;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    return ms / reps;
}

static float time_tc(hzb_ctx *c, int R, int ns, const double2 *x, double2 *y, int reps)
{
    if (interbody_tc(c, R, x, y, ns)) return -1.f;
    cudaEventRecord(c->ev0, c->stream);
    for (int q = 0; q < reps; ++q)
        if (interbody_tc(c, R, x, y, ns)) return -1.f;
    cudaEventRecord(c->ev1, c->stream);
    if (cudaEventSynchronize(c->ev1) != cudaSuccess) return -1.f;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    return ms / reps;
}

hzb_status autotune(hzb_ctx *c, int R, int which, double *best_ms)
{
    if (!c->nodes_ready) {
        hzb_status st = make_nodes(c);
        if (st) return st;
    }
    const size_t n = (size_t)c->N * R;
    if (check_cuda(c, c->io_in.ensure(n), "alloc") || check_cuda(c, c->io_out.ensure(n), "alloc")) return HZB_ENOMEM;
    cudaMemsetAsync(c->io_in.ptr, 0, n * sizeof(double2), c->stream);
    const long long calls = c->interbody_calls, launches = c->launches;
    for (int prec = 1; prec >= 0; --prec) {
        if (!(which & (prec ? 1 : 2))) continue;
        int bt = 0, bs = 0, bx = 0;
        float bm = 1e30f;
        const int tpts[3] = {1, 2, 4};
        // FP32 kernel variants: 0 scalar, 1 packed pairs, 2 pair-symmetric packed
        // (one of them when the engine fixes it)
        int xmin = 0, xmax = prec ? 2 : 0;
        if (prec && c->nbody_engine >= 2 && c->nbody_engine <= 4) xmin = xmax = c->nbody_engine - 2;
        for (int xv = xmin; xv <= xmax; ++xv) {
            if (xv == 2) {                  // no source split; TP = 1 or 2 packed target pairs
                for (int tp = 1; tp <= 2; ++tp) {
                    float ms = time_cfg(c, prec, R, tp, 1, xv, c->io_in.ptr, c->io_out.ptr, 3);
                    if (ms < 0) return fail(c, HZB_ECUDA, "autotune launch failed");
                    if (ms < bm) { bm = ms; bt = tp; bs = 1; bx = xv; }
                }
                continue;
            }
            for (int a = 0; a < 3; ++a) {
                int tpt = tpts[a];
                if (prec == 0 && tpt == 4) continue;
                int d = default_nsplit(c, R, tpt);
                int cand[5] = {1, 2, d, 2 * d, 4 * d};
                for (int b = 0; b < 5; ++b) {
                    if (b > 0 && cand[b] == cand[b - 1]) continue;
                    if (cand[b] > 64) continue;
                    float ms = time_cfg(c, prec, R, tpt, cand[b], xv, c->io_in.ptr, c->io_out.ptr, prec ? 3 : 1);
                    if (ms < 0) return fail(c, HZB_ECUDA, "autotune launch failed");
                    if (ms < bm) { bm = ms; bt = tpt; bs = cand[b]; bx = xv; }
                }
            }
        }
        if (prec && R >= 8 && c->nbody_engine < 0) {
            // the tensor-core contractions (mma.sync, tcgen05) compete for the FP32 sum
            const int d = default_nsplit_tc(c, R);
            const int cand[4] = {1, 2, d, 2 * d};
            int tbs = 0;
            float tbm = 1e30f;
            for (int b = 0; b < 4; ++b) {
                if ((b > 0 && cand[b] == cand[b - 1]) || cand[b] > 64) continue;
                float ms = time_tc(c, R, cand[b], c->io_in.ptr, c->io_out.ptr, 3);
                if (ms < 0) return fail(c, HZB_ECUDA, "autotune launch failed");
                if (ms < tbm) { tbm = ms; tbs = cand[b]; }
            }
            float t5 = 1e30f;
            {
                if (interbody_tc5(c, R, c->io_in.ptr, c->io_out.ptr, default_nsplit_tc5(c, R), T5_SPLIT3))
                    return fail(c, HZB_ECUDA, "autotune launch failed");
                cudaEventRecord(c->ev0, c->stream);
                for (int q = 0; q < 3; ++q)
                    if (interbody_tc5(c, R, c->io_in.ptr, c->io_out.ptr, default_nsplit_tc5(c, R), T5_SPLIT3))
                        return fail(c, HZB_ECUDA, "autotune launch failed");
                cudaEventRecord(c->ev1, c->stream);
                if (cudaEventSynchronize(c->ev1) != cudaSuccess) return fail(c, HZB_ECUDA, "autotune launch failed");
                cudaEventElapsedTime(&t5, c->ev0, c->ev1);
                t5 /= 3;
            }
            c->tunetc_split = tbs;
            c->tune32_tc = (t5 < tbm && t5 < bm) ? 2 : (tbm < bm ? 1 : 0);
            c->tune32_tc_R = R;
            bm = std::min(bm, std::min(tbm, t5));
        }
        if (prec) { c->tune32_tpt = bt; c->tune32_split = bs; c->tune32_x2 = bx; c->tune32_R = R; }
        else { c->tune64_tpt = bt; c->tune64_split = bs; }
        if (best_ms) best_ms[prec ? 0 : 1] = bm;
    }
    c->interbody_calls = calls;       // tuning launches are not solve work
    c->launches = launches;
    return HZB_OK;
}

}  // namespace hzb
