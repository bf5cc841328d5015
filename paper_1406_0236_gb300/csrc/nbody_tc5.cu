// Inter-body sum y = B sigma (Sec. 3.3, Eq. (nystromnaive)) for many right-hand sides
// with the contraction over sources on the 5th-generation tensor cores (tcgen05,
// accumulators in tensor memory).
//
// A CTA of 256 threads owns 128 targets of one TargetBlock (4 CTAs per block) and RC = 16
// or 32 right-hand sides.  For every tile of 32 sources:
//   * two threads per target form the pair kernels
//     G(t, s) = e^{ikr}[n_s.d/r^3 - i(k n_s.d/r^2 + eta/r)] in FP32 for the 32 sources, two
//     sources per f32x2 instruction, and store Re G, Im G, each split into TF32 hi + lo,
//     as row t of four 128 x 32 K-major operand tiles in shared memory (128-byte swizzle);
//   * the weighted densities sigma'_{s,r} = w_s sigma_{s,r}/(4 pi) of the RC RHS form
//     two 2RC x 32 operand tiles B1 = [Re s' ; Im s'] and B2 = [-Im s' ; Re s'] (rows =
//     output columns, hi + lo each), so that Y = Re G B1 + Im G B2 gives
//     [Re y | Im y] in the 128 x 2RC accumulator;
//   * one thread issues 24 MMAs (4 k-steps of 8 sources x {Ahi Bhi, Ahi Blo, Alo Bhi}
//     for both products) with tcgen05.mma.kind::tf32 into tensor memory and commits
//     them to an mbarrier; the tile's accumulator starts from zero.  The single-term
//     form (TERMS = 1, opt-in engine) keeps only the hi parts: 8 MMAs, half the operand
//     stores, about 3e-4 relative error in the sum;
//   * after the commit, each warp reads 32 lanes x RC columns of the accumulator
//     (tcgen05.ld) and adds them to running FP32 sums in registers: the tensor cores'
//     internal accumulation is not rounded to nearest, so chaining ~10^4 tiles in tensor
//     memory would drift.
// TF32 rounding is done by two integer operations on the bit pattern (t5_tf32i), which
// measured faster than the conversion instruction.  The next tile's positions and
// densities are loaded into registers while the current tile's pair kernels and MMAs run.  Every mbarrier wait is bounded; on a timeout the CTA
// sets an error flag, writes NaN outputs, frees its tensor memory and returns.
#include <algorithm>

#include "f32x2.cuh"
#include "tcgen05.cuh"
#include "hzb_internal.h"
#include "kernel_math.cuh"

namespace hzb {

static const int T5_M = 128;              // targets per CTA = MMA M = TMEM lanes
static const int T5_K = 32;               // sources per tile: one 128-byte row of TF32
// right-hand sides per CTA: RC = 16 or 32 (template), MMA N = 2 RC (real and imaginary columns)
static const int T5_TMEM_COLS = 128;      // allocated tensor-memory columns (>= 2 RC, power of 2)
static const int T5_THREADS = 256;        // two threads per target row
static const int T5_A_BYTES = T5_M * T5_K * 4;          // one A operand tile (16 KB)
static const int T5_B_BYTES = 64 * T5_K * 4;            // one B operand tile (8 KB at RC = 32)
static const int T5_SMEM = 4 * T5_A_BYTES + 4 * T5_B_BYTES + 1024 + 1024;   // + source tile, alignment
static const int T5_STAGE = 4 * T5_A_BYTES + 4 * T5_B_BYTES;              // one operand stage (96 KB)

// Pair kernels of one target and two sources (packed f32x2); e^{ikr} straight from the
// transcendental unit, which scales its argument to turns itself (that rounding is the
// one an explicit reduction to a fraction of a turn would make).
__device__ __forceinline__ void t5_pair2(f2x tx, f2x ty, f2x tz, f2x sx, f2x sy, f2x sz, f2x nx, f2x ny, f2x nz,
                                         f2x k2, f2x eta2, f2x &gre, f2x &gim)
{
    const f2x dx = f2_sub(tx, sx), dy = f2_sub(ty, sy), dz = f2_sub(tz, sz);
    const f2x r2 = f2_fma(dx, dx, f2_fma(dy, dy, f2_mul(dz, dz)));
    float ra, rb;
    f2_unpack(r2, ra, rb);
    const f2x ir = f2_pack(rsqrtf(ra), rsqrtf(rb));
    const f2x X = f2_mul(f2_fma(nx, dx, f2_fma(ny, dy, f2_mul(nz, dz))), f2_mul(ir, ir));
    const f2x A = f2_mul(X, ir), B = f2_fma(k2, X, f2_mul(eta2, ir));
    const f2x kr = f2_mul(f2_mul(r2, ir), k2);
    float ta, tb, sa, ca, sb, cb;
    f2_unpack(kr, ta, tb);
    __sincosf(ta, &sa, &ca);
    __sincosf(tb, &sb, &cb);
    const f2x s2 = f2_pack(sa, sb), c2 = f2_pack(ca, cb);
    gre = f2_fma(c2, A, f2_mul(s2, B));
    gim = f2_sub(f2_mul(s2, A), f2_mul(c2, B));
}

// TF32 hi + lo split of a packed pair: hi rounded to TF32, lo = x - hi rounded to TF32
// (integer rounding, t5_tf32i).
__device__ __forceinline__ void t5_split2(f2x x, uint32_t &h0, uint32_t &h1, uint32_t &l0, uint32_t &l1)
{
    float a, b;
    f2_unpack(x, a, b);
    h0 = t5_tf32i(a);
    h1 = t5_tf32i(b);
    const f2x lo = f2_sub(x, f2_pack(__uint_as_float(h0), __uint_as_float(h1)));
    f2_unpack(lo, a, b);
    l0 = t5_tf32i(a);
    l1 = t5_tf32i(b);
}

template <int RC, int TERMS>
__global__ void __launch_bounds__(T5_THREADS, 1)
nbody_tc5_kernel(const TargetBlock *__restrict__ blocks, int N, int R, int chunk, const float4 *__restrict__ pos,
                 const float4 *__restrict__ nrm, const float2 *__restrict__ sw, float k, float eta,
                 float2 *__restrict__ ypart, double2 *__restrict__ y, size_t split_stride, int *__restrict__ err)
{
    extern __shared__ __align__(1024) unsigned char t5_smem_raw[];
    __shared__ uint32_t s_taddr;
    __shared__ __align__(8) unsigned long long s_mbar;
    __shared__ int s_forced;                           // host-set flag: take the timeout exit
    __shared__ __align__(16) float s_src[6][T5_K];     // x, y, z, nx, ny, nz of the tile's sources
    // operand tiles on a 1024-byte boundary (the swizzle atom)
    const uint32_t raw = (uint32_t)__cvta_generic_to_shared(t5_smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const uint32_t sA = base;                          // rh, rl, ih, il: 4 x 16 KB
    const uint32_t sB = base + 4 * T5_A_BYTES;         // b1h, b1l, b2h, b2l: 4 x 8 KB
    const uint32_t mbar = (uint32_t)__cvta_generic_to_shared(&s_mbar);

    const TargetBlock tb = blocks[blockIdx.x >> 2];
    const int sub = blockIdx.x & 3;
    if (sub * T5_M >= tb.count) return;                // whole CTA past the block's end
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr int NC = 2 * RC;                         // accumulator columns
    const int r0 = blockIdx.y * RC;
    // pair-kernel duty: row (target) `row`, sources 16 `half` .. 16 `half` + 15 of a tile
    const int row = tid & (T5_M - 1), half = tid >> 7;
    f2x tx = f2_splat(1e18f), ty = tx, tz = tx;
    if (sub * T5_M + row < tb.count) {
        const float4 p = pos[tb.start + sub * T5_M + row];
        tx = f2_splat(p.x); ty = f2_splat(p.y); tz = f2_splat(p.z);
    }
    const f2x k2 = f2_splat(k), eta2 = f2_splat(eta);
    // B-operand duty: right-hand side bn, sources 4 bc .. 4 bc + 3 (threads with bc < 8)
    const int bn = tid % RC, bc = tid / RC;
    const bool bduty = bc < T5_K / 4;
    const int rb = r0 + bn;
    // accumulator duty: TMEM lanes 32 (warp mod 4) .., columns RC (warp / 4) ..: real parts
    // in warps 0-3, imaginary parts in warps 4-7
    const int orow = 32 * (warp & 3) + lane, ocol = RC * (warp >> 2);
    if (warp == 0) {
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&s_taddr);
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst),
                     "r"(T5_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_forced = *(volatile int *)err < 0 ? 1 : 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_taddr;
    const uint32_t tmem_warp = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)ocol;

    float acc[RC];
#pragma unroll
    for (int q = 0; q < RC; ++q) acc[q] = 0.f;
    uint32_t phase = 0;
    // a negative error flag set by the host before the launch (injected fault) sends the CTA
    // to its timeout exit before any MMA is issued: nothing asynchronous is then in flight
    // (read once by thread 0 before the set-up barrier, so the whole CTA takes one branch)
    bool failed = s_forced != 0;
    const int c0 = blockIdx.z * chunk, c1 = min(N, c0 + chunk);
    // the tile sequence: range 0 = [c0, min(c1, excl_lo)), range 1 = [max(c0, excl_hi), c1)
    const int lo0 = c0, hi0 = min(c1, tb.excl_lo), lo1 = max(c0, tb.excl_hi), hi1 = c1;
    const int n0 = hi0 > lo0 ? (hi0 - lo0 + T5_K - 1) / T5_K : 0;
    const int n1 = hi1 > lo1 ? (hi1 - lo1 + T5_K - 1) / T5_K : 0;
    // registers prefetched for the next tile
    float4 pa = make_float4(-1e18f, -1e18f, -1e18f, 0.f), pn = make_float4(0.f, 0.f, 0.f, 0.f);
    float2 bv[4];
    auto tile_of = [&](int i, int &j0, int &cnt) {
        if (i < n0) { j0 = lo0 + i * T5_K; cnt = min(T5_K, hi0 - j0); }
        else { j0 = lo1 + (i - n0) * T5_K; cnt = min(T5_K, hi1 - j0); }
    };
    auto prefetch = [&](int i) {
        int j0, cnt;
        tile_of(i, j0, cnt);
        pa = make_float4(-1e18f, -1e18f, -1e18f, 0.f);
        pn = make_float4(0.f, 0.f, 0.f, 0.f);
        if (tid < T5_K && tid < cnt) { pa = pos[j0 + tid]; pn = nrm[j0 + tid]; }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int s = 4 * bc + q;
            bv[q] = (bduty && s < cnt && rb < R) ? sw[(size_t)(j0 + s) * R + rb] : make_float2(0.f, 0.f);
        }
    };
    const int ntile = failed ? 0 : n0 + n1;
    if (ntile > 0) prefetch(0);
    for (int it = 0; it < ntile; ++it) {
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();                               // previous tile's operands and accumulator consumed
        if (tid < T5_K) {
            s_src[0][tid] = pa.x; s_src[1][tid] = pa.y; s_src[2][tid] = pa.z;
            s_src[3][tid] = pn.x; s_src[4][tid] = pn.y; s_src[5][tid] = pn.z;
        }
        if (bduty) {   // B operands: rows bn (B1 = Re s', B2 = -Im s') and bn + RC (B1 = Im s', B2 = Re s')
            uint32_t h[4], l[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) { h[q] = t5_tf32i(bv[q].x); l[q] = t5_tf32i(bv[q].x - __uint_as_float(h[q])); }
            t5_st4(sB + 0 * T5_B_BYTES + t5_chunk_off(bn, bc), h[0], h[1], h[2], h[3]);
            if (TERMS == 3) t5_st4(sB + 1 * T5_B_BYTES + t5_chunk_off(bn, bc), l[0], l[1], l[2], l[3]);
            t5_st4(sB + 2 * T5_B_BYTES + t5_chunk_off(bn + RC, bc), h[0], h[1], h[2], h[3]);
            if (TERMS == 3) t5_st4(sB + 3 * T5_B_BYTES + t5_chunk_off(bn + RC, bc), l[0], l[1], l[2], l[3]);
#pragma unroll
            for (int q = 0; q < 4; ++q) { h[q] = t5_tf32i(bv[q].y); l[q] = t5_tf32i(bv[q].y - __uint_as_float(h[q])); }
            t5_st4(sB + 0 * T5_B_BYTES + t5_chunk_off(bn + RC, bc), h[0], h[1], h[2], h[3]);
            if (TERMS == 3) t5_st4(sB + 1 * T5_B_BYTES + t5_chunk_off(bn + RC, bc), l[0], l[1], l[2], l[3]);
#pragma unroll
            for (int q = 0; q < 4; ++q) { h[q] ^= 0x80000000u; l[q] ^= 0x80000000u; }
            t5_st4(sB + 2 * T5_B_BYTES + t5_chunk_off(bn, bc), h[0], h[1], h[2], h[3]);
            if (TERMS == 3) t5_st4(sB + 3 * T5_B_BYTES + t5_chunk_off(bn, bc), l[0], l[1], l[2], l[3]);
        }
        __syncthreads();                               // source tile staged
        if (it + 1 < ntile) prefetch(it + 1);          // overlaps the pair kernels and the MMAs
        // A operands: row `row`, chunks 4 half .. 4 half + 3
#pragma unroll 1
        for (int cc = 0; cc < 4; ++cc) {
            const int c = 4 * half + cc;
            uint32_t rh[4], rl[4], ih[4], il[4];
#pragma unroll
            for (int p = 0; p < 2; ++p) {              // sources 4c + 2p, 4c + 2p + 1
                const int q = 4 * c + 2 * p;
                f2x gr, gi;
                t5_pair2(tx, ty, tz, *reinterpret_cast<const f2x *>(&s_src[0][q]),
                         *reinterpret_cast<const f2x *>(&s_src[1][q]), *reinterpret_cast<const f2x *>(&s_src[2][q]),
                         *reinterpret_cast<const f2x *>(&s_src[3][q]), *reinterpret_cast<const f2x *>(&s_src[4][q]),
                         *reinterpret_cast<const f2x *>(&s_src[5][q]), k2, eta2, gr, gi);
                t5_split2(gr, rh[2 * p], rh[2 * p + 1], rl[2 * p], rl[2 * p + 1]);
                t5_split2(gi, ih[2 * p], ih[2 * p + 1], il[2 * p], il[2 * p + 1]);
            }
            const uint32_t off = t5_chunk_off(row, c);
            t5_st4(sA + 0 * T5_A_BYTES + off, rh[0], rh[1], rh[2], rh[3]);
            if (TERMS == 3) t5_st4(sA + 1 * T5_A_BYTES + off, rl[0], rl[1], rl[2], rl[3]);
            t5_st4(sA + 2 * T5_A_BYTES + off, ih[0], ih[1], ih[2], ih[3]);
            if (TERMS == 3) t5_st4(sA + 3 * T5_A_BYTES + off, il[0], il[1], il[2], il[3]);
        }
        // make the generic-proxy stores visible to the tensor cores, then issue
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            // products: (A tile, B tile) = Re G x B1 and Im G x B2, each hi.hi, hi.lo, lo.hi
            // (TERMS = 3) or hi.hi alone (TERMS = 1: the first and fourth of these)
            constexpr int NP = TERMS == 3 ? 6 : 2;
            const int am[6] = {0, TERMS == 3 ? 0 : 2, 1, 2, 2, 3}, bm[6] = {0, TERMS == 3 ? 1 : 2, 0, 2, 3, 2};
#pragma unroll
            for (int ks = 0; ks < T5_K / 8; ++ks)
#pragma unroll
                for (int p = 0; p < NP; ++p)
                    t5_mma(tmem, t5_desc(sA + am[p] * T5_A_BYTES + 32 * ks), t5_desc(sB + bm[p] * T5_B_BYTES + 32 * ks),
                           t5_idesc(NC), (ks | p) ? 1u : 0u);
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                         : "memory");
        }
        const bool ok = t5_wait(mbar, phase);
        phase ^= 1u;
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (RC == 32) t5_ld32(tmem_warp, acc);
        else t5_ld16(tmem_warp, acc);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(T5_TMEM_COLS) : "memory");
    if (failed && tid == 0) atomicExch(err, 1);
    const int t = sub * T5_M + orow;
    if (t >= tb.count) return;
    // columns ocol .. ocol + RC - 1: real parts (ocol = 0) or imaginary parts (ocol = RC)
#pragma unroll
    for (int r = 0; r < RC; ++r) {
        if (r0 + r >= R) break;
        const size_t e = (size_t)(tb.start + t) * R + r0 + r;
        const float v = failed ? __int_as_float(0x7fc00000) : acc[r];
        if (ypart) reinterpret_cast<float *>(ypart + blockIdx.z * split_stride + e)[ocol ? 1 : 0] = v;
        else reinterpret_cast<double *>(y + e)[ocol ? 1 : 0] = (double)v;
    }
}

// ---------------------------------------------------------------- warp-specialised form
//
// The same contraction with the tile phases on separate warps, synchronised by
// mbarriers only (no block barrier inside the tile loop):
//   warps 0-15  producers (four per target row): stage the tile's sources (producer-only
//               named barrier), write the density (B) and pair-kernel (A) operands of
//               stage s = i mod 2 once the MMAs of tile i - 2 released it (`empty[s]`),
//               then arrive on `full[s]` (512 arrivals);
//   warp 20     one thread issues the 24 MMAs of tile i into accumulator b = i mod 2 once
//               `full[s]` completed and the epilogue released b (`accempty[b]`), then
//               commits to `empty[s]` and `accfull[b]`;
//   warps 16-19 epilogue: wait `accfull[b]`, read the 128 lanes x 2RC columns
//               (tcgen05.ld), add them to FP32 sums, arrive on `accempty[b]` (128).
// A wait that runs out sets a shared abort flag that every other wait polls; producer
// decisions to stop are made together (bar.red.or on the producers' barrier), so no
// named barrier is left waiting.
static const int WS_PROD_WARPS = 16;
static const int WS_PROD = WS_PROD_WARPS * 32;      // producer threads
static const int WS_THREADS = (WS_PROD_WARPS + 5) * 32;
static const int WS_SMEM = 2 * T5_STAGE + 1024;

__device__ __forceinline__ bool ws_wait(uint32_t mbar, uint32_t parity, volatile int *abort_flag)
{
    for (int it = 0; it < (1 << 22); ++it) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (ok) return true;
        if (*abort_flag) return false;
    }
    *abort_flag = 1;
    return false;
}

__device__ __forceinline__ void ws_arrive(uint32_t mbar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}

// producers' named barrier (id 1, all producer threads) that also ORs a flag across them
__device__ __forceinline__ bool ws_prod_sync_or(bool v)
{
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(WS_PROD)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void ws_prod_sync()
{
    asm volatile("bar.sync 1, %0;" ::"n"(WS_PROD) : "memory");
}

template <int RC>
__global__ void __launch_bounds__(WS_THREADS, 1)
nbody_tc5ws_kernel(const TargetBlock *__restrict__ blocks, int N, int R, int chunk, const float4 *__restrict__ pos,
                   const float4 *__restrict__ nrm, const float2 *__restrict__ sw, float k, float eta,
                   float2 *__restrict__ ypart, double2 *__restrict__ y, size_t split_stride, int *__restrict__ err)
{
    constexpr int NC = 2 * RC;                         // accumulator columns: [Re y | Im y]
    extern __shared__ __align__(1024) unsigned char ws_smem_raw[];
    __shared__ uint32_t s_taddr;
    __shared__ __align__(8) unsigned long long s_bar[8];   // full[2], empty[2], accfull[2], accempty[2]
    __shared__ int s_abort;
    __shared__ __align__(16) float s_src[6][T5_K];
    const uint32_t raw = (uint32_t)__cvta_generic_to_shared(ws_smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const uint32_t bar0 = (uint32_t)__cvta_generic_to_shared(&s_bar[0]);
    const uint32_t full0 = bar0, empty0 = bar0 + 16, accfull0 = bar0 + 32, accempty0 = bar0 + 48;
    volatile int *abort_flag = &s_abort;

    const TargetBlock tb = blocks[blockIdx.x >> 2];
    const int sub = blockIdx.x & 3;
    if (sub * T5_M >= tb.count) return;                // whole CTA past the block's end
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int r0 = blockIdx.y * RC;
    if (warp == 0) {
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&s_taddr);
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst),
                     "r"(T5_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int q = 0; q < 2; ++q) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(full0 + 8 * q), "r"(WS_PROD)
                         : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(empty0 + 8 * q), "r"(1) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(accfull0 + 8 * q), "r"(1) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(accempty0 + 8 * q), "r"(128) : "memory");
        }
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_taddr;

    const int c0 = blockIdx.z * chunk, c1 = min(N, c0 + chunk);
    const int lo0 = c0, hi0 = min(c1, tb.excl_lo), lo1 = max(c0, tb.excl_hi), hi1 = c1;
    const int n0 = hi0 > lo0 ? (hi0 - lo0 + T5_K - 1) / T5_K : 0;
    const int n1 = hi1 > lo1 ? (hi1 - lo1 + T5_K - 1) / T5_K : 0;
    const int ntile = n0 + n1;

    if (warp < WS_PROD_WARPS) {
        // ------------------------------------------------ producers
        const int row = tid & (T5_M - 1), quarter = tid >> 7;   // sources 8 quarter .. 8 quarter + 7
        f2x tx = f2_splat(1e18f), ty = tx, tz = tx;
        if (sub * T5_M + row < tb.count) {
            const float4 p = pos[tb.start + sub * T5_M + row];
            tx = f2_splat(p.x); ty = f2_splat(p.y); tz = f2_splat(p.z);
        }
        const f2x k2 = f2_splat(k), eta2 = f2_splat(eta);
        const int bn = tid % RC, bc = tid / RC;
        const bool bduty = bc < T5_K / 4;
        const int rb = r0 + bn;
        float4 pa = make_float4(-1e18f, -1e18f, -1e18f, 0.f), pn = make_float4(0.f, 0.f, 0.f, 0.f);
        float2 bv[4];
        auto prefetch = [&](int i) {
            int j0, cnt;
            if (i < n0) { j0 = lo0 + i * T5_K; cnt = min(T5_K, hi0 - j0); }
            else { j0 = lo1 + (i - n0) * T5_K; cnt = min(T5_K, hi1 - j0); }
            pa = make_float4(-1e18f, -1e18f, -1e18f, 0.f);
            pn = make_float4(0.f, 0.f, 0.f, 0.f);
            if (tid < T5_K && tid < cnt) { pa = pos[j0 + tid]; pn = nrm[j0 + tid]; }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int sidx = 4 * bc + q;
                bv[q] = (bduty && sidx < cnt && rb < R) ? sw[(size_t)(j0 + sidx) * R + rb] : make_float2(0.f, 0.f);
            }
        };
        if (ntile > 0) prefetch(0);
        for (int it = 0; it < ntile; ++it) {
            const int st = it & 1, u = it >> 1;
            const bool ok = (u == 0) || ws_wait(empty0 + 8 * st, (uint32_t)((u - 1) & 1), abort_flag);
            // all producers agree to go on; also: every producer finished reading s_src
            if (ws_prod_sync_or(!ok || *abort_flag)) break;
            const uint32_t sA = base + (uint32_t)st * T5_STAGE;
            const uint32_t sB = sA + 4 * T5_A_BYTES;
            if (tid < T5_K) {
                s_src[0][tid] = pa.x; s_src[1][tid] = pa.y; s_src[2][tid] = pa.z;
                s_src[3][tid] = pn.x; s_src[4][tid] = pn.y; s_src[5][tid] = pn.z;
            }
            if (bduty) {
                uint32_t h[4], l[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) { h[q] = t5_tf32i(bv[q].x); l[q] = t5_tf32i(bv[q].x - __uint_as_float(h[q])); }
                t5_st4(sB + 0 * T5_B_BYTES + t5_chunk_off(bn, bc), h[0], h[1], h[2], h[3]);
                t5_st4(sB + 1 * T5_B_BYTES + t5_chunk_off(bn, bc), l[0], l[1], l[2], l[3]);
                t5_st4(sB + 2 * T5_B_BYTES + t5_chunk_off(bn + RC, bc), h[0], h[1], h[2], h[3]);
                t5_st4(sB + 3 * T5_B_BYTES + t5_chunk_off(bn + RC, bc), l[0], l[1], l[2], l[3]);
#pragma unroll
                for (int q = 0; q < 4; ++q) { h[q] = t5_tf32i(bv[q].y); l[q] = t5_tf32i(bv[q].y - __uint_as_float(h[q])); }
                t5_st4(sB + 0 * T5_B_BYTES + t5_chunk_off(bn + RC, bc), h[0], h[1], h[2], h[3]);
                t5_st4(sB + 1 * T5_B_BYTES + t5_chunk_off(bn + RC, bc), l[0], l[1], l[2], l[3]);
#pragma unroll
                for (int q = 0; q < 4; ++q) { h[q] ^= 0x80000000u; l[q] ^= 0x80000000u; }
                t5_st4(sB + 2 * T5_B_BYTES + t5_chunk_off(bn, bc), h[0], h[1], h[2], h[3]);
                t5_st4(sB + 3 * T5_B_BYTES + t5_chunk_off(bn, bc), l[0], l[1], l[2], l[3]);
            }
            ws_prod_sync();                            // source tile staged
            if (it + 1 < ntile) prefetch(it + 1);
#pragma unroll
            for (int cc = 0; cc < 2; ++cc) {
                const int c = 2 * quarter + cc;
                uint32_t rh[4], rl[4], ih[4], il[4];
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    const int q = 4 * c + 2 * p;
                    f2x gr, gi;
                    t5_pair2(tx, ty, tz, *reinterpret_cast<const f2x *>(&s_src[0][q]),
                             *reinterpret_cast<const f2x *>(&s_src[1][q]),
                             *reinterpret_cast<const f2x *>(&s_src[2][q]),
                             *reinterpret_cast<const f2x *>(&s_src[3][q]),
                             *reinterpret_cast<const f2x *>(&s_src[4][q]),
                             *reinterpret_cast<const f2x *>(&s_src[5][q]), k2, eta2, gr, gi);
                    t5_split2(gr, rh[2 * p], rh[2 * p + 1], rl[2 * p], rl[2 * p + 1]);
                    t5_split2(gi, ih[2 * p], ih[2 * p + 1], il[2 * p], il[2 * p + 1]);
                }
                const uint32_t off = t5_chunk_off(row, c);
                t5_st4(sA + 0 * T5_A_BYTES + off, rh[0], rh[1], rh[2], rh[3]);
                t5_st4(sA + 1 * T5_A_BYTES + off, rl[0], rl[1], rl[2], rl[3]);
                t5_st4(sA + 2 * T5_A_BYTES + off, ih[0], ih[1], ih[2], ih[3]);
                t5_st4(sA + 3 * T5_A_BYTES + off, il[0], il[1], il[2], il[3]);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            ws_arrive(full0 + 8 * st);
        }
    } else if (warp < WS_PROD_WARPS + 4) {
        // ------------------------------------------------ epilogue
        const int q4 = warp - WS_PROD_WARPS;           // TMEM lane quarter (warp mod 4)
        const uint32_t tl = tmem + ((uint32_t)(32 * q4) << 16);
        float acc[NC];
#pragma unroll
        for (int q = 0; q < NC; ++q) acc[q] = 0.f;
        for (int it = 0; it < ntile; ++it) {
            const int b = it & 1, v = it >> 1;
            if (!ws_wait(accfull0 + 8 * b, (uint32_t)(v & 1), abort_flag)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int q = 0; q < NC / 16; ++q) t5_ld16(tl + 64 * b + 16 * q, acc + 16 * q);
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            ws_arrive(accempty0 + 8 * b);
        }
        const bool failed = *abort_flag != 0;
        const int t = sub * T5_M + 32 * q4 + lane;
        if (t < tb.count) {
#pragma unroll
            for (int r = 0; r < RC; ++r) {
                if (r0 + r >= R) break;
                const size_t e = (size_t)(tb.start + t) * R + r0 + r;
                float2 v = make_float2(acc[r], acc[RC + r]);
                if (failed) v = make_float2(__int_as_float(0x7fc00000), __int_as_float(0x7fc00000));
                if (ypart) ypart[blockIdx.z * split_stride + e] = v;
                else y[e] = make_double2((double)v.x, (double)v.y);
            }
        }
    } else if (lane == 0) {
        // ------------------------------------------------ MMA issue
        const int am[6] = {0, 0, 1, 2, 2, 3}, bm[6] = {0, 1, 0, 2, 3, 2};
        for (int it = 0; it < ntile; ++it) {
            const int st = it & 1, u = it >> 1;
            if (!ws_wait(full0 + 8 * st, (uint32_t)(u & 1), abort_flag)) break;
            if (u >= 1 && !ws_wait(accempty0 + 8 * st, (uint32_t)((u - 1) & 1), abort_flag)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sA = base + (uint32_t)st * T5_STAGE;
            const uint32_t sB = sA + 4 * T5_A_BYTES;
#pragma unroll
            for (int ks = 0; ks < T5_K / 8; ++ks)
#pragma unroll
                for (int p = 0; p < 6; ++p)
                    t5_mma(tmem + 64 * st, t5_desc(sA + am[p] * T5_A_BYTES + 32 * ks),
                           t5_desc(sB + bm[p] * T5_B_BYTES + 32 * ks), t5_idesc(NC), (ks | p) ? 1u : 0u);
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             empty0 + 8 * st)
                         : "memory");
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             accfull0 + 8 * st)
                         : "memory");
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(T5_TMEM_COLS) : "memory");
    if (tid == 0 && s_abort) atomicExch(err, 1);
}

// mode: T5_SPLIT3 (three-term TF32 split, FP32-level products), T5_WS (the same, warp-
// specialised), T5_SINGLE (TF32 products alone: about 3e-4 relative error in the sum, 1.4x
// faster; for inner solves whose refinement tolerates it)
hzb_status interbody_tc5(hzb_ctx *c, int R, const double2 *sigma, double2 *y, int nsplit, int mode)
{
    const bool ws = mode == T5_WS;
    if (!c->nodes_ready) return fail(c, HZB_ESTATE, "nodes not built");
    const int N = (int)c->N;
    int chunk = (N + nsplit - 1) / nsplit;
    chunk = ((chunk + T5_K - 1) / T5_K) * T5_K;
    nsplit = (N + chunk - 1) / chunk;
    const size_t n = (size_t)N * R;
    float2 *part = nullptr;
    if (nsplit > 1) {
        if (check_cuda(c, c->nb_part32.ensure(n * nsplit), "alloc partial sums")) return HZB_ENOMEM;
        part = c->nb_part32.ptr;
    }
    if (check_cuda(c, c->kerr.ensure(1), "alloc error flag")) return HZB_ENOMEM;
    if (!c->kerr_ready) {
        if (check_cuda(c, cudaMemsetAsync(c->kerr.ptr, 0, sizeof(int), c->stream), "clear error flag"))
            return HZB_ECUDA;
        c->kerr_ready = true;
    }
    static bool attr_done[64] = {false};
    const int dev = c->opt.device;
    if (dev >= 0 && dev < 64 && !attr_done[dev]) {
        if (check_cuda(c, cudaFuncSetAttribute(nbody_tc5_kernel<16, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               T5_SMEM), "tcgen05 kernel shared memory") ||
            check_cuda(c, cudaFuncSetAttribute(nbody_tc5_kernel<32, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               T5_SMEM), "tcgen05 kernel shared memory") ||
            check_cuda(c, cudaFuncSetAttribute(nbody_tc5_kernel<16, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               T5_SMEM), "tcgen05 kernel shared memory") ||
            check_cuda(c, cudaFuncSetAttribute(nbody_tc5_kernel<32, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               T5_SMEM), "tcgen05 kernel shared memory") ||
            check_cuda(c, cudaFuncSetAttribute(nbody_tc5ws_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               WS_SMEM), "tcgen05 kernel shared memory") ||
            check_cuda(c, cudaFuncSetAttribute(nbody_tc5ws_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               WS_SMEM), "tcgen05 kernel shared memory"))
            return HZB_ECUDA;
        attr_done[dev] = true;
    }
    if ((c->fault & FAULT_TIMEOUT) && !(c->fault_spent & FAULT_TIMEOUT) && !c->capturing && !ws) {
        c->fault_spent |= FAULT_TIMEOUT;   // injected: every CTA takes the timeout exit (flag -1)
        if (check_cuda(c, cudaMemsetAsync(c->kerr.ptr, 0xff, sizeof(int), c->stream), "inject timeout"))
            return HZB_ECUDA;
    }
    c->interbody_calls++;
    c->launches += (nsplit > 1) ? 3 : 2;
    const int slot = prof_begin(c, 1);
    const float2 *sw = weighted_sigma32(c, R, sigma);
    if (!sw) return HZB_ENOMEM;
    const int rc = (R <= 16) ? 16 : 32;
    dim3 grid(c->n_tblocks * 4, (R + rc - 1) / rc, nsplit);
    const float k = (float)c->k, eta = (float)c->eta;
    if (ws && rc == 16)
        nbody_tc5ws_kernel<16><<<grid, WS_THREADS, WS_SMEM, c->stream>>>(c->tblocks.ptr, N, R, chunk, c->pos32.ptr,
                                                                        c->nrm32.ptr, sw, k, eta, part, y, n,
                                                                        c->kerr.ptr);
    else if (ws)
        nbody_tc5ws_kernel<32><<<grid, WS_THREADS, WS_SMEM, c->stream>>>(c->tblocks.ptr, N, R, chunk, c->pos32.ptr,
                                                                        c->nrm32.ptr, sw, k, eta, part, y, n,
                                                                        c->kerr.ptr);
    else {
        auto launch = [&](auto kern) {
            kern<<<grid, T5_THREADS, T5_SMEM, c->stream>>>(c->tblocks.ptr, N, R, chunk, c->pos32.ptr, c->nrm32.ptr, sw,
                                                           k, eta, part, y, n, c->kerr.ptr);
        };
        const bool single = mode == T5_SINGLE;
        if (rc == 16) launch(single ? nbody_tc5_kernel<16, 1> : nbody_tc5_kernel<16, 3>);
        else launch(single ? nbody_tc5_kernel<32, 1> : nbody_tc5_kernel<32, 3>);
    }
    if (nsplit > 1) split_reduce_f2(c, n, nsplit, part, y);
    cudaError_t e = cudaGetLastError();
    prof_end(c, slot);
    if (check_cuda(c, e, "nbody_tc5_kernel")) return HZB_ECUDA;
    if (!c->capturing && !c->in_solve) {   // a bounded wait that ran out: outputs are NaN (a solve
                                           // reads the flag once at its end instead)
        int flag = 0;
        if (check_cuda(c, cudaMemcpyAsync(&flag, c->kerr.ptr, sizeof(int), cudaMemcpyDeviceToHost, c->stream),
                       "read error flag") ||
            check_cuda(c, cudaStreamSynchronize(c->stream), "nbody_tc5_kernel"))
            return HZB_ECUDA;
        if (flag) {                    // report once; the context stays usable for the next call
            if (check_cuda(c, cudaMemsetAsync(c->kerr.ptr, 0, sizeof(int), c->stream), "clear error flag"))
                return HZB_ECUDA;
            return fail(c, HZB_ETIMEOUT, "tensor-core wait timed out in nbody_tc5_kernel");
        }
    }
    return HZB_OK;
}

}  // namespace hzb
