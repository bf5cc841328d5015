// Throughput microbenchmarks of the GPU's arithmetic pipes, the denominators of the
// inter-body and modal kernels' rooflines: FP32 fused multiply-add (scalar and packed
// f32x2), FP64 fused multiply-add, the transcendental unit (rsqrt, sin, cos) and the
// TF32 tensor cores through tcgen05.  Each kernel runs independent dependency chains
// long enough (tens of milliseconds) that launch and tail effects are below 1 %, on
// every SM, and is timed with CUDA events on the context's stream.  Not part of the
// paper: measurement infrastructure for this GPU.
#include <cstdint>

#include "f32x2.cuh"
#include "hzb_internal.h"
#include "tcgen05.cuh"

namespace hzb {

static const int PK_THREADS = 256;
static const int PK_CHAINS = 8;          // independent chains per thread

// a x + b in PK_CHAINS chains, `iters` rounds; the result is stored only when it is
// exactly `never` (which it is not), so the loop is kept without a memory stream
__global__ void __launch_bounds__(PK_THREADS) peak_ffma_kernel(int iters, float a, float b, float never, float *out)
{
    float v[PK_CHAINS];
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) v[c] = threadIdx.x * 1e-3f + c;
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int c = 0; c < PK_CHAINS; ++c) v[c] = fmaf(v[c], a, b);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) s += v[c];
    if (s == never) out[0] = s;
}

__global__ void __launch_bounds__(PK_THREADS) peak_ffma2_kernel(int iters, float a, float b, float never, float *out)
{
    f2x v[PK_CHAINS];
    const f2x a2 = f2_splat(a), b2 = f2_splat(b);
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) v[c] = f2_pack(threadIdx.x * 1e-3f + c, c * 0.5f);
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int c = 0; c < PK_CHAINS; ++c) v[c] = f2_fma(v[c], a2, b2);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) {
        float lo, hi;
        f2_unpack(v[c], lo, hi);
        s += lo + hi;
    }
    if (s == never) out[0] = s;
}

__global__ void __launch_bounds__(PK_THREADS) peak_dfma_kernel(int iters, double a, double b, double never, double *out)
{
    double v[PK_CHAINS];
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) v[c] = threadIdx.x * 1e-3 + c;
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int c = 0; c < PK_CHAINS; ++c) v[c] = fma(v[c], a, b);
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) s += v[c];
    if (s == never) out[0] = s;
}

// one rsqrt, one sin and one cos per chain and round (the three transcendental-unit
// operations of an FP32 pair kernel); the adds keep the arguments in range
__global__ void __launch_bounds__(PK_THREADS) peak_mufu_kernel(int iters, float never, float *out)
{
    float v[PK_CHAINS];
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) v[c] = 1.0f + threadIdx.x * 1e-4f + c * 1e-2f;
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int c = 0; c < PK_CHAINS; ++c) v[c] = 1.5f + rsqrtf(v[c]) + __sinf(v[c]) * __cosf(v[c]);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) s += v[c];
    if (s == never) out[0] = s;
}

// tcgen05.mma.kind::tf32, M = 128, N = 256, K = 8, cta_group::1, operands resident in
// shared memory (K-major, 128-byte swizzle, 128 x 32 and 256 x 32 tiles of TF32 ones),
// accumulator in 256 tensor-memory columns.  One thread issues `iters` rounds of the
// tile's 4 k-steps; every 16 rounds it commits to an mbarrier and waits (bounded), so
// the issue queue never runs far ahead.  A wait that runs out sets *err and ends the
// loop; tensor memory is freed on every path.
static const int PT_A = 128 * 32 * 4, PT_B = 256 * 32 * 4;
static const int PT_SMEM = 120 * 1024;      // 49 KB used; the rest keeps one CTA per SM

__global__ void __launch_bounds__(128, 1) peak_tf32_kernel(int iters, int *err)
{
    extern __shared__ __align__(1024) unsigned char pt_raw[];
    __shared__ uint32_t s_taddr;
    __shared__ __align__(8) unsigned long long s_mbar;
    __shared__ int s_fail;
    const uint32_t raw = (uint32_t)__cvta_generic_to_shared(pt_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const uint32_t sA = base, sB = base + PT_A;
    const uint32_t mbar = (uint32_t)__cvta_generic_to_shared(&s_mbar);
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t one = t5_tf32(1.0f);
    for (int q = tid; q < (PT_A + PT_B) / 16; q += blockDim.x)
        t5_st4(base + 16 * q, one, one, one, one);
    if (warp == 0) {
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&s_taddr);
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst), "r"(256)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        s_fail = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_taddr;
    if (tid == 0) {
        uint32_t phase = 0;
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int ks = 0; ks < 4; ++ks)
                t5_mma(tmem, t5_desc(sA + 32 * ks), t5_desc(sB + 32 * ks), t5_idesc(256), (it | ks) ? 1u : 0u);
            if ((it & 15) == 15 || it + 1 == iters) {
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                             : "memory");
                if (!t5_wait(mbar, phase)) {
                    s_fail = 1;
                    break;
                }
                phase ^= 1u;
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256) : "memory");
    if (tid == 0 && s_fail) atomicExch(err, 1);
}

}  // namespace hzb

using namespace hzb;

extern "C" hzb_status hzb_measure_peak(hzb_ctx *c, int kind, double *value)
{
    HZB_GUARD(c);
    if (!value || kind < 0 || kind > 4) return fail(c, HZB_EINVAL, "kind in 0..4 and a non-null output");
    int nsm = 0;
    if (check_cuda(c, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->opt.device), "SM count"))
        return HZB_ECUDA;
    if (check_cuda(c, c->red.ensure(4), "alloc") || check_cuda(c, c->kerr.ensure(1), "alloc"))
        return HZB_ENOMEM;
    if (!c->kerr_ready) {
        if (check_cuda(c, cudaMemsetAsync(c->kerr.ptr, 0, sizeof(int), c->stream), "clear error flag"))
            return HZB_ECUDA;
        c->kerr_ready = true;
    }
    const dim3 grid(nsm * 8), block(PK_THREADS);
    double ops = 0.0;                       // operations (FMA = 2 flops) or instructions per launch
    auto launch = [&](int iters) {
        switch (kind) {
        case 0: peak_ffma_kernel<<<grid, block, 0, c->stream>>>(iters, 0.999f, 1e-3f, -1.f, (float *)c->red.ptr); break;
        case 1: peak_ffma2_kernel<<<grid, block, 0, c->stream>>>(iters, 0.999f, 1e-3f, -1.f, (float *)c->red.ptr); break;
        case 2: peak_dfma_kernel<<<grid, block, 0, c->stream>>>(iters, 0.999, 1e-3, -1.0, c->red.ptr); break;
        case 3: peak_mufu_kernel<<<grid, block, 0, c->stream>>>(iters, -1.f, (float *)c->red.ptr); break;
        default: peak_tf32_kernel<<<nsm, 128, PT_SMEM, c->stream>>>(iters, c->kerr.ptr); break;
        }
    };
    int iters = 0;
    const double thr = (double)grid.x * PK_THREADS * PK_CHAINS;
    switch (kind) {
    case 0: iters = 1 << 19; ops = 2.0 * thr * iters; break;                 // flops
    case 1: iters = 1 << 18; ops = 4.0 * thr * iters; break;                 // flops (two lanes)
    case 2: iters = 1 << 13; ops = 2.0 * thr * iters; break;                 // flops
    case 3: iters = 1 << 14; ops = 3.0 * thr * iters; break;                 // rsqrt + sin + cos
    default: iters = 1 << 17; ops = 4.0 * 2.0 * 128 * 256 * 8 * (double)nsm * iters; break;   // flops
    }
    if (kind == 4 &&
        check_cuda(c, cudaFuncSetAttribute(peak_tf32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, PT_SMEM),
                   "peak kernel shared memory"))
        return HZB_ECUDA;
    launch(iters / 16);                     // warm-up
    cudaEventRecord(c->ev0, c->stream);
    launch(iters);
    cudaEventRecord(c->ev1, c->stream);
    if (check_cuda(c, cudaGetLastError(), "peak kernel") || check_cuda(c, cudaEventSynchronize(c->ev1), "peak kernel"))
        return HZB_ECUDA;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    c->launches += 2;
    if (kind == 4) {
        int flag = 0;
        if (check_cuda(c, cudaMemcpy(&flag, c->kerr.ptr, sizeof(int), cudaMemcpyDeviceToHost), "error flag"))
            return HZB_ECUDA;
        if (flag) {
            cudaMemsetAsync(c->kerr.ptr, 0, sizeof(int), c->stream);
            return fail(c, HZB_ETIMEOUT, "tcgen05 wait timed out in the peak kernel");
        }
    }
    *value = ops / (ms * 1e-3) / 1e12;      // T(FL)OP/s, or T operations/s of the transcendental unit
    return HZB_OK;
}
