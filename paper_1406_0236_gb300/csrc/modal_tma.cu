// FP32 per-mode scattering GEMM (Eq. (singleinverse), step (2) of the D^{-1} apply) on
// the 5th-generation tensor cores with operands brought in by the tensor memory
// accelerator (TMA).
//
// With the real embedding  [Cr; Ci] = [[Sr, -Si], [Si, Sr]] [Xr; Xi]  (M = K = 2n) and the
// TF32 three-term split x = hi + lo (A B ~ Ahi Bhi + Ahi Blo + Alo Bhi):
//   * once per shape, embed_split_S_kernel writes the embedded S_p as two TF32 planes
//     (hi, lo) per mode, K-major rows of pitch KP = 2n rounded up to 4 floats;
//   * per apply, embed_split_X_kernel writes the panel X_p the same way (rows = panel
//     columns, K = 2n along the row);
//   * modal_gemm_tma_kernel: a CTA owns a 128 x 64 tile of the embedded C of one mode.
//     Warp 8 (one thread) streams 32-wide K chunks of the four operand tiles with
//     cp.async.bulk.tensor (3-D tensor maps, 128-byte swizzle: the tiles land in the
//     K-major layout the MMA descriptors describe) into two shared-memory stages, and
//     issues 12 tcgen05.mma.kind::tf32 per chunk into one of two tensor-memory
//     accumulators; warps 0-7 drain an accumulator (tcgen05.ld, 32 lanes x 32 columns
//     per warp) into FP32 registers every two chunks, so no chain of tensor-core
//     accumulations is longer than 24 MMAs.  Stages, accumulators and drains hand over
//     through mbarriers; every wait is bounded and a timeout writes NaN and sets the
//     context's device error flag.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <mutex>

#include "hzb_internal.h"
#include "tcgen05.cuh"

namespace hzb {

static const int MT_M = 128, MT_N = 64, MT_K = 32, MT_FLUSH = 2;
static const int MT_A = MT_M * MT_K * 4, MT_B = MT_N * MT_K * 4;          // 16 KB, 8 KB
static const int MT_STAGE = 2 * MT_A + 2 * MT_B;                          // hi/lo of A and B
static const int MT_SMEM = 2 * MT_STAGE + 1024;
static const int MT_THREADS = 9 * 32;

static inline int kpitch(int n) { return (2 * n + 3) & ~3; }

__device__ __forceinline__ void mt_split(double a, float &hi, float &lo)
{
    hi = __uint_as_float(t5_tf32i((float)a));
    lo = __uint_as_float(t5_tf32i((float)(a - (double)hi)));
}

// plane (2p + h), row m, column k of the embedded, split S_p
__global__ void embed_split_S_kernel(int n, int KP, int M1, const double2 *__restrict__ S, float *__restrict__ img)
{
    const int n2 = 2 * n;
    const size_t total = (size_t)M1 * n2 * KP;
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    const int k = (int)(e % KP);
    const size_t rest = e / KP;
    const int m = (int)(rest % n2), p = (int)(rest / n2);
    float hi = 0.f, lo = 0.f;
    if (k < n2) {
        const int mr = m < n ? m : m - n, kr = k < n ? k : k - n;
        const double2 v = S[((size_t)p * n + mr) * n + kr];
        const double a = (m < n) ? (k < n ? v.x : -v.y) : (k < n ? v.y : v.x);
        mt_split(a, hi, lo);
    }
    img[((size_t)(2 * p) * n2 + m) * KP + k] = hi;
    img[((size_t)(2 * p + 1) * n2 + m) * KP + k] = lo;
}

// plane (2p + h), row = panel column c, column k of [Xr; Xi] split
__global__ void embed_split_X_kernel(int n, int KP, int nc, int M1, const float2 *__restrict__ X,
                                     float *__restrict__ img)
{
    const int n2 = 2 * n;
    const size_t total = (size_t)M1 * nc * KP;
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    const int k = (int)(e % KP);
    const size_t rest = e / KP;
    const int col = (int)(rest % nc), p = (int)(rest / nc);
    float hi = 0.f, lo = 0.f;
    if (k < n2) {
        const float2 v = X[((size_t)p * n + (k < n ? k : k - n)) * nc + col];
        mt_split((double)(k < n ? v.x : v.y), hi, lo);
    }
    img[((size_t)(2 * p) * nc + col) * KP + k] = hi;
    img[((size_t)(2 * p + 1) * nc + col) * KP + k] = lo;
}

__device__ __forceinline__ void mt_tma3(uint32_t dst, const CUtensorMap *map, int x, int y, int z, uint32_t mbar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(mbar)
        : "memory");
}

__device__ __forceinline__ bool mt_wait(uint32_t mbar, uint32_t parity, volatile int *abort_flag)
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

__global__ void __launch_bounds__(MT_THREADS, 1)
modal_gemm_tma_kernel(int n, int nc, const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                      float2 *__restrict__ C, int *__restrict__ err)
{
    extern __shared__ __align__(1024) unsigned char mt_smem_raw[];
    __shared__ uint32_t s_taddr;
    __shared__ __align__(8) unsigned long long s_bar[8];   // tma_full[2], mma_done[2], acc_full[2], acc_free[2]
    __shared__ int s_abort;
    const uint32_t raw = (uint32_t)__cvta_generic_to_shared(mt_smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const uint32_t bar0 = (uint32_t)__cvta_generic_to_shared(&s_bar[0]);
    const uint32_t tma_full0 = bar0, mma_done0 = bar0 + 16, acc_full0 = bar0 + 32, acc_free0 = bar0 + 48;
    volatile int *abort_flag = &s_abort;
    const int p = blockIdx.z, m0 = blockIdx.y * MT_M, c0 = blockIdx.x * MT_N;
    const int n2 = 2 * n;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) {
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&s_taddr);
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst), "r"(2 * MT_N)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int q = 0; q < 2; ++q) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tma_full0 + 8 * q), "r"(1) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mma_done0 + 8 * q), "r"(1) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(acc_full0 + 8 * q), "r"(1) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(acc_free0 + 8 * q), "r"(256) : "memory");
        }
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_taddr;
    const int nk = (n2 + MT_K - 1) / MT_K;
    const int ng = (nk + MT_FLUSH - 1) / MT_FLUSH;

    if (warp == 8) {
        if (lane == 0) {
            // ---------------------------------------------- TMA and MMA issue
            auto issue_tma = [&](int kc) {
                const int st = kc & 1;
                const uint32_t sA = base + (uint32_t)st * MT_STAGE;
                const uint32_t fb = tma_full0 + 8 * st;
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(MT_STAGE)
                             : "memory");
                mt_tma3(sA, &tmA, kc * MT_K, m0, 2 * p, fb);
                mt_tma3(sA + MT_A, &tmA, kc * MT_K, m0, 2 * p + 1, fb);
                mt_tma3(sA + 2 * MT_A, &tmB, kc * MT_K, c0, 2 * p, fb);
                mt_tma3(sA + 2 * MT_A + MT_B, &tmB, kc * MT_K, c0, 2 * p + 1, fb);
            };
            bool ok = true;
            if (nk > 0) issue_tma(0);
            for (int kc = 0; kc < nk && ok; ++kc) {
                if (kc + 1 < nk) {
                    // stage of chunk kc + 1 was read by the MMAs of chunk kc - 1
                    if (kc >= 1 && !mt_wait(mma_done0 + 8 * ((kc + 1) & 1), (uint32_t)(((kc - 1) >> 1) & 1),
                                            abort_flag)) { ok = false; break; }
                    issue_tma(kc + 1);
                }
                const int st = kc & 1;
                if (!mt_wait(tma_full0 + 8 * st, (uint32_t)((kc >> 1) & 1), abort_flag)) { ok = false; break; }
                const int g = kc / MT_FLUSH, b = g & 1;
                const bool first = (kc % MT_FLUSH) == 0;
                if (first && g >= 2 &&
                    !mt_wait(acc_free0 + 8 * b, (uint32_t)(((g >> 1) - 1) & 1), abort_flag)) { ok = false; break; }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t sA = base + (uint32_t)st * MT_STAGE;
                const uint32_t as[3] = {sA, sA, sA + MT_A};
                const uint32_t bs[3] = {sA + 2 * MT_A, sA + 2 * MT_A + MT_B, sA + 2 * MT_A};
#pragma unroll
                for (int ks = 0; ks < MT_K / 8; ++ks)
#pragma unroll
                    for (int t = 0; t < 3; ++t)
                        t5_mma(tmem + MT_N * b, t5_desc(as[t] + 32 * ks), t5_desc(bs[t] + 32 * ks), t5_idesc(MT_N),
                               (first && ks == 0 && t == 0) ? 0u : 1u);
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 mma_done0 + 8 * st)
                             : "memory");
                if ((kc % MT_FLUSH) == MT_FLUSH - 1 || kc == nk - 1)
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                     acc_full0 + 8 * b)
                                 : "memory");
            }
        }
    } else {
        // -------------------------------------------------- drain (warps 0-7)
        float acc[32];
#pragma unroll
        for (int q = 0; q < 32; ++q) acc[q] = 0.f;
        const uint32_t tl = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(32 * (warp >> 2));
        for (int g = 0; g < ng; ++g) {
            const int b = g & 1;
            if (!mt_wait(acc_full0 + 8 * b, (uint32_t)((g >> 1) & 1), abort_flag)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            t5_ld16(tl + MT_N * b, acc);
            t5_ld16(tl + MT_N * b + 16, acc + 16);
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(acc_free0 + 8 * b) : "memory");
        }
        const bool failed = *abort_flag != 0;
        const int r = m0 + 32 * (warp & 3) + lane;
        if (r < n2) {
            const int rr = r < n ? r : r - n, comp = r < n ? 0 : 1;
            float2 *Cp = C + (size_t)p * n * nc;
#pragma unroll
            for (int q = 0; q < 32; ++q) {
                const int col = c0 + 32 * (warp >> 2) + q;
                if (col < nc)
                    reinterpret_cast<float *>(&Cp[(size_t)rr * nc + col])[comp] =
                        failed ? __int_as_float(0x7fc00000) : acc[q];
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * MT_N) : "memory");
    if (tid == 0 && s_abort) atomicExch(err, 1);
}

// ---------------------------------------------------------------- host

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, []() {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// 3-D FP32 tensor map: dims {KP, rows, planes}, box {32, box_rows, 1}, 128-byte swizzle,
// zero fill outside the tensor.
static bool make_map(CUtensorMap *map, float *ptr, int KP, int rows, int planes, int box_rows)
{
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[3] = {(cuuint64_t)KP, (cuuint64_t)rows, (cuuint64_t)planes};
    cuuint64_t strides[2] = {(cuuint64_t)KP * 4, (cuuint64_t)KP * rows * 4};
    cuuint32_t box[3] = {(cuuint32_t)MT_K, (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, ptr, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

hzb_status modal_gemm_tma(hzb_ctx *c, ShapeDev &sd, int ncols, const float2 *X, float2 *Cout)
{
    const int n = sd.geom.NG, M1 = sd.geom.M + 1, KP = kpitch(n);
    static_assert(sizeof(CUtensorMap) <= sizeof(ShapeDev::tmA), "tensor map storage");
    // the shape's embedded, split S_p (once)
    if (!sd.tmA_ready) {
        const size_t na = (size_t)2 * M1 * 2 * n * KP;
        if (check_cuda(c, sd.Aimg.ensure(na), "alloc modal operand image")) return HZB_ENOMEM;
        const size_t total = (size_t)M1 * 2 * n * KP;
        embed_split_S_kernel<<<(unsigned)((total + 255) / 256), 256, 0, c->stream>>>(n, KP, M1, sd.S64.ptr,
                                                                                       sd.Aimg.ptr);
        c->launches++;
        if (!make_map(reinterpret_cast<CUtensorMap *>(sd.tmA), sd.Aimg.ptr, KP, 2 * n, 2 * M1, MT_M))
            return fail(c, HZB_ECUDA, "tensor map of the modal matrices");
        sd.tmA_ready = true;
    }
    const size_t nb = (size_t)2 * M1 * ncols * KP;
    if (check_cuda(c, c->Ximg.ensure(nb), "alloc panel image")) return HZB_ENOMEM;
    const size_t total = (size_t)M1 * ncols * KP;
    embed_split_X_kernel<<<(unsigned)((total + 255) / 256), 256, 0, c->stream>>>(n, KP, ncols, M1, X, c->Ximg.ptr);
    CUtensorMap tmB;
    if (!make_map(&tmB, c->Ximg.ptr, KP, ncols, 2 * M1, MT_N)) return fail(c, HZB_ECUDA, "tensor map of the panel");
    if (check_cuda(c, c->kerr.ensure(1), "alloc error flag")) return HZB_ENOMEM;
    if (!c->kerr_ready) {
        if (check_cuda(c, cudaMemsetAsync(c->kerr.ptr, 0, sizeof(int), c->stream), "clear error flag"))
            return HZB_ECUDA;
        c->kerr_ready = true;
    }
    static bool attr_done[64] = {false};
    const int dev = c->opt.device;
    if (dev >= 0 && dev < 64 && !attr_done[dev]) {
        if (check_cuda(c, cudaFuncSetAttribute(modal_gemm_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               MT_SMEM), "TMA modal GEMM shared memory"))
            return HZB_ECUDA;
        attr_done[dev] = true;
    }
    dim3 grid((ncols + MT_N - 1) / MT_N, (2 * n + MT_M - 1) / MT_M, M1);
    modal_gemm_tma_kernel<<<grid, MT_THREADS, MT_SMEM, c->stream>>>(
        n, ncols, *reinterpret_cast<const CUtensorMap *>(sd.tmA), tmB, Cout, c->kerr.ptr);
    c->launches += 2;
    return check_cuda(c, cudaGetLastError(), "modal_gemm_tma_kernel");
}

}  // namespace hzb
