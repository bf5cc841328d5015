// Learned warm start: a multilayer perceptron that maps an incident direction to
// the POD coefficients of the density (not part of the paper; it only seeds GMRES,
// whose zero-guess solve remains the fallback).  Weights are held in BF16 for the
// forward and backward products, with FP32 master copies for the optimiser;
// activations and all accumulations are FP32.
//
// Layer l: a_l = h_{l-1} W_l^T + b_l; hidden layers h_l = GELU(a_l) = a Phi(a);
// output y = a_last.  Loss (1/B) sum (y - t)^2.  Adam with bias correction.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "hzb_internal.h"
#include "tcgen05.cuh"

struct hzb_mlp {
    int device = 0;
    cudaStream_t stream = nullptr;
    int n_in = 0, width = 0, depth = 0, n_out = 0;
    std::vector<int> din, dout;            // per layer
    std::vector<size_t> woff, boff;        // offsets into the parameter vector
    size_t nparams = 0;
    float *master = nullptr;               // FP32 parameters
    float *grad = nullptr;
    float *m = nullptr, *v = nullptr;      // Adam moments
    __nv_bfloat16 *wbf = nullptr;          // BF16 copy of the parameters
    long long step = 0;
    // activations for a batch
    int cap_batch = 0;
    std::vector<float *> act_a, act_h;     // pre- and post-activation per layer
    float *gbuf0 = nullptr, *gbuf1 = nullptr;
    float *xbuf = nullptr, *tbuf = nullptr, *loss = nullptr;
    // tensor-core products (layers whose sizes are multiples of the tile): BF16 operands
    __nv_bfloat16 *hbf = nullptr;          // a layer input (B x I) or gradient (B x O) in BF16
    __nv_bfloat16 *tA = nullptr, *tB = nullptr;   // transposed BF16 operands of the weight gradient
    __nv_bfloat16 *wtbf = nullptr;         // transposed BF16 weights W^T (I x O) of the layer being back-propagated
    int *kerr = nullptr;                   // bounded-wait flag of the tensor-core kernel
    int use_tc = 1;                        // 0: CUDA-core products only
    std::string err;
};

namespace hzb {

// C(m, n) = sum_k A(m, k) B(k, n) (+ bias[n]); A(m, k) = A[m * sam + k * sak],
// B(k, n) = B[k * sbk + n * sbn]; FP32 accumulation; optional accumulate into C.
template <typename TA, typename TB>
__global__ void gemm_kernel(int M, int Nn, int K, const TA *__restrict__ A, long sam, long sak,
                            const TB *__restrict__ B, long sbk, long sbn, const float *__restrict__ bias,
                            float *__restrict__ C, long scm, long scn)
{
    __shared__ float As[32][33];
    __shared__ float Bs[32][33];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;      // 256 threads: 16 x 16
    const int m0 = blockIdx.y * 32, n0 = blockIdx.x * 32;
    float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
    for (int k0 = 0; k0 < K; k0 += 32) {
        for (int e = threadIdx.x; e < 32 * 32; e += 256) {
            int r = e / 32, q = e % 32;
            int gm = m0 + r, gk = k0 + q;
            As[r][q] = (gm < M && gk < K) ? (float)A[gm * sam + gk * sak] : 0.f;
            int gk2 = k0 + r, gn = n0 + q;
            Bs[r][q] = (gk2 < K && gn < Nn) ? (float)B[gk2 * sbk + gn * sbn] : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int q = 0; q < 32; ++q) {
            float a0 = As[ty][q], a1 = As[ty + 16][q];
            float b0 = Bs[q][tx], b1 = Bs[q][tx + 16];
            acc[0][0] = fmaf(a0, b0, acc[0][0]);
            acc[0][1] = fmaf(a0, b1, acc[0][1]);
            acc[1][0] = fmaf(a1, b0, acc[1][0]);
            acc[1][1] = fmaf(a1, b1, acc[1][1]);
        }
        __syncthreads();
    }
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            int gm = m0 + ty + 16 * a, gn = n0 + tx + 16 * b;
            if (gm < M && gn < Nn) C[gm * scm + gn * scn] = acc[a][b] + (bias ? bias[gn] : 0.f);
        }
}

__device__ inline float gelu_f(float a) { return a * 0.5f * (1.f + erff(a * 0.70710678118654752f)); }
__device__ inline float gelu_grad_f(float a)
{
    return 0.5f * (1.f + erff(a * 0.70710678118654752f)) + a * 0.3989422804014327f * expf(-0.5f * a * a);
}

__global__ void gelu_kernel(size_t n, const float *a, float *h)
{
    size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) h[e] = gelu_f(a[e]);
}

// g = 2 (y - t) / B; loss partials
__global__ void loss_grad_kernel(size_t n, int B, const float *y, const float *t, float *g, float *loss)
{
    __shared__ float red[256];
    size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    float d = 0.f;
    if (e < n) {
        d = y[e] - t[e];
        g[e] = 2.f * d / B;
    }
    red[threadIdx.x] = d * d;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, red[0] / B);
}

__global__ void gelu_back_kernel(size_t n, const float *a, float *g)
{
    size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) g[e] *= gelu_grad_f(a[e]);
}

// db[o] = sum_b g[b][o]
__global__ void bias_grad_kernel(int B, int O, const float *g, float *db)
{
    int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= O) return;
    float s = 0.f;
    for (int b = 0; b < B; ++b) s += g[(size_t)b * O + o];
    db[o] = s;
}

__global__ void adam_kernel(size_t n, float lr, float b1, float b2, float eps, float c1, float c2, float *p,
                            const float *g, float *m, float *v, __nv_bfloat16 *pb)
{
    size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    float gg = g[e];
    float mm = b1 * m[e] + (1.f - b1) * gg;
    float vv = b2 * v[e] + (1.f - b2) * gg * gg;
    m[e] = mm;
    v[e] = vv;
    float pp = p[e] - lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    p[e] = pp;
    pb[e] = __float2bfloat16_rn(pp);
}

__global__ void to_bf16_kernel(size_t n, const float *p, __nv_bfloat16 *pb)
{
    size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) pb[e] = __float2bfloat16_rn(p[e]);
}

// ------------------------------------------------------------------ tensor-core products
//
// C (M x N, FP32, row-major, ldc) = A (M x K) B (N x K)^T (+ bias[n]) with A and B BF16,
// row-major (K contiguous), on tcgen05.mma.kind::f16 (BF16 operands, FP32 accumulation
// in tensor memory).  M % 128 == 0, N % 128 == 0, K % 64 == 0.  A CTA of 128 threads owns
// a 128 x 128 tile of C: per 64-wide K chunk its threads copy the two 128 x 64 operand
// tiles into shared memory in the 128-byte-swizzled K-major layout, thread 0 issues four
// MMAs (K = 16 each) and commits them to an mbarrier; after the last chunk the four warps
// read their 32 rows x 128 columns of the accumulator (tcgen05.ld).  Every wait is bounded;
// one that runs out sets *err, writes NaN and frees the tensor memory.
static const int MM_M = 128, MM_N = 128, MM_KC = 64;
static const int MM_TILE = MM_M * MM_KC * 2;           // 16 KB per operand tile
static const int MM_SMEM = 2 * MM_TILE + 1024;

__host__ __device__ constexpr uint32_t bf16_idesc(int n, int m)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
        : "memory");
}

__global__ void __launch_bounds__(128, 1)
mlp_tc_gemm_kernel(int M, int N, int K, const __nv_bfloat16 *__restrict__ A, const __nv_bfloat16 *__restrict__ B,
                   const float *__restrict__ bias, float *__restrict__ C, int ldc, int *err)
{
    extern __shared__ __align__(1024) unsigned char mm_raw[];
    __shared__ uint32_t s_taddr;
    __shared__ __align__(8) unsigned long long s_mbar;
    const uint32_t raw = (uint32_t)__cvta_generic_to_shared(mm_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const uint32_t sA = base, sB = base + MM_TILE;
    const uint32_t mbar = (uint32_t)__cvta_generic_to_shared(&s_mbar);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * MM_M, n0 = blockIdx.x * MM_N;
    if (warp == 0) {
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&s_taddr);
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst), "r"(MM_N)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_taddr;
    uint32_t phase = 0;
    bool failed = false;
    for (int k0 = 0; k0 < K; k0 += MM_KC) {
        // operand tiles: row r, 16-byte chunk c (8 BF16) of the 64-wide K chunk
        for (int e = tid; e < MM_M * 8; e += 128) {
            const int r = e >> 3, c = e & 7;
            const uint4 va = *reinterpret_cast<const uint4 *>(A + (size_t)(m0 + r) * K + k0 + 8 * c);
            const uint4 vb = *reinterpret_cast<const uint4 *>(B + (size_t)(n0 + r) * K + k0 + 8 * c);
            t5_st4(sA + t5_chunk_off(r, c), va.x, va.y, va.z, va.w);
            t5_st4(sB + t5_chunk_off(r, c), vb.x, vb.y, vb.z, vb.w);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int ks = 0; ks < MM_KC / 16; ++ks)
                mma_bf16(tmem, t5_desc(sA + 32 * ks), t5_desc(sB + 32 * ks), bf16_idesc(MM_N, MM_M),
                         (k0 | ks) ? 1u : 0u);
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
    }
    // epilogue: warp w holds rows 32 w .. 32 w + 31 of the tile, 128 columns
    const int row = m0 + 32 * warp + lane;
#pragma unroll 1
    for (int cb = 0; cb < MM_N; cb += 32) {
        float v[32];
#pragma unroll
        for (int q = 0; q < 32; ++q) v[q] = 0.f;
        if (!failed) t5_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)cb, v);
        float *out = C + (size_t)row * ldc + n0 + cb;
#pragma unroll
        for (int q = 0; q < 32; ++q)
            out[q] = failed ? __int_as_float(0x7fc00000) : v[q] + (bias ? bias[n0 + cb + q] : 0.f);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(MM_N) : "memory");
    if (failed && tid == 0) atomicExch(err, 1);
}

// out (C x R, BF16) = in^T for in (R x C, FP32 or BF16), 32 x 32 tiles through shared memory
template <typename T>
__global__ void transpose_bf16_kernel(int R, int Cn, const T *__restrict__ in, __nv_bfloat16 *__restrict__ out)
{
    __shared__ float tile[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int q = threadIdx.y; q < 32; q += blockDim.y) {
        const int r = r0 + q, c = c0 + threadIdx.x;
        tile[q][threadIdx.x] = (r < R && c < Cn) ? (float)in[(size_t)r * Cn + c] : 0.f;
    }
    __syncthreads();
    for (int q = threadIdx.y; q < 32; q += blockDim.y) {
        const int c = c0 + q, r = r0 + threadIdx.x;
        if (c < Cn && r < R) out[(size_t)c * R + r] = __float2bfloat16_rn(tile[threadIdx.x][q]);
    }
}

static unsigned nb(size_t n) { return (unsigned)((n + 255) / 256); }

template <typename TA, typename TB>
static void gemm(cudaStream_t s, int M, int Nn, int K, const TA *A, long sam, long sak, const TB *B, long sbk, long sbn,
                 const float *bias, float *C, long scm, long scn)
{
    dim3 g((Nn + 31) / 32, (M + 31) / 32);
    gemm_kernel<TA, TB><<<g, 256, 0, s>>>(M, Nn, K, A, sam, sak, B, sbk, sbn, bias, C, scm, scn);
}

static void tc_gemm(hzb_mlp *m, int M, int Nn, int K, const __nv_bfloat16 *A, const __nv_bfloat16 *B, const float *bias,
                    float *C, int ldc)
{
    mlp_tc_gemm_kernel<<<dim3(Nn / MM_N, M / MM_M), 128, MM_SMEM, m->stream>>>(M, Nn, K, A, B, bias, C, ldc, m->kerr);
}

// a layer's products go to the tensor cores when the batch, its inputs and its outputs
// are whole tiles
static bool layer_tc(const hzb_mlp *m, int B, int l)
{
    return m->use_tc && B % 128 == 0 && m->din[l] % 128 == 0 && m->dout[l] % 128 == 0;
}

static void transpose_bf16(cudaStream_t st, int R, int Cn, const float *in, __nv_bfloat16 *out)
{
    transpose_bf16_kernel<float><<<dim3((Cn + 31) / 32, (R + 31) / 32), dim3(32, 8), 0, st>>>(R, Cn, in, out);
}

static void transpose_bf16(cudaStream_t st, int R, int Cn, const __nv_bfloat16 *in, __nv_bfloat16 *out)
{
    transpose_bf16_kernel<__nv_bfloat16><<<dim3((Cn + 31) / 32, (R + 31) / 32), dim3(32, 8), 0, st>>>(R, Cn, in, out);
}

static hzb_status mfail(hzb_mlp *m, hzb_status s, const std::string &msg)
{
    if (m) m->err = msg;
    return s;
}

static hzb_status ensure_batch(hzb_mlp *m, int B)
{
    if (B <= m->cap_batch) return HZB_OK;
    for (float *p : m->act_a) cudaFree(p);
    for (float *p : m->act_h) cudaFree(p);
    cudaFree(m->gbuf0); cudaFree(m->gbuf1); cudaFree(m->xbuf); cudaFree(m->tbuf);
    cudaFree(m->hbf); cudaFree(m->tA); cudaFree(m->tB);
    m->act_a.assign(m->din.size(), nullptr);
    m->act_h.assign(m->din.size(), nullptr);
    int wmax = std::max(std::max(m->width, m->n_out), m->n_in);
    bool ok = true;
    for (size_t l = 0; l < m->din.size(); ++l) {
        ok &= cudaMalloc(&m->act_a[l], (size_t)B * m->dout[l] * sizeof(float)) == cudaSuccess;
        ok &= cudaMalloc(&m->act_h[l], (size_t)B * m->dout[l] * sizeof(float)) == cudaSuccess;
    }
    ok &= cudaMalloc(&m->gbuf0, (size_t)B * wmax * sizeof(float)) == cudaSuccess;
    ok &= cudaMalloc(&m->gbuf1, (size_t)B * wmax * sizeof(float)) == cudaSuccess;
    ok &= cudaMalloc(&m->xbuf, (size_t)B * m->n_in * sizeof(float)) == cudaSuccess;
    ok &= cudaMalloc(&m->tbuf, (size_t)B * m->n_out * sizeof(float)) == cudaSuccess;
    ok &= cudaMalloc(&m->hbf, (size_t)B * wmax * sizeof(__nv_bfloat16)) == cudaSuccess;
    ok &= cudaMalloc(&m->tA, (size_t)B * wmax * sizeof(__nv_bfloat16)) == cudaSuccess;
    ok &= cudaMalloc(&m->tB, (size_t)B * wmax * sizeof(__nv_bfloat16)) == cudaSuccess;
    if (!ok) return mfail(m, HZB_ENOMEM, "MLP activation buffers");
    m->cap_batch = B;
    return HZB_OK;
}

// forward through all layers; x device (B x n_in); returns pointer to the output
static const float *forward(hzb_mlp *m, int B, const float *x)
{
    const float *h = x;
    int L = (int)m->din.size();
    for (int l = 0; l < L; ++l) {
        const __nv_bfloat16 *W = m->wbf + m->woff[l];
        const float *b = m->master + m->boff[l];
        if (layer_tc(m, B, l)) {                      // a = bf16(h) W^T + b on the tensor cores
            const size_t n = (size_t)B * m->din[l];
            to_bf16_kernel<<<nb(n), 256, 0, m->stream>>>(n, h, m->hbf);
            tc_gemm(m, B, m->dout[l], m->din[l], m->hbf, W, b, m->act_a[l], m->dout[l]);
        } else {
            gemm<float, __nv_bfloat16>(m->stream, B, m->dout[l], m->din[l], h, m->din[l], 1, W, 1, m->din[l], b,
                                       m->act_a[l], m->dout[l], 1);
        }
        if (l < L - 1) {
            size_t n = (size_t)B * m->dout[l];
            gelu_kernel<<<nb(n), 256, 0, m->stream>>>(n, m->act_a[l], m->act_h[l]);
            h = m->act_h[l];
        } else {
            h = m->act_a[l];
        }
    }
    return h;
}

// loss and gradients into m->grad
static void backward(hzb_mlp *m, int B, const float *x, const float *t)
{
    int L = (int)m->din.size();
    const float *y = m->act_a[L - 1];
    size_t n = (size_t)B * m->n_out;
    cudaMemsetAsync(m->loss, 0, sizeof(float), m->stream);
    loss_grad_kernel<<<nb(n), 256, 0, m->stream>>>(n, B, y, t, m->gbuf0, m->loss);
    float *g = m->gbuf0, *g2 = m->gbuf1;
    for (int l = L - 1; l >= 0; --l) {
        int I = m->din[l], O = m->dout[l];
        if (l < L - 1) gelu_back_kernel<<<nb((size_t)B * O), 256, 0, m->stream>>>((size_t)B * O, m->act_a[l], g);
        const float *hin = (l == 0) ? x : m->act_h[l - 1];
        const bool tc = layer_tc(m, B, l);
        // dW (O x I) = g^T (O x B) h_in (B x I)
        if (tc) {                                     // bf16(g)^T bf16(h_in) on the tensor cores
            transpose_bf16(m->stream, B, O, g, m->tA);
            transpose_bf16(m->stream, B, I, hin, m->tB);
            tc_gemm(m, O, I, B, m->tA, m->tB, nullptr, m->grad + m->woff[l], I);
        } else {
            gemm<float, float>(m->stream, O, I, B, g, 1, O, hin, I, 1, nullptr, m->grad + m->woff[l], I, 1);
        }
        bias_grad_kernel<<<(O + 255) / 256, 256, 0, m->stream>>>(B, O, g, m->grad + m->boff[l]);
        if (l > 0) {
            // dh_in (B x I) = g (B x O) W (O x I)
            if (tc) {                                 // bf16(g) W with W^T (I x O) as the K-major operand
                const size_t n = (size_t)B * O;
                to_bf16_kernel<<<nb(n), 256, 0, m->stream>>>(n, g, m->hbf);
                transpose_bf16(m->stream, O, I, m->wbf + m->woff[l], m->wtbf);
                tc_gemm(m, B, I, O, m->hbf, m->wtbf, nullptr, g2, I);
            } else {
                gemm<float, __nv_bfloat16>(m->stream, B, I, O, g, O, 1, m->wbf + m->woff[l], I, 1, nullptr, g2, I,
                                           1);
            }
            std::swap(g, g2);
        }
    }
}

}  // namespace hzb

using namespace hzb;

extern "C" {

hzb_status hzb_mlp_create(int device, void *stream, int n_in, int width, int depth, int n_out,
                          unsigned long long seed, hzb_mlp **out)
{
    if (!out || n_in < 1 || width < 1 || depth < 1 || n_out < 1 || n_in > 65536 || width > 65536 || n_out > 65536 ||
        depth > 64)
        return HZB_EINVAL;
    *out = nullptr;
    if (cudaSetDevice(device) != cudaSuccess) return HZB_ECUDA;
    hzb_mlp *m = new (std::nothrow) hzb_mlp();
    if (!m) return HZB_ENOMEM;
    m->device = device;
    m->stream = (cudaStream_t)stream;
    m->n_in = n_in; m->width = width; m->depth = depth; m->n_out = n_out;
    for (int l = 0; l <= depth; ++l) {
        int i = (l == 0) ? n_in : width, o = (l == depth) ? n_out : width;
        m->din.push_back(i);
        m->dout.push_back(o);
        m->woff.push_back(m->nparams);
        m->nparams += (size_t)i * o;
        m->boff.push_back(m->nparams);
        m->nparams += o;
    }
    // deterministic initialisation: splitmix64 stream, W ~ U(-1/sqrt(in), 1/sqrt(in)), b = 0
    std::vector<float> p(m->nparams, 0.f);
    unsigned long long st = seed;
    auto next = [&]() {
        unsigned long long z = (st += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return (double)(z >> 11) * (1.0 / 9007199254740992.0);
    };
    for (size_t l = 0; l < m->din.size(); ++l) {
        double s = 1.0 / std::sqrt((double)m->din[l]);
        for (size_t e = 0; e < (size_t)m->din[l] * m->dout[l]; ++e) p[m->woff[l] + e] = (float)((2.0 * next() - 1.0) * s);
    }
    size_t wmax = 0;
    for (size_t l = 0; l < m->din.size(); ++l) wmax = std::max(wmax, (size_t)m->din[l] * m->dout[l]);
    bool ok = cudaMalloc(&m->master, m->nparams * 4) == cudaSuccess && cudaMalloc(&m->grad, m->nparams * 4) == cudaSuccess &&
              cudaMalloc(&m->m, m->nparams * 4) == cudaSuccess && cudaMalloc(&m->v, m->nparams * 4) == cudaSuccess &&
              cudaMalloc(&m->wbf, m->nparams * 2) == cudaSuccess && cudaMalloc(&m->loss, 4) == cudaSuccess &&
              cudaMalloc(&m->wtbf, wmax * 2) == cudaSuccess && cudaMalloc(&m->kerr, sizeof(int)) == cudaSuccess &&
              cudaFuncSetAttribute(mlp_tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, MM_SMEM) ==
                  cudaSuccess;
    if (!ok) {
        *out = m;
        return HZB_ENOMEM;
    }
    cudaMemcpyAsync(m->master, p.data(), m->nparams * 4, cudaMemcpyHostToDevice, m->stream);
    cudaMemsetAsync(m->m, 0, m->nparams * 4, m->stream);
    cudaMemsetAsync(m->v, 0, m->nparams * 4, m->stream);
    cudaMemsetAsync(m->kerr, 0, sizeof(int), m->stream);
    to_bf16_kernel<<<nb(m->nparams), 256, 0, m->stream>>>(m->nparams, m->master, m->wbf);
    if (cudaStreamSynchronize(m->stream) != cudaSuccess) {
        *out = m;
        return HZB_ECUDA;
    }
    *out = m;
    return HZB_OK;
}

hzb_status hzb_mlp_destroy(hzb_mlp *m)
{
    if (!m) return HZB_EINVAL;
    cudaSetDevice(m->device);
    cudaDeviceSynchronize();              // the caller's stream may already be gone
    for (float *p : m->act_a) cudaFree(p);
    for (float *p : m->act_h) cudaFree(p);
    cudaFree(m->gbuf0); cudaFree(m->gbuf1); cudaFree(m->xbuf); cudaFree(m->tbuf);
    cudaFree(m->master); cudaFree(m->grad); cudaFree(m->m); cudaFree(m->v); cudaFree(m->wbf); cudaFree(m->loss);
    cudaFree(m->hbf); cudaFree(m->tA); cudaFree(m->tB); cudaFree(m->wtbf); cudaFree(m->kerr);
    delete m;
    cudaGetLastError();
    return HZB_OK;
}

const char *hzb_mlp_last_error(const hzb_mlp *m) { return m ? m->err.c_str() : "null network"; }

hzb_status hzb_mlp_set_tensor_cores(hzb_mlp *m, int on)
{
    if (!m || (on != 0 && on != 1)) return HZB_EINVAL;
    m->use_tc = on;
    return HZB_OK;
}

hzb_status hzb_mlp_num_params(const hzb_mlp *m, long long *n)
{
    if (!m || !n) return HZB_EINVAL;
    *n = (long long)m->nparams;
    return HZB_OK;
}

hzb_status hzb_mlp_get_params(hzb_mlp *m, float *out)
{
    if (!m || !out) return HZB_EINVAL;
    cudaSetDevice(m->device);
    if (cudaMemcpyAsync(out, m->master, m->nparams * 4, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
        cudaStreamSynchronize(m->stream) != cudaSuccess)
        return mfail(m, HZB_ECUDA, "copy params");
    return HZB_OK;
}

hzb_status hzb_mlp_set_params(hzb_mlp *m, const float *in)
{
    if (!m || !in) return HZB_EINVAL;
    cudaSetDevice(m->device);
    cudaMemcpyAsync(m->master, in, m->nparams * 4, cudaMemcpyHostToDevice, m->stream);
    to_bf16_kernel<<<nb(m->nparams), 256, 0, m->stream>>>(m->nparams, m->master, m->wbf);
    if (cudaStreamSynchronize(m->stream) != cudaSuccess) return mfail(m, HZB_ECUDA, "set params");
    return HZB_OK;
}

// a bounded tensor-core wait that ran out (outputs NaN): report once and clear
static hzb_status check_tc_flag(hzb_mlp *m)
{
    int flag = 0;
    if (cudaMemcpy(&flag, m->kerr, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return mfail(m, HZB_ECUDA, "read error flag");
    if (flag) {
        cudaMemset(m->kerr, 0, sizeof(int));
        return mfail(m, HZB_ETIMEOUT, "tensor-core wait timed out in mlp_tc_gemm_kernel");
    }
    return HZB_OK;
}

static hzb_status stage(hzb_mlp *m, float *dst, const float *src, size_t n, int on_device, const float **use)
{
    if (on_device) {
        *use = src;
        return HZB_OK;
    }
    if (cudaMemcpyAsync(dst, src, n * 4, cudaMemcpyHostToDevice, m->stream) != cudaSuccess)
        return mfail(m, HZB_ECUDA, "copy input");
    *use = dst;
    return HZB_OK;
}

hzb_status hzb_mlp_forward(hzb_mlp *m, int B, const float *x, float *y, int on_device)
{
    if (!m || !x || !y || B < 1) return HZB_EINVAL;
    cudaSetDevice(m->device);
    hzb_status st = ensure_batch(m, B);
    if (st) return st;
    const float *xd;
    if ((st = stage(m, m->xbuf, x, (size_t)B * m->n_in, on_device, &xd))) return st;
    const float *yd = forward(m, B, xd);
    cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (cudaMemcpyAsync(y, yd, (size_t)B * m->n_out * 4, kind, m->stream) != cudaSuccess ||
        cudaStreamSynchronize(m->stream) != cudaSuccess)
        return mfail(m, HZB_ECUDA, "forward");
    return check_tc_flag(m);
}

hzb_status hzb_mlp_gradients(hzb_mlp *m, int B, const float *x, const float *t, float *loss, float *grads,
                             int on_device)
{
    if (!m || !x || !t || B < 1) return HZB_EINVAL;
    cudaSetDevice(m->device);
    hzb_status st = ensure_batch(m, B);
    if (st) return st;
    const float *xd, *td;
    if ((st = stage(m, m->xbuf, x, (size_t)B * m->n_in, on_device, &xd)) ||
        (st = stage(m, m->tbuf, t, (size_t)B * m->n_out, on_device, &td)))
        return st;
    forward(m, B, xd);
    backward(m, B, xd, td);
    if (grads) {
        cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        cudaMemcpyAsync(grads, m->grad, m->nparams * 4, kind, m->stream);
    }
    if (loss) cudaMemcpyAsync(loss, m->loss, 4, cudaMemcpyDeviceToHost, m->stream);
    if (cudaStreamSynchronize(m->stream) != cudaSuccess || cudaGetLastError() != cudaSuccess)
        return mfail(m, HZB_ECUDA, "gradients");
    return check_tc_flag(m);
}

hzb_status hzb_mlp_train_step(hzb_mlp *m, int B, const float *x, const float *t, float lr, float *loss, int on_device)
{
    if (!m || !x || !t || B < 1 || !(lr > 0)) return HZB_EINVAL;
    cudaSetDevice(m->device);
    hzb_status st = ensure_batch(m, B);
    if (st) return st;
    const float *xd, *td;
    if ((st = stage(m, m->xbuf, x, (size_t)B * m->n_in, on_device, &xd)) ||
        (st = stage(m, m->tbuf, t, (size_t)B * m->n_out, on_device, &td)))
        return st;
    forward(m, B, xd);
    backward(m, B, xd, td);
    m->step++;
    const float b1 = 0.9f, b2 = 0.999f;
    float c1 = 1.f - std::pow(b1, (float)m->step), c2 = 1.f - std::pow(b2, (float)m->step);
    adam_kernel<<<nb(m->nparams), 256, 0, m->stream>>>(m->nparams, lr, b1, b2, 1e-8f, c1, c2, m->master, m->grad,
                                                       m->m, m->v, m->wbf);
    if (loss) cudaMemcpyAsync(loss, m->loss, 4, cudaMemcpyDeviceToHost, m->stream);
    if (cudaStreamSynchronize(m->stream) != cudaSuccess || cudaGetLastError() != cudaSuccess)
        return mfail(m, HZB_ECUDA, "train step");
    return check_tc_flag(m);
}

}  // extern "C"
