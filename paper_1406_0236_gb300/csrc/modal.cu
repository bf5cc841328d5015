// Block-diagonal inverse D^{-1} (Sec. 4, Remark after Eq. (precond); Eq. (singleinverse)):
// for each body, (1) DFT over the azimuth of every ring,
//     y^_p(i) = sum_l y(i, l) e^{-2 pi i p l / N_F},  p = -M..M,
// (2) tau^_p = S_|p| y^_p (S_{-p} = S_p because the modal kernels are even in psi),
// (3) inverse DFT with the 1/N_F factor, and tau = alpha sigma + beta tau.
// Step (2) is a batched complex GEMM per (shape, |p|): the columns stack, for every
// body of that shape, the +p and -p coefficient vectors of all right-hand sides.
// Column layout of a shape's mode-p panel: col = (2 * body_in_shape + sign) * R + r,
// sign 0 for +p and 1 for -p (the -0 columns are zero).
#include <algorithm>

#include "hzb_internal.h"
#include "tcgen05.cuh"
#include "kernel_math.cuh"

namespace hzb {

template <typename T> struct C2;
template <> struct C2<double> { typedef double2 t; };
template <> struct C2<float> { typedef float2 t; };

static const int DFT_THREADS = 128;

void launch_modal_gemm_tc(hzb_ctx *c, int n, int nc, int modes, const float2 *A, const float2 *B, float2 *C);
hzb_status launch_modal_gemm_tc5(hzb_ctx *c, int n, int nc, int modes, const float2 *A, const float2 *B,
                                 float2 *C);


// One block per (body of the shape, ring).  y is N x R (FP64); out is the shape's
// panel array (M+1) x NG x ncols in precision T, which is also the arithmetic precision
// (twiddles rounded from FP64 values; the FP32 path's DFT then runs on the FP32 pipe).
template <typename T>
__global__ void dft_forward_kernel(int NG, int NF, int R, int ncols, const long long *__restrict__ body_off,
                                   const double2 *__restrict__ y, typename C2<T>::t *__restrict__ yh)
{
    typedef typename C2<T>::t ct;
    extern __shared__ double smem_d[];
    ct *tw = (ct *)smem_d;                           // NF: e^{-2 pi i m / NF}
    ct *ring = tw + NF;                              // NF x R
    const int bs = blockIdx.y, i = blockIdx.x;
    const int M = (NF - 1) / 2;
    const long long base = body_off[bs] + (long long)i * NF;
    for (int m = threadIdx.x; m < NF; m += blockDim.x) {
        double s, c;
        sincospi(-2.0 * m / NF, &s, &c);
        tw[m].x = (T)c;
        tw[m].y = (T)s;
    }
    for (int e = threadIdx.x; e < NF * R; e += blockDim.x) {
        const double2 v = y[base * R + e];
        ring[e].x = (T)v.x;
        ring[e].y = (T)v.y;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < NF * R; e += blockDim.x) {
        const int pidx = e / R, r = e % R;
        const int p = pidx - M;
        const int pm = ((p % NF) + NF) % NF;
        T sx = (T)0, sy = (T)0;
        int idx = 0;
        for (int l = 0; l < NF; ++l) {
            const ct v = ring[l * R + r], w = tw[idx];
            sx = fma(v.x, w.x, fma(-v.y, w.y, sx));
            sy = fma(v.x, w.y, fma(v.y, w.x, sy));
            idx += pm;
            if (idx >= NF) idx -= NF;
        }
        const int ap = p < 0 ? -p : p;
        const int sg = p < 0 ? 1 : 0;
        ct o;
        o.x = (T)sx;
        o.y = (T)sy;
        yh[((size_t)ap * NG + i) * ncols + (2 * bs + sg) * R + r] = o;
        if (p == 0) {
            ct z;
            z.x = (T)0;
            z.y = (T)0;
            yh[((size_t)0 * NG + i) * ncols + (2 * bs + 1) * R + r] = z;
        }
    }
}

// tau(i, l) = alpha sigma(i, l) + beta / NF * sum_p tau^_p(i) e^{2 pi i p l / NF}
template <typename T>
__global__ void dft_inverse_kernel(int NG, int NF, int R, int ncols, const long long *__restrict__ body_off,
                                   const typename C2<T>::t *__restrict__ th, const double2 *__restrict__ sigma,
                                   double alpha, double beta, double2 *__restrict__ out)
{
    typedef typename C2<T>::t ct;
    extern __shared__ double smem_d[];
    ct *tw = (ct *)smem_d;                           // NF: e^{+2 pi i m / NF}
    ct *co = tw + NF;                                // NF x R coefficients, p = -M..M
    const int bs = blockIdx.y, i = blockIdx.x;
    const int M = (NF - 1) / 2;
    const long long base = body_off[bs] + (long long)i * NF;
    for (int m = threadIdx.x; m < NF; m += blockDim.x) {
        double s, c;
        sincospi(2.0 * m / NF, &s, &c);
        tw[m].x = (T)c;
        tw[m].y = (T)s;
    }
    for (int e = threadIdx.x; e < NF * R; e += blockDim.x) {
        const int pidx = e / R, r = e % R, p = pidx - M;
        const int ap = p < 0 ? -p : p, sg = p < 0 ? 1 : 0;
        co[e] = th[((size_t)ap * NG + i) * ncols + (2 * bs + sg) * R + r];
    }
    __syncthreads();
    const double sc = beta / NF;
    for (int e = threadIdx.x; e < NF * R; e += blockDim.x) {
        const int l = e / R, r = e % R;
        T sx = (T)0, sy = (T)0;
        // p = -M .. M  ->  twiddle index (p l) mod NF, starting at (-M l) mod NF
        int idx = (int)(((long long)(NF - M) * l) % NF);
        for (int pidx = 0; pidx < NF; ++pidx) {
            const ct v = co[pidx * R + r], w = tw[idx];
            sx = fma(v.x, w.x, fma(-v.y, w.y, sx));
            sy = fma(v.x, w.y, fma(v.y, w.x, sy));
            idx += l;
            if (idx >= NF) idx -= NF;
        }
        double2 o = make_double2((double)sx * sc, (double)sy * sc);
        if (alpha != 0.0) {
            const double2 s = sigma[base * R + e];
            o.x = fma(alpha, s.x, o.x);
            o.y = fma(alpha, s.y, o.y);
        }
        out[base * R + e] = o;
    }
}

// The DFT kernels' dynamic shared memory: beyond the default 48 KB, raise their
// limit once to the largest size any call uses (200 KB).  The limit is never set
// lower, so calls with different sizes (and both D^{-1} entry points) cannot
// invalidate each other's launches.
template <typename T>
static void dft_smem_limit(size_t bytes)
{
    if (bytes <= 48 * 1024) return;
    cudaFuncSetAttribute(dft_forward_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(dft_inverse_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

// Batched complex GEMM C[p] = A[p] B[p], A: n x n, B and C: n x nc, row-major.
// 32 x 32 output tile per block, 256 threads, 2 x 2 outputs per thread, K step 16.
template <typename T>
__global__ void __launch_bounds__(256)
modal_gemm_kernel(int n, int nc, const typename C2<T>::t *__restrict__ A, const typename C2<T>::t *__restrict__ B,
                  typename C2<T>::t *__restrict__ C)
{
    typedef typename C2<T>::t ct;
    __shared__ ct As[32][17];
    __shared__ ct Bs[16][33];
    const int p = blockIdx.z;
    const ct *Ap = A + (size_t)p * n * n;
    const ct *Bp = B + (size_t)p * n * nc;
    ct *Cp = C + (size_t)p * n * nc;
    const int row0 = blockIdx.y * 32, col0 = blockIdx.x * 32;
    const int tid = threadIdx.x;
    const int tr = tid / 16, tc = tid % 16;     // rows tr, tr+16; cols tc, tc+16
    T accr[2][2] = {{0, 0}, {0, 0}}, acci[2][2] = {{0, 0}, {0, 0}};
    for (int k0 = 0; k0 < n; k0 += 16) {
        for (int e = tid; e < 32 * 16; e += 256) {
            int r = e / 16, kk = e % 16;
            int gr = row0 + r, gk = k0 + kk;
            ct v;
            v.x = (T)0; v.y = (T)0;
            if (gr < n && gk < n) v = Ap[(size_t)gr * n + gk];
            As[r][kk] = v;
        }
        for (int e = tid; e < 16 * 32; e += 256) {
            int kk = e / 32, cc = e % 32;
            int gk = k0 + kk, gc = col0 + cc;
            ct v;
            v.x = (T)0; v.y = (T)0;
            if (gk < n && gc < nc) v = Bp[(size_t)gk * nc + gc];
            Bs[kk][cc] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            ct a0 = As[tr][kk], a1 = As[tr + 16][kk];
            ct b0 = Bs[kk][tc], b1 = Bs[kk][tc + 16];
            accr[0][0] += a0.x * b0.x - a0.y * b0.y; acci[0][0] += a0.x * b0.y + a0.y * b0.x;
            accr[0][1] += a0.x * b1.x - a0.y * b1.y; acci[0][1] += a0.x * b1.y + a0.y * b1.x;
            accr[1][0] += a1.x * b0.x - a1.y * b0.y; acci[1][0] += a1.x * b0.y + a1.y * b0.x;
            accr[1][1] += a1.x * b1.x - a1.y * b1.y; acci[1][1] += a1.x * b1.y + a1.y * b1.x;
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            int gr = row0 + tr + 16 * a, gc = col0 + tc + 16 * b;
            if (gr < n && gc < nc) {
                ct v;
                v.x = accr[a][b];
                v.y = acci[a][b];
                Cp[(size_t)gr * nc + gc] = v;
            }
        }
}

template <typename T>
static hzb_status local_inverse_t(hzb_ctx *c, int R, const double2 *y, const double2 *sigma, double alpha,
                                  double beta, double2 *tau)
{
    typedef typename C2<T>::t ct;
    for (ShapeDev *sp : c->shapes) {
        ShapeDev &sd = *sp;
        const int NG = sd.geom.NG, NF = sd.geom.NF, M = sd.geom.M;
        const int ms = (int)sd.bodies.size();
        const int ncols = 2 * ms * R;
        const size_t panel = (size_t)(M + 1) * NG * ncols;
        ct *yh, *th;
        const ct *S;
        if (sizeof(T) == 8) {
            if (check_cuda(c, c->yhat64.ensure(panel), "alloc") || check_cuda(c, c->that64.ensure(panel), "alloc"))
                return HZB_ENOMEM;
            yh = (ct *)c->yhat64.ptr;
            th = (ct *)c->that64.ptr;
            S = (const ct *)sd.S64.ptr;
        } else {
            if (check_cuda(c, c->yhat32.ensure(panel), "alloc") || check_cuda(c, c->that32.ensure(panel), "alloc"))
                return HZB_ENOMEM;
            yh = (ct *)c->yhat32.ptr;
            th = (ct *)c->that32.ptr;
            S = (const ct *)sd.S32.ptr;
        }
        const long long *doff = sd.body_offs.ptr;        // first node of each body of the shape
        size_t smem = (size_t)NF * (R + 1) * sizeof(ct);
        if (smem > 200 * 1024) return fail(c, HZB_EINVAL, "n_modes * R too large for the modal apply");
        dft_smem_limit<T>(smem);
        dft_forward_kernel<T><<<dim3(NG, ms), DFT_THREADS, smem, c->stream>>>(NG, NF, R, ncols, doff, y, yh);
        // FP32 path: tensor cores (TF32 x 3) once the panels are wide enough to fill them
        const bool tc = (sizeof(T) == 4) && (c->modal_engine == 1 || (c->modal_engine < 0 && ncols >= 32));
        if (sizeof(T) == 4 && c->modal_engine == 2) {
            hzb_status st = launch_modal_gemm_tc5(c, NG, ncols, M + 1, (const float2 *)S, (const float2 *)yh, (float2 *)th);
            if (st) return st;
        } else if (tc)
            launch_modal_gemm_tc(c, NG, ncols, M + 1, (const float2 *)S, (const float2 *)yh, (float2 *)th);
        else
            modal_gemm_kernel<T><<<dim3((ncols + 31) / 32, (NG + 31) / 32, M + 1), 256, 0, c->stream>>>(NG, ncols, S, yh, th);
        dft_inverse_kernel<T><<<dim3(NG, ms), DFT_THREADS, smem, c->stream>>>(NG, NF, R, ncols, doff, th, sigma,
                                                                               alpha, beta, tau);
        c->launches += 3;
        if (check_cuda(c, cudaGetLastError(), "modal apply")) return HZB_ECUDA;
    }
    return HZB_OK;
}

hzb_status local_inverse64(hzb_ctx *c, int R, const double2 *y, const double2 *sigma, double alpha, double beta,
                           double2 *tau)
{
    return local_inverse_t<double>(c, R, y, sigma, alpha, beta, tau);
}

hzb_status local_inverse32(hzb_ctx *c, int R, const double2 *y, const double2 *sigma, double alpha, double beta,
                           double2 *tau)
{
    return local_inverse_t<float>(c, R, y, sigma, alpha, beta, tau);
}

}  // namespace hzb

namespace hzb {

// The FP64 D^{-1} apply with caller-provided scratch: yh and th each hold at least
// (M+1) x N_G x (2 m_s R) complex values for every shape (shapes run one after the
// other on the stream, reusing them).  Launches the same kernels as local_inverse64
// and allocates nothing.
hzb_status local_inverse64_scratch(hzb_ctx *c, int R, const double2 *y, const double2 *sigma, double alpha,
                                   double beta, double2 *tau, double2 *yh, double2 *th)
{
    for (ShapeDev *sp : c->shapes) {
        ShapeDev &sd = *sp;
        const int NG = sd.geom.NG, NF = sd.geom.NF, M = sd.geom.M;
        const int ms = (int)sd.bodies.size();
        const int ncols = 2 * ms * R;
        const long long *doff = sd.body_offs.ptr;
        size_t smem = (size_t)NF * (R + 1) * sizeof(double2);
        if (smem > 200 * 1024) return fail(c, HZB_EINVAL, "n_modes * R too large for the modal apply");
        dft_smem_limit<double>(smem);
        dft_forward_kernel<double><<<dim3(NG, ms), DFT_THREADS, smem, c->stream>>>(NG, NF, R, ncols, doff, y, yh);
        modal_gemm_kernel<double><<<dim3((ncols + 31) / 32, (NG + 31) / 32, M + 1), 256, 0, c->stream>>>(
            NG, ncols, sd.S64.ptr, yh, th);
        dft_inverse_kernel<double><<<dim3(NG, ms), DFT_THREADS, smem, c->stream>>>(NG, NF, R, ncols, doff, th,
                                                                                    sigma, alpha, beta, tau);
        c->launches += 3;
        if (check_cuda(c, cudaGetLastError(), "modal apply")) return HZB_ECUDA;
    }
    return HZB_OK;
}

// Largest per-shape panel (M+1) x N_G x (2 m_s R) of the context, in complex values.
size_t modal_panel_elems(const hzb_ctx *c, int R)
{
    size_t mx = 0;
    for (const ShapeDev *sp : c->shapes)
        mx = std::max(mx, (size_t)(sp->geom.M + 1) * sp->geom.NG * (2 * sp->bodies.size() * (size_t)R));
    return mx;
}

}  // namespace hzb

namespace hzb {

// ---------------------------------------------------------------- tensor-core modal GEMM
// FP32 path, many columns: C = A B for complex A (n x n) and B (n x nc) through the
// real embedding  [Cr; Ci] = [[Ar, -Ai], [Ai, Ar]] [Br; Bi]  (a 2n x 2n x nc real GEMM)
// on the tensor cores in TF32 with a three-term split, x = hi + lo with hi, lo TF32:
// A B ~ Ahi Bhi + Ahi Blo + Alo Bhi, FP32 accumulation (about FP32 accuracy).
// mma.sync m16n8k8; 64 x 64 output tile per CTA, 4 warps of 32 x 32, K step 32.

__device__ __forceinline__ uint32_t to_tf32(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void mma_tf32(float *d, const uint32_t *a, const uint32_t *b)
{
    asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__global__ void __launch_bounds__(128)
modal_gemm_tc_kernel(int n, int nc, const float2 *__restrict__ A, const float2 *__restrict__ B, float2 *__restrict__ C)
{
    __shared__ float As[64][33];
    __shared__ float Bs[32][72];
    const int p = blockIdx.z;
    const float2 *Ap = A + (size_t)p * n * n;
    const float2 *Bp = B + (size_t)p * n * nc;
    float2 *Cp = C + (size_t)p * n * nc;
    const int n2 = 2 * n;
    const int row0 = blockIdx.y * 64, col0 = blockIdx.x * 64;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp >> 1, wn = warp & 1;
    const int g = lane >> 2, t = lane & 3;
    float acc[2][4][4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
    for (int k0 = 0; k0 < n2; k0 += 32) {
        for (int e = tid; e < 64 * 32; e += 128) {
            const int r = e >> 5, kk = e & 31;
            const int R = row0 + r, K = k0 + kk;
            float v = 0.f;
            if (R < n2 && K < n2) {
                const float2 a = Ap[(size_t)(R < n ? R : R - n) * n + (K < n ? K : K - n)];
                v = (R < n) ? (K < n ? a.x : -a.y) : (K < n ? a.y : a.x);
            }
            As[r][kk] = v;
        }
        for (int e = tid; e < 32 * 64; e += 128) {
            const int kk = e >> 6, c = e & 63;
            const int K = k0 + kk, col = col0 + c;
            float v = 0.f;
            if (K < n2 && col < nc) {
                const float2 b = Bp[(size_t)(K < n ? K : K - n) * nc + col];
                v = (K < n) ? b.x : b.y;
            }
            Bs[kk][c] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 32; kk += 8) {
            uint32_t ah[2][4], al[2][4];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                const int r = wm * 32 + mt * 16 + g;
                const float v[4] = {As[r][kk + t], As[r + 8][kk + t], As[r][kk + t + 4], As[r + 8][kk + t + 4]};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    ah[mt][q] = to_tf32(v[q]);
                    al[mt][q] = to_tf32(v[q] - __uint_as_float(ah[mt][q]));
                }
            }
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const int c = wn * 32 + nt * 8 + g;
                const float v0 = Bs[kk + t][c], v1 = Bs[kk + t + 4][c];
                uint32_t bh[2] = {to_tf32(v0), to_tf32(v1)};
                uint32_t bl[2] = {to_tf32(v0 - __uint_as_float(bh[0])), to_tf32(v1 - __uint_as_float(bh[1]))};
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    mma_tf32(acc[mt][nt], al[mt], bh);
                    mma_tf32(acc[mt][nt], ah[mt], bl);
                    mma_tf32(acc[mt][nt], ah[mt], bh);
                }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int R = row0 + wm * 32 + mt * 16 + g + 8 * h;
                const int col = col0 + wn * 32 + nt * 8 + 2 * t;
                if (R >= n2) continue;
                float *base = (R < n) ? &Cp[(size_t)R * nc].x : &Cp[(size_t)(R - n) * nc].y;
                if (col < nc) base[2 * col] = acc[mt][nt][2 * h];
                if (col + 1 < nc) base[2 * (col + 1)] = acc[mt][nt][2 * h + 1];
            }
}

// ---------------------------------------------------------------- tcgen05 modal GEMM
//
// C[p] = A[p] B[p] (A = S_p: n x n complex; B, C: n x nc complex, row-major) on the
// 5th-generation tensor cores through the real embedding
//     [Cr; Ci] = [[Ar, -Ai], [Ai, Ar]] [Br; Bi]      (M = K = 2n, N = nc),
// each real product in TF32 with a three-term hi/lo split.  A CTA of 256 threads owns a
// 128 x 64 tile of the embedded C for one mode; per 32-wide K chunk the threads write the
// A tile (128 rows x 32, K-major) and the B tile (64 columns x 32, K-major) with the
// 128-byte swizzle, one thread issues 12 tcgen05 MMAs into tensor memory and commits them
// to an mbarrier (bounded wait); every two chunks the eight warps add the accumulator
// (32 lanes x 32 columns each) into FP32 registers and the next chunk starts from zero.
static const int MG_M = 128, MG_N = 64, MG_K = 32, MG_THREADS = 256, MG_FLUSH = 2;
static const int MG_A = MG_M * MG_K * 4, MG_B = MG_N * MG_K * 4;
static const int MG_SMEM = 2 * MG_A + 2 * MG_B + 1024;

__global__ void __launch_bounds__(MG_THREADS)
modal_gemm_tc5_kernel(int n, int nc, const float2 *__restrict__ A, const float2 *__restrict__ B,
                      float2 *__restrict__ C, int *__restrict__ err)
{
    extern __shared__ __align__(1024) unsigned char mg_smem_raw[];
    __shared__ uint32_t s_taddr;
    __shared__ __align__(8) unsigned long long s_mbar;
    const uint32_t raw = (uint32_t)__cvta_generic_to_shared(mg_smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const uint32_t sAh = base, sAl = base + MG_A, sBh = base + 2 * MG_A, sBl = sBh + MG_B;
    const uint32_t mbar = (uint32_t)__cvta_generic_to_shared(&s_mbar);
    const int p = blockIdx.z, m0 = blockIdx.y * MG_M, c0 = blockIdx.x * MG_N;
    const int n2 = 2 * n;
    const float2 *Ap = A + (size_t)p * n * n;
    const float2 *Bp = B + (size_t)p * n * nc;
    float2 *Cp = C + (size_t)p * n * nc;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) {
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&s_taddr);
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst), "r"(MG_N)
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
    const uint32_t tmem_warp = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(32 * (warp >> 2));
    float acc[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) acc[q] = 0.f;
    // A duty: row `arow`, chunks 4 ahalf .. +3; B duty: column `bcol`, chunks 2 bq, 2 bq + 1
    const int arow = tid & (MG_M - 1), ahalf = tid >> 7;
    const int bcol = tid & (MG_N - 1), bq = tid >> 6;
    const int m = m0 + arow, mr = m < n ? m : m - n;
    const int cg = c0 + bcol;
    const int nk = (n2 + MG_K - 1) / MG_K;
    uint32_t phase = 0;
    bool failed = false;
    for (int kc = 0; kc < nk; ++kc) {
        const int k0 = kc * MG_K;
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();                               // previous chunk's operands consumed
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
            const int c = 4 * ahalf + cc;
            uint32_t h[4], l[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int k = k0 + 4 * c + q;
                float a = 0.f;
                if (m < n2 && k < n2) {
                    const float2 v = Ap[(size_t)mr * n + (k < n ? k : k - n)];
                    a = (m < n) ? (k < n ? v.x : -v.y) : (k < n ? v.y : v.x);
                }
                h[q] = t5_tf32(a);
                l[q] = t5_tf32(a - __uint_as_float(h[q]));
            }
            t5_st4(sAh + t5_chunk_off(arow, c), h[0], h[1], h[2], h[3]);
            t5_st4(sAl + t5_chunk_off(arow, c), l[0], l[1], l[2], l[3]);
        }
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
            const int c = 2 * bq + cc;
            uint32_t h[4], l[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int k = k0 + 4 * c + q;
                float b = 0.f;
                if (k < n2 && cg < nc) {
                    const float2 v = Bp[(size_t)(k < n ? k : k - n) * nc + cg];
                    b = (k < n) ? v.x : v.y;
                }
                h[q] = t5_tf32(b);
                l[q] = t5_tf32(b - __uint_as_float(h[q]));
            }
            t5_st4(sBh + t5_chunk_off(bcol, c), h[0], h[1], h[2], h[3]);
            t5_st4(sBl + t5_chunk_off(bcol, c), l[0], l[1], l[2], l[3]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t as[3] = {sAh, sAh, sAl}, bs[3] = {sBh, sBl, sBh};
            const bool first = (kc % MG_FLUSH) == 0;
#pragma unroll
            for (int ks = 0; ks < MG_K / 8; ++ks)
#pragma unroll
                for (int t = 0; t < 3; ++t)
                    t5_mma(tmem, t5_desc(as[t] + 32 * ks), t5_desc(bs[t] + 32 * ks), t5_idesc(MG_N),
                           (first && ks == 0 && t == 0) ? 0u : 1u);
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
        if ((kc % MG_FLUSH) == MG_FLUSH - 1 || kc == nk - 1) t5_ld32(tmem_warp, acc);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(MG_N) : "memory");
    if (failed && tid == 0) atomicExch(err, 1);
    const int r = m0 + 32 * (warp & 3) + lane;
    if (r >= n2) return;
    const int rr = r < n ? r : r - n, comp = r < n ? 0 : 1;
#pragma unroll
    for (int q = 0; q < 32; ++q) {
        const int col = c0 + 32 * (warp >> 2) + q;
        if (col < nc)
            reinterpret_cast<float *>(&Cp[(size_t)rr * nc + col])[comp] =
                failed ? __int_as_float(0x7fc00000) : acc[q];
    }
}

hzb_status launch_modal_gemm_tc5(hzb_ctx *c, int n, int nc, int modes, const float2 *A, const float2 *B, float2 *C)
{
    if (check_cuda(c, c->kerr.ensure(1), "alloc error flag")) return HZB_ENOMEM;
    if (!c->kerr_ready) {
        if (check_cuda(c, cudaMemsetAsync(c->kerr.ptr, 0, sizeof(int), c->stream), "clear error flag"))
            return HZB_ECUDA;
        c->kerr_ready = true;
    }
    static bool attr_done[64] = {false};
    const int dev = c->opt.device;
    if (dev >= 0 && dev < 64 && !attr_done[dev]) {
        if (check_cuda(c, cudaFuncSetAttribute(modal_gemm_tc5_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               MG_SMEM), "tcgen05 modal GEMM shared memory"))
            return HZB_ECUDA;
        attr_done[dev] = true;
    }
    dim3 grid((nc + MG_N - 1) / MG_N, (2 * n + MG_M - 1) / MG_M, modes);
    modal_gemm_tc5_kernel<<<grid, MG_THREADS, MG_SMEM, c->stream>>>(n, nc, A, B, C, c->kerr.ptr);
    return HZB_OK;
}

void launch_modal_gemm_tc(hzb_ctx *c, int n, int nc, int modes, const float2 *A, const float2 *B, float2 *C)
{
    dim3 grid((nc + 63) / 64, (2 * n + 63) / 64, modes);
    modal_gemm_tc_kernel<<<grid, 128, 0, c->stream>>>(n, nc, A, B, C);
}

}  // namespace hzb
