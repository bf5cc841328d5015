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
#include "kernel_math.cuh"

namespace hzb {

template <typename T> struct C2;
template <> struct C2<double> { typedef double2 t; };
template <> struct C2<float> { typedef float2 t; };

static const int DFT_THREADS = 128;

void launch_modal_gemm_tc(hzb_ctx *c, int n, int nc, int modes, const float2 *A, const float2 *B, float2 *C);


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
// 32 x (16 TB) output tile per block, 256 threads, 2 x TB outputs per thread, K step 16;
// TB = 1 for panels of at most 16 columns (one body of a shape and R = 1 ... 8 bodies
// with R = 1 fill 16), so no half of the tile multiplies zeros.
template <typename T, int TB>
__global__ void __launch_bounds__(256)
modal_gemm_kernel(int n, int nc, const typename C2<T>::t *__restrict__ A, const typename C2<T>::t *__restrict__ B,
                  typename C2<T>::t *__restrict__ C)
{
    typedef typename C2<T>::t ct;
    __shared__ ct As[32][17];
    __shared__ ct Bs[16][16 * TB + 1];
    const int p = blockIdx.z;
    const ct *Ap = A + (size_t)p * n * n;
    const ct *Bp = B + (size_t)p * n * nc;
    ct *Cp = C + (size_t)p * n * nc;
    const int row0 = blockIdx.y * 32, col0 = blockIdx.x * (16 * TB);
    const int tid = threadIdx.x;
    const int tr = tid / 16, tc = tid % 16;     // rows tr, tr+16; cols tc (, tc+16)
    T accr[2][TB], acci[2][TB];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < TB; ++b) accr[a][b] = acci[a][b] = (T)0;
    for (int k0 = 0; k0 < n; k0 += 16) {
        for (int e = tid; e < 32 * 16; e += 256) {
            int r = e / 16, kk = e % 16;
            int gr = row0 + r, gk = k0 + kk;
            ct v;
            v.x = (T)0; v.y = (T)0;
            if (gr < n && gk < n) v = Ap[(size_t)gr * n + gk];
            As[r][kk] = v;
        }
        for (int e = tid; e < 16 * 16 * TB; e += 256) {
            int kk = e / (16 * TB), cc = e % (16 * TB);
            int gk = k0 + kk, gc = col0 + cc;
            ct v;
            v.x = (T)0; v.y = (T)0;
            if (gk < n && gc < nc) v = Bp[(size_t)gk * nc + gc];
            Bs[kk][cc] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            const ct a[2] = {As[tr][kk], As[tr + 16][kk]};
#pragma unroll
            for (int b = 0; b < TB; ++b) {
                const ct bb = Bs[kk][tc + 16 * b];
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    accr[q][b] += a[q].x * bb.x - a[q].y * bb.y;
                    acci[q][b] += a[q].x * bb.y + a[q].y * bb.x;
                }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < TB; ++b) {
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
static void modal_gemm(cudaStream_t st, int n, int nc, int modes, const typename C2<T>::t *A,
                       const typename C2<T>::t *B, typename C2<T>::t *C)
{
    if (nc <= 16)
        modal_gemm_kernel<T, 1><<<dim3((nc + 15) / 16, (n + 31) / 32, modes), 256, 0, st>>>(n, nc, A, B, C);
    else
        modal_gemm_kernel<T, 2><<<dim3((nc + 31) / 32, (n + 31) / 32, modes), 256, 0, st>>>(n, nc, A, B, C);
}

template <typename T>
static hzb_status local_inverse_t(hzb_ctx *c, int R, const double2 *y, const double2 *sigma, double alpha,
                                  double beta, double2 *tau)
{
    typedef typename C2<T>::t ct;
    if (c->reduced) return reduced_local(c, R, y, sigma, alpha, beta, tau, sizeof(T) == 4);
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
        // FP32 path: tcgen05 fed by TMA (modal_tma.cu) once the panels are wide enough to
        // fill the tensor cores, or as chosen; mma.sync TF32 x 3 on request
        const bool f32 = sizeof(T) == 4;
        if (f32 && (c->modal_engine == 2 || (c->modal_engine < 0 && ncols >= 32))) {
            hzb_status st = modal_gemm_tma(c, sd, ncols, (const float2 *)yh, (float2 *)th);
            if (st) return st;
        } else if (f32 && c->modal_engine == 1)
            launch_modal_gemm_tc(c, NG, ncols, M + 1, (const float2 *)S, (const float2 *)yh, (float2 *)th);
        else
            modal_gemm<T>(c->stream, NG, ncols, M + 1, S, yh, th);
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
        modal_gemm<double>(c->stream, NG, ncols, M + 1, sd.S64.ptr, yh, th);
        dft_inverse_kernel<double><<<dim3(NG, ms), DFT_THREADS, smem, c->stream>>>(NG, NF, R, ncols, doff, th,
                                                                                    sigma, alpha, beta, tau);
        c->launches += 3;
        if (check_cuda(c, cudaGetLastError(), "modal apply")) return HZB_ECUDA;
    }
    return HZB_OK;
}

// Y = A_pp^{-1} X for a single body of the shape placed at offset 0 (X, Y: n x R,
// node-major), FP64: the same three kernels as local_inverse64.
hzb_status shape_inverse64(hzb_ctx *c, ShapeDev &sd, int R, const double2 *X, double2 *Y)
{
    const int NG = sd.geom.NG, NF = sd.geom.NF, M = sd.geom.M;
    const int ncols = 2 * R;
    const size_t panel = (size_t)(M + 1) * NG * ncols;
    if (check_cuda(c, c->yhat64.ensure(panel), "alloc") || check_cuda(c, c->that64.ensure(panel), "alloc") ||
        check_cuda(c, c->zero_off.ensure(1), "alloc"))
        return HZB_ENOMEM;
    if (check_cuda(c, cudaMemsetAsync(c->zero_off.ptr, 0, sizeof(long long), c->stream), "memset")) return HZB_ECUDA;
    size_t smem = (size_t)NF * (R + 1) * sizeof(double2);
    if (smem > 200 * 1024) return fail(c, HZB_EINVAL, "n_modes * R too large for the modal apply");
    dft_smem_limit<double>(smem);
    dft_forward_kernel<double><<<dim3(NG, 1), DFT_THREADS, smem, c->stream>>>(NG, NF, R, ncols, c->zero_off.ptr, X,
                                                                             c->yhat64.ptr);
    modal_gemm<double>(c->stream, NG, ncols, M + 1, sd.S64.ptr, c->yhat64.ptr, c->that64.ptr);
    dft_inverse_kernel<double><<<dim3(NG, 1), DFT_THREADS, smem, c->stream>>>(NG, NF, R, ncols, c->zero_off.ptr,
                                                                             c->that64.ptr, nullptr, 0.0, 1.0, Y);
    c->launches += 3;
    return check_cuda(c, cudaGetLastError(), "shape inverse");
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

__device__ __forceinline__ uint32_t to_tf32(float x)       // = cvt.rna.tf32.f32 for finite x
{
    return (__float_as_uint(x) + 0x1000u) & 0xFFFFE000u;
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

void launch_modal_gemm_tc(hzb_ctx *c, int n, int nc, int modes, const float2 *A, const float2 *B, float2 *C)
{
    dim3 grid((nc + 63) / 64, (2 * n + 63) / 64, modes);
    modal_gemm_tc_kernel<<<grid, 128, 0, c->stream>>>(n, nc, A, B, C);
}

}  // namespace hzb
