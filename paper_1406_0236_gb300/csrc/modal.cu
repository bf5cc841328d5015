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

// One block per (body of the shape, ring).  y is N x R (FP64); out is the shape's
// panel array (M+1) x NG x ncols in precision T.
template <typename T>
__global__ void dft_forward_kernel(int NG, int NF, int R, int ncols, const long long *__restrict__ body_off,
                                   const double2 *__restrict__ y, typename C2<T>::t *__restrict__ yh)
{
    typedef typename C2<T>::t ct;
    extern __shared__ double smem_d[];
    double2 *tw = (double2 *)smem_d;                 // NF: e^{-2 pi i m / NF}
    double2 *ring = tw + NF;                         // NF x R
    const int bs = blockIdx.y, i = blockIdx.x;
    const int M = (NF - 1) / 2;
    const long long base = body_off[bs] + (long long)i * NF;
    for (int m = threadIdx.x; m < NF; m += blockDim.x) {
        double s, c;
        sincospi(-2.0 * m / NF, &s, &c);
        tw[m] = make_double2(c, s);
    }
    for (int e = threadIdx.x; e < NF * R; e += blockDim.x) ring[e] = y[base * R + e];
    __syncthreads();
    for (int e = threadIdx.x; e < NF * R; e += blockDim.x) {
        const int pidx = e / R, r = e % R;
        const int p = pidx - M;
        const int pm = ((p % NF) + NF) % NF;
        double sx = 0.0, sy = 0.0;
        int idx = 0;
        for (int l = 0; l < NF; ++l) {
            const double2 v = ring[l * R + r], w = tw[idx];
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
    extern __shared__ double smem_d[];
    double2 *tw = (double2 *)smem_d;                 // NF: e^{+2 pi i m / NF}
    double2 *co = tw + NF;                           // NF x R coefficients, p = -M..M
    const int bs = blockIdx.y, i = blockIdx.x;
    const int M = (NF - 1) / 2;
    const long long base = body_off[bs] + (long long)i * NF;
    for (int m = threadIdx.x; m < NF; m += blockDim.x) {
        double s, c;
        sincospi(2.0 * m / NF, &s, &c);
        tw[m] = make_double2(c, s);
    }
    for (int e = threadIdx.x; e < NF * R; e += blockDim.x) {
        const int pidx = e / R, r = e % R, p = pidx - M;
        const int ap = p < 0 ? -p : p, sg = p < 0 ? 1 : 0;
        const auto v = th[((size_t)ap * NG + i) * ncols + (2 * bs + sg) * R + r];
        co[e] = make_double2((double)v.x, (double)v.y);
    }
    __syncthreads();
    const double sc = beta / NF;
    for (int e = threadIdx.x; e < NF * R; e += blockDim.x) {
        const int l = e / R, r = e % R;
        double sx = 0.0, sy = 0.0;
        // p = -M .. M  ->  twiddle index (p l) mod NF, starting at (-M l) mod NF
        int idx = (int)(((long long)(NF - M) * l) % NF);
        for (int pidx = 0; pidx < NF; ++pidx) {
            const double2 v = co[pidx * R + r], w = tw[idx];
            sx = fma(v.x, w.x, fma(-v.y, w.y, sx));
            sy = fma(v.x, w.y, fma(v.y, w.x, sy));
            idx += l;
            if (idx >= NF) idx -= NF;
        }
        double2 o = make_double2(sx * sc, sy * sc);
        if (alpha != 0.0) {
            const double2 s = sigma[base * R + e];
            o.x = fma(alpha, s.x, o.x);
            o.y = fma(alpha, s.y, o.y);
        }
        out[base * R + e] = o;
    }
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
        size_t smem = (size_t)NF * (R + 1) * sizeof(double2);
        if (smem > 200 * 1024) return fail(c, HZB_EINVAL, "n_modes * R too large for the modal apply");
        if (smem > 48 * 1024) {        // opt-in beyond the default 48 KB (not needed, and not issued, below it)
            cudaFuncSetAttribute(dft_forward_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            cudaFuncSetAttribute(dft_inverse_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        }
        dft_forward_kernel<T><<<dim3(NG, ms), DFT_THREADS, smem, c->stream>>>(NG, NF, R, ncols, doff, y, yh);
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
        cudaFuncSetAttribute(dft_forward_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(dft_inverse_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
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
