// Block-diagonal inverse D^{-1} (Sec. 4, Remark after Eq. (precond); Eq. (singleinverse))
// in lean double-float arithmetic on the FP32 pipe: the same three steps as modal.cu
// (azimuthal DFT of every ring, tau^_p = S_|p| y^_p, inverse DFT with the 1/N_F factor
// and tau = alpha sigma + beta tau), for the refinement residual of the mixed solve.
// GB300 runs FP64 at 1/64 of the FP32 rate; a complex multiply-add in double-float
// takes 48 FP32 operations against 4 FP64 fused multiply-adds, so at the two pipes'
// peaks these kernels run about six times faster than the FP64 ones, at about 1e-13
// relative error instead of 1e-16.
//
// Complex values travel as float4 (re.hi, re.lo, im.hi, im.lo): the inputs y and sigma
// and the output tau are FP64 and converted once per element; the mode panels and the
// scattering matrices S_p (split once per build into a cached copy) are double-float.
// Accumulators are renormalised every 16 terms.
#include <algorithm>

#include "hzb_internal.h"
#include "lean_df.cuh"

namespace hzb {

using namespace lean;

static const int DFLM_THREADS = 128;

__global__ void csplit_kernel(size_t n, const double2 *__restrict__ in, float4 *__restrict__ out)
{
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) out[e] = csplit(in[e]);
}

// twiddles e^{sgn 2 pi i m / NF}, m < NF, in double-float
__device__ __forceinline__ void dfl_twiddles(int NF, double sgn, float4 *tw)
{
    for (int m = threadIdx.x; m < NF; m += blockDim.x) {
        double s, c;
        sincospi(sgn * 2.0 * m / NF, &s, &c);
        tw[m] = csplit(make_double2(c, s));
    }
}

// One block per (body of the shape, ring): yh_p = sum_l y(i, l) e^{-2 pi i p l / NF}
__global__ void dfl_dft_forward_kernel(int NG, int NF, int R, int ncols, const long long *__restrict__ body_off,
                                       const double2 *__restrict__ y, float4 *__restrict__ yh)
{
    extern __shared__ float4 smem_f4[];
    float4 *tw = smem_f4;                            // NF
    float4 *ring = tw + NF;                          // NF x R
    const int bs = blockIdx.y, i = blockIdx.x;
    const int M = (NF - 1) / 2;
    const long long base = body_off[bs] + (long long)i * NF;
    dfl_twiddles(NF, -1.0, tw);
    for (int e = threadIdx.x; e < NF * R; e += blockDim.x) ring[e] = csplit(y[base * R + e]);
    __syncthreads();
    for (int e = threadIdx.x; e < NF * R; e += blockDim.x) {
        const int pidx = e / R, r = e % R;
        const int p = pidx - M;
        const int pm = ((p % NF) + NF) % NF;
        dd sr = {0.f, 0.f}, si = {0.f, 0.f};
        int idx = 0;
        for (int l = 0; l < NF; ++l) {
            cmac(sr, si, ring[l * R + r], tw[idx]);
            if ((l & 15) == 15) { sr = norm(sr); si = norm(si); }
            idx += pm;
            if (idx >= NF) idx -= NF;
        }
        sr = norm(sr);
        si = norm(si);
        const int ap = p < 0 ? -p : p;
        const int sg = p < 0 ? 1 : 0;
        yh[((size_t)ap * NG + i) * ncols + (2 * bs + sg) * R + r] = make_float4(sr.h, sr.l, si.h, si.l);
        if (p == 0) yh[((size_t)0 * NG + i) * ncols + (2 * bs + 1) * R + r] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// tau(i, l) = alpha sigma(i, l) + beta / NF * sum_p tau^_p(i) e^{2 pi i p l / NF}
__global__ void dfl_dft_inverse_kernel(int NG, int NF, int R, int ncols, const long long *__restrict__ body_off,
                                       const float4 *__restrict__ th, const double2 *__restrict__ sigma,
                                       double alpha, double beta, double2 *__restrict__ out)
{
    extern __shared__ float4 smem_f4[];
    float4 *tw = smem_f4;                            // NF
    float4 *co = tw + NF;                            // NF x R coefficients, p = -M..M
    const int bs = blockIdx.y, i = blockIdx.x;
    const int M = (NF - 1) / 2;
    const long long base = body_off[bs] + (long long)i * NF;
    dfl_twiddles(NF, 1.0, tw);
    for (int e = threadIdx.x; e < NF * R; e += blockDim.x) {
        const int pidx = e / R, r = e % R, p = pidx - M;
        const int ap = p < 0 ? -p : p, sg = p < 0 ? 1 : 0;
        co[e] = th[((size_t)ap * NG + i) * ncols + (2 * bs + sg) * R + r];
    }
    __syncthreads();
    const double sc = beta / NF;
    for (int e = threadIdx.x; e < NF * R; e += blockDim.x) {
        const int l = e / R, r = e % R;
        dd sr = {0.f, 0.f}, si = {0.f, 0.f};
        int idx = (int)(((long long)(NF - M) * l) % NF);
        for (int pidx = 0; pidx < NF; ++pidx) {
            cmac(sr, si, co[pidx * R + r], tw[idx]);
            if ((pidx & 15) == 15) { sr = norm(sr); si = norm(si); }
            idx += l;
            if (idx >= NF) idx -= NF;
        }
        double2 o = make_double2(value(norm(sr)) * sc, value(norm(si)) * sc);
        if (alpha != 0.0) {
            const double2 s = sigma[base * R + e];
            o.x = fma(alpha, s.x, o.x);
            o.y = fma(alpha, s.y, o.y);
        }
        out[base * R + e] = o;
    }
}

// Batched complex GEMM C[p] = A[p] B[p] in double-float: A n x n, B and C n x nc,
// row-major.  32 x 32 output tile per block of 256 threads, each 2 x 2 outputs
// (rows tr, tr + 16; columns tc, tc + 16), K step 16.
__global__ void __launch_bounds__(256)
dfl_modal_gemm_kernel(int n, int nc, const float4 *__restrict__ A, const float4 *__restrict__ B, float4 *__restrict__ C)
{
    __shared__ float4 As[32][17];
    __shared__ float4 Bs[16][33];
    const int p = blockIdx.z;
    const float4 *Ap = A + (size_t)p * n * n;
    const float4 *Bp = B + (size_t)p * n * nc;
    float4 *Cp = C + (size_t)p * n * nc;
    const int row0 = blockIdx.y * 32, col0 = blockIdx.x * 32;
    const int tid = threadIdx.x, tr = tid / 16, tc = tid % 16;
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    dd ar[2][2], ai[2][2];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) ar[a][b] = ai[a][b] = {0.f, 0.f};
    for (int k0 = 0; k0 < n; k0 += 16) {
        for (int e = tid; e < 32 * 16; e += 256) {
            const int r = e / 16, kk = e % 16, gr = row0 + r, gk = k0 + kk;
            As[r][kk] = (gr < n && gk < n) ? Ap[(size_t)gr * n + gk] : zero;
        }
        for (int e = tid; e < 16 * 32; e += 256) {
            const int kk = e / 32, cc = e % 32, gk = k0 + kk, gc = col0 + cc;
            Bs[kk][cc] = (gk < n && gc < nc) ? Bp[(size_t)gk * nc + gc] : zero;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < 16; ++kk) {
            const float4 a0 = As[tr][kk], a1 = As[tr + 16][kk];
            const float4 b0 = Bs[kk][tc], b1 = Bs[kk][tc + 16];
            cmac(ar[0][0], ai[0][0], a0, b0);
            cmac(ar[0][1], ai[0][1], a0, b1);
            cmac(ar[1][0], ai[1][0], a1, b0);
            cmac(ar[1][1], ai[1][1], a1, b1);
        }
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                ar[a][b] = norm(ar[a][b]);
                ai[a][b] = norm(ai[a][b]);
            }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int gr = row0 + tr + 16 * a, gc = col0 + tc + 16 * b;
            if (gr < n && gc < nc) Cp[(size_t)gr * nc + gc] = make_float4(ar[a][b].h, ar[a][b].l, ai[a][b].h, ai[a][b].l);
        }
}

// the shape's S_p split into double-float, built on first use after each (re)build
static hzb_status ensure_sdd(hzb_ctx *c, ShapeDev &sd)
{
    if (sd.Sdd_ready) return HZB_OK;
    if (c->capturing) return fail(c, HZB_ESTATE, "double-float scattering matrices not built before capture");
    const size_t nmat = (size_t)(sd.geom.M + 1) * sd.geom.NG * sd.geom.NG;
    if (check_cuda(c, sd.Sdd.ensure(nmat), "alloc double-float S")) return HZB_ENOMEM;
    csplit_kernel<<<(unsigned)((nmat + 255) / 256), 256, 0, c->stream>>>(nmat, sd.S64.ptr, sd.Sdd.ptr);
    c->launches++;
    if (check_cuda(c, cudaGetLastError(), "split S")) return HZB_ECUDA;
    sd.Sdd_ready = true;
    return HZB_OK;
}

// The DFT kernels' dynamic shared memory beyond the default 48 KB: raised once to the
// largest size any call uses (200 KB), never lowered.
static void dfl_dft_smem_limit(size_t bytes)
{
    if (bytes <= 48 * 1024) return;
    cudaFuncSetAttribute(dfl_dft_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(dfl_dft_inverse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

// tau = alpha sigma + beta D^{-1} y with the DFTs and the mode GEMMs in double-float;
// the mode panels live in the FP64 panel buffers (16 bytes per value either way)
hzb_status local_inverse_dfl(hzb_ctx *c, int R, const double2 *y, const double2 *sigma, double alpha, double beta,
                             double2 *tau)
{
    if (c->reduced) return reduced_local(c, R, y, sigma, alpha, beta, tau, false);
    for (ShapeDev *sp : c->shapes) {
        ShapeDev &sd = *sp;
        const int NG = sd.geom.NG, NF = sd.geom.NF, M = sd.geom.M;
        const int ms = (int)sd.bodies.size();
        const int ncols = 2 * ms * R;
        const size_t panel = (size_t)(M + 1) * NG * ncols;
        hzb_status st = ensure_sdd(c, sd);
        if (st) return st;
        if (check_cuda(c, c->yhat64.ensure(panel), "alloc") || check_cuda(c, c->that64.ensure(panel), "alloc"))
            return HZB_ENOMEM;
        float4 *yh = reinterpret_cast<float4 *>(c->yhat64.ptr);
        float4 *th = reinterpret_cast<float4 *>(c->that64.ptr);
        const size_t smem = (size_t)NF * (R + 1) * sizeof(float4);
        if (smem > 200 * 1024) return fail(c, HZB_EINVAL, "n_modes * R too large for the modal apply");
        dfl_dft_smem_limit(smem);
        const long long *doff = sd.body_offs.ptr;
        dfl_dft_forward_kernel<<<dim3(NG, ms), DFLM_THREADS, smem, c->stream>>>(NG, NF, R, ncols, doff, y, yh);
        dfl_modal_gemm_kernel<<<dim3((ncols + 31) / 32, (NG + 31) / 32, M + 1), 256, 0, c->stream>>>(
            NG, ncols, sd.Sdd.ptr, yh, th);
        dfl_dft_inverse_kernel<<<dim3(NG, ms), DFLM_THREADS, smem, c->stream>>>(NG, NF, R, ncols, doff, th, sigma,
                                                                                alpha, beta, tau);
        c->launches += 3;
        if (check_cuda(c, cudaGetLastError(), "double-float modal apply")) return HZB_ECUDA;
    }
    return HZB_OK;
}

}  // namespace hzb
