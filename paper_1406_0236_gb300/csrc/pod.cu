// POD basis and guess of the learned warm start (no counterpart in the paper; it only
// seeds GMRES).  Given the N x T snapshot matrix X of training densities, the basis U
// (N x k, orthonormal columns) spans the dominant left singular subspace of X, found
// by subspace iteration from a Gaussian sketch (the randomized range finder of Halko,
// Martinsson and Tropp, with q power steps):
//     Z = X Omega  (Omega: T x k standard complex Gaussian),
//     repeat q times:  Z = X (X^H Z),
//     U = orth(Z)   (classical Gram-Schmidt applied twice, FP64).
// The coefficients of a density in the basis are c = U^H x, and the network's guess is
// x0 = U c.  The products run in FP32 (complex, CUDA cores) with FP64 inputs and
// outputs: the guess needs a few digits, the solve that follows fixes the rest.
#include <cstdint>

#include "hzb_internal.h"

namespace hzb {

static const int CG_T = 64;           // output tile (rows and columns)
static const int CG_K = 16;           // k-slab staged in shared memory

// C (M x N) = op(A) op(B), complex.  op(A)(m, k) = A[m * sam + k * sak] (conjugated when
// CA), op(B)(k, n) = B[k * sbk + n * sbn] (conjugated when CB); C[m * ldc + n].
// 256 threads, each 4 x 4 outputs of a 64 x 64 tile; FP32 accumulation.
template <bool CA, bool CB>
__global__ void __launch_bounds__(256) cgemm_kernel(int M, int N, int K, const double2 *__restrict__ A, long long sam,
                                                    long long sak, const double2 *__restrict__ B, long long sbk,
                                                    long long sbn, double2 *__restrict__ C, long long ldc)
{
    __shared__ float2 As[CG_K][CG_T + 1];
    __shared__ float2 Bs[CG_K][CG_T + 1];
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    const int m0 = blockIdx.y * CG_T, n0 = blockIdx.x * CG_T;
    float2 acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = make_float2(0.f, 0.f);
    for (int k0 = 0; k0 < K; k0 += CG_K) {
        // consecutive threads walk the operand's contiguous index (coalesced loads)
        for (int e = tid; e < CG_K * CG_T; e += 256) {
            const int kk = (sak == 1) ? e % CG_K : e / CG_T, mm = (sak == 1) ? e / CG_K : e % CG_T;
            const int gm = m0 + mm, gk = k0 + kk;
            const double2 a = (gm < M && gk < K) ? A[gm * sam + gk * sak] : make_double2(0.0, 0.0);
            As[kk][mm] = make_float2((float)a.x, CA ? -(float)a.y : (float)a.y);
        }
        for (int e = tid; e < CG_K * CG_T; e += 256) {
            const int kk = (sbn == 1) ? e / CG_T : e % CG_K, nn = (sbn == 1) ? e % CG_T : e / CG_K;
            const int gk = k0 + kk, gn = n0 + nn;
            const double2 b = (gk < K && gn < N) ? B[gk * sbk + gn * sbn] : make_double2(0.0, 0.0);
            Bs[kk][nn] = make_float2((float)b.x, CB ? -(float)b.y : (float)b.y);
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < CG_K; ++kk) {
            float2 a[4], b[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                a[q] = As[kk][ty + 16 * q];
                b[q] = Bs[kk][tx + 16 * q];
            }
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    acc[p][q].x = fmaf(a[p].x, b[q].x, fmaf(-a[p].y, b[q].y, acc[p][q].x));
                    acc[p][q].y = fmaf(a[p].x, b[q].y, fmaf(a[p].y, b[q].x, acc[p][q].y));
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int gm = m0 + ty + 16 * p, gn = n0 + tx + 16 * q;
            if (gm < M && gn < N) C[gm * ldc + gn] = make_double2(acc[p][q].x, acc[p][q].y);
        }
}

static void cgemm(cudaStream_t st, int M, int N, int K, const double2 *A, long long sam, long long sak, bool ca,
                  const double2 *B, long long sbk, long long sbn, bool cb, double2 *C, long long ldc)
{
    dim3 g((N + CG_T - 1) / CG_T, (M + CG_T - 1) / CG_T);
    if (ca && cb) cgemm_kernel<true, true><<<g, 256, 0, st>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc);
    else if (ca) cgemm_kernel<true, false><<<g, 256, 0, st>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc);
    else if (cb) cgemm_kernel<false, true><<<g, 256, 0, st>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc);
    else cgemm_kernel<false, false><<<g, 256, 0, st>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc);
}

// Standard complex Gaussian entries (unit variance per component) from a counter-based
// generator: splitmix64 of (seed, index) gives two uniforms, Box-Muller two normals.
__device__ __forceinline__ uint64_t pod_splitmix(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void gauss_fill_kernel(long long n, uint64_t seed, double2 *out)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const uint64_t a = pod_splitmix(seed ^ pod_splitmix(2 * (uint64_t)e));
    const uint64_t b = pod_splitmix(seed ^ pod_splitmix(2 * (uint64_t)e + 1));
    const double u1 = ((a >> 11) + 1) * (1.0 / 9007199254740993.0);      // (0, 1]
    const double u2 = (b >> 11) * (1.0 / 9007199254740992.0);
    const double rr = sqrt(-2.0 * log(u1));
    double s, c;
    sincospi(2.0 * u2, &s, &c);
    out[e] = make_double2(rr * c, rr * s);
}

// Gram-Schmidt pieces on the columns of Z (N x k, row-major, leading dimension k), FP64.
// dots: h[i] = sum_r conj(Z[r][i]) Z[r][j] for the columns i = blockIdx.x < j, and the
// squared norm of column j itself when launched with i = j (block reduction over rows)
__global__ void gs_dots_kernel(int N, int k, int j, int i0, const double2 *__restrict__ Z, double2 *__restrict__ h)
{
    __shared__ double2 red[256];
    const int i = i0 + blockIdx.x;
    double2 s = make_double2(0.0, 0.0);
    for (int r = threadIdx.x; r < N; r += blockDim.x) {
        const double2 a = Z[(size_t)r * k + i], b = Z[(size_t)r * k + j];
        s.x += a.x * b.x + a.y * b.y;
        s.y += a.x * b.y - a.y * b.x;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            red[threadIdx.x].x += red[threadIdx.x + w].x;
            red[threadIdx.x].y += red[threadIdx.x + w].y;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) h[i] = red[0];
}

// Z[:, j] -= sum_{i<j} Z[:, i] h[i]
__global__ void gs_update_kernel(int N, int k, int j, double2 *__restrict__ Z, const double2 *__restrict__ h)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N) return;
    double2 z = Z[(size_t)r * k + j];
    for (int i = 0; i < j; ++i) {
        const double2 q = Z[(size_t)r * k + i], c = h[i];
        z.x -= q.x * c.x - q.y * c.y;
        z.y -= q.x * c.y + q.y * c.x;
    }
    Z[(size_t)r * k + j] = z;
}

// Z[:, j] /= ||Z[:, j]|| (h[j] = Z[:, j]^H Z[:, j]); a zero column stays zero
__global__ void gs_scale_kernel(int N, int k, int j, double2 *__restrict__ Z, const double2 *__restrict__ h)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N) return;
    const double nn = h[j].x;
    const double s = nn > 0.0 ? 1.0 / sqrt(nn) : 0.0;
    const double2 z = Z[(size_t)r * k + j];
    Z[(size_t)r * k + j] = make_double2(z.x * s, z.y * s);
}

// orthonormal columns, in order, by classical Gram-Schmidt applied twice per column
static int orthonormalise(cudaStream_t st, int N, int k, double2 *Z, double2 *h)
{
    const unsigned gb = (unsigned)((N + 255) / 256);
    int launches = 0;
    for (int j = 0; j < k; ++j) {
        for (int pass = 0; pass < 2 && j > 0; ++pass) {
            gs_dots_kernel<<<j, 256, 0, st>>>(N, k, j, 0, Z, h);
            gs_update_kernel<<<gb, 256, 0, st>>>(N, k, j, Z, h);
            launches += 2;
        }
        gs_dots_kernel<<<1, 256, 0, st>>>(N, k, j, j, Z, h);
        gs_scale_kernel<<<gb, 256, 0, st>>>(N, k, j, Z, h);
        launches += 2;
    }
    return launches;
}

}  // namespace hzb

using namespace hzb;

extern "C" hzb_status hzb_pod_basis(hzb_ctx *c, int N, int T, const double *X, int k, int power_steps,
                                    unsigned long long seed, double *U)
{
    HZB_GUARD(c);
    if (N < 1 || T < 1 || k < 1 || k > N || k > T || power_steps < 0 || power_steps > 8 || !X || !U)
        return fail(c, HZB_EINVAL, "need 1 <= k <= min(N, T), 0 <= power_steps <= 8 and device pointers");
    DevBuf<double2> om, w, h;
    if (check_cuda(c, om.ensure((size_t)T * k), "alloc sketch") || check_cuda(c, w.ensure((size_t)T * k), "alloc") ||
        check_cuda(c, h.ensure((size_t)k), "alloc")) {
        om.release(); w.release(); h.release();
        return HZB_ENOMEM;
    }
    const double2 *Xd = (const double2 *)X;
    double2 *Z = (double2 *)U;
    const long long nk = (long long)T * k;
    gauss_fill_kernel<<<(unsigned)((nk + 255) / 256), 256, 0, c->stream>>>(nk, seed, om.ptr);
    cgemm(c->stream, N, k, T, Xd, T, 1, false, om.ptr, k, 1, false, Z, k);                 // Z = X Omega
    c->launches += 2;
    for (int q = 0; q < power_steps; ++q) {
        c->launches += orthonormalise(c->stream, N, k, Z, h.ptr);                         // keeps the scale sane
        cgemm(c->stream, T, k, N, Xd, 1, T, true, Z, k, 1, false, w.ptr, k);              // W = X^H Z
        cgemm(c->stream, N, k, T, Xd, T, 1, false, w.ptr, k, 1, false, Z, k);             // Z = X W
        c->launches += 2;
    }
    c->launches += orthonormalise(c->stream, N, k, Z, h.ptr);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    om.release(); w.release(); h.release();
    return check_cuda(c, e, "POD basis");
}

extern "C" hzb_status hzb_pod_project(hzb_ctx *c, int N, int k, int T, const double *U, const double *X, double *C)
{
    HZB_GUARD(c);
    if (N < 1 || k < 1 || T < 1 || !U || !X || !C) return fail(c, HZB_EINVAL, "bad sizes or null pointer");
    cgemm(c->stream, k, T, N, (const double2 *)U, 1, k, true, (const double2 *)X, T, 1, false, (double2 *)C, T);
    c->launches++;
    return check_cuda(c, cudaGetLastError(), "POD projection");
}

// coef[j][r] = scale (y[r][2j] + i y[r][2j+1]): the network's real outputs as complex POD
// coefficients, k x R
__global__ void net_coef_kernel(int k, int R, const float *__restrict__ y, double scale, double2 *__restrict__ coef)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= k * R) return;
    const int j = e / R, r = e % R;
    coef[e] = make_double2(scale * y[(size_t)r * 2 * k + 2 * j], scale * y[(size_t)r * 2 * k + 2 * j + 1]);
}

extern "C" hzb_status hzb_pod_expand(hzb_ctx *c, int N, int k, int R, const double *U, const double *coef, double *x0)
{
    HZB_GUARD(c);
    if (N < 1 || k < 1 || R < 1 || !U || !coef || !x0) return fail(c, HZB_EINVAL, "bad sizes or null pointer");
    cgemm(c->stream, N, R, k, (const double2 *)U, k, 1, false, (const double2 *)coef, R, 1, false, (double2 *)x0, R);
    c->launches++;
    return check_cuda(c, cudaGetLastError(), "POD expansion");
}

extern "C" hzb_status hzb_pod_guess(hzb_ctx *c, int N, int k, int R, const double *U, const float *y, double scale,
                                    double *x0)
{
    HZB_GUARD(c);
    if (N < 1 || k < 1 || R < 1 || !U || !y || !x0) return fail(c, HZB_EINVAL, "bad sizes or null pointer");
    if (check_cuda(c, c->w_d.ensure((size_t)k * R), "alloc coefficients")) return HZB_ENOMEM;
    net_coef_kernel<<<(unsigned)((k * R + 255) / 256), 256, 0, c->stream>>>(k, R, y, scale, c->w_d.ptr);
    cgemm(c->stream, N, R, k, (const double2 *)U, k, 1, false, c->w_d.ptr, R, 1, false, (double2 *)x0, R);
    c->launches += 2;
    return check_cuda(c, cudaGetLastError(), "POD guess");
}
