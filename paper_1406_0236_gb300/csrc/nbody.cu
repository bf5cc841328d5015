// Inter-body combined-field sum (Sec. 3.3: off-diagonal blocks by the plain Nystrom
// formula, Eq. (nystromnaive); the paper applies B with an FMM, here it is a tiled
// direct sum):
//     y_i = sum_{j not on body(i)} w_j K(x_i, x_j) sigma_j,
//     w_j K(x_i, x_j) = w_j / (4 pi) * e^{ikr} [ n_j.d / r^3 - i (k n_j.d / r^2 + eta / r) ],
// d = x_i - x_j, r = |d|.  Also: the field at off-surface points and the far field.
//
// Work decomposition: one CTA per TargetBlock (a run of <= 512 targets inside one
// body), so the sources of the target's own body are one contiguous range skipped
// uniformly by the whole CTA; source tiles are staged in shared memory with the
// density pre-multiplied by w_j / (4 pi); each thread owns TPT targets.
#include "hzb_internal.h"
#include "kernel_math.cuh"

namespace hzb {

static const int NB_THREADS = 128;
static const int NB_TPT = 4;            // targets per thread; 128 x 4 = 512 = TargetBlock size
static const int NB_TILE = 128;

// ------------------------------------------------------------------ FP64

template <int RC>
__global__ void __launch_bounds__(NB_THREADS)
nbody64_kernel(const TargetBlock *__restrict__ blocks, int N, int R, const double4 *__restrict__ pos,
               const double4 *__restrict__ nrm, const double2 *__restrict__ sigma, double k, double eta,
               double2 *__restrict__ y)
{
    __shared__ double4 s_pos[NB_TILE];
    __shared__ double4 s_nrm[NB_TILE];
    __shared__ double2 s_sig[NB_TILE * RC];
    const TargetBlock tb = blocks[blockIdx.x];
    const int r0 = blockIdx.y * RC;
    const int tid = threadIdx.x;
    double tx[NB_TPT], ty[NB_TPT], tz[NB_TPT];
    double2 acc[NB_TPT][RC];
#pragma unroll
    for (int m = 0; m < NB_TPT; ++m) {
        int t = tid + m * NB_THREADS;
        double4 p = (t < tb.count) ? pos[tb.start + t] : make_double4(1e30, 1e30, 1e30, 0.0);
        tx[m] = p.x; ty[m] = p.y; tz[m] = p.z;
#pragma unroll
        for (int c = 0; c < RC; ++c) acc[m][c] = make_double2(0.0, 0.0);
    }
    for (int range = 0; range < 2; ++range) {
        const int lo = range ? tb.excl_hi : 0;
        const int hi = range ? N : tb.excl_lo;
        for (int j0 = lo; j0 < hi; j0 += NB_TILE) {
            const int cnt = min(NB_TILE, hi - j0);
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
                for (int m = 0; m < NB_TPT; ++m) {
                    const double dx = tx[m] - p.x, dy = ty[m] - p.y, dz = tz[m] - p.z;
                    const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
                    const double ir = rsqrt(r2);
                    const double r = r2 * ir;
                    const double nd = fma(n.x, dx, fma(n.y, dy, n.z * dz));
                    const double ndir2 = nd * ir * ir;
                    const double A = ndir2 * ir;
                    const double B = fma(k, ndir2, eta * ir);
                    double s, c;
                    sincos(k * r, &s, &c);
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
#pragma unroll
    for (int m = 0; m < NB_TPT; ++m) {
        int t = tid + m * NB_THREADS;
        if (t < tb.count)
#pragma unroll
            for (int c = 0; c < RC; ++c)
                if (r0 + c < R) y[(size_t)(tb.start + t) * R + r0 + c] = acc[m][c];
    }
}

// ------------------------------------------------------------------ FP32

// Phase of e^{ikr}: r k / (2 pi) is reduced to [-1/2, 1/2] turns before the
// hardware sine and cosine, whose error grows with the argument.
template <int RC>
__global__ void __launch_bounds__(NB_THREADS)
nbody32_kernel(const TargetBlock *__restrict__ blocks, int N, int R, const float4 *__restrict__ pos,
               const float4 *__restrict__ nrm, const double2 *__restrict__ sigma, float k, float eta,
               float k_turns, double2 *__restrict__ y)
{
    __shared__ float4 s_a[NB_TILE];           // x, y, z, nx
    __shared__ float2 s_b[NB_TILE];           // ny, nz
    __shared__ float2 s_sig[NB_TILE * RC];
    const TargetBlock tb = blocks[blockIdx.x];
    const int r0 = blockIdx.y * RC;
    const int tid = threadIdx.x;
    float tx[NB_TPT], ty[NB_TPT], tz[NB_TPT];
    float2 acc[NB_TPT][RC];
#pragma unroll
    for (int m = 0; m < NB_TPT; ++m) {
        int t = tid + m * NB_THREADS;
        float4 p = (t < tb.count) ? pos[tb.start + t] : make_float4(1e18f, 1e18f, 1e18f, 0.f);
        tx[m] = p.x; ty[m] = p.y; tz[m] = p.z;
#pragma unroll
        for (int c = 0; c < RC; ++c) acc[m][c] = make_float2(0.f, 0.f);
    }
    for (int range = 0; range < 2; ++range) {
        const int lo = range ? tb.excl_hi : 0;
        const int hi = range ? N : tb.excl_lo;
        for (int j0 = lo; j0 < hi; j0 += NB_TILE) {
            const int cnt = min(NB_TILE, hi - j0);
            __syncthreads();
            if (tid < cnt) {
                const float4 p = pos[j0 + tid];
                const float4 n = nrm[j0 + tid];
                s_a[tid] = make_float4(p.x, p.y, p.z, n.x);
                s_b[tid] = make_float2(n.y, n.z);
                const double wq = (double)p.w * HZB_INV4PI;
#pragma unroll
                for (int c = 0; c < RC; ++c) {
                    double2 s = (r0 + c < R) ? sigma[(size_t)(j0 + tid) * R + r0 + c] : make_double2(0.0, 0.0);
                    s_sig[tid * RC + c] = make_float2((float)(s.x * wq), (float)(s.y * wq));
                }
            }
            __syncthreads();
#pragma unroll 2
            for (int jj = 0; jj < cnt; ++jj) {
                const float4 a = s_a[jj];
                const float2 b = s_b[jj];
#pragma unroll
                for (int m = 0; m < NB_TPT; ++m) {
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
    for (int m = 0; m < NB_TPT; ++m) {
        int t = tid + m * NB_THREADS;
        if (t < tb.count)
#pragma unroll
            for (int c = 0; c < RC; ++c)
                if (r0 + c < R)
                    y[(size_t)(tb.start + t) * R + r0 + c] = make_double2((double)acc[m][c].x, (double)acc[m][c].y);
    }
}

template <typename F>
static hzb_status launch_rc(hzb_ctx *c, int R, F f1, F f4, F f8)
{
    (void)c;
    if (R == 1) return f1(1);
    if (R <= 4) return f4(4);
    return f8(8);
}

hzb_status interbody64(hzb_ctx *c, int R, const double2 *sigma, double2 *y)
{
    if (!c->nodes_ready) return fail(c, HZB_ESTATE, "nodes not built");
    int N = (int)c->N;
    c->interbody_calls++;
    c->launches++;
    const int slot = prof_begin(c, 0);
    cudaError_t e;
    if (R == 1) {
        nbody64_kernel<1><<<dim3(c->n_tblocks, 1), NB_THREADS, 0, c->stream>>>(
            c->tblocks.ptr, N, R, c->pos64.ptr, c->nrm64.ptr, sigma, c->k, c->eta, y);
    } else if (R <= 4) {
        nbody64_kernel<4><<<dim3(c->n_tblocks, 1), NB_THREADS, 0, c->stream>>>(
            c->tblocks.ptr, N, R, c->pos64.ptr, c->nrm64.ptr, sigma, c->k, c->eta, y);
    } else {
        nbody64_kernel<8><<<dim3(c->n_tblocks, (R + 7) / 8), NB_THREADS, 0, c->stream>>>(
            c->tblocks.ptr, N, R, c->pos64.ptr, c->nrm64.ptr, sigma, c->k, c->eta, y);
    }
    e = cudaGetLastError();
    prof_end(c, slot);
    return check_cuda(c, e, "nbody64_kernel");
}

hzb_status interbody32(hzb_ctx *c, int R, const double2 *sigma, double2 *y)
{
    if (!c->nodes_ready) return fail(c, HZB_ESTATE, "nodes not built");
    int N = (int)c->N;
    c->interbody_calls++;
    c->launches++;
    const int slot = prof_begin(c, 1);
    const float k = (float)c->k, eta = (float)c->eta, kt = (float)(c->k / (2.0 * M_PI));
    if (R == 1) {
        nbody32_kernel<1><<<dim3(c->n_tblocks, 1), NB_THREADS, 0, c->stream>>>(
            c->tblocks.ptr, N, R, c->pos32.ptr, c->nrm32.ptr, sigma, k, eta, kt, y);
    } else if (R <= 4) {
        nbody32_kernel<4><<<dim3(c->n_tblocks, 1), NB_THREADS, 0, c->stream>>>(
            c->tblocks.ptr, N, R, c->pos32.ptr, c->nrm32.ptr, sigma, k, eta, kt, y);
    } else {
        nbody32_kernel<8><<<dim3(c->n_tblocks, (R + 7) / 8), NB_THREADS, 0, c->stream>>>(
            c->tblocks.ptr, N, R, c->pos32.ptr, c->nrm32.ptr, sigma, k, eta, kt, y);
    }
    cudaError_t e = cudaGetLastError();
    prof_end(c, slot);
    return check_cuda(c, e, "nbody32_kernel");
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
