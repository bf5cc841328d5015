// GMRES on the block-diagonally preconditioned system (Sec. 4, Eq. (precond))
//     sigma + D^{-1} B sigma = -D^{-1} v,
// batched over R right-hand sides that each have their own Krylov space (one
// operator apply serves all of them).  Arnoldi uses classical Gram-Schmidt with
// one re-orthogonalisation (CGS2); the Hessenberg least-squares problem is updated
// by complex Givens rotations on the device; the host reads back only the R
// residual estimates per iteration.  The paper stops at a residual of 1e-9 and does
// not state restart or orthogonalisation; zero initial guess unless one is given.
//
// Mixed precision (FP64 outer refinement): r = b - A x with the FP64 operator (or its
// double-float form on the FP32 pipe), an inner GMRES on A d = r whose operator
// applies run the FP32 inter-body sum and FP32 modal GEMMs (Arnoldi and least squares
// stay FP64), x += d, repeat.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "hzb_internal.h"
#include "kernel_math.cuh"

namespace hzb {

static const int RED_THREADS = 256;

// partial[(v * R + r) * nblk + blk] = sum over this block's nodes of conj(V_v) w
__global__ void cdot_partial_kernel(long long N, int R, const double2 *__restrict__ V, long long vstride,
                                    const double2 *__restrict__ w, double2 *partial)
{
    __shared__ double2 red[RED_THREADS];
    const int v = blockIdx.y, r = blockIdx.z, nblk = gridDim.x;
    const double2 *Vv = V + v * vstride;
    double2 acc = make_double2(0.0, 0.0);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)nblk * blockDim.x) {
        double2 a = Vv[i * R + r], b = w[i * R + r];
        acc.x = fma(a.x, b.x, fma(a.y, b.y, acc.x));
        acc.y = fma(a.x, b.y, fma(-a.y, b.x, acc.y));
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = RED_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] = cadd(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[((size_t)v * R + r) * nblk + blockIdx.x] = red[0];
}

__global__ void cdot_final_kernel(int nvr, int nblk, const double2 *partial, double2 *out)
{
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nvr) return;
    double2 s = make_double2(0.0, 0.0);
    for (int b = 0; b < nblk; ++b) s = cadd(s, partial[(size_t)e * nblk + b]);
    out[e] = s;
}

// w[i][r] -= sum_{v < nv} V_v[i][r] h[v][r]
__global__ void caxpy_multi_kernel(long long N, int R, int nv, const double2 *__restrict__ V, long long vstride,
                                   const double2 *__restrict__ h, double2 *w)
{
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N * R) return;
    int r = (int)(e % R);
    double2 acc = w[e];
    for (int v = 0; v < nv; ++v) {
        double2 hv = h[v * R + r];
        cfma(acc, make_double2(-hv.x, -hv.y), V[v * vstride + e]);
    }
    w[e] = acc;
}

// x[i][r] += sum_{v < jdone[r]} V_v[i][r] y[v][r]
__global__ void update_x_kernel(long long N, int R, int nv, const double2 *__restrict__ V, long long vstride,
                                const double2 *__restrict__ y, const int *__restrict__ jdone, double2 *x)
{
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N * R) return;
    int r = (int)(e % R);
    int nj = min(jdone[r], nv);
    double2 acc = x[e];
    for (int v = 0; v < nj; ++v) cfma(acc, y[v * R + r], V[v * vstride + e]);
    x[e] = acc;
}

__global__ void scale_kernel(long long N, int R, const double2 *w, const double *inv, double2 *out)
{
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N * R) return;
    out[e] = cscale(w[e], inv[e % R]);
}

__global__ void axpby_kernel(long long n, double a, const double2 *x, double b, const double2 *y, double2 *out)
{
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    double2 u = x[e], v = y[e];
    out[e] = make_double2(a * u.x + b * v.x, a * u.y + b * v.y);
}

struct GmresState {
    double2 *H;      // m x m x R: H[(row * m + col) * R + r]  (upper triangle after rotations)
    double2 *cs, *sn;  // m x R
    double2 *g;      // (m + 1) x R
    double2 *h1, *h2;  // (m + 1) x R
    double2 *nrm2;   // R  (w^H w)
    double *bnorm;   // R
    double *res;     // R relative residual estimate
    double *inv;     // R scale of the next basis vector
    int *active;     // R
    int *jdone;      // R
};

// Start of a cycle: beta = ||r0||, g = (beta, 0, ...), 1/beta as the scale of V_0.
__global__ void cycle_start_kernel(int R, int m, GmresState s, double tol, int first)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    // a non-finite norm (NaN or Inf in b, the guess or the operator) must reach the host
    // as a non-finite residual: fmax(NaN, 0) would turn it into a zero, i.e. "converged"
    const double n2 = s.nrm2[r].x;
    const double qnan = __longlong_as_double(0x7ff8000000000000ll);
    double beta = isfinite(n2) ? sqrt(fmax(n2, 0.0)) : qnan;
    if (first) s.bnorm[r] = beta;
    double bn = s.bnorm[r];
    double rel = (isfinite(beta) && isfinite(bn)) ? (bn > 0.0 ? beta / bn : 0.0) : qnan;
    s.res[r] = rel;
    int act = (bn > 0.0 && rel > tol && isfinite(beta)) ? 1 : 0;
    s.active[r] = act;
    s.jdone[r] = 0;
    for (int q = 0; q <= m; ++q) s.g[q * R + r] = make_double2(0.0, 0.0);
    s.g[r] = make_double2(beta, 0.0);
    s.inv[r] = (act && beta > 0.0) ? 1.0 / beta : 0.0;
}

// Arnoldi column j: h = h1 + h2 (CGS2), h_{j+1,j} = ||w||; apply the previous
// rotations, form the one that zeroes h_{j+1,j}, update g and the residual.
__global__ void givens_kernel(int R, int m, int j, GmresState s, double tol)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    if (!s.active[r]) {
        s.inv[r] = 0.0;
        return;
    }
    if (!isfinite(s.nrm2[r].x)) {          // non-finite basis vector: report, do not treat as breakdown
        s.res[r] = __longlong_as_double(0x7ff8000000000000ll);
        s.inv[r] = 0.0;
        s.active[r] = 0;
        return;
    }
    double hn = sqrt(fmax(s.nrm2[r].x, 0.0));
    for (int i = 0; i <= j; ++i) {
        double2 v = cadd(s.h1[i * R + r], s.h2[i * R + r]);
        s.H[((size_t)i * m + j) * R + r] = v;
    }
    for (int i = 0; i < j; ++i) {
        double2 a = s.H[((size_t)i * m + j) * R + r], b = s.H[((size_t)(i + 1) * m + j) * R + r];
        double2 c = s.cs[i * R + r], sn = s.sn[i * R + r];
        double2 t = cadd(cmul(c, a), cmul(sn, b));
        double2 u = csub(cmul(cconj(c), b), cmul(cconj(sn), a));
        s.H[((size_t)i * m + j) * R + r] = t;
        s.H[((size_t)(i + 1) * m + j) * R + r] = u;
    }
    double2 a = s.H[((size_t)j * m + j) * R + r];
    double den = sqrt(a.x * a.x + a.y * a.y + hn * hn);
    double2 c, sn;
    if (den > 0.0) {
        c = make_double2(a.x / den, -a.y / den);      // conj(a) / den
        sn = make_double2(hn / den, 0.0);             // conj(h_{j+1,j}) / den, h real
    } else {
        c = make_double2(1.0, 0.0);
        sn = make_double2(0.0, 0.0);
    }
    s.cs[j * R + r] = c;
    s.sn[j * R + r] = sn;
    s.H[((size_t)j * m + j) * R + r] = make_double2(den, 0.0);
    double2 gj = s.g[j * R + r];
    s.g[(j + 1) * R + r] = cscale(cmul(cconj(sn), gj), -1.0);
    s.g[j * R + r] = cmul(c, gj);
    double2 gn = s.g[(j + 1) * R + r];
    double rel = sqrt(gn.x * gn.x + gn.y * gn.y) / s.bnorm[r];
    s.res[r] = rel;
    s.jdone[r] = j + 1;
    bool done = !(rel > tol) || !(hn > 1e-300) || !isfinite(rel);
    s.inv[r] = done ? 0.0 : 1.0 / hn;
    if (done) s.active[r] = 0;
}

// y = H^{-1} g on the leading jdone x jdone upper triangle.
__global__ void backsolve_kernel(int R, int m, GmresState s, double2 *y)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    int n = s.jdone[r];
    for (int i = n - 1; i >= 0; --i) {
        double2 acc = s.g[i * R + r];
        for (int q = i + 1; q < n; ++q) cfma(acc, make_double2(-1.0, 0.0), cmul(s.H[((size_t)i * m + q) * R + r], y[q * R + r]));
        double2 d = s.H[((size_t)i * m + i) * R + r];
        double dd = d.x * d.x + d.y * d.y;
        y[i * R + r] = dd > 0.0 ? make_double2((acc.x * d.x + acc.y * d.y) / dd, (acc.y * d.x - acc.x * d.y) / dd)
                                : make_double2(0.0, 0.0);
    }
}

int prof_begin(hzb_ctx *c, int kind)
{
    if (!c->prof_on || c->capturing) return -1;
    const size_t slot = c->evkind.size();
    if (slot >= 4096) return -1;
    while (c->evpool.size() < 2 * (slot + 1)) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return -1;
        c->evpool.push_back(e);
    }
    c->evkind.push_back(kind);
    cudaEventRecord(c->evpool[2 * slot], c->stream);
    return (int)slot;
}

void prof_end(hzb_ctx *c, int slot)
{
    if (slot >= 0) cudaEventRecord(c->evpool[2 * slot + 1], c->stream);
}

hzb_status vec_copy(hzb_ctx *c, double2 *dst, const double2 *src, size_t n)
{
    return check_cuda(c, cudaMemcpyAsync(dst, src, n * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream), "copy");
}

hzb_status vec_zero(hzb_ctx *c, double2 *dst, size_t n)
{
    return check_cuda(c, cudaMemsetAsync(dst, 0, n * sizeof(double2), c->stream), "memset");
}

static unsigned nblocks(long long n, int th = 256) { return (unsigned)((n + th - 1) / th); }

// out[v * R + r] = sum_i conj(V_v[i][r]) w[i][r], v < nv
static hzb_status cdots(hzb_ctx *c, int R, int nv, const double2 *V, long long vstride, const double2 *w,
                        double2 *out)
{
    long long N = c->N;
    int nblk = (int)std::min<long long>(120, std::max<long long>(1, N / (RED_THREADS * 8)));
    size_t need = (size_t)nv * R * nblk;
    if (check_cuda(c, c->w_d.ensure(std::max<size_t>(need, (size_t)N * R)), "alloc partial")) return HZB_ENOMEM;
    cdot_partial_kernel<<<dim3(nblk, nv, R), RED_THREADS, 0, c->stream>>>(N, R, V, vstride, w, c->w_d.ptr);
    cdot_final_kernel<<<nblocks(nv * R), 256, 0, c->stream>>>(nv * R, nblk, c->w_d.ptr, out);
    c->launches += 2;
    return check_cuda(c, cudaGetLastError(), "cdot");
}

hzb_status apply_op(hzb_ctx *c, int R, const double2 *x, double2 *z, int precision)
{
    size_t n = (size_t)c->N * R;
    if (check_cuda(c, c->w_c.ensure(n), "alloc apply")) return HZB_ENOMEM;
    hzb_status st;
    if (precision == HZB_PREC_MIXED_FP32) {
        if ((st = interbody32(c, R, x, c->w_c.ptr))) return st;
        return local_inverse32(c, R, c->w_c.ptr, x, 1.0, 1.0, z);
    }
    if (precision == HZB_PREC_DOUBLE_FLOAT) {
        if ((st = interbody_df(c, R, x, c->w_c.ptr))) return st;
        return local_inverse_dfl(c, R, c->w_c.ptr, x, 1.0, 1.0, z);
    }
    if ((st = interbody64(c, R, x, c->w_c.ptr))) return st;
    return local_inverse64(c, R, c->w_c.ptr, x, 1.0, 1.0, z);
}

static hzb_status ensure_pinned(hzb_ctx *c, size_t n)
{
    if (c->host_pinned_n >= n) return HZB_OK;
    if (c->host_pinned) cudaFreeHost(c->host_pinned);
    c->host_pinned = nullptr;
    c->host_pinned_n = 0;
    if (check_cuda(c, cudaMallocHost(&c->host_pinned, n * sizeof(double)), "pinned")) return HZB_ENOMEM;
    c->host_pinned_n = n;
    return HZB_OK;
}

// Pointers and sizes a captured Arnoldi step depends on: a change invalidates the graphs.
struct GraphKey {
    static const int NP = 22;
    const void *p[NP];
    long long N;
    int R, m, precision, tpt32, split32, tpt64, split64, modal_engine, nbody_engine, splittc, tc32, x2, engine64;
    bool operator==(const GraphKey &o) const { return std::memcmp(this, &o, sizeof(GraphKey)) == 0; }
};
static_assert(sizeof(GraphKey) <= sizeof(((hzb_ctx *)nullptr)->gkey), "graph key storage");

static void drop_graphs(hzb_ctx *c)
{
    for (cudaGraphExec_t g : c->gexec)
        if (g) cudaGraphExecDestroy(g);
    c->gexec.clear();
    c->glaunch.clear();
}

// Replay the captured graph of Arnoldi step j (capturing it on first use).
template <typename F>
static hzb_status graph_step(hzb_ctx *c, int j, F &step, const GraphKey &key)
{
    if (!c->gkey_valid || std::memcmp(c->gkey, &key, sizeof(GraphKey)) != 0) {
        drop_graphs(c);
        std::memcpy(c->gkey, &key, sizeof(GraphKey));
        c->gkey_valid = true;
    }
    if ((int)c->gexec.size() <= j) {
        c->gexec.resize(j + 1, nullptr);
        c->glaunch.resize(j + 1, 0);
    }
    if (!c->gexec[j]) {
        const long long l0 = c->launches, i0 = c->interbody_calls;
        if (check_cuda(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "begin capture"))
            return HZB_ECUDA;
        c->capturing = true;
        hzb_status st = step(j);
        c->capturing = false;
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(c->stream, &g);
        if (st || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return st ? st : check_cuda(c, e, "end capture");
        }
        cudaGraphExec_t ex = nullptr;
        e = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (check_cuda(c, e, "graph instantiate")) return HZB_ECUDA;
        c->gexec[j] = ex;
        c->glaunch[j] = c->launches - l0;
        c->launches = l0;
        c->interbody_calls = i0;
    }
    c->launches += c->glaunch[j];
    c->interbody_calls += 1;
    return check_cuda(c, cudaGraphLaunch(c->gexec[j], c->stream), "graph launch");
}

void release_graphs(hzb_ctx *c) { drop_graphs(c); }

hzb_status gmres_solve(hzb_ctx *c, int R, const double2 *b, double2 *x, int x_is_zero, int precision, double tol,
                       int maxit, int restart, int *iters, double *relres, int *converged)
{
    const long long N = c->N;
    const size_t NR = (size_t)N * R;
    int m = (restart > 0) ? std::min(restart, maxit) : maxit;
    // keep the Krylov basis within 32 GB of HBM: restart earlier for large N x R
    const double basis_budget = 32.0 * (1ull << 30);
    const long long m_fit = (long long)(basis_budget / (16.0 * (double)NR)) - 1;
    m = (int)std::max<long long>(std::min<long long>(m, m_fit), 8);
    hzb_status st;
    if (check_cuda(c, c->krylov.ensure((size_t)(m + 1) * NR), "alloc krylov basis") ||
        check_cuda(c, c->w_a.ensure(NR), "alloc") || check_cuda(c, c->w_b.ensure(NR), "alloc"))
        return HZB_ENOMEM;
    // small state, laid out in one buffer
    size_t nsmall = (size_t)m * m * R + 2 * (size_t)m * R + 3 * (size_t)(m + 1) * R + R + (size_t)m * R + 4 * R;
    if (check_cuda(c, c->small.ensure(nsmall), "alloc hessenberg")) return HZB_ENOMEM;
    if (ensure_pinned(c, 2 * (size_t)R + 4)) return HZB_ENOMEM;
    GmresState s;
    double2 *p = c->small.ptr;
    s.H = p; p += (size_t)m * m * R;
    s.cs = p; p += (size_t)m * R;
    s.sn = p; p += (size_t)m * R;
    s.g = p; p += (size_t)(m + 1) * R;
    s.h1 = p; p += (size_t)(m + 1) * R;
    s.h2 = p; p += (size_t)(m + 1) * R;
    s.nrm2 = p; p += R;
    double2 *y = p; p += (size_t)m * R;
    s.bnorm = (double *)p; p += R;
    s.res = (double *)p; p += R;
    s.inv = (double *)p; p += R;
    int *ip = (int *)p;
    s.active = ip;
    s.jdone = ip + R;

    double2 *V = c->krylov.ptr;
    double2 *w = c->w_a.ptr;
    const unsigned gN = nblocks((long long)NR);
    const unsigned gR = nblocks(R, 64);
    int total = 0, real_iters = 0;
    bool first = true, all_done = false;
    double *hres = c->host_pinned;
    int *hact = (int *)(c->host_pinned + R);
    int *hjd = hact + R;
    // dot-product partial sums sized for the largest step, so that a captured step
    // never reallocates
    {
        int nblk = (int)std::min<long long>(120, std::max<long long>(1, N / (RED_THREADS * 8)));
        if (check_cuda(c, c->w_d.ensure(std::max<size_t>((size_t)(m + 1) * R * nblk, NR)), "alloc partial"))
            return HZB_ENOMEM;
    }
    // CUDA graphs need a capturable (non-legacy) stream; auto = small problems only
    bool graphs = c->use_graphs > 0 || (c->use_graphs < 0 && (long long)NR <= 4000000);
    if (c->stream == nullptr) graphs = false;
    // The key is taken right before each captured step, after the eager step 0 has
    // made every allocation the step needs, so it names the buffers the graph uses.
    GraphKey graph_key;
    auto make_key = [&]() {
        std::memset(&graph_key, 0, sizeof(graph_key));
        const void *ps[GraphKey::NP] = {V, w, c->small.ptr, c->w_c.ptr, c->w_d.ptr, c->yhat64.ptr, c->that64.ptr,
                                        c->yhat32.ptr, c->that32.ptr, c->nb_part32.ptr, c->nb_part64.ptr,
                                        c->sctab.ptr, (const void *)c->stream, c->tblocks.ptr, c->sig32.ptr,
                                        c->w_a.ptr, c->w_b.ptr, c->f_a.ptr, c->f_b.ptr, c->dfa.ptr,
                                        c->blockpairs.ptr, c->Ximg.ptr};
        std::memcpy(graph_key.p, ps, sizeof(ps));
        graph_key.N = N; graph_key.R = R; graph_key.m = m; graph_key.precision = precision;
        graph_key.tpt32 = c->tune32_tpt; graph_key.split32 = c->tune32_split;
        graph_key.tpt64 = c->tune64_tpt; graph_key.split64 = c->tune64_split;
        graph_key.modal_engine = c->modal_engine; graph_key.nbody_engine = c->nbody_engine;
        graph_key.splittc = c->tunetc_split; graph_key.tc32 = c->tune32_tc * 1000000 + c->tune32_tc_R;
        graph_key.x2 = c->tune32_x2 * 10000 + c->tune32_R; graph_key.engine64 = c->nbody64_engine;
    };
    if (x_is_zero && (st = vec_zero(c, x, NR))) return st;
    // ||b|| once
    if ((st = cdots(c, R, 1, b, 0, b, s.nrm2))) return st;
    while (true) {
        // r0 = b - A x  (b itself for a zero start)
        if (first && x_is_zero) {
            if ((st = vec_copy(c, w, b, NR))) return st;
        } else {
            if ((st = apply_op(c, R, x, c->w_b.ptr, precision))) return st;
            axpby_kernel<<<gN, 256, 0, c->stream>>>((long long)NR, 1.0, b, -1.0, c->w_b.ptr, w);
            c->launches++;
        }
        if (!(first)) {
            if ((st = cdots(c, R, 1, w, 0, w, s.nrm2))) return st;
        }
        cycle_start_kernel<<<gR, 64, 0, c->stream>>>(R, m, s, tol, first ? 1 : 0);
        if (first && !x_is_zero) {
            // the first norm above was ||b||; the residual norm of a non-zero start is needed too
            if ((st = cdots(c, R, 1, w, 0, w, s.nrm2))) return st;
            cycle_start_kernel<<<gR, 64, 0, c->stream>>>(R, m, s, tol, 0);
        }
        first = false;
        scale_kernel<<<gN, 256, 0, c->stream>>>(N, R, w, s.inv, V);
        c->launches += 2;
        cudaMemcpyAsync(hres, s.res, R * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
        cudaMemcpyAsync(hact, s.active, R * sizeof(int), cudaMemcpyDeviceToHost, c->stream);
        if (check_cuda(c, cudaStreamSynchronize(c->stream), "gmres start")) return HZB_ECUDA;
        bool any = false;
        for (int r = 0; r < R; ++r) any |= hact[r] != 0;
        if (!any || total >= maxit) {
            all_done = !any;
            break;
        }
        // One Arnoldi step: z = A V_j, CGS2 against V_0..V_j, norm, Givens, V_{j+1}.
        auto arnoldi_step = [&](int jj) -> hzb_status {
            hzb_status e2;
            double2 *Vj = V + (size_t)jj * NR;
            if ((e2 = apply_op(c, R, Vj, w, precision))) return e2;
            if ((e2 = cdots(c, R, jj + 1, V, (long long)NR, w, s.h1))) return e2;
            caxpy_multi_kernel<<<gN, 256, 0, c->stream>>>(N, R, jj + 1, V, (long long)NR, s.h1, w);
            if ((e2 = cdots(c, R, jj + 1, V, (long long)NR, w, s.h2))) return e2;
            caxpy_multi_kernel<<<gN, 256, 0, c->stream>>>(N, R, jj + 1, V, (long long)NR, s.h2, w);
            if ((e2 = cdots(c, R, 1, w, 0, w, s.nrm2))) return e2;
            givens_kernel<<<gR, 64, 0, c->stream>>>(R, m, jj, s, tol);
            c->launches += 4;                  // two caxpy, givens, scale
            scale_kernel<<<gN, 256, 0, c->stream>>>(N, R, w, s.inv, V + (size_t)(jj + 1) * NR);
            return HZB_OK;
        };
        // Steps run in chunks of `every` without host synchronisation: a right-hand
        // side that converges inside a chunk is frozen by givens_kernel (its next basis
        // vectors are zero and its jdone stays), so the extra steps change nothing.
        // automatic: chunks of 4 where an apply is cheap next to a host round trip; every
        // step where an apply costs milliseconds (a converged chunk's extra steps would
        // each cost a full apply)
        const double pair_work = (double)c->N * (double)c->N * R;
        const int every = c->check_every > 0 ? c->check_every : ((long long)NR <= 1000000 && pair_work < 4e9 ? 4 : 1);
        int j = 0;
        while (j < m && total < maxit) {
            const int q = std::min(every, std::min(m - j, maxit - total));
            for (int t = 0; t < q; ++t, ++j, ++total) {
                if (graphs && j > 0) {
                    make_key();
                    if ((st = graph_step(c, j, arnoldi_step, graph_key))) return st;
                } else if ((st = arnoldi_step(j))) {
                    return st;
                }
            }
            cudaMemcpyAsync(hres, s.res, R * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
            cudaMemcpyAsync(hact, s.active, R * sizeof(int), cudaMemcpyDeviceToHost, c->stream);
            cudaMemcpyAsync(hjd, s.jdone, R * sizeof(int), cudaMemcpyDeviceToHost, c->stream);
            if (check_cuda(c, cudaStreamSynchronize(c->stream), "gmres iteration")) return HZB_ECUDA;
            bool anyact = false;
            for (int r = 0; r < R; ++r) anyact |= hact[r] != 0;
            if (!anyact) break;
        }
        {
            int jmax = 0;
            for (int r = 0; r < R; ++r) jmax = std::max(jmax, hjd[r]);
            real_iters += jmax;
        }
        backsolve_kernel<<<gR, 64, 0, c->stream>>>(R, m, s, y);
        update_x_kernel<<<gN, 256, 0, c->stream>>>(N, R, m, V, (long long)NR, y, s.jdone, x);
        c->launches += 2;
        if (check_cuda(c, cudaGetLastError(), "gmres update")) return HZB_ECUDA;
        bool anyact = false;
        for (int r = 0; r < R; ++r) anyact |= hact[r] != 0;
        if (!anyact) {
            all_done = true;
            break;
        }
        if (total >= maxit) break;
    }
    if (check_cuda(c, cudaStreamSynchronize(c->stream), "gmres end")) return HZB_ECUDA;
    double worst = 0.0;
    bool bad = false;
    for (int r = 0; r < R; ++r) {
        if (!std::isfinite(hres[r])) bad = true;
        worst = std::max(worst, hres[r]);
    }
    *iters = real_iters;
    *relres = worst;
    *converged = all_done && worst <= tol && !bad;
    if (bad) return fail(c, HZB_ENAN, "non-finite residual in GMRES");
    return HZB_OK;
}

// ||b - A x|| / ||b|| per right-hand side with the operator of the given precision;
// r_out (N x R) receives b - A x
static hzb_status residual_with(hzb_ctx *c, int R, const double2 *b, const double2 *x, double2 *r_out,
                                std::vector<double> &rel, int precision)
{
    const size_t NR = (size_t)c->N * R;
    hzb_status st;
    if ((st = apply_op(c, R, x, r_out, precision))) return st;
    axpby_kernel<<<nblocks((long long)NR), 256, 0, c->stream>>>((long long)NR, 1.0, b, -1.0, r_out, r_out);
    c->launches++;
    DevBuf<double2> &tmp = c->tiny;
    if (check_cuda(c, tmp.ensure(2 * (size_t)R), "alloc")) return HZB_ENOMEM;
    if ((st = cdots(c, R, 1, r_out, 0, r_out, tmp.ptr)) || (st = cdots(c, R, 1, b, 0, b, tmp.ptr + R))) return st;
    std::vector<double2> h(2 * R);
    cudaMemcpyAsync(h.data(), tmp.ptr, 2 * R * sizeof(double2), cudaMemcpyDeviceToHost, c->stream);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (check_cuda(c, e, "residual")) return HZB_ECUDA;
    rel.assign(R, 0.0);
    for (int r = 0; r < R; ++r) rel[r] = h[R + r].x > 0 ? std::sqrt(std::max(h[r].x, 0.0) / h[R + r].x) : 0.0;
    return HZB_OK;
}

// the refinement residual: FP64 operator (or double-float inter-body sum)
static hzb_status true_residual(hzb_ctx *c, int R, const double2 *b, const double2 *x, double2 *r_out,
                                std::vector<double> &rel)
{
    return residual_with(c, R, b, x, r_out, rel, c->opt.residual);
}

hzb_status solve_driver(hzb_ctx *c, int R, const double2 *v, const double2 *x0, hzb_stats *stats,
                        const double2 *b_given)
{
    const size_t NR = (size_t)c->N * R;
    hzb_status st;
    DevBuf<double2> &bbuf = c->s_b, &rbuf = c->s_r, &dbuf = c->s_d;
    // kernels with bounded waits leave their error flag for the end of the solve (no
    // per-launch synchronisation inside the iteration)
    c->in_solve = true;
    auto cleanup = [&]() { c->in_solve = false; };
    if (check_cuda(c, c->sol.ensure(NR), "alloc densities") || check_cuda(c, bbuf.ensure(NR), "alloc rhs")) {
        cleanup();
        return HZB_ENOMEM;
    }
    c->sol_R = R;
    long long calls0 = c->interbody_calls, launches0 = c->launches;
    c->evkind.clear();
    c->prof_on = true;
    cudaEventRecord(c->ev0, c->stream);
    // b = -D^{-1} v, unless given
    if (b_given) {
        if ((st = vec_copy(c, bbuf.ptr, b_given, NR))) { cleanup(); return st; }
    } else if ((st = (c->opt.precision != HZB_PREC_FP64 && c->opt.residual == HZB_PREC_DOUBLE_FLOAT)
                         ? local_inverse_dfl(c, R, v, nullptr, 0.0, -1.0, bbuf.ptr)
                         : local_inverse64(c, R, v, nullptr, 0.0, -1.0, bbuf.ptr))) {
        cleanup();
        return st;
    }
    if ((c->fault & FAULT_NAN) && !(c->fault_spent & FAULT_NAN)) {         // injected: NaN in b
        c->fault_spent |= FAULT_NAN;
        static const double2 qnan2 = {std::nan(""), 0.0};
        if (check_cuda(c, cudaMemcpyAsync(bbuf.ptr, &qnan2, sizeof(double2), cudaMemcpyHostToDevice, c->stream),
                       "inject NaN")) {
            cleanup();
            return HZB_ECUDA;
        }
    }
    double2 *x = c->sol.ptr;
    int it = 0, conv = 0, outer = 0;
    double rr = 0.0;
    hzb_status solve_status = HZB_OK;
    if (x0) {
        if ((st = vec_copy(c, x, x0, NR))) { cleanup(); return st; }
    }
    if (c->opt.precision == HZB_PREC_FP64) {
        st = gmres_solve(c, R, bbuf.ptr, x, x0 ? 0 : 1, HZB_PREC_FP64, c->opt.gmres_tol, c->opt.maxit,
                         c->opt.restart, &it, &rr, &conv);
        if (st) { cleanup(); return st; }
        outer = 1;
        if (!conv) solve_status = HZB_ENOCONV;
    } else {
        if (check_cuda(c, rbuf.ensure(NR), "alloc") || check_cuda(c, dbuf.ensure(NR), "alloc")) {
            cleanup();
            return HZB_ENOMEM;
        }
        std::vector<double> rel(R, 1.0);
        if (x0) {
            // A guess starts refinement with the inner (FP32) operator's residual: the first
            // correction then lands on the FP32-operator solution, as from a zero start, and
            // the high-precision residuals that follow are the same in number.
            if ((st = residual_with(c, R, bbuf.ptr, x, rbuf.ptr, rel, HZB_PREC_MIXED_FP32))) { cleanup(); return st; }
        } else {
            if ((st = vec_zero(c, x, NR)) || (st = vec_copy(c, rbuf.ptr, bbuf.ptr, NR))) { cleanup(); return st; }
        }
        double worst = *std::max_element(rel.begin(), rel.end());
        conv = worst <= c->opt.gmres_tol;
        double c1 = -1.0;            // contraction observed in the first refinement step
        // From a guess, the first correction solves with the FP32 operator's residual and
        // lands on the FP32-operator solution whatever the tolerance, so reducing that
        // residual below inner_tol * |b| buys nothing: in this step the inner tolerance is
        // absolute (relative to b), and a good guess needs fewer inner iterations.  A guess
        // whose FP32 residual is already below that level is better than any such
        // correction would leave it: the step is skipped and refinement starts from the
        // guess's high-precision residual.
        bool guess_step = x0 != nullptr;
        while (!conv && outer < c->opt.max_outer && it < c->opt.maxit) {
            const double want = c->opt.verify_final ? 0.3 : 0.1;
            double tin = std::max(c->opt.inner_tol, want * c->opt.gmres_tol / std::max(worst, 1e-300));
            bool skip = false;
            if (guess_step) {
                const double t_abs = c->opt.inner_tol / std::max(worst, 1e-300);
                skip = t_abs >= 1.0;
                tin = std::max(tin, t_abs);
            }
            tin = std::min(tin, 0.5);
            int iin = 0, cin = 1;
            double rin = 0.0;
            if (!skip) {
                cin = 0;
                st = gmres_solve(c, R, rbuf.ptr, dbuf.ptr, 1, HZB_PREC_MIXED_FP32, tin, c->opt.maxit - it,
                                 c->opt.restart, &iin, &rin, &cin);
                if (st && st != HZB_ENOCONV) { cleanup(); return st; }
                it += iin;
                axpby_kernel<<<nblocks((long long)NR), 256, 0, c->stream>>>((long long)NR, 1.0, x, 1.0, dbuf.ptr, x);
                c->launches++;
            }
            ++outer;
            if (!c->opt.verify_final && c1 >= 0.0) {
                // the residual after this correction is bounded by worst * max(c1, tin);
                // a factor 10 covers the variation of the contraction between steps
                const double pred = worst * std::max(c1, tin) * 10.0;
                if (pred <= c->opt.gmres_tol && cin) {
                    worst = pred;
                    conv = 1;
                    break;
                }
            }
            if ((st = true_residual(c, R, bbuf.ptr, x, rbuf.ptr, rel))) { cleanup(); return st; }
            double nw = *std::max_element(rel.begin(), rel.end());
            if (!std::isfinite(nw)) { cleanup(); return fail(c, HZB_ENAN, "non-finite refinement residual"); }
            // c1 bounds the contraction of later steps by where the FP32 operator's solution
            // lands: from zero that is nw / 1; after a guess's first step, which aimed at the
            // absolute level inner_tol * |b|, it is nw itself, not nw over the guess's FP32
            // residual.  A skipped step observes no contraction: the next one sets c1.
            if (c1 < 0.0 && !skip) c1 = guess_step ? nw : nw / std::max(worst, 1e-300);
            guess_step = false;
            worst = nw;
            conv = worst <= c->opt.gmres_tol;
        }
        rr = worst;
        if (!conv) solve_status = HZB_ENOCONV;
    }
    cudaEventRecord(c->ev1, c->stream);
    if (check_cuda(c, cudaEventSynchronize(c->ev1), "solve")) { cleanup(); return HZB_ECUDA; }
    cleanup();
    if (c->kerr_ready) {                          // a bounded tensor-core wait that ran out during the solve
        int flag = 0;
        if (check_cuda(c, cudaMemcpy(&flag, c->kerr.ptr, sizeof(int), cudaMemcpyDeviceToHost), "read error flag"))
            return HZB_ECUDA;
        if (flag) {
            cudaMemset(c->kerr.ptr, 0, sizeof(int));
            return fail(c, HZB_ETIMEOUT, "tensor-core wait timed out during the solve");
        }
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    c->prof_on = false;
    double tk[3] = {0.0, 0.0, 0.0};
    long long nk[3] = {0, 0, 0};
    for (size_t q = 0; q < c->evkind.size(); ++q) {
        float e = 0.f;
        if (cudaEventElapsedTime(&e, c->evpool[2 * q], c->evpool[2 * q + 1]) == cudaSuccess) {
            tk[c->evkind[q]] += e;
            nk[c->evkind[q]]++;
        }
    }
    c->evkind.clear();
    if (stats) {
        stats->t_nbody64_ms = tk[0];
        stats->t_nbody32_ms = tk[1];
        stats->t_nbodydf_ms = tk[2];
        stats->n_nbodydf = nk[2];
        stats->n_nbody64 = nk[0];
        stats->n_nbody32 = nk[1];
        stats->kernel_launches = c->launches - launches0;
        stats->iterations = it;
        stats->outer_iterations = outer;
        stats->converged = conv;
        stats->rel_residual = rr;
        stats->t_solve_ms = ms;
        stats->t_setup_ms = c->t_setup_ms;
        stats->interbody_applies = c->interbody_calls - calls0;
    }
    cleanup();
    if (solve_status == HZB_ENOCONV) return fail(c, HZB_ENOCONV, "GMRES did not reach the tolerance");
    return HZB_OK;
}

}  // namespace hzb
