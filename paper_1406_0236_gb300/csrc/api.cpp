// C ABI of the library (include/hzb.h): context, call order, argument checks and
// host <-> device marshalling.  All arithmetic runs in the CUDA kernels.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "hzb_internal.h"

using namespace hzb;

namespace hzb {

hzb_status fail(hzb_ctx *c, hzb_status s, const std::string &msg)
{
    if (c) c->err = msg;
    return s;
}

hzb_status check_cuda(hzb_ctx *c, cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return HZB_OK;
    if (c) c->err = std::string(what) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return HZB_ENOMEM;
    }
    return HZB_ECUDA;
}

thread_local bool g_fail_alloc = false;

int parse_fault_spec(const char *spec)
{
    int f = 0;
    if (!spec) return 0;
    std::string s(spec);
    size_t a = 0;
    while (a <= s.size()) {
        size_t b = s.find(',', a);
        if (b == std::string::npos) b = s.size();
        const std::string t = s.substr(a, b - a);
        if (t == "alloc") f |= FAULT_ALLOC;
        else if (t == "geom") f |= FAULT_GEOM;
        else if (t == "nan") f |= FAULT_NAN;
        else if (t == "timeout") f |= FAULT_TIMEOUT;
        a = b + 1;
    }
    return f;
}

}  // namespace hzb


extern "C" {

void hzb_default_options(hzb_options *o)
{
    if (!o) return;
    o->device = 0;
    o->cuda_stream = nullptr;
    o->precision = HZB_PREC_FP64;
    o->gmres_tol = 1e-10;
    o->restart = 0;
    o->maxit = 500;
    o->inner_tol = 1e-5;
    o->max_outer = 10;
    o->verify_final = 1;
    o->residual = HZB_PREC_FP64;
}

const char *hzb_status_string(hzb_status s)
{
    switch (s) {
    case HZB_OK: return "ok";
    case HZB_EINVAL: return "invalid argument";
    case HZB_ENOMEM: return "out of memory";
    case HZB_ECUDA: return "CUDA error";
    case HZB_ENOCONV: return "GMRES did not converge";
    case HZB_ENAN: return "non-finite value";
    case HZB_ETIMEOUT: return "device wait timed out";
    case HZB_ESTATE: return "call out of order";
    }
    return "unknown status";
}

static bool valid_options(const hzb_options *o)
{
    return o && o->device >= 0 && (o->precision == HZB_PREC_FP64 || o->precision == HZB_PREC_MIXED_FP32) &&
           (o->residual == HZB_PREC_FP64 || o->residual == HZB_PREC_DOUBLE_FLOAT) &&
           o->gmres_tol > 0 && o->maxit > 0 && o->max_outer > 0 && o->inner_tol > 0 && o->inner_tol < 1;
}

hzb_status hzb_create(const hzb_options *options, hzb_ctx **out)
{
    if (!out) return HZB_EINVAL;
    *out = nullptr;
    hzb_options o;
    hzb_default_options(&o);
    if (options) o = *options;
    if (!valid_options(&o)) return HZB_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || o.device >= ndev) {
        cudaGetLastError();
        return HZB_ECUDA;
    }
    if (cudaSetDevice(o.device) != cudaSuccess) return HZB_ECUDA;
    hzb_ctx *c = new (std::nothrow) hzb_ctx();
    if (!c) return HZB_ENOMEM;
    c->opt = o;
    c->stream = (cudaStream_t)o.cuda_stream;
    c->fault = parse_fault_spec(std::getenv("HZB_FAULT"));
    if (cudaEventCreate(&c->ev0) != cudaSuccess || cudaEventCreate(&c->ev1) != cudaSuccess) {
        delete c;
        return HZB_ECUDA;
    }
    *out = c;
    return HZB_OK;
}

hzb_status hzb_destroy(hzb_ctx *c)
{
    if (!c) return HZB_EINVAL;
    cudaSetDevice(c->opt.device);
    g_fail_alloc = false;
    // the caller's stream may already be gone: wait for the whole device instead
    cudaDeviceSynchronize();
    release_compression(c);
    for (ShapeDev *s : c->shapes) {
        s->ring.release(); s->body_offs.release(); s->A64.release(); s->S64.release(); s->S32.release();
        s->Sdd.release();
        s->Aimg.release();
        delete s;
    }
    c->pos64.release(); c->nrm64.release(); c->pos32.release(); c->nrm32.release(); c->body_of.release();
    c->tblocks.release(); c->body_xf.release(); c->w_a.release(); c->w_b.release(); c->w_c.release();
    c->w_d.release(); c->f_a.release(); c->f_b.release(); c->yhat64.release(); c->that64.release();
    c->yhat32.release(); c->that32.release(); c->s_b.release(); c->s_r.release(); c->s_d.release();
    c->io_in.release(); c->io_out.release(); c->io_small.release(); c->tiny.release(); c->sol.release();
    c->red.release(); c->krylov.release(); c->small.release();
    c->sctab.release(); c->nb_part64.release(); c->nb_part32.release(); c->sig32.release(); c->blockpairs.release(); c->kerr.release(); c->Ximg.release();
    c->dfa.release(); c->dfb.release(); c->dfc.release(); c->dftab.release(); c->nodecheck.release();
    c->dfltab.release();
    if (c->host_pinned) cudaFreeHost(c->host_pinned);
    release_graphs(c);
    for (cudaEvent_t e : c->evpool) cudaEventDestroy(e);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    delete c;
    cudaGetLastError();
    return HZB_OK;
}

const char *hzb_last_error(const hzb_ctx *c) { return c ? c->err.c_str() : "null context"; }

hzb_status hzb_set_stream(hzb_ctx *c, void *stream)
{
    if (!c) return HZB_EINVAL;
    c->stream = (cudaStream_t)stream;
    c->opt.cuda_stream = stream;
    return HZB_OK;
}

hzb_status hzb_set_options(hzb_ctx *c, const hzb_options *o)
{
    if (!c) return HZB_EINVAL;
    if (!valid_options(o) || o->device != c->opt.device) return fail(c, HZB_EINVAL, "invalid options");
    c->opt = *o;
    c->stream = (cudaStream_t)o->cuda_stream;
    return HZB_OK;
}

hzb_status hzb_set_wave(hzb_ctx *c, double k, double eta)
{
    if (!c) return HZB_EINVAL;
    if (c->state > 1) return fail(c, HZB_ESTATE, "hzb_set_wave must precede hzb_add_body");
    if (!(k >= 0.0) || !std::isfinite(k) || !std::isfinite(eta)) return fail(c, HZB_EINVAL, "k must be >= 0");
    c->k = k;
    c->eta = eta;
    c->state = 1;
    return HZB_OK;
}

static bool same_shape(const hzb_shape &a, const hzb_shape &b)
{
    if (a.kind != b.kind || a.n_panels != b.n_panels || a.gl_order != b.gl_order || a.n_modes != b.n_modes) return false;
    for (int q = 0; q < 4; ++q)
        if (a.p[q] != b.p[q]) return false;
    return true;
}

static hzb_status add_body_impl(hzb_ctx *c, const hzb_shape *shape, const std::vector<double> &curve,
                                const double cen[3], const double rot[9], int *body_id);

hzb_status hzb_add_body(hzb_ctx *c, const hzb_shape *shape, const double cen[3], const double rot[9], int *body_id)
{
    if (!c) return HZB_EINVAL;
    if (shape && shape->kind == HZB_CURVE_SPLINE) return fail(c, HZB_EINVAL, "spline curves go through hzb_add_body_curve");
    return add_body_impl(c, shape, std::vector<double>(), cen, rot, body_id);
}

hzb_status hzb_add_body_curve(hzb_ctx *c, const double *rz, int n_points, int gl_order, int n_modes,
                              const double cen[3], const double rot[9], int *body_id)
{
    if (!c) return HZB_EINVAL;
    if (!rz || n_points < 3 || n_points > 4097) return fail(c, HZB_EINVAL, "curve needs 3..4097 points");
    hzb_shape sh;
    std::memset(&sh, 0, sizeof(sh));
    sh.kind = HZB_CURVE_SPLINE;
    sh.n_panels = n_points - 1;
    sh.gl_order = gl_order;
    sh.n_modes = n_modes;
    return add_body_impl(c, &sh, std::vector<double>(rz, rz + 2 * (size_t)n_points), cen, rot, body_id);
}

static hzb_status add_body_impl(hzb_ctx *c, const hzb_shape *shape, const std::vector<double> &curve,
                                const double cen[3], const double rot[9], int *body_id)
{
    if (c->state < 1 || c->state > 2) return fail(c, HZB_ESTATE, "hzb_add_body needs hzb_set_wave and no build yet");
    if (!shape || !cen || !rot) return fail(c, HZB_EINVAL, "null argument");
    for (int q = 0; q < 3; ++q)
        if (!std::isfinite(cen[q])) return fail(c, HZB_EINVAL, "non-finite centre");
    // rot must be orthonormal with det +1
    double R[9];
    std::memcpy(R, rot, sizeof(R));
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double s = 0;
            for (int q = 0; q < 3; ++q) s += R[3 * q + a] * R[3 * q + b];
            if (std::fabs(s - (a == b ? 1.0 : 0.0)) > 1e-9) return fail(c, HZB_EINVAL, "rotation is not orthonormal");
        }
    double det = R[0] * (R[4] * R[8] - R[5] * R[7]) - R[1] * (R[3] * R[8] - R[5] * R[6]) + R[2] * (R[3] * R[7] - R[4] * R[6]);
    if (det < 0) return fail(c, HZB_EINVAL, "rotation has determinant -1");
    int sidx = -1;
    for (size_t s = 0; s < c->shapes.size(); ++s)
        if (same_shape(c->shapes[s]->geom.spec, *shape) && c->shapes[s]->geom.curve_rz == curve) sidx = (int)s;
    if (sidx < 0) {
        ShapeDev *sd = new (std::nothrow) ShapeDev();
        if (!sd) return HZB_ENOMEM;
        std::string err;
        if (!build_shape_geometry(*shape, curve, sd->geom, err)) {
            delete sd;
            return fail(c, HZB_EINVAL, err);
        }
        c->shapes.push_back(sd);
        sidx = (int)c->shapes.size() - 1;
    }
    ShapeDev &sd = *c->shapes[sidx];
    long long n = (long long)sd.geom.NG * sd.geom.NF;
    if (c->N + n > (long long)0x7fffffff) return fail(c, HZB_EINVAL, "too many nodes");
    BodyRec b;
    b.shape = sidx;
    std::memcpy(b.c, cen, sizeof(b.c));
    std::memcpy(b.rot, rot, sizeof(b.rot));
    b.offset = c->N;
    b.n_nodes = (int)n;
    b.index_in_shape = (int)sd.bodies.size();
    sd.bodies.push_back((int)c->bodies.size());
    c->bodies.push_back(b);
    c->N += n;
    c->state = 2;
    if (body_id) *body_id = (int)c->bodies.size() - 1;
    return HZB_OK;
}

hzb_status hzb_num_nodes(const hzb_ctx *c, long long *n)
{
    if (!c || !n) return HZB_EINVAL;
    *n = c->N;
    return HZB_OK;
}

hzb_status hzb_get_nodes(hzb_ctx *c, double *xyz, double *nrm, double *w)
{
    HZB_GUARD(c);
    if (c->state < 2) return fail(c, HZB_ESTATE, "no bodies");
    hzb_status st = make_nodes(c);
    if (st) return st;
    std::vector<double4> p((size_t)c->N), q((size_t)c->N);
    if (check_cuda(c, cudaMemcpyAsync(p.data(), c->pos64.ptr, c->N * sizeof(double4), cudaMemcpyDeviceToHost, c->stream), "copy") ||
        check_cuda(c, cudaMemcpyAsync(q.data(), c->nrm64.ptr, c->N * sizeof(double4), cudaMemcpyDeviceToHost, c->stream), "copy") ||
        check_cuda(c, cudaStreamSynchronize(c->stream), "copy"))
        return HZB_ECUDA;
    for (long long i = 0; i < c->N; ++i) {
        if (xyz) { xyz[3 * i] = p[i].x; xyz[3 * i + 1] = p[i].y; xyz[3 * i + 2] = p[i].z; }
        if (nrm) { nrm[3 * i] = q[i].x; nrm[3 * i + 1] = q[i].y; nrm[3 * i + 2] = q[i].z; }
        if (w) w[i] = p[i].w;
    }
    return HZB_OK;
}

hzb_status hzb_build_scattering_matrices(hzb_ctx *c)
{
    HZB_GUARD(c);
    if (c->state != 2) return fail(c, HZB_ESTATE, "hzb_build_scattering_matrices needs bodies and no earlier build");
    hzb_status st = make_nodes(c);
    if (st) return st;
    cudaEventRecord(c->ev0, c->stream);
    for (ShapeDev *s : c->shapes)
        if ((st = build_shape_matrices(c, *s))) return st;
    cudaEventRecord(c->ev1, c->stream);
    if (check_cuda(c, cudaEventSynchronize(c->ev1), "setup")) return HZB_ECUDA;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    c->t_setup_ms = ms;
    c->state = 3;
    return HZB_OK;
}

hzb_status hzb_get_modal_block(hzb_ctx *c, int body, int p, int which, double *out)
{
    HZB_GUARD(c);
    if (c->state != 3) return fail(c, HZB_ESTATE, "scattering matrices not built");
    if (body < 0 || body >= (int)c->bodies.size() || !out || (which != 0 && which != 1))
        return fail(c, HZB_EINVAL, "bad body, mode selector or output");
    ShapeDev &sd = *c->shapes[c->bodies[body].shape];
    if (p < 0 || p > sd.geom.M) return fail(c, HZB_EINVAL, "mode out of range");
    size_t blk = (size_t)sd.geom.NG * sd.geom.NG;
    const double2 *src = (which ? sd.S64.ptr : sd.A64.ptr) + (size_t)p * blk;
    if (check_cuda(c, cudaMemcpyAsync(out, src, blk * sizeof(double2), cudaMemcpyDeviceToHost, c->stream), "copy") ||
        check_cuda(c, cudaStreamSynchronize(c->stream), "copy"))
        return HZB_ECUDA;
    return HZB_OK;
}

// Stage an N x R complex input: device pointers pass through, host ones are copied.
static hzb_status stage_in(hzb_ctx *c, DevBuf<double2> &buf, const double *src, size_t n, int on_device,
                           const double2 **dst)
{
    if (on_device) {
        *dst = (const double2 *)src;
        return HZB_OK;
    }
    if (check_cuda(c, buf.ensure(n), "alloc staging")) return HZB_ENOMEM;
    if (check_cuda(c, cudaMemcpyAsync(buf.ptr, src, n * sizeof(double2), cudaMemcpyHostToDevice, c->stream), "copy in"))
        return HZB_ECUDA;
    *dst = buf.ptr;
    return HZB_OK;
}

static hzb_status finish_out(hzb_ctx *c, const double2 *dev, double *dst, size_t n, int on_device)
{
    if (on_device) return HZB_OK;
    if (check_cuda(c, cudaMemcpyAsync(dst, dev, n * sizeof(double2), cudaMemcpyDeviceToHost, c->stream), "copy out") ||
        check_cuda(c, cudaStreamSynchronize(c->stream), "sync"))
        return HZB_ECUDA;
    return HZB_OK;
}

static hzb_status check_apply_args(hzb_ctx *c, int R, const void *a, const void *b, int precision, bool need_build)
{
    if (c->state < 2) return fail(c, HZB_ESTATE, "no bodies");
    if (need_build && c->state != 3) return fail(c, HZB_ESTATE, "scattering matrices not built");
    if (R < 1 || R > 4096 || !a || !b) return fail(c, HZB_EINVAL, "bad R or null pointer");
    if (precision != HZB_PREC_FP64 && precision != HZB_PREC_MIXED_FP32 && precision != HZB_PREC_DOUBLE_FLOAT)
        return fail(c, HZB_EINVAL, "bad precision");
    return HZB_OK;
}

hzb_status hzb_interbody(hzb_ctx *c, int R, const double *sigma, double *y, int on_device, int precision)
{
    HZB_GUARD(c);
    hzb_status st = check_apply_args(c, R, sigma, y, precision, false);
    if (st) return st;
    if ((st = make_nodes(c))) return st;
    size_t n = (size_t)c->N * R;
    const double2 *s;
    if ((st = stage_in(c, c->io_in, sigma, n, on_device, &s))) return st;
    double2 *out = (double2 *)y;
    if (!on_device) {
        if (check_cuda(c, c->io_out.ensure(n), "alloc")) return HZB_ENOMEM;
        out = c->io_out.ptr;
    }
    st = (precision == HZB_PREC_FP64) ? interbody64(c, R, s, out)
         : (precision == HZB_PREC_DOUBLE_FLOAT) ? interbody_df(c, R, s, out) : interbody32(c, R, s, out);
    if (st) return st;
    return finish_out(c, out, y, n, on_device);
}

hzb_status hzb_interbody_bodies(hzb_ctx *c, int R, const double *sigma, int body_begin, int body_end, double *y,
                                int on_device, int precision)
{
    HZB_GUARD(c);
    hzb_status st = check_apply_args(c, R, sigma, y, precision, false);
    if (st) return st;
    if (precision == HZB_PREC_DOUBLE_FLOAT) return fail(c, HZB_EINVAL, "body-range sums run in FP64 or FP32");
    if (body_begin < 0 || body_end > (int)c->bodies.size() || body_begin >= body_end)
        return fail(c, HZB_EINVAL, "body range out of bounds or empty");
    if ((st = make_nodes(c))) return st;
    const size_t n = (size_t)c->N * R;
    const double2 *s;
    if ((st = stage_in(c, c->io_in, sigma, n, on_device, &s))) return st;
    if (check_cuda(c, c->w_c.ensure(n), "alloc")) return HZB_ENOMEM;
    const long long r0 = c->bodies[body_begin].offset;
    const long long r1 = c->bodies[body_end - 1].offset + c->bodies[body_end - 1].n_nodes;
    // the one-directional kernels over the TargetBlocks of the range only
    c->tblock_off = c->body_block0[body_begin];
    c->tune_limit_blocks = c->body_block0[body_end] - c->body_block0[body_begin];
    if (precision == HZB_PREC_FP64) {
        const int tpt = c->tune64_tpt > 0 ? c->tune64_tpt : 1;
        const int ns = c->tune64_split > 0 ? c->tune64_split : default_nsplit(c, R, tpt);
        st = interbody64_cfg(c, R, s, c->w_c.ptr, tpt, ns);
    } else {
        const int tpt = c->tune32_tpt > 0 ? c->tune32_tpt : 4;
        const int ns = c->tune32_split > 0 ? c->tune32_split : default_nsplit(c, R, tpt);
        st = interbody32_cfg(c, R, s, c->w_c.ptr, tpt, ns, true);
    }
    c->tblock_off = 0;
    c->tune_limit_blocks = 0;
    if (st) return st;
    const size_t nr = (size_t)(r1 - r0) * R;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (check_cuda(c, cudaMemcpyAsync(y, c->w_c.ptr + (size_t)r0 * R, nr * sizeof(double2), kind, c->stream),
                   "copy rows") ||
        check_cuda(c, cudaStreamSynchronize(c->stream), "body-range sum"))
        return HZB_ECUDA;
    return HZB_OK;
}

hzb_status hzb_local_inverse(hzb_ctx *c, int R, const double *y, const double *sigma, double alpha, double beta,
                             double *tau, int on_device, int precision)
{
    HZB_GUARD(c);
    hzb_status st = check_apply_args(c, R, y, tau, precision, true);
    if (st) return st;
    if (alpha != 0.0 && !sigma) return fail(c, HZB_EINVAL, "sigma is required when alpha != 0");
    size_t n = (size_t)c->N * R;
    const double2 *dy, *ds = nullptr;
    if ((st = stage_in(c, c->io_in, y, n, on_device, &dy))) return st;
    if (alpha != 0.0 && (st = stage_in(c, c->s_r, sigma, n, on_device, &ds))) return st;
    double2 *out = (double2 *)tau;
    if (!on_device) {
        if (check_cuda(c, c->io_out.ensure(n), "alloc")) return HZB_ENOMEM;
        out = c->io_out.ptr;
    }
    st = (precision == HZB_PREC_MIXED_FP32)     ? local_inverse32(c, R, dy, ds, alpha, beta, out)
         : (precision == HZB_PREC_DOUBLE_FLOAT) ? local_inverse_dfl(c, R, dy, ds, alpha, beta, out)
                                                : local_inverse64(c, R, dy, ds, alpha, beta, out);
    if (st) return st;
    return finish_out(c, out, tau, n, on_device);
}

hzb_status hzb_apply(hzb_ctx *c, int R, const double *sigma, double *z, int on_device, int precision)
{
    HZB_GUARD(c);
    hzb_status st = check_apply_args(c, R, sigma, z, precision, true);
    if (st) return st;
    size_t n = (size_t)c->N * R;
    const double2 *s;
    if ((st = stage_in(c, c->io_in, sigma, n, on_device, &s))) return st;
    double2 *out = (double2 *)z;
    if (!on_device) {
        if (check_cuda(c, c->io_out.ensure(n), "alloc")) return HZB_ENOMEM;
        out = c->io_out.ptr;
    }
    if ((st = apply_op(c, R, s, out, precision))) return st;
    return finish_out(c, out, z, n, on_device);
}

hzb_status hzb_solve_plane_waves(hzb_ctx *c, int R, const double *dirs, hzb_stats *stats)
{
    HZB_GUARD(c);
    c->prof_on = false;
    if (c->state != 3) return fail(c, HZB_ESTATE, "scattering matrices not built");
    if (R < 1 || R > 4096 || !dirs) return fail(c, HZB_EINVAL, "bad R or directions");
    for (int r = 0; r < R; ++r) {
        double nn = dirs[3 * r] * dirs[3 * r] + dirs[3 * r + 1] * dirs[3 * r + 1] + dirs[3 * r + 2] * dirs[3 * r + 2];
        if (!(std::fabs(nn - 1.0) < 1e-8)) return fail(c, HZB_EINVAL, "directions must be unit vectors");
    }
    size_t n = (size_t)c->N * R;
    if (check_cuda(c, c->io_small.ensure(3 * (size_t)R), "alloc") || check_cuda(c, c->io_in.ensure(n), "alloc"))
        return HZB_ENOMEM;
    if (check_cuda(c, cudaMemcpyAsync(c->io_small.ptr, dirs, 3 * R * sizeof(double), cudaMemcpyHostToDevice, c->stream),
                   "copy dirs"))
        return HZB_ECUDA;
    hzb_status st = plane_waves(c, R, c->io_small.ptr, c->io_in.ptr);
    if (st) return st;
    if (c->accel && c->rctx) return solve_reduced(c, R, c->io_in.ptr, nullptr, stats);
    return solve_driver(c, R, c->io_in.ptr, nullptr, stats);
}

hzb_status hzb_incident_plane_waves(hzb_ctx *c, int R, const double *dirs, double *v, int on_device)
{
    HZB_GUARD(c);
    if (c->state < 2) return fail(c, HZB_ESTATE, "no bodies");
    if (R < 1 || R > 4096 || !dirs || !v) return fail(c, HZB_EINVAL, "bad R or null pointer");
    for (int r = 0; r < R; ++r) {
        double nn = dirs[3 * r] * dirs[3 * r] + dirs[3 * r + 1] * dirs[3 * r + 1] + dirs[3 * r + 2] * dirs[3 * r + 2];
        if (!(std::fabs(nn - 1.0) < 1e-8)) return fail(c, HZB_EINVAL, "directions must be unit vectors");
    }
    hzb_status st = make_nodes(c);
    if (st) return st;
    const size_t n = (size_t)c->N * R;
    if (check_cuda(c, c->io_small.ensure(3 * (size_t)R), "alloc")) return HZB_ENOMEM;
    double2 *out = (double2 *)v;
    if (!on_device) {
        if (check_cuda(c, c->io_out.ensure(n), "alloc")) return HZB_ENOMEM;
        out = c->io_out.ptr;
    }
    if (check_cuda(c, cudaMemcpyAsync(c->io_small.ptr, dirs, 3 * R * sizeof(double), cudaMemcpyHostToDevice, c->stream),
                   "copy dirs"))
        return HZB_ECUDA;
    if ((st = plane_waves(c, R, c->io_small.ptr, out))) return st;
    if (!on_device) return finish_out(c, out, v, n, 0);
    return check_cuda(c, cudaStreamSynchronize(c->stream), "plane waves");
}

hzb_status hzb_solve_data(hzb_ctx *c, int R, const double *v, const double *x0, int on_device, hzb_stats *stats)
{
    HZB_GUARD(c);
    c->prof_on = false;
    if (c->state != 3) return fail(c, HZB_ESTATE, "scattering matrices not built");
    if (R < 1 || R > 4096 || !v) return fail(c, HZB_EINVAL, "bad R or data");
    size_t n = (size_t)c->N * R;
    const double2 *dv, *dx0 = nullptr;
    hzb_status st;
    if ((st = stage_in(c, c->io_in, v, n, on_device, &dv))) return st;
    if (x0 && (st = stage_in(c, c->io_out, x0, n, on_device, &dx0))) return st;
    if (c->accel && c->rctx) return solve_reduced(c, R, dv, dx0, stats);
    return solve_driver(c, R, dv, dx0, stats);
}

hzb_status hzb_get_density(hzb_ctx *c, double *sigma, int on_device)
{
    HZB_GUARD(c);
    if (!sigma) return fail(c, HZB_EINVAL, "null output");
    if (c->sol_R <= 0) return fail(c, HZB_ESTATE, "no solve yet");
    size_t n = (size_t)c->N * c->sol_R;
    cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (check_cuda(c, cudaMemcpyAsync(sigma, c->sol.ptr, n * sizeof(double2), kind, c->stream), "copy density") ||
        check_cuda(c, cudaStreamSynchronize(c->stream), "sync"))
        return HZB_ECUDA;
    return HZB_OK;
}

static hzb_status point_query(hzb_ctx *c, int n, const double *pts, double *out, bool far)
{
    HZB_GUARD(c);
    if (c->sol_R <= 0) return fail(c, HZB_ESTATE, "no solve yet");
    if (n < 1 || n > (1 << 20) || !pts || !out) return fail(c, HZB_EINVAL, "bad point count or null pointer");
    int R = c->sol_R;
    size_t no = (size_t)n * R;
    if (check_cuda(c, c->io_small.ensure(3 * (size_t)n), "alloc") || check_cuda(c, c->io_out.ensure(no), "alloc"))
        return HZB_ENOMEM;
    if (check_cuda(c, cudaMemcpyAsync(c->io_small.ptr, pts, 3 * n * sizeof(double), cudaMemcpyHostToDevice, c->stream), "copy"))
        return HZB_ECUDA;
    hzb_status st = far ? far_field64(c, R, c->sol.ptr, n, c->io_small.ptr, c->io_out.ptr)
                        : field_points64(c, R, c->sol.ptr, n, c->io_small.ptr, c->io_out.ptr);
    if (st) return st;
    return finish_out(c, c->io_out.ptr, out, no, 0);
}

hzb_status hzb_autotune(hzb_ctx *c, int R, int which, double best_ms[2])
{
    HZB_GUARD(c);
    if (c->state < 2) return fail(c, HZB_ESTATE, "no bodies");
    if (R < 1 || R > 4096 || which < 1 || which > 3) return fail(c, HZB_EINVAL, "bad R or selector");
    return autotune(c, R, which, best_ms);
}

hzb_status hzb_tuned_config(const hzb_ctx *c, int R, int out[6])
{
    if (!c || !out) return HZB_EINVAL;
    // the FP32 engine interbody32 takes for R right-hand sides
    int e = -1;
    if (c->nbody_engine == 1) e = 1;
    else if (c->nbody_engine == 5 || c->nbody_engine == 6) e = 2;
    else if (c->nbody_engine < 0) e = (c->tune32_tc >= 0 && c->tune32_tc_R == R) ? c->tune32_tc : (R >= 16 ? 2 : 0);
    int v = (c->tune32_x2 >= 0 && c->tune32_R == R) ? c->tune32_x2 : (R <= 2 ? 2 : 1);
    if (c->nbody_engine >= 2 && c->nbody_engine <= 4) v = c->nbody_engine - 2;
    out[0] = e == 2 ? 4 : (e == 1 ? 3 : v);
    out[1] = c->tune32_tpt;
    out[2] = c->tune32_split;
    out[3] = (c->nbody64_engine >= 1 || (c->nbody64_engine < 0 && R <= 4)) ? 1 : 0;
    out[4] = c->tune64_tpt;
    out[5] = c->tune64_split;
    return HZB_OK;
}

hzb_status hzb_set_execution(hzb_ctx *c, int check_every, int use_graphs)
{
    if (!c) return HZB_EINVAL;
    if (check_every < 0 || check_every > 64 || use_graphs < -1 || use_graphs > 1)
        return fail(c, HZB_EINVAL, "check_every in [0, 64], use_graphs in {-1, 0, 1}");
    c->check_every = check_every;
    c->use_graphs = use_graphs;
    return HZB_OK;
}

hzb_status hzb_set_modal_engine(hzb_ctx *c, int engine)
{
    if (!c) return HZB_EINVAL;
    if (engine < -1 || engine > 2) return fail(c, HZB_EINVAL, "engine in {-1, 0, 1, 2}");
    c->modal_engine = engine;
    return HZB_OK;
}

hzb_status hzb_set_fp64_interbody_engine(hzb_ctx *c, int engine)
{
    if (!c) return HZB_EINVAL;
    if (engine < -1 || engine > 2) return fail(c, HZB_EINVAL, "engine in {-1, 0, 1, 2}");
    c->nbody64_engine = engine;
    return HZB_OK;
}

hzb_status hzb_set_interbody_engine(hzb_ctx *c, int engine)
{
    if (!c) return HZB_EINVAL;
    if (engine < -1 || engine > 7) return fail(c, HZB_EINVAL, "engine in {-1, 0, ..., 7}");
    c->nbody_engine = engine;
    return HZB_OK;
}

hzb_status hzb_far_field(hzb_ctx *c, int n, const double *xhat, double *out)
{
    return point_query(c, n, xhat, out, true);
}

hzb_status hzb_eval_field(hzb_ctx *c, int n, const double *x, double *out)
{
    return point_query(c, n, x, out, false);
}

}  // extern "C"
