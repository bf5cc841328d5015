// Saving and loading the per-shape modal matrices A~_p and S_p = A~_p^{-1} (Sec. 3.2:
// computed once per distinct body shape and reusable for any arrangement of bodies of
// that shape at the same wavenumber), so that a later context skips the setup.
//
// File layout (little-endian, as the host writes it):
//   char magic[8] = "HZBSCAT1"; int32 version = 3; int32 n_shapes;
//   double k, eta;
//   per shape: hzb_shape spec (the struct as laid out by this library, padding zeroed),
//              int32 NG, int32 M, int32 n_curve, n_curve doubles (the spline curve's
//              (r, z) points, none for the analytic shapes), then (M+1) NG NG complex
//              doubles of A~_p, then the same of S_p, p = 0..M, each matrix row-major
//              (row = target ring);
//   then per shape the skeleton of the accelerated scheme (Sec. 5): int32 k (0: none),
//              double rho (the proxy radius it was computed for, 0 if given by the
//              caller), double eps (the ID tolerance, 0 if given by the caller); for a
//              caller's skeleton int32 m and the m bodies of the shape it was set for
//              (centre, rotation: 12 doubles each); if k > 0: k int32 skeleton nodes
//              (ascending), k n complex doubles of T (row-major), k k complex doubles of
//              the reduced S_p.
// Version 2 files (no skeleton section) and version 3 files (no eps, no arrangement)
// load too.  A computed skeleton loads only where its proxy sphere still separates the
// bodies of the new arrangement, a caller's skeleton only into the arrangement it was
// set for (it carries no proxy sphere that would validate another); when every shape
// has one, the reduced system is built and solves use it.  hzb_get_skeleton_info
// reports the restored skeleton's eps.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "hzb_internal.h"

namespace hzb {

static const char HZB_SCAT_MAGIC[8] = {'H', 'Z', 'B', 'S', 'C', 'A', 'T', '1'};

__global__ void to_fp32_copy_kernel(size_t n, const double2 *a, float2 *b)
{
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) b[e] = make_float2((float)a[e].x, (float)a[e].y);
}

// field by field: the struct's padding bytes are not part of the shape
static bool same_shape(const hzb_shape &a, const hzb_shape &b)
{
    if (a.kind != b.kind || a.n_panels != b.n_panels || a.gl_order != b.gl_order || a.n_modes != b.n_modes) return false;
    for (int q = 0; q < 4; ++q)
        if (a.p[q] != b.p[q]) return false;
    return true;
}

}  // namespace hzb

using namespace hzb;

extern "C" hzb_status hzb_save_scattering(hzb_ctx *c, const char *path)
{
    if (!path) return HZB_EINVAL;
    HZB_GUARD(c);
    if (c->state != 3) return fail(c, HZB_ESTATE, "scattering matrices not built");
    FILE *f = std::fopen(path, "wb");
    if (!f) return fail(c, HZB_EINVAL, std::string("cannot open for writing: ") + path);
    bool ok = true;
    const int version = 4, ns = (int)c->shapes.size();
    ok &= std::fwrite(HZB_SCAT_MAGIC, 1, 8, f) == 8;
    ok &= std::fwrite(&version, sizeof(int), 1, f) == 1;
    ok &= std::fwrite(&ns, sizeof(int), 1, f) == 1;
    ok &= std::fwrite(&c->k, sizeof(double), 1, f) == 1;
    ok &= std::fwrite(&c->eta, sizeof(double), 1, f) == 1;
    std::vector<double2> host;
    for (int s = 0; s < ns && ok; ++s) {
        const ShapeDev &sd = *c->shapes[s];
        const int NG = sd.geom.NG, M = sd.geom.M;
        hzb_shape spec;
        std::memset(&spec, 0, sizeof(spec));
        spec.kind = sd.geom.spec.kind;
        for (int q = 0; q < 4; ++q) spec.p[q] = sd.geom.spec.p[q];
        spec.n_panels = sd.geom.spec.n_panels;
        spec.gl_order = sd.geom.spec.gl_order;
        spec.n_modes = sd.geom.spec.n_modes;
        ok &= std::fwrite(&spec, sizeof(hzb_shape), 1, f) == 1;
        ok &= std::fwrite(&NG, sizeof(int), 1, f) == 1;
        ok &= std::fwrite(&M, sizeof(int), 1, f) == 1;
        const int ncv = (int)sd.geom.curve_rz.size();
        ok &= std::fwrite(&ncv, sizeof(int), 1, f) == 1;
        if (ncv > 0) ok &= std::fwrite(sd.geom.curve_rz.data(), sizeof(double), ncv, f) == (size_t)ncv;
        const size_t nmat = (size_t)(M + 1) * NG * NG;
        host.resize(nmat);
        for (const DevBuf<double2> *b : {&sd.A64, &sd.S64}) {
            if (check_cuda(c, cudaMemcpyAsync(host.data(), b->ptr, nmat * sizeof(double2), cudaMemcpyDeviceToHost,
                                              c->stream), "copy matrices") ||
                check_cuda(c, cudaStreamSynchronize(c->stream), "copy matrices")) {
                std::fclose(f);
                return HZB_ECUDA;
            }
            ok &= std::fwrite(host.data(), sizeof(double2), nmat, f) == nmat;
        }
    }
    for (int s = 0; s < ns && ok; ++s) {
        const ShapeDev &sd = *c->shapes[s];
        const int k = sd.skel_k, n = sd.geom.NG * sd.geom.NF;
        ok &= std::fwrite(&k, sizeof(int), 1, f) == 1;
        ok &= std::fwrite(&sd.skel_rho, sizeof(double), 1, f) == 1;
        ok &= std::fwrite(&sd.skel_eps, sizeof(double), 1, f) == 1;
        if (sd.skel_rho == 0.0) {                          // the arrangement a caller's skeleton is for
            const int m = (int)sd.bodies.size();
            ok &= std::fwrite(&m, sizeof(int), 1, f) == 1;
            for (int b : sd.bodies) {
                ok &= std::fwrite(c->bodies[b].c, sizeof(double), 3, f) == 3;
                ok &= std::fwrite(c->bodies[b].rot, sizeof(double), 9, f) == 9;
            }
        }
        if (k == 0 || !ok) continue;
        ok &= std::fwrite(sd.skel_J.data(), sizeof(int), k, f) == (size_t)k;
        const size_t nt = (size_t)k * n, ns2 = (size_t)k * k;
        host.resize(std::max(nt, ns2));
        for (int which = 0; which < 2 && ok; ++which) {
            const size_t cnt = which ? ns2 : nt;
            const double2 *src = which ? sd.St64.ptr : sd.T64.ptr;
            if (check_cuda(c, cudaMemcpyAsync(host.data(), src, cnt * sizeof(double2), cudaMemcpyDeviceToHost,
                                              c->stream), "copy skeleton") ||
                check_cuda(c, cudaStreamSynchronize(c->stream), "copy skeleton")) {
                std::fclose(f);
                return HZB_ECUDA;
            }
            ok &= std::fwrite(host.data(), sizeof(double2), cnt, f) == cnt;
        }
    }
    ok &= std::fclose(f) == 0;
    if (!ok) return fail(c, HZB_EINVAL, std::string("write failed: ") + path);
    return HZB_OK;
}

extern "C" hzb_status hzb_load_scattering(hzb_ctx *c, const char *path)
{
    if (!path) return HZB_EINVAL;
    HZB_GUARD(c);
    if (c->state != 2) return fail(c, HZB_ESTATE, "hzb_load_scattering needs bodies and no earlier build");
    FILE *f = std::fopen(path, "rb");
    if (!f) return fail(c, HZB_EINVAL, std::string("cannot open: ") + path);
    char magic[8];
    int version = 0, ns = 0;
    double k = 0.0, eta = 0.0;
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, HZB_SCAT_MAGIC, 8) == 0;
    ok = ok && std::fread(&version, sizeof(int), 1, f) == 1 && version >= 2 && version <= 4;
    ok = ok && std::fread(&ns, sizeof(int), 1, f) == 1 && std::fread(&k, sizeof(double), 1, f) == 1 &&
         std::fread(&eta, sizeof(double), 1, f) == 1;
    if (!ok) {
        std::fclose(f);
        return fail(c, HZB_EINVAL, "not a scattering-matrix file of this version");
    }
    if (k != c->k || eta != c->eta || ns != (int)c->shapes.size()) {
        std::fclose(f);
        return fail(c, HZB_EINVAL, "file was written for another wavenumber, coupling or set of shapes");
    }
    std::vector<double2> host;
    for (int s = 0; s < ns; ++s) {
        ShapeDev &sd = *c->shapes[s];
        hzb_shape spec;
        int NG = 0, M = 0;
        int ncv = 0;
        ok = std::fread(&spec, sizeof(hzb_shape), 1, f) == 1 && std::fread(&NG, sizeof(int), 1, f) == 1 &&
             std::fread(&M, sizeof(int), 1, f) == 1 && std::fread(&ncv, sizeof(int), 1, f) == 1 && ncv >= 0 &&
             ncv <= 2 * 4097;
        std::vector<double> curve(ok ? ncv : 0);
        if (ok && ncv > 0) ok = std::fread(curve.data(), sizeof(double), ncv, f) == (size_t)ncv;
        if (!ok || !same_shape(spec, sd.geom.spec) || NG != sd.geom.NG || M != sd.geom.M || curve != sd.geom.curve_rz) {
            std::fclose(f);
            return fail(c, HZB_EINVAL, "shape " + std::to_string(s) + " differs from the file's");
        }
        const size_t nmat = (size_t)(M + 1) * NG * NG;
        if (check_cuda(c, sd.A64.ensure(nmat), "alloc A") || check_cuda(c, sd.S64.ensure(nmat), "alloc S") ||
            check_cuda(c, sd.S32.ensure(nmat), "alloc S32")) {
            std::fclose(f);
            return HZB_ENOMEM;
        }
        host.resize(nmat);
        for (DevBuf<double2> *b : {&sd.A64, &sd.S64}) {
            if (std::fread(host.data(), sizeof(double2), nmat, f) != nmat) {
                std::fclose(f);
                return fail(c, HZB_EINVAL, "file ends early");
            }
            if (check_cuda(c, cudaMemcpyAsync(b->ptr, host.data(), nmat * sizeof(double2), cudaMemcpyHostToDevice,
                                              c->stream), "upload matrices") ||
                check_cuda(c, cudaStreamSynchronize(c->stream), "upload matrices")) {
                std::fclose(f);
                return HZB_ECUDA;
            }
        }
        to_fp32_copy_kernel<<<(unsigned)((nmat + 255) / 256), 256, 0, c->stream>>>(nmat, sd.S64.ptr, sd.S32.ptr);
        sd.tmA_ready = false;
        sd.Sdd_ready = false;
        if (check_cuda(c, cudaGetLastError(), "to_fp32_copy_kernel")) {
            std::fclose(f);
            return HZB_ECUDA;
        }
    }
    hzb_status st = make_nodes(c);
    if (st) {
        std::fclose(f);
        return st;
    }
    if (check_cuda(c, cudaStreamSynchronize(c->stream), "load")) {
        std::fclose(f);
        return HZB_ECUDA;
    }
    c->t_setup_ms = 0.0;
    c->state = 3;
    if (version >= 3) {
        // skeletons: each is restored where its proxy sphere still fits the arrangement, a
        // caller's skeleton only into the arrangement it was set for
        bool all = true;
        for (int s = 0; s < ns; ++s) {
            ShapeDev &sd = *c->shapes[s];
            const int n = sd.geom.NG * sd.geom.NF;
            int k = 0;
            double rho = 0.0, eps = 0.0;
            bool same_arrangement = true;
            if (std::fread(&k, sizeof(int), 1, f) != 1 || std::fread(&rho, sizeof(double), 1, f) != 1 || k < 0 ||
                k > n || (version >= 4 && std::fread(&eps, sizeof(double), 1, f) != 1)) {
                std::fclose(f);
                release_compression(c);
                return fail(c, HZB_EINVAL, "file ends early or holds a bad skeleton size");
            }
            if (version >= 4 && rho == 0.0) {
                int m = 0;
                if (std::fread(&m, sizeof(int), 1, f) != 1 || m < 0 || m > (1 << 20)) {
                    std::fclose(f);
                    release_compression(c);
                    return fail(c, HZB_EINVAL, "file ends early or holds a bad body count");
                }
                same_arrangement = m == (int)sd.bodies.size();
                for (int q = 0; q < m; ++q) {
                    double xf[12];
                    if (std::fread(xf, sizeof(double), 12, f) != 12) {
                        std::fclose(f);
                        release_compression(c);
                        return fail(c, HZB_EINVAL, "file ends early");
                    }
                    if (same_arrangement) {
                        const BodyRec &b = c->bodies[sd.bodies[q]];
                        same_arrangement = std::memcmp(xf, b.c, 3 * sizeof(double)) == 0 &&
                                           std::memcmp(xf + 3, b.rot, 9 * sizeof(double)) == 0;
                    }
                }
            } else if (version == 3 && rho == 0.0) {
                same_arrangement = false;                  // no record of the arrangement: not restored
            }
            if (k == 0) {
                all = false;
                continue;
            }
            std::vector<int> J(k);
            std::vector<double2> T((size_t)k * n), S((size_t)k * k);
            if (std::fread(J.data(), sizeof(int), k, f) != (size_t)k ||
                std::fread(T.data(), sizeof(double2), T.size(), f) != T.size() ||
                std::fread(S.data(), sizeof(double2), S.size(), f) != S.size()) {
                std::fclose(f);
                release_compression(c);
                return fail(c, HZB_EINVAL, "file ends early");
            }
            bool valid = std::is_sorted(J.begin(), J.end()) && J.front() >= 0 && J.back() < n &&
                         std::adjacent_find(J.begin(), J.end()) == J.end();
            if (!valid) {
                std::fclose(f);
                release_compression(c);
                return fail(c, HZB_EINVAL, "bad skeleton indices in the file");
            }
            if ((rho > 0.0 && !proxy_fits(c, s, rho)) || (rho == 0.0 && !same_arrangement)) {
                all = false;
                continue;
            }
            DevBuf<double2> Td;
            if (check_cuda(c, Td.ensure(T.size()), "alloc T")) {
                std::fclose(f);
                return HZB_ENOMEM;
            }
            st = check_cuda(c, cudaMemcpyAsync(Td.ptr, T.data(), T.size() * sizeof(double2), cudaMemcpyHostToDevice,
                                               c->stream), "upload T");
            if (!st) st = install_skeleton(c, sd, J, Td, S.data());
            Td.release();
            if (st) {
                std::fclose(f);
                release_compression(c);
                return st;
            }
            sd.skel_rho = rho;
            sd.skel_eps = eps;
        }
        if (all) {
            if ((st = build_reduced(c))) {
                std::fclose(f);
                release_compression(c);
                return st;
            }
            c->accel = true;
        }
    }
    std::fclose(f);
    return HZB_OK;
}
