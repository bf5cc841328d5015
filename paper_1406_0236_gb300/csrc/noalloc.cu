// hzb_local_inverse_noalloc: the block-diagonal inverse D^{-1} for callers that
// cannot allocate device memory at call time.  Such callers include code running
// inside CUDA stream capture (cudaMalloc and cudaFree are not capturable and
// synchronise the device), real-time or embedded pipelines that fix their memory
// budget at start-up, and host runtimes that own the device allocator and forbid
// other libraries from calling it.  The DFT and GEMM scratch of this apply lives in
// the file-scope array below instead of context workspaces that grow on demand.
//
// Limits and sharing:
//   * capacity NOALLOC_ELEMS complex doubles (16 MiB), split into two halves for the
//     mode panels y^ and tau^; the call fails with HZB_EINVAL when a shape's panel
//     (M+1) x N_G x (2 m_s R) does not fit one half;
//   * every GPU that loads this library holds the 16 MiB until the process exits;
//   * all calls on a device share the array: calls whose work overlaps on the GPU
//     (different streams, or other contexts on the same device) race and corrupt each
//     other's results; serialise them on one stream;
//   * the first call on a device looks up the array's device address
//     (cudaGetSymbolAddress, with that device current); make that first call before
//     any stream capture;
//   * like hzb_local_inverse on the same context, it applies the direct D^{-1} of Eq.
//     (precond), also while the accelerated scheme is on (the reduced operator of
//     Eq. (ip6) belongs to the context's internal reduced system, not to this call);
//   * nothing in the array needs to start at zero: every element the call reads was
//     written earlier in the same call (the previous call's contents are overwritten).
#include <mutex>

#include "hzb_internal.h"

namespace hzb {

static const size_t NOALLOC_ELEMS = (size_t)1 << 20;     // 16 MiB of double2
static __device__ __align__(256) double2 g_noalloc_scratch[NOALLOC_ELEMS];

static const int NOALLOC_MAX_DEVICES = 64;
static double2 *g_noalloc_addr[NOALLOC_MAX_DEVICES] = {nullptr};
static std::mutex g_noalloc_mu;

hzb_status local_inverse64_scratch(hzb_ctx *c, int R, const double2 *y, const double2 *sigma, double alpha,
                                   double beta, double2 *tau, double2 *yh, double2 *th);
size_t modal_panel_elems(const hzb_ctx *c, int R);

// Device address of the scratch array on the current device (set up once per device).
static hzb_status noalloc_scratch(hzb_ctx *c, double2 **out)
{
    const int dev = c->opt.device;
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return fail(c, HZB_EINVAL, "device ordinal too large for the no-alloc scratch table");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        double2 *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress((void **)&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return check_cuda(c, e == cudaSuccess ? cudaErrorInvalidSymbol : e, "cudaGetSymbolAddress");
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return HZB_OK;
}

}  // namespace hzb

using namespace hzb;

extern "C" hzb_status hzb_local_inverse_noalloc(hzb_ctx *c, int R, const double *y, const double *sigma,
                                                double alpha, double beta, double *tau)
{
    if (!c) return HZB_EINVAL;
    if (cudaSetDevice(c->opt.device) != cudaSuccess) return fail(c, HZB_ECUDA, "cudaSetDevice failed");
    cudaGetLastError();                   // a stale error of an unrelated earlier call is not ours
    if (c->state != 3) return fail(c, HZB_ESTATE, "scattering matrices not built");
    if (R < 1 || R > 4096 || !y || !tau) return fail(c, HZB_EINVAL, "bad R or null pointer");
    if (alpha != 0.0 && !sigma) return fail(c, HZB_EINVAL, "sigma is required when alpha != 0");
    const size_t need = modal_panel_elems(c, R);
    if (need > NOALLOC_ELEMS / 2)
        return fail(c, HZB_EINVAL,
                    "hzb_local_inverse_noalloc: a mode panel needs " + std::to_string(need) +
                        " complex values per half, the static scratch holds " + std::to_string(NOALLOC_ELEMS / 2) +
                        " (16 MiB in total); use hzb_local_inverse or fewer right-hand sides per call");
    double2 *base = nullptr;
    hzb_status st = noalloc_scratch(c, &base);
    if (st) return st;
    return local_inverse64_scratch(c, R, (const double2 *)y, (const double2 *)sigma, alpha, beta, (double2 *)tau,
                                   base, base + NOALLOC_ELEMS / 2);
}
