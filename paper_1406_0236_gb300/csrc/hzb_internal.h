// Internal declarations of the hzb library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/hzb.h"

namespace hzb {

// ---------------------------------------------------------------- geometry (host)

// One smooth piece of a generating curve.  type 0: (a sin t, c cos t);
// type 1: arc of radius R at polar angle th0 + sg * t; type 2: rim semicircle.
struct Piece {
    int type;
    double p[10];
    double t0, t1;
};

struct Panel {
    int piece;
    double ta, tb;
};

// Discretised generating curve of one distinct shape.
struct ShapeGeom {
    hzb_shape spec;
    std::vector<double> curve_rz;         // HZB_CURVE_SPLINE: the n_panels + 1 points (r, z)
    int NG = 0, NF = 0, M = 0;
    std::vector<Piece> pieces;
    std::vector<Panel> panels;
    // per ring node
    std::vector<double> t, r, z, nr, nz, ds, speed;
    std::vector<int> piece_of, panel_of;
    std::vector<double> panel_len;
    // near-panel list: for ring i, near_start[i] .. near_start[i+1]-1 index into near_panel
    std::vector<int> near_start, near_panel;
    std::vector<double> near_tstar;       // closest parameter on that panel
};

bool build_shape_geometry(const hzb_shape &spec, const std::vector<double> &curve_rz, ShapeGeom &g,
                          std::string &err);
void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w);
// evaluate gamma and gamma' of a piece at t
void piece_eval(const Piece &pc, double t, double &r, double &z, double &dr, double &dz);

// ---------------------------------------------------------------- host fault injection

// Faults injected on the host for tests of the error paths (environment variable
// HZB_FAULT, read once by hzb_create: a comma-separated list of the names below).
// No fault touches the GPU's state beyond the context's own buffers and flags.
enum {
    FAULT_ALLOC = 1,     // "alloc": every device allocation of the context fails (HZB_ENOMEM)
    FAULT_GEOM = 2,      // "geom": the first node generation writes a NaN weight (HZB_EINVAL)
    FAULT_NAN = 4,       // "nan": the first solve's preconditioned right-hand side gets a NaN (HZB_ENAN)
    FAULT_TIMEOUT = 8    // "timeout": the first tcgen05 inter-body launch takes its bounded-wait
                         // exit before any MMA is issued (HZB_ETIMEOUT)
};
int parse_fault_spec(const char *spec);
// set by every ABI entry from its context: DevBuf::ensure fails while it is true
extern thread_local bool g_fail_alloc;

// ---------------------------------------------------------------- device buffers

template <typename T>
struct DevBuf {
    T *ptr = nullptr;
    size_t n = 0;
    cudaError_t ensure(size_t count) {
        if (count <= n) return cudaSuccess;
        if (g_fail_alloc) return cudaErrorMemoryAllocation;
        if (ptr) cudaFree(ptr);
        ptr = nullptr;
        n = 0;
        cudaError_t e = cudaMalloc(&ptr, count * sizeof(T) + 256);
        if (e == cudaSuccess) n = count;
        return e;
    }
    void release() {
        if (ptr) cudaFree(ptr);
        ptr = nullptr;
        n = 0;
    }
};

struct ShapeDev {
    ShapeGeom geom;
    std::vector<int> bodies;              // bodies using this shape, in order
    DevBuf<double> ring;                  // NG x 8: r, z, nr, nz, ds, t, (unused)
    DevBuf<long long> body_offs;          // first node of each body of this shape
    DevBuf<double2> A64;                  // (M+1) x NG x NG: A~_p
    DevBuf<double2> S64;                  // (M+1) x NG x NG: S_p = A~_p^{-1}
    DevBuf<float2> S32;                   // FP32 copy of S64
    DevBuf<float4> Sdd;                   // S64 split into double-float (re.hi, re.lo, im.hi, im.lo), on first use
    bool Sdd_ready = false;               // cleared whenever S64 is rewritten
    DevBuf<float> Aimg;                   // embedded, TF32-split S_p for the TMA modal GEMM (modal_tma.cu)
    alignas(64) unsigned char tmA[128];   // its TMA tensor map (CUtensorMap)
    bool tmA_ready = false;
    // accelerated scheme (compress.cu, Sec. 5): the shape's skeleton and reduced blocks
    int skel_k = 0;                       // skeleton size k (0: none)
    double skel_rho = 0.0;                // proxy radius it was computed for (0: given by the caller)
    double skel_eps = 0.0;                // ID tolerance it was computed for (0: given by the caller)
    std::vector<int> skel_J;              // skeleton nodes, shape-local, ascending
    DevBuf<double2> T64;                  // k x n row-major: V_p^* = T
    DevBuf<double2> U64;                  // n x k row-major: U_p = T^T
    DevBuf<float4> Tdf, Udf;              // T and U split into FP32 (hi.re, hi.im, lo.re, lo.im)
    DevBuf<double2> St64;                 // k x k row-major: S_p = T A_pp^{-1} T^T
    DevBuf<float2> St32;                  // its FP32 copy
    DevBuf<long long> red_offs;           // first reduced-system node of each body of the shape
};

struct BodyRec {
    int shape;
    double c[3];
    double rot[9];
    long long offset;   // first node
    int n_nodes;
    int index_in_shape;
};

// CTA work item of the inter-body sum: a contiguous target range inside one body.
struct TargetBlock {
    int start;      // first target node
    int count;      // targets in this block
    int excl_lo;    // source range of the target's own body [excl_lo, excl_hi)
    int excl_hi;
};

}  // namespace hzb

struct hzb_ctx {
    hzb_options opt;
    cudaStream_t stream = nullptr;
    std::string err;
    int state = 0;          // 0 created, 1 wave set, 2 bodies being added, 3 built
    double k = 0.0, eta = 0.0;
    std::vector<hzb::ShapeDev *> shapes;
    std::vector<hzb::BodyRec> bodies;
    long long N = 0;
    bool nodes_ready = false;
    double center[3] = {0, 0, 0};  // origin of the FP32 coordinates
    double t_setup_ms = 0.0;

    // geometry on the device
    hzb::DevBuf<double4> pos64;     // x, y, z, w
    hzb::DevBuf<double4> nrm64;     // nx, ny, nz, 0
    hzb::DevBuf<float4> pos32;      // x - center (FP32), w
    hzb::DevBuf<float4> nrm32;
    hzb::DevBuf<int> body_of;
    hzb::DevBuf<hzb::TargetBlock> tblocks;
    int n_tblocks = 0;
    std::vector<int> body_block0;   // first TargetBlock of each body (and the total at the end)
    int tblock_off = 0;             // one-directional kernels: first TargetBlock launched (body-range sums)
    hzb::DevBuf<double> body_xf;    // per body: c[3], rot[9]

    // workspaces
    hzb::DevBuf<double2> w_a, w_b, w_c, w_d;   // N x R
    hzb::DevBuf<float2> f_a, f_b;              // N x R (FP32)
    hzb::DevBuf<double2> yhat64;               // modal workspace FP64
    hzb::DevBuf<double2> that64;
    hzb::DevBuf<float2> yhat32, that32;
    hzb::DevBuf<double2> s_b, s_r, s_d;        // solve: right-hand side, residual, correction
    hzb::DevBuf<double2> io_in, io_out;        // staging of host inputs and outputs
    hzb::DevBuf<double> io_small;              // staging of directions and points
    hzb::DevBuf<double2> tiny;                 // residual norms
    hzb::DevBuf<double2> sol;                  // densities of the last solve, N x R
    int sol_R = 0;
    hzb::DevBuf<double> red;                   // reduction scratch
    hzb::DevBuf<double2> krylov;               // (m+1) x N x R
    hzb::DevBuf<double2> small;                // Hessenberg etc.
    double *host_pinned = nullptr;             // small pinned host buffer
    size_t host_pinned_n = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    long long interbody_calls = 0;
    long long launches = 0;                    // kernels launched (all wrappers)
    // inter-body kernels: FP64 cos/sin table, split partial sums, launch shape
    hzb::DevBuf<double2> sctab;
    hzb::DevBuf<double2> nb_part64;
    hzb::DevBuf<float2> nb_part32;
    hzb::DevBuf<int2> blockpairs;              // unordered TargetBlock pairs on different bodies (nbody_sym.cu)
    long long n_blockpairs = 0;                // 0: not built, -1: none (one body)
    int nbody64_engine = -1;                   // FP64/double-float sums: -1 auto (pair-symmetric for R <= 4),
                                               // 0 one-directional, 1 pair-symmetric (double-float: lean forms),
                                               // 2 as -1 with the normalised double-float kernels
    hzb::DevBuf<int> kerr;                     // device error flag of kernels with bounded waits
    hzb::DevBuf<float> Ximg;                   // embedded, TF32-split modal panel (TMA modal GEMM)
    bool kerr_ready = false;
    hzb::DevBuf<float2> sig32;                 // w_j sigma_j / (4 pi) in FP32, N x R (FP32 inter-body kernels)
    int tune64_tpt = 0, tune64_split = 0;      // 0: default
    int tune32_tpt = 0, tune32_split = 0;
    int tune32_R = 0;                          // R the FP32 variant was tuned for
    int tune32_x2 = -1;                        // FP32 CUDA-core kernel: -1 default (packed), 0 scalar, 1 packed,
                                               // 2 pair-symmetric packed
    int tune_limit_blocks = 0;                 // autotuner: time only the first blocks (0 = all)
    // double-float inter-body kernel: split positions/normals, cos/sin table, launch shape
    hzb::DevBuf<float4> dfa, dfb, dfc, dftab;
    bool df_ready = false;
    hzb::DevBuf<float4> dfltab;                // lean double-float kernel: cos/sin(2 pi m / 1024)
    bool dfltab_ready = false;
    int tunedf_tpt = 0, tunedf_split = 0;
    // GMRES execution: steps between host checks (0 = auto) and CUDA graphs (-1 auto, 0 off, 1 on)
    int check_every = 0;
    int use_graphs = -1;
    int modal_engine = -1;                     // FP32 modal GEMM: -1 auto, 0 CUDA cores, 1 tensor cores
    int nbody_engine = -1;                     // FP32 inter-body sum: -1 auto, 0 CUDA cores, 1 tensor cores,
                                               // 2 CUDA cores scalar kernel, 3 CUDA cores packed-pair kernel,
                                               // 4 CUDA cores pair-symmetric packed kernel,
                                               // 5 tensor cores with tcgen05 (TMEM accumulators),
                                               // 6 tcgen05, warp-specialised pipeline
    int tunetc_split = 0;                      // tensor-core inter-body source split (0: default)
    int tune32_tc = -1, tune32_tc_R = 0;       // autotuner's engine choice for R = tune32_tc_R (-1: none)
    std::vector<cudaGraphExec_t> gexec;        // captured Arnoldi step j
    std::vector<long long> glaunch;            // kernels per captured step
    unsigned char gkey[256];
    bool gkey_valid = false;
    bool capturing = false;
    bool in_solve = false;                     // inside solve_driver: error flags are read at its end
    // accelerated scheme (compress.cu): the reduced system of Eq. (ip6) as a context of its
    // own over the skeleton nodes; its local operator is the dense S_p of each body
    hzb_ctx *rctx = nullptr;
    bool reduced = false;                      // this context is a reduced system
    bool accel = false;                        // solves go through the reduced system
    double t_compress_ms = 0.0;
    struct RShape {
        int k, ms;
        const double2 *S64;
        const float2 *S32;
        const long long *offs;                 // first reduced node of each body of the shape
    };
    std::vector<RShape> rshapes;               // reduced context: one per shape
    hzb::DevBuf<double2> rb, rx;               // reduced right-hand side and guess (parent)
    hzb::DevBuf<float4> ysplit;                // a vector split into FP32 hi/lo (double-float GEMV)
    hzb::DevBuf<long long> zero_off;           // {0}: one body at offset 0
    // device timing of the inter-body kernels during a solve: event pairs
    std::vector<cudaEvent_t> evpool;
    std::vector<int> evkind;                   // 0: FP64, 1: FP32, per recorded pair
    bool prof_on = false;
    // host fault injection (FAULT_* bits from HZB_FAULT) and the one-shot faults already fired
    int fault = 0;
    int fault_spent = 0;
    hzb::DevBuf<int> nodecheck;                // node validation: [bad count, first bad node]
};

// Entry of every ABI call: valid context, its device current, the context's injected
// allocation fault (if any) armed, and no stale (non-sticky) error of an unrelated
// earlier runtime call left for this call's checks to report.
#define HZB_GUARD(c)                                                     \
    do {                                                                 \
        if (!(c)) return HZB_EINVAL;                                     \
        if (cudaSetDevice((c)->opt.device) != cudaSuccess)               \
            return hzb::fail((c), HZB_ECUDA, "cudaSetDevice failed");    \
        hzb::g_fail_alloc = ((c)->fault & hzb::FAULT_ALLOC) != 0;        \
        cudaGetLastError();                                              \
    } while (0)

// ---------------------------------------------------------------- kernels' host entry points
namespace hzb {

hzb_status fail(hzb_ctx *c, hzb_status s, const std::string &msg);
// event pair around one inter-body launch (no-op unless a solve is profiling)
int prof_begin(hzb_ctx *c, int kind);
void prof_end(hzb_ctx *c, int slot);
hzb_status check_cuda(hzb_ctx *c, cudaError_t e, const char *what);

// setup.cu
hzb_status make_nodes(hzb_ctx *c);
hzb_status build_shape_matrices(hzb_ctx *c, ShapeDev &s);

// nbody.cu: y = B sigma; sigma, y device N x R complex FP64 (FP32 path converts internally)
hzb_status interbody64(hzb_ctx *c, int R, const double2 *sigma, double2 *y);
hzb_status interbody32(hzb_ctx *c, int R, const double2 *sigma, double2 *y);
hzb_status interbody_df(hzb_ctx *c, int R, const double2 *sigma, double2 *y);   // nbody_df.cu
hzb_status interbody_dfl_sym(hzb_ctx *c, int R, const double2 *sigma, double2 *y);   // nbody_dfl.cu
hzb_status interbody_dfl(hzb_ctx *c, int R, const double2 *sigma, double2 *y, int nsplit);   // nbody_dfl.cu
int dfl_default_nsplit(hzb_ctx *c, int R);                                                  // nbody_dfl.cu
hzb_status interbody_tc(hzb_ctx *c, int R, const double2 *sigma, double2 *y, int nsplit);
hzb_status modal_gemm_tma(hzb_ctx *c, ShapeDev &sd, int ncols, const float2 *X, float2 *Cout);  // modal_tma.cu
enum { T5_SPLIT3 = 0, T5_WS = 1, T5_SINGLE = 2 };   // forms of the tcgen05 inter-body kernel
hzb_status interbody_tc5(hzb_ctx *c, int R, const double2 *sigma, double2 *y, int nsplit,
                         int mode);  // nbody_tc5.cu
const float2 *weighted_sigma32(hzb_ctx *c, int R, const double2 *sigma);      // nbody.cu; nullptr on failure
hzb_status ensure_sctab(hzb_ctx *c);                                          // nbody.cu: FP64 cos/sin table
hzb_status interbody64_sym(hzb_ctx *c, int R, const double2 *sigma, double2 *y);  // nbody_sym.cu
hzb_status interbody32_sym(hzb_ctx *c, int R, const double2 *sigma, double2 *y, int tp);  // nbody_sym.cu
hzb_status ensure_block_pairs(hzb_ctx *c);                                    // nbody_sym.cu  // nbody_tc.cu
void split_reduce_f2(hzb_ctx *c, size_t n, int nsplit, const float2 *part, double2 *y);
hzb_status interbody64_cfg(hzb_ctx *c, int R, const double2 *sigma, double2 *y, int tpt, int nsplit);
hzb_status interbody32_cfg(hzb_ctx *c, int R, const double2 *sigma, double2 *y, int tpt, int nsplit, bool x2);
int default_nsplit(hzb_ctx *c, int R, int tpt);
hzb_status autotune(hzb_ctx *c, int R, int which, double *best_ms);
// field at external points (no exclusion): out T x R (device), pts T x 3 (device)
hzb_status field_points64(hzb_ctx *c, int R, const double2 *sigma, int T, const double *pts,
                          double2 *out);

// modal.cu: tau = alpha sigma + beta D^{-1} y
hzb_status local_inverse64(hzb_ctx *c, int R, const double2 *y, const double2 *sigma,
                           double alpha, double beta, double2 *tau);
hzb_status local_inverse32(hzb_ctx *c, int R, const double2 *y, const double2 *sigma,
                           double alpha, double beta, double2 *tau);
// the same in double-float on the FP32 pipe (modal_dfl.cu), for the refinement residual
hzb_status local_inverse_dfl(hzb_ctx *c, int R, const double2 *y, const double2 *sigma, double alpha, double beta,
                             double2 *tau);

// krylov.cu
hzb_status apply_op(hzb_ctx *c, int R, const double2 *x, double2 *z, int precision);
hzb_status gmres_solve(hzb_ctx *c, int R, const double2 *b, double2 *x, int x_is_zero,
                       int precision, double tol, int maxit, int restart,
                       int *iters, double *relres, int *converged);
// b_given: the preconditioned right-hand side itself (then v is not read)
hzb_status solve_driver(hzb_ctx *c, int R, const double2 *v, const double2 *x0, hzb_stats *st,
                        const double2 *b_given = nullptr);
void release_graphs(hzb_ctx *c);

// modal.cu: Y = A_pp^{-1} X for one body of the shape, X and Y n x R (node-major)
hzb_status shape_inverse64(hzb_ctx *c, ShapeDev &sd, int R, const double2 *X, double2 *Y);

// compress.cu: the reduced system's local operator tau = alpha sigma + beta S y
hzb_status reduced_local(hzb_ctx *c, int R, const double2 *y, const double2 *sigma, double alpha,
                         double beta, double2 *tau, bool fp32);
hzb_status solve_reduced(hzb_ctx *c, int R, const double2 *v, const double2 *x0, hzb_stats *st);
void release_compression(hzb_ctx *c);
// install J (distinct, any order) and T (device, k x n, rows in J's order) for a shape; its
// S_p from S_host (k x k, rows and columns in ascending J order) or computed when NULL
hzb_status install_skeleton(hzb_ctx *c, ShapeDev &sd, const std::vector<int> &J, DevBuf<double2> &T,
                            const double2 *S_host = nullptr);
hzb_status build_reduced(hzb_ctx *c);
// whether a proxy sphere of radius rho encloses every body of the shape and excludes the others
bool proxy_fits(const hzb_ctx *c, int shape, double rho);

// fields.cu
hzb_status plane_waves(hzb_ctx *c, int R, const double *dirs_dev, double2 *v);
hzb_status far_field64(hzb_ctx *c, int R, const double2 *sigma, int n, const double *xhat_dev,
                       double2 *out);

// small device helpers
hzb_status vec_copy(hzb_ctx *c, double2 *dst, const double2 *src, size_t n);
hzb_status vec_zero(hzb_ctx *c, double2 *dst, size_t n);

}  // namespace hzb
