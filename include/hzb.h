/*
 * hzb.h — C ABI of the GB300 (sm_103a) multibody axisymmetric Helmholtz solver.
 *
 * Method: Hao, Martinsson, Young, "An efficient and highly accurate solver for
 * multi-body acoustic scattering problems involving rotationally symmetric
 * scatterers".  A sound-soft scattering problem (Sec. 2, Eq. (basic)) on m
 * rotationally symmetric bodies is written as the combined-field BIE (Eq.
 * (intHelm2))
 *       1/2 sigma(x) + int_Gamma K(x,y) sigma(y) dA(y) = -v(x),
 *       K(x,y) = d phi(x,y)/d n(y) - i eta phi(x,y),  phi = e^{ik|x-y|}/(4 pi |x-y|)
 * (eta is a signed real coupling; the paper's Eq. (Gkappa) is eta = -k).  Each body
 * is discretised by Gauss-Legendre panels on its generating curve times an
 * equispaced azimuthal rule (Sec. 3.2); its diagonal block is inverted once per
 * azimuthal Fourier mode (Eqs. (FAF), (singleinverse)); GMRES then solves the
 * block-diagonally preconditioned system (Sec. 4, Eq. (precond))
 *       sigma + D^{-1} B sigma = -D^{-1} v,
 * where B holds the inter-body interactions K(x_i, x_j) w_j (Eq. (nystromnaive)).
 *
 * Conventions used by every call:
 *   - Complex numbers are interleaved (re, im) doubles.
 *   - Nodes are ordered body-major (order of hzb_add_body), then ring i along the
 *     generating curve (from its first end), then azimuth l fastest; N is the
 *     total node count.  A block of R vectors is stored node-major with the R
 *     values of one node contiguous ("N x R").
 *   - Host pointers are read or written before the call returns; the library
 *     keeps no reference to them.  Device pointers (flag *_on_device = 1) must be
 *     device memory of the context's GPU, and are accessed in stream order on the
 *     context's stream.
 *   - Every call returns an hzb_status; on failure hzb_last_error() describes it.
 *   - The context owns all device memory it allocates; hzb_destroy frees it.
 *   - A context is used by one host thread at a time.
 *   - Order: hzb_create -> hzb_set_wave -> hzb_add_body* ->
 *     hzb_build_scattering_matrices -> solves/applies/fields (any number).
 *     Calls out of order return HZB_ESTATE.
 */
#ifndef HZB_H
#define HZB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hzb_ctx hzb_ctx;

typedef enum {
    HZB_OK = 0,
    HZB_EINVAL = -1,     /* bad argument (null pointer, even N_F, size out of range ...) */
    HZB_ENOMEM = -2,     /* device or host allocation failed */
    HZB_ECUDA = -3,      /* a CUDA runtime call failed */
    HZB_ENOCONV = -4,    /* GMRES reached maxit; best iterate is stored */
    HZB_ENAN = -5,       /* NaN or Inf met in a residual */
    HZB_ETIMEOUT = -6,   /* a bounded device wait gave up */
    HZB_ESTATE = -7      /* call out of order */
} hzb_status;

/* Failure detection.  GMRES reports a non-finite residual as HZB_ENAN (a NaN or Inf in
 * the data, the guess or the operator), and non-convergence as HZB_ENOCONV.  Every
 * wait of a kernel on an mbarrier is bounded: when one runs out the kernel frees its
 * tensor memory, writes NaN to its outputs and sets a flag that the call reports as
 * HZB_ETIMEOUT (the flag is then cleared, so the context stays usable); inside a solve
 * the flag is read once, at the end of the solve (no synchronisation per launch), unless
 * the NaN outputs stopped GMRES first (HZB_ENAN).  Geometry is
 * checked when the nodes are generated: intersecting bodies and non-finite or
 * degenerate nodes give HZB_EINVAL.
 *
 * Host fault injection, for tests of these paths: the environment variable HZB_FAULT,
 * read by hzb_create, is a comma-separated list of
 *   alloc    every device allocation of the context fails (HZB_ENOMEM);
 *   geom     the first node generation writes a NaN weight (HZB_EINVAL);
 *   nan      the first solve's preconditioned right-hand side gets a NaN (HZB_ENAN);
 *   timeout  the first tcgen05 inter-body launch (FP32 engine 5) finds its error flag
 *            set before it starts and takes its timeout exit before issuing any MMA
 *            (HZB_ETIMEOUT).
 * The last three fire once per context.  Nothing is injected on the GPU itself. */

typedef enum {
    HZB_PREC_FP64 = 0,        /* every kernel in FP64 */
    HZB_PREC_MIXED_FP32 = 1,  /* FP64 outer refinement, FP32 inter-body sum and modal apply inside */
    HZB_PREC_DOUBLE_FLOAT = 2 /* inter-body sum in double-float (two FP32 numbers, ~48-bit
                                 significand, ~1e-13 relative per term) on the FP32 pipe;
                                 valid for hzb_interbody/hzb_apply and as the refinement residual */
} hzb_precision;

typedef enum {
    HZB_SPHERE = 0,
    HZB_SPHEROID = 1,
    HZB_OPEN_SHELL = 2,
    HZB_CURVE_SPLINE = 3   /* generating curve given by points: added with hzb_add_body_curve */
} hzb_shape_kind;

typedef struct {
    int device;            /* CUDA device ordinal */
    void *cuda_stream;     /* cudaStream_t to launch on; NULL = the legacy default stream.  The
                              stream must stay valid while the context uses it (change it with
                              hzb_set_stream before destroying it) */
    int precision;         /* hzb_precision */
    double gmres_tol;      /* relative residual of the preconditioned system */
    int restart;           /* GMRES restart length (<= 0: no restart, up to maxit) */
    int maxit;             /* total GMRES iterations (inner iterations in mixed mode) */
    double inner_tol;      /* mixed mode: relative tolerance of each inner FP32 solve; with a
                              guess x0, the first inner solve stops at inner_tol * |b| (absolute)
                              instead, since it starts from the FP32 operator's residual */
    int max_outer;         /* mixed mode: maximum refinement steps */
    int verify_final;      /* mixed mode: 1 (default) = stop only on a computed FP64 residual;
                              0 = after an FP64 residual r_k, stop once the bound
                              rel_k * max(c_1, inner_tol) * 10 <= gmres_tol holds for the next
                              correction (c_1: contraction observed in the first refinement
                              step; from a guess, the first step's residual rel_1 itself),
                              saving the last FP64 apply */
    int residual;          /* mixed mode: precision of the refinement residual (its inter-body
                              sum and D^{-1}, and b = -D^{-1} v), HZB_PREC_FP64 (default) or
                              HZB_PREC_DOUBLE_FLOAT */
} hzb_options;

typedef struct {
    int kind;              /* hzb_shape_kind (HZB_CURVE_SPLINE bodies: hzb_add_body_curve) */
    double p[4];           /* SPHERE: (a); SPHEROID: (a, c) semi-axes (a,a,c);
                              OPEN_SHELL: (R_out, R_in, opening half-angle [rad],
                              rim radius = (R_out - R_in)/2), opening centred on body -z */
    int n_panels;          /* Gauss-Legendre panels on the generating curve */
    int gl_order;          /* nodes per panel, 2..32 */
    int n_modes;           /* N_F, odd, 3..1023: azimuthal nodes = Fourier modes -M..M */
} hzb_shape;

typedef struct {
    int iterations;          /* GMRES iterations (FP64 path) or total inner iterations (mixed) */
    int outer_iterations;    /* refinement steps (mixed), 1 for the FP64 path */
    int converged;           /* 1 if every right-hand side met the tolerance */
    double rel_residual;     /* max over right-hand sides of the final ||b - A x|| / ||b|| */
    double t_solve_ms;       /* device time of the solve (CUDA events) */
    double t_setup_ms;       /* device time of hzb_build_scattering_matrices */
    long long interbody_applies;  /* inter-body sums launched during the solve */
    double t_nbody64_ms;     /* summed device time of the FP64 inter-body kernel (CUDA events) */
    double t_nbody32_ms;     /* summed device time of the FP32 inter-body kernel */
    long long n_nbody64;     /* its launches during the solve */
    long long n_nbody32;
    long long kernel_launches;    /* kernels of this library launched during the solve */
    double t_nbodydf_ms;     /* summed device time of the double-float inter-body kernel */
    long long n_nbodydf;
} hzb_stats;

/* Fill *o with defaults: device 0, default stream, FP64, tol 1e-10, no restart,
 * maxit 500, inner_tol 1e-5, max_outer 10. */
void hzb_default_options(hzb_options *o);

/* Create a context on options->device.  Allocates nothing on the device yet.
 * Errors: HZB_EINVAL (null), HZB_ECUDA (device unavailable). */
hzb_status hzb_create(const hzb_options *options, hzb_ctx **out);
hzb_status hzb_destroy(hzb_ctx *ctx);
const char *hzb_last_error(const hzb_ctx *ctx);
const char *hzb_status_string(hzb_status s);

/* Change the stream later calls launch on. */
hzb_status hzb_set_stream(hzb_ctx *ctx, void *cuda_stream);
/* Change precision, tolerances and limits after creation. */
hzb_status hzb_set_options(hzb_ctx *ctx, const hzb_options *options);

/* Wavenumber k >= 0 and signed coupling eta (Sec. 2, Eq. (Gkappa) with +i k
 * replaced by -i eta).  Must precede hzb_add_body. */
hzb_status hzb_set_wave(hzb_ctx *ctx, double k, double eta);

/* Add body number *body_id (0, 1, ...): shape in its own frame (symmetry axis =
 * body z), centre c[3], rotation rot[9] row-major whose columns are the body x, y,
 * z axes in world coordinates (x_world = c + rot * x_body).  Azimuth theta_l =
 * 2 pi l / N_F is measured from the body x axis.  Bodies with identical hzb_shape
 * share one set of scattering matrices (the remark on repeated shapes in Sec. 6). */
hzb_status hzb_add_body(hzb_ctx *ctx, const hzb_shape *shape, const double c[3],
                        const double rot[9], int *body_id);

/* Add a body whose generating curve (Sec. 3.2) is the cubic spline through n_points
 * points rz[2k] = r_k >= 0, rz[2k+1] = z_k in the body frame, listed from the top pole
 * (r_0 = 0) down to the bottom pole (r_{n-1} = 0, z_{n-1} < z_0), with r_k > 0 between:
 * parameter = cumulative chord length t; r(t) with r'' = 0 and z(t) with z' = 0 at both
 * poles (so the surface closes smoothly on the axis); one Gauss-Legendre panel of
 * gl_order nodes per spline segment (n_points - 1 panels); n_modes as for hzb_add_body;
 * c, rot and body_id as for hzb_add_body.  Bodies with the same points, gl_order and
 * n_modes share their scattering matrices.  Errors: HZB_EINVAL (fewer than 3 or more
 * than 4097 points, ends off the axis, coincident points, r <= 0 inside, wrong
 * direction, bad rotation), HZB_ESTATE as hzb_add_body. */
hzb_status hzb_add_body_curve(hzb_ctx *ctx, const double *rz, int n_points, int gl_order, int n_modes,
                              const double c[3], const double rot[9], int *body_id);

/* Total node count N (valid after the last hzb_add_body). */
hzb_status hzb_num_nodes(const hzb_ctx *ctx, long long *n);

/* Copy the surface rule to host arrays: xyz N x 3, normals N x 3 (outward unit),
 * weights N (w = w_GL |gamma'| r 2 pi / N_F, Sec. 3.2).  Any pointer may be NULL.
 * Forces node generation (device) if it has not happened yet. */
hzb_status hzb_get_nodes(hzb_ctx *ctx, double *xyz, double *normals, double *weights);

/* Setup, once: per distinct shape the modal kernels, the near-panel product
 * integration, A~_p = 1/2 I + K_p and S_p = A~_p^{-1} for p = 0..M, all in FP64
 * on the device (Sec. 3.2, Remark on the cost of precomputation). */
hzb_status hzb_build_scattering_matrices(hzb_ctx *ctx);

/* Write the FP64 modal matrices A~_p and S_p (p = 0..M) of every distinct shape, with
 * k, eta and the shapes, to the file `path` (Sec. 3.2: the precomputation depends on
 * the shape and the wavenumber only, not on where the bodies sit), and each shape's
 * skeleton of the accelerated scheme when it has one (J, T, the reduced S_p and the
 * proxy radius; Sec. 5: the ID is local to the shape).  Needs a built context.  The
 * format is this library's own (magic "HZBSCAT1", version 4, host byte order): each
 * skeleton is stored with its ID tolerance and proxy radius, and a skeleton the caller
 * set (hzb_set_skeleton) with the arrangement of its shape's bodies.
 * Errors: HZB_ESTATE (not built), HZB_EINVAL (cannot write), HZB_ECUDA. */
hzb_status hzb_save_scattering(hzb_ctx *ctx, const char *path);

/* Instead of hzb_build_scattering_matrices: read the matrices written by
 * hzb_save_scattering for the same k, eta and the same list of distinct shapes (in
 * the order of their first hzb_add_body), then proceed as after a build.  The bodies'
 * positions and rotations may differ from the saving context's.  Saved skeletons
 * are restored where their proxy sphere still encloses every body of the shape and
 * excludes all others, caller-given skeletons only when the shape's bodies sit where they
 * sat when the file was written (hzb_get_skeleton_info reports each restored skeleton's
 * eps); when every shape has one, the acceleration is on as after hzb_compress.
 * Version 2 files (no skeletons) and version 3 files load too.
 * Errors: HZB_ESTATE (no bodies, or already built), HZB_EINVAL (unreadable file, other
 * version, or a k / eta / shape mismatch: nothing is loaded), HZB_ENOMEM, HZB_ECUDA. */
hzb_status hzb_load_scattering(hzb_ctx *ctx, const char *path);

/* Autotuner of the inter-body kernels' launch shape (targets per thread, source
 * chunks per target block) for R right-hand sides: times each candidate with CUDA
 * events on the context's stream and keeps the fastest for later calls.
 * which: bit 0 = FP32 kernel, bit 1 = FP64 kernel.  For the FP32 sum with R >= 8 and
 * the engine on automatic (hzb_set_interbody_engine -1) the tensor-core contractions
 * (mma.sync and tcgen05) are timed as well and, for this R, the fastest engine is kept.  best_ms (may be NULL):
 * the fastest time per launch [FP32, FP64].  Not part of the paper: a GB300 tuning aid. */
hzb_status hzb_autotune(hzb_ctx *ctx, int R, int which, double best_ms[2]);

/* The inter-body kernels the context will launch for R right-hand sides (host only,
 * no GPU work), written to out[6]: [0] FP32 kernel: 0 scalar, 1 packed pairs,
 * 2 pair-symmetric packed, 3 tensor cores (mma.sync), 4 tensor cores (tcgen05); [1] its targets (or packed target pairs)
 * per thread, 0 = default; [2] its source chunks, 0 = default; [3] FP64 kernel:
 * 0 one-directional, 1 pair-symmetric; [4], [5] the one-directional FP64 kernel's
 * targets per thread and source chunks (0 = default).  HZB_EINVAL on NULL. */
hzb_status hzb_tuned_config(const hzb_ctx *ctx, int R, int out[6]);

/* GMRES execution controls (no effect on results beyond rounding of where a
 * converged right-hand side stops):
 *   check_every: Arnoldi steps issued between host reads of the residual estimates
 *                (0 = auto: 4 when N x R <= 1e6 and N^2 x R < 4e9, else 1, since a
 *                chunk's steps after convergence each cost one apply); a right-hand side that
 *                converges inside a chunk is frozen on the device, so later steps of
 *                the chunk change nothing for it;
 *   use_graphs:  capture each Arnoldi step j (operator apply, CGS2, Givens) once as a
 *                CUDA graph and replay it in later iterations and solves (-1 auto:
 *                on when N x R <= 4e6; needs a non-default stream). */
hzb_status hzb_set_execution(hzb_ctx *ctx, int check_every, int use_graphs);

/* Engine of the FP32 per-mode scattering GEMM (Eq. (singleinverse) step (2)):
 * 0 = CUDA cores; 1 = tensor cores through mma.sync, TF32 with a three-term hi/lo split
 * and FP32 accumulation (about FP32 accuracy); 2 = the same contraction on tcgen05 with
 * the operands streamed by TMA (embedded, split S_p images built once per shape: about
 * 32 N_G^2 (M+1) bytes; accumulators in tensor memory drained into FP32 registers every
 * 64 of the K = 2 N_G terms); -1 (default) = 2 when a shape's panel has at least 32
 * columns (2 x bodies of the shape x right-hand sides), else 0.  Returns HZB_EINVAL for
 * other values. */
hzb_status hzb_set_modal_engine(hzb_ctx *ctx, int engine);

/* Engine of the FP32 inter-body sum (Sec. 3.3): 0 = CUDA cores (one pair kernel per
 * target-source pair, complex multiply-accumulate per right-hand side; the kernel
 * variant the autotuner picked, else the packed-pair one); 1 = tensor cores: pair
 * kernels generated on the CUDA cores, the contraction with the densities of up to 32
 * right-hand sides on the tensor cores (TF32, three-term split, FP32 accumulation);
 * 2 = CUDA cores, scalar FP32 kernel; 3 = CUDA cores, packed-pair kernel (two sources
 * per f32x2 instruction); 4 = CUDA cores, pair-symmetric packed kernel (each unordered
 * node pair evaluated once for both directions, results added with FP64 atomics: equal
 * to rounding between runs, not bit for bit); 5 = tensor cores through tcgen05 (TF32
 * three-term split, accumulators in tensor memory, 16 or 32 right-hand sides per CTA);
 * 6 = the same contraction as a warp-specialised pipeline (producer, MMA and epilogue
 * warps synchronised by mbarriers, two operand stages, two accumulators);
 * 7 = engine 5 with single-term TF32 products (no hi/lo split: about 3e-4 relative
 * error in the sum instead of ~3e-6, about 1.4x faster; only ever chosen here, never by
 * the default or the autotuner, for inner solves whose refinement absorbs it);
 * -1 (default) = tcgen05 tensor cores when R >= 16, else as 0, unless hzb_autotune
 * timed the engines for this R.  Returns HZB_EINVAL for other values. */
hzb_status hzb_set_interbody_engine(hzb_ctx *ctx, int engine);

/* Engine of the FP64 and double-float inter-body sums (Sec. 3.3): 0 = one-directional
 * kernels (each ordered pair on its own, source chunks added in a fixed order:
 * bit-reproducible); 1 = pair-symmetric kernels: each unordered pair of nodes on
 * different bodies is evaluated once for both directions (r, 1/r and e^{ikr} are
 * shared), about 1.5x fewer operations; both directions are added into y with FP64
 * atomics, so runs agree to rounding but not bit for bit; -1 (default) = 1 for R <= 4
 * right-hand sides, 0 above (the one-directional kernels amortise the pair geometry over
 * up to 8 right-hand sides per CTA); 2 = pair-symmetric, with the double-float sum in its
 * earlier form (every double-float operation renormalised; the FP64 sum as for 1).  The
 * pair-symmetric double-float sum of engine 1 leaves its products and sums unnormalised
 * and takes e^{ikr} from a 1024-entry table (about 1.7x fewer FP32 operations).  Returns
 * HZB_EINVAL for other values.  Not part of the paper: a GB300 choice (FP64 runs at
 * 1/64 of the FP32 rate). */
hzb_status hzb_set_fp64_interbody_engine(hzb_ctx *ctx, int engine);

/* Measured throughput of one arithmetic pipe of the context's GPU, the denominators of
 * the kernels' rooflines (not part of the paper): kind 0 = FP32 fused multiply-add
 * (TFLOP/s, FMA = 2), 1 = the same with packed f32x2 instructions, 2 = FP64 fused
 * multiply-add (TFLOP/s), 3 = transcendental unit (T operations/s: one rsqrt, sin and
 * cos per round), 4 = TF32 tensor cores through tcgen05.mma (dense TFLOP/s, M = 128,
 * N = 256, operands resident in shared memory).  Each runs for tens of milliseconds on
 * every SM, timed with CUDA events on the context's stream.  Errors: HZB_EINVAL (kind
 * or null value), HZB_ETIMEOUT (a tensor-core wait ran out), HZB_ECUDA. */
hzb_status hzb_measure_peak(hzb_ctx *ctx, int kind, double *value);

/* Copy A~_p (which = 0) or S_p (which = 1) of the shape of body `body`, mode p in
 * 0..M, to host out (N_G x N_G complex, row-major). */
hzb_status hzb_get_modal_block(hzb_ctx *ctx, int body, int p, int which, double *out);

/* y = B sigma (inter-body sum only, Sec. 3.3).  sigma and y: N x R complex.
 * precision: hzb_precision of the kernel used (FP64 or FP32 with FP64 in/out). */
hzb_status hzb_interbody(hzb_ctx *ctx, int R, const double *sigma, double *y,
                         int on_device, int precision);

/* Rows of y = B sigma (Sec. 3.3) for the targets of bodies [body_begin, body_end) only,
 * against all sources: sigma is the full N x R block, y receives the rows of those
 * bodies (n_rows x R, in node order).  The rank-local inter-body sum of a solve whose
 * bodies are partitioned over several GPUs (each rank owns a contiguous body range and
 * all-gathers sigma before this call).  precision: HZB_PREC_FP64 or HZB_PREC_MIXED_FP32
 * (one-directional kernels).  Errors: HZB_EINVAL (empty or out-of-range body range,
 * double-float precision), HZB_ESTATE (no bodies). */
hzb_status hzb_interbody_bodies(hzb_ctx *ctx, int R, const double *sigma, int body_begin, int body_end, double *y,
                                int on_device, int precision);

/* tau = alpha * sigma + beta * D^{-1} y (the per-body FFT -> S_p -> inverse FFT of
 * the Remark after Eq. (precond)).  sigma may be NULL when alpha = 0.  Always the
 * direct D^{-1} on all N nodes, also while the accelerated scheme is on.  precision:
 * HZB_PREC_FP64, HZB_PREC_MIXED_FP32 (DFTs and GEMMs in FP32) or HZB_PREC_DOUBLE_FLOAT
 * (DFTs and GEMMs in double-float on the FP32 pipe, about 1e-13 relative; the first
 * such call after a build splits the scattering matrices into a cached copy). */
hzb_status hzb_local_inverse(hzb_ctx *ctx, int R, const double *y, const double *sigma,
                             double alpha, double beta, double *tau, int on_device,
                             int precision);

/* The same FP64 D^{-1} apply as hzb_local_inverse (device pointers, N x R complex),
 * for callers that cannot allocate device memory when they call: code inside CUDA
 * stream capture (allocation is not capturable), real-time or embedded pipelines
 * with a memory budget fixed at start-up, runtimes that own the device allocator.
 * It allocates nothing: its scratch is a static 16 MiB device array of the library
 * (held by every GPU that loads it until exit), so a call fails with HZB_EINVAL when
 * a shape's mode panel (M+1) x N_G x (2 m_s R) exceeds 524,288 complex values.  All
 * calls on a device share that array: calls that overlap on the GPU race.  The first
 * call on a device looks up the array's address; make it before any stream capture.
 * Like hzb_local_inverse, it applies the direct D^{-1}, also while the accelerated
 * scheme is on.  The paper has no counterpart of this entry point. */
hzb_status hzb_local_inverse_noalloc(hzb_ctx *ctx, int R, const double *y, const double *sigma,
                                     double alpha, double beta, double *tau);

/* z = sigma + D^{-1} B sigma, the preconditioned operator of Eq. (precond). */
hzb_status hzb_apply(hzb_ctx *ctx, int R, const double *sigma, double *z, int on_device,
                     int precision);

/* Solve for R incident plane waves v = exp(i k d.x), dirs R x 3 unit vectors (host).
 * The densities stay in the context (hzb_get_density).  Returns HZB_ENOCONV if
 * some right-hand side missed the tolerance (best iterate kept). */
hzb_status hzb_solve_plane_waves(hzb_ctx *ctx, int R, const double *dirs, hzb_stats *stats);

/* The incident plane waves v = exp(i k d.x) at the nodes (Eq. (basic)) for R unit
 * directions dirs (host, R x 3), written to v (N x R complex, host or device per the
 * flag): the data hzb_solve_plane_waves solves for, for callers that pass it to
 * hzb_solve_data with a guess.  Errors: HZB_EINVAL (non-unit direction), HZB_ESTATE. */
hzb_status hzb_incident_plane_waves(hzb_ctx *ctx, int R, const double *dirs, double *v, int on_device);

/* Solve for R general Dirichlet data sets: v is N x R complex (u = -v on Gamma).
 * x0 (N x R complex, may be NULL) is an initial guess in the same memory space. */
hzb_status hzb_solve_data(hzb_ctx *ctx, int R, const double *v, const double *x0,
                          int on_device, hzb_stats *stats);

/* Copy the densities of the last solve (N x R complex) to sigma. */
hzb_status hzb_get_density(hzb_ctx *ctx, double *sigma, int on_device);

/* Far-field pattern u_inf(xhat) = (1/4pi) sum_j w_j e^{-ik xhat.x_j}
 * (-ik xhat.n_j - i eta) sigma_j of the last solve's densities, for n unit
 * directions xhat (host, n x 3); out: n x R complex (host). */
hzb_status hzb_far_field(hzb_ctx *ctx, int n, const double *xhat, double *out);

/* Scattered field u(x) = sum_j w_j K(x, x_j) sigma_j at n exterior points x (host,
 * n x 3), smooth rule (Eq. (intHelm1)); out: n x R complex (host). */
hzb_status hzb_eval_field(hzb_ctx *ctx, int n, const double *x, double *out);

/* ------------------------------------------------------------------------------
 * Accelerated scheme (Sec. 5, Eqs. (ip0)-(ip6)).  For bodies that are not tightly
 * packed, each shape gets an interpolative decomposition (ID): a skeleton J of k of
 * its n nodes and T (k x n, T(:, J) = I) with V_p^* = T and U_p = T^T, such that every
 * off-diagonal block factors as A_pq ~ U_p A_pq(J_p, J_q) V_q^* (Eq. (ip0)).  GMRES
 * then runs on the reduced system (Eq. (ip6))
 *       sig~ + S B~ sig~ = -v~,  S_p = T A_pp^{-1} T^T,  v~_p = T A_pp^{-1} v_p,
 * whose inter-body sum B~ = B(J, J) is the direct sum over skeleton nodes only, and
 * the density on all nodes follows from Eq. (ip1): sig = D^{-1} (-v - U B~ sig~), so
 * hzb_get_density, hzb_far_field and hzb_eval_field work unchanged.  While the
 * acceleration is on, hzb_solve_plane_waves and hzb_solve_data solve this way in the
 * context's precision (FP64, or mixed: FP32 reduced applies with FP64 refinement);
 * the result differs from the direct solve by about eps times the conditioning.
 * ------------------------------------------------------------------------------ */

/* Compute every shape's ID on the GPU and switch the acceleration on.  The ID is of
 * the proxy matrix [K(z, y_j) w_j ; G(x_i, z) ; dG/dn_z(x_i, z)] (rows: points z of a
 * sphere of radius rho about the body centre, n_theta Gauss-Legendre rings in
 * cos(theta) times the body's N_F azimuths, or for an open shell 3 N_F azimuths in three
 * classes offset by 0, 1/3 and 2/3 of the azimuthal step, which removes the ~1e-6 error
 * floor that N_F azimuths leave on a shell's off-diagonal blocks; each block scaled to
 * unit Frobenius norm);
 * its rank k counts the pivots of a column-pivoted QR with |R_jj| > eps |R_11|.
 *   eps:          tolerance in [0, 1); 0 keeps every column of nonzero pivot
 *   n_theta:      proxy rings, 0 = max(16, ceil(1.2 N_G)), at most 4096
 *   proxy_radius: rho for every shape, or 0 = per shape midway between its largest
 *                 node radius and the nearest other body's bounding sphere
 * Needs hzb_build_scattering_matrices.  HZB_EINVAL if a proxy sphere cannot enclose
 * its body while excluding every other body (bodies too close).  Device memory: about
 * 3 k n complex doubles per shape while it is compressed, then k n + 1.5 k^2. */
hzb_status hzb_compress(hzb_ctx *ctx, double eps, int n_theta, double proxy_radius);

/* Install a skeleton for the shape of `body` (shared by every body of that shape):
 * J holds k distinct node indices of the shape (0..n-1, any order), T the k x n
 * complex matrix row-major with row s belonging to J[s].  Once every shape has one,
 * the reduced system is built and the acceleration switched on. */
hzb_status hzb_set_skeleton(hzb_ctx *ctx, int body, int k, const int *J, const double *T);

/* The skeleton of the shape of `body`: *k (0: none); J (k ints, ascending) and T
 * (k x n complex, row-major, rows in the order of J) are filled when not NULL. */
hzb_status hzb_get_skeleton(hzb_ctx *ctx, int body, int *k, int *J, double *T);

/* The skeleton of the shape of `body`: *k its size (0: none), *eps the ID tolerance and
 * *rho the proxy radius it was computed for (both 0 for a skeleton the caller set);
 * after hzb_load_scattering, the values stored with the restored skeleton.  Any output
 * may be NULL. */
hzb_status hzb_get_skeleton_info(hzb_ctx *ctx, int body, int *k, double *eps, double *rho);

/* on = 1: solves go through the reduced system (HZB_ESTATE without skeletons);
 * on = 0: the direct solve of Eq. (precond). */
hzb_status hzb_set_acceleration(hzb_ctx *ctx, int on);

/* *n = unknowns of the reduced system (sum of k over the bodies), 0 without one. */
hzb_status hzb_reduced_size(const hzb_ctx *ctx, long long *n);

/* out = sig~ + S B~ sig~, the reduced operator of Eq. (ip6), on host arrays of
 * (reduced size) x R complex in the reduced numbering (body by body, each body's
 * skeleton in ascending order); precision: hzb_precision. */
hzb_status hzb_apply_reduced(hzb_ctx *ctx, int R, const double *sig, double *out, int precision);

/* Interpolative decomposition of a rows x cols complex matrix Z (host, column-major)
 * on the GPU: column-pivoted QR stopped at |R_jj| <= eps |R_11|, T = [I, R11^{-1} R12]
 * in the original column order.  Out: *k; J (cols ints; the first k are the skeleton
 * columns in pivot order); T (room for min(rows, cols) x cols complex; k x cols
 * row-major, row s for column J[s], T(:, J) = I). */
hzb_status hzb_interp_decomp(hzb_ctx *ctx, int rows, int cols, const double *Z, double eps, int *k,
                             int *J, double *T);

/* ------------------------------------------------------------------------------
 * Learned warm start (no counterpart in the paper; it only seeds GMRES through the
 * x0 of hzb_solve_data, and the zero-guess solve remains the fallback).
 * A multilayer perceptron: n_in inputs -> depth hidden layers of `width` units with
 * GELU(a) = a Phi(a) -> n_out linear outputs.  Parameters are stored layer by layer
 * as W (n_out_l x n_in_l, row-major) then b (n_out_l), FP32 masters with a BF16
 * copy used by the forward and backward products; activations and accumulations
 * are FP32.  Loss: (1/B) sum over the batch and outputs of (y - t)^2.  Optimiser:
 * Adam (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected).  Batches: B x n_in
 * inputs and B x n_out targets, row-major FP32, host or device (flag).
 * ------------------------------------------------------------------------------ */
typedef struct hzb_mlp hzb_mlp;

/* Products of the layers whose batch, inputs and outputs are multiples of 128 (the
 * 512-wide hidden and output layers at batch sizes 128, 256, ...) run on the tensor
 * cores (tcgen05.mma kind::f16: BF16 operands, FP32 accumulation in tensor memory): the
 * layer input and the back-propagated gradient are rounded to BF16 for the product; the
 * other layers (e.g. the first, 3 inputs) on the CUDA cores with FP32 activations.
 * on = 0 forces the CUDA cores everywhere (default 1).  A bounded tensor-core wait that
 * runs out makes the call return HZB_ETIMEOUT. */
hzb_status hzb_mlp_set_tensor_cores(hzb_mlp *m, int on);

/* Create on `device` launching on `stream` (NULL = default stream); weights drawn
 * uniformly in +-1/sqrt(fan_in) from a splitmix64 stream seeded by `seed`, biases 0. */
hzb_status hzb_mlp_create(int device, void *stream, int n_in, int width, int depth, int n_out,
                          unsigned long long seed, hzb_mlp **out);
hzb_status hzb_mlp_destroy(hzb_mlp *m);
const char *hzb_mlp_last_error(const hzb_mlp *m);
hzb_status hzb_mlp_num_params(const hzb_mlp *m, long long *n);
/* FP32 master parameters to / from host memory (set also refreshes the BF16 copy). */
hzb_status hzb_mlp_get_params(hzb_mlp *m, float *out);
hzb_status hzb_mlp_set_params(hzb_mlp *m, const float *in);
/* y = network(x) for a batch of B rows. */
hzb_status hzb_mlp_forward(hzb_mlp *m, int B, const float *x, float *y, int on_device);
/* Loss (host float) and the gradient of every parameter (same layout as the
 * parameters; host or device per the flag; either output may be NULL). */
hzb_status hzb_mlp_gradients(hzb_mlp *m, int B, const float *x, const float *t, float *loss,
                             float *grads, int on_device);
/* One Adam step on the batch; *loss (may be NULL) receives the loss before the step. */
hzb_status hzb_mlp_train_step(hzb_mlp *m, int B, const float *x, const float *t, float lr,
                              float *loss, int on_device);

/* POD basis and guess of the warm start (no counterpart in the paper).  All arrays are
 * device memory of the context's GPU, complex interleaved, row-major.
 *   hzb_pod_basis:   U (N x k) with orthonormal columns spanning the dominant left
 *                    singular subspace of the snapshot matrix X (N x T): a complex
 *                    Gaussian sketch Z = X Omega (counter-based generator seeded by
 *                    `seed`), power_steps rounds of Z = X (X^H Z) (0..8), then classical
 *                    Gram-Schmidt applied twice in FP64 (the randomized range finder of
 *                    Halko, Martinsson and Tropp).  1 <= k <= min(N, T).
 *   hzb_pod_project: C (k x T) = U^H X.
 *   hzb_pod_expand:  x0 (N x R) = U coef (coef k x R).
 *   hzb_pod_guess:   x0 (N x R) = U coef with coef[j][r] = scale (y[r][2j] + i y[r][2j+1]),
 *                    y (R x 2k, FP32) the network's outputs (hzb_mlp_forward).
 * The products run in FP32 on complex operands (FP64 in and out).  Errors: HZB_EINVAL
 * (sizes, null pointers), HZB_ENOMEM, HZB_ECUDA. */
hzb_status hzb_pod_basis(hzb_ctx *ctx, int N, int T, const double *X, int k, int power_steps,
                         unsigned long long seed, double *U);
hzb_status hzb_pod_project(hzb_ctx *ctx, int N, int k, int T, const double *U, const double *X, double *C);
hzb_status hzb_pod_expand(hzb_ctx *ctx, int N, int k, int R, const double *U, const double *coef, double *x0);
hzb_status hzb_pod_guess(hzb_ctx *ctx, int N, int k, int R, const double *U, const float *y, double scale,
                         double *x0);

#ifdef __cplusplus
}
#endif
#endif /* HZB_H */
