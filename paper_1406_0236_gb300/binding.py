"""ctypes binding of include/hzb.h (names follow the C ABI; marshalling only).

Host arrays are numpy complex128 / float64; device arrays are torch CUDA tensors
(complex128), passed by data_ptr() with the on_device flag.  Nothing here computes
any part of the method.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
_LIBPATH = os.path.join(HERE, "libhzb.so")

HZB_PREC_FP64 = 0
HZB_PREC_MIXED_FP32 = 1
HZB_PREC_DOUBLE_FLOAT = 2
HZB_SPHERE, HZB_SPHEROID, HZB_OPEN_SHELL = 0, 1, 2

_STATUS = {0: "ok", -1: "invalid argument", -2: "out of memory", -3: "CUDA error",
           -4: "GMRES did not converge", -5: "non-finite value", -6: "device wait timed out",
           -7: "call out of order"}


class HzbError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("hzb status %d (%s): %s" % (status, _STATUS.get(status, "?"), msg))
        self.status = status


class _Options(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("cuda_stream", ctypes.c_void_p), ("precision", ctypes.c_int),
                ("gmres_tol", ctypes.c_double), ("restart", ctypes.c_int), ("maxit", ctypes.c_int),
                ("inner_tol", ctypes.c_double), ("max_outer", ctypes.c_int), ("verify_final", ctypes.c_int),
                ("residual", ctypes.c_int)]


class _Shape(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("p", ctypes.c_double * 4), ("n_panels", ctypes.c_int),
                ("gl_order", ctypes.c_int), ("n_modes", ctypes.c_int)]


class _Stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("outer_iterations", ctypes.c_int), ("converged", ctypes.c_int),
                ("rel_residual", ctypes.c_double), ("t_solve_ms", ctypes.c_double),
                ("t_setup_ms", ctypes.c_double), ("interbody_applies", ctypes.c_longlong),
                ("t_nbody64_ms", ctypes.c_double), ("t_nbody32_ms", ctypes.c_double),
                ("n_nbody64", ctypes.c_longlong), ("n_nbody32", ctypes.c_longlong),
                ("kernel_launches", ctypes.c_longlong), ("t_nbodydf_ms", ctypes.c_double),
                ("n_nbodydf", ctypes.c_longlong)]


@dataclass
class Stats:
    iterations: int
    outer_iterations: int
    converged: bool
    rel_residual: float
    t_solve_ms: float
    t_setup_ms: float
    interbody_applies: int
    t_nbody64_ms: float = 0.0
    t_nbody32_ms: float = 0.0
    n_nbody64: int = 0
    n_nbody32: int = 0
    kernel_launches: int = 0
    t_nbodydf_ms: float = 0.0
    n_nbodydf: int = 0
    status: int = 0


@dataclass
class Options:
    device: int = 0
    precision: int = HZB_PREC_FP64
    gmres_tol: float = 1e-10
    restart: int = 0
    maxit: int = 500
    inner_tol: float = 1e-5
    max_outer: int = 10
    verify_final: int = 1
    residual: int = HZB_PREC_FP64


def library_path() -> str:
    return _LIBPATH


_lib = None
_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)


def lib():
    """Load libhzb.so (raises if it is missing: there is no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIBPATH):
        raise ImportError("libhzb.so is not built (run paper_1406_0236_gb300/build.py); no CPU fallback exists")
    L = ctypes.CDLL(_LIBPATH)
    i, d, p = ctypes.c_int, ctypes.c_double, ctypes.c_void_p
    sig = {
        "hzb_default_options": (None, [ctypes.POINTER(_Options)]),
        "hzb_create": (i, [ctypes.POINTER(_Options), ctypes.POINTER(p)]),
        "hzb_destroy": (i, [p]),
        "hzb_last_error": (ctypes.c_char_p, [p]),
        "hzb_status_string": (ctypes.c_char_p, [i]),
        "hzb_set_stream": (i, [p, p]),
        "hzb_set_options": (i, [p, ctypes.POINTER(_Options)]),
        "hzb_set_wave": (i, [p, d, d]),
        "hzb_add_body": (i, [p, ctypes.POINTER(_Shape), _D, _D, ctypes.POINTER(i)]),
        "hzb_num_nodes": (i, [p, ctypes.POINTER(ctypes.c_longlong)]),
        "hzb_get_nodes": (i, [p, p, p, p]),
        "hzb_build_scattering_matrices": (i, [p]),
        "hzb_get_modal_block": (i, [p, i, i, i, p]),
        "hzb_interbody": (i, [p, i, p, p, i, i]),
        "hzb_local_inverse": (i, [p, i, p, p, d, d, p, i, i]),
        "hzb_apply": (i, [p, i, p, p, i, i]),
        "hzb_solve_plane_waves": (i, [p, i, p, ctypes.POINTER(_Stats)]),
        "hzb_solve_data": (i, [p, i, p, p, i, ctypes.POINTER(_Stats)]),
        "hzb_get_density": (i, [p, p, i]),
        "hzb_far_field": (i, [p, i, p, p]),
        "hzb_eval_field": (i, [p, i, p, p]),
        "hzb_autotune": (i, [p, i, i, p]),
        "hzb_local_inverse_noalloc": (i, [p, i, p, p, d, d, p]),
        "hzb_set_execution": (i, [p, i, i]),
        "hzb_set_modal_engine": (i, [p, i]),
        "hzb_set_interbody_engine": (i, [p, i]),
        "hzb_set_fp64_interbody_engine": (i, [p, i]),
        "hzb_tuned_config": (i, [p, i, p]),
        "hzb_save_scattering": (i, [p, ctypes.c_char_p]),
        "hzb_add_body_curve": (i, [p, _D, i, i, i, _D, _D, ctypes.POINTER(i)]),
        "hzb_load_scattering": (i, [p, ctypes.c_char_p]),
        "hzb_compress": (i, [p, d, i, d]),
        "hzb_set_skeleton": (i, [p, i, i, p, p]),
        "hzb_get_skeleton": (i, [p, i, ctypes.POINTER(i), p, p]),
        "hzb_set_acceleration": (i, [p, i]),
        "hzb_reduced_size": (i, [p, ctypes.POINTER(ctypes.c_longlong)]),
        "hzb_apply_reduced": (i, [p, i, p, p, i]),
        "hzb_interp_decomp": (i, [p, i, i, p, d, ctypes.POINTER(i), p, p]),
        "hzb_measure_peak": (i, [p, i, ctypes.POINTER(d)]),
        "hzb_interbody_bodies": (i, [p, i, p, i, i, p, i, i]),
        "hzb_pod_basis": (i, [p, i, i, p, i, i, ctypes.c_ulonglong, p]),
        "hzb_incident_plane_waves": (i, [p, i, p, p, i]),
        "hzb_get_skeleton_info": (i, [p, i, ctypes.POINTER(i), ctypes.POINTER(d), ctypes.POINTER(d)]),
        "hzb_pod_project": (i, [p, i, i, i, p, p, p]),
        "hzb_pod_expand": (i, [p, i, i, i, p, p, p]),
        "hzb_pod_guess": (i, [p, i, i, i, p, p, d, p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _is_dev(a) -> bool:
    return hasattr(a, "is_cuda") and bool(a.is_cuda)


def _ptr(a):
    if _is_dev(a):
        return ctypes.c_void_p(a.data_ptr())
    return a.ctypes.data_as(ctypes.c_void_p)



def check_device_vectors(N: int, device: int, first, *others, expect_cuda: bool = True):
    """Raise ValueError unless `first` and every non-None tensor in `others` is a
    contiguous complex128 tensor of shape (N,) or (N, R), all of the same shape, on
    CUDA device `device` (expect_cuda=False checks CPU tensors the same way, for
    tests on machines without a GPU).  The C entry points take raw device addresses
    and trust the sizes, so a short, strided or complex64 tensor would make the
    kernels read and write outside the caller's buffers."""
    import torch
    for t in (first,) + tuple(x for x in others if x is not None):
        if not isinstance(t, torch.Tensor):
            raise ValueError("expected a torch tensor, got %s" % type(t).__name__)
        if expect_cuda and (not t.is_cuda or t.device.index != int(device)):
            raise ValueError("expected a CUDA tensor on cuda:%d, got one on %s" % (device, t.device))
        if not expect_cuda and t.is_cuda:
            raise ValueError("expected a CPU tensor")
        if t.dtype != torch.complex128:
            raise ValueError("expected complex128, got %s" % t.dtype)
        if not t.is_contiguous():
            raise ValueError("device tensors must be contiguous")
        if t.dim() not in (1, 2) or t.shape[0] != N:
            raise ValueError("expected shape (N,) or (N, R) with N = %d, got %s" % (N, tuple(t.shape)))
        if t.shape != first.shape:
            raise ValueError("operands differ in shape: %s and %s" % (tuple(first.shape), tuple(t.shape)))


class Solver:
    """One context of the C library.  Typical use:

        s = Solver(k, eta); s.add_body(...); s.build_scattering_matrices()
        st = s.solve_plane_waves(dirs); sigma = s.get_density(); u = s.far_field(xhat)
    """

    def __init__(self, k: float, eta: float, options: Options = None, stream=None):
        L = lib()
        o = options or Options()
        co = _Options()
        L.hzb_default_options(ctypes.byref(co))
        co.device, co.precision, co.gmres_tol = o.device, o.precision, o.gmres_tol
        co.restart, co.maxit, co.inner_tol, co.max_outer = o.restart, o.maxit, o.inner_tol, o.max_outer
        co.verify_final = o.verify_final
        co.residual = o.residual
        co.cuda_stream = stream
        self._opt = co
        h = ctypes.c_void_p()
        self._check(L.hzb_create(ctypes.byref(co), ctypes.byref(h)), ctx=None)
        self._h = h
        self._check(L.hzb_set_wave(h, float(k), float(eta)))
        self.k, self.eta = float(k), float(eta)
        self.bodies = 0
        self._body_n = []                   # node count of each body

    # ------------------------------------------------------------ plumbing
    def _check(self, status: int, ctx="self"):
        if status != 0:
            msg = lib().hzb_last_error(self._h).decode() if ctx is not None and getattr(self, "_h", None) else ""
            raise HzbError(status, msg)

    def close(self):
        if getattr(self, "_h", None):
            lib().hzb_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream_handle: int):
        self._check(lib().hzb_set_stream(self._h, ctypes.c_void_p(stream_handle)))

    def set_execution(self, check_every: int = 0, use_graphs: int = -1):
        """GMRES steps between host checks (0 = auto) and CUDA graphs (-1 auto, 0 off, 1 on)."""
        self._check(lib().hzb_set_execution(self._h, int(check_every), int(use_graphs)))

    def set_modal_engine(self, engine: int):
        """FP32 modal GEMM engine: 0 CUDA cores, 1 mma.sync TF32 x 3, 2 tcgen05 fed by TMA, -1 auto."""
        self._check(lib().hzb_set_modal_engine(self._h, int(engine)))

    def set_interbody_engine(self, engine: int):
        """FP32 inter-body sum engine: 0 CUDA cores, 1 tensor cores, 2 scalar CUDA-core kernel,
        3 packed-pair CUDA-core kernel, 4 pair-symmetric packed kernel, 5 tcgen05 tensor cores,
        6 tcgen05 warp-specialised pipeline, 7 tcgen05 with single-term TF32 products (opt-in,
        ~3e-4 relative error), -1 auto (tensor cores for R >= 16 or as tuned)."""
        self._check(lib().hzb_set_interbody_engine(self._h, int(engine)))

    def set_fp64_interbody_engine(self, engine: int):
        """FP64/double-float inter-body engine: 0 one-directional, 1 pair-symmetric, -1 auto (1 for R <= 4)."""
        self._check(lib().hzb_set_fp64_interbody_engine(self._h, int(engine)))

    def set_options(self, **kw):
        for k_, v in kw.items():
            setattr(self._opt, k_, v)
        self._check(lib().hzb_set_options(self._h, ctypes.byref(self._opt)))

    # ------------------------------------------------------------ geometry
    def add_body(self, kind: int, params, n_panels: int, gl_order: int, n_modes: int, center, rot) -> int:
        if int(kind) == 3:                  # spline generating curve: params = (r0, z0, r1, z1, ...)
            rz = np.ascontiguousarray(np.asarray(params, dtype=np.float64).reshape(-1))
            if rz.size // 2 - 1 != int(n_panels):
                raise ValueError("a spline curve has one panel per segment: n_panels = points - 1")
            return self.add_body_curve(rz.reshape(-1, 2), gl_order, n_modes, center, rot)
        s = _Shape()
        s.kind = int(kind)
        pp = list(params) + [0.0] * (4 - len(params))
        for q in range(4):
            s.p[q] = float(pp[q])
        s.n_panels, s.gl_order, s.n_modes = int(n_panels), int(gl_order), int(n_modes)
        c = np.ascontiguousarray(center, dtype=np.float64)
        r = np.ascontiguousarray(np.asarray(rot, dtype=np.float64).reshape(9))
        bid = ctypes.c_int()
        self._check(lib().hzb_add_body(self._h, ctypes.byref(s), c.ctypes.data_as(_D), r.ctypes.data_as(_D),
                                       ctypes.byref(bid)))
        self.bodies += 1
        self._body_n.append(int(n_panels) * int(gl_order) * int(n_modes))
        return bid.value

    @classmethod
    def from_workload(cls, wl, options: Options = None, stream=None) -> "Solver":
        s = cls(wl.k, wl.eta, options, stream)
        for b in wl.bodies:
            sh = b.shape
            s.add_body(sh.kind, sh.params, sh.n_panels, sh.gl_order, sh.n_modes, b.center, b.rot)
        return s

    def add_body_curve(self, rz, gl_order: int, n_modes: int, center, rot) -> int:
        """Body whose generating curve is the cubic spline through the (r, z) points rz
        (top pole first, both ends on the axis); one panel per spline segment."""
        pts = np.ascontiguousarray(np.asarray(rz, dtype=np.float64).reshape(-1, 2))
        c = np.ascontiguousarray(center, dtype=np.float64)
        r = np.ascontiguousarray(np.asarray(rot, dtype=np.float64).reshape(9))
        bid = ctypes.c_int()
        self._check(lib().hzb_add_body_curve(self._h, pts.ctypes.data_as(_D), int(pts.shape[0]), int(gl_order),
                                             int(n_modes), c.ctypes.data_as(_D), r.ctypes.data_as(_D),
                                             ctypes.byref(bid)))
        self.bodies += 1
        self._body_n.append((int(pts.shape[0]) - 1) * int(gl_order) * int(n_modes))
        return bid.value

    @property
    def N(self) -> int:
        n = ctypes.c_longlong()
        self._check(lib().hzb_num_nodes(self._h, ctypes.byref(n)))
        return n.value

    def get_nodes(self):
        N = self.N
        x = np.zeros((N, 3)); n = np.zeros((N, 3)); w = np.zeros(N)
        self._check(lib().hzb_get_nodes(self._h, _ptr(x), _ptr(n), _ptr(w)))
        return x, n, w

    def autotune(self, R: int = 1, which: int = 1):
        """Pick the inter-body kernels' launch shape by timing (bit 0: FP32, bit 1: FP64).
        Returns the best time per launch in ms, [FP32, FP64]."""
        best = np.zeros(2)
        self._check(lib().hzb_autotune(self._h, int(R), int(which), _ptr(best)))
        return best

    # ------------------------------------------------------------ warm-start linear algebra
    def pod_basis(self, X, k: int, power_steps: int = 2, seed: int = 7):
        """U (N x k, orthonormal columns) of the dominant subspace of X (N x T CUDA complex128)."""
        import torch
        if not (_is_dev(X) and X.dtype == torch.complex128 and X.is_contiguous() and X.dim() == 2):
            raise ValueError("X must be a contiguous N x T complex128 CUDA tensor")
        U = X.new_empty((X.shape[0], int(k)))
        self._check(lib().hzb_pod_basis(self._h, int(X.shape[0]), int(X.shape[1]), _ptr(X), int(k),
                                        int(power_steps), int(seed), _ptr(U)))
        return U

    def pod_project(self, U, X):
        """C = U^H X (k x T) for CUDA complex128 U (N x k) and X (N x T)."""
        if U.shape[0] != X.shape[0] or not (U.is_contiguous() and X.is_contiguous()):
            raise ValueError("U (N x k) and X (N x T) must be contiguous with the same N")
        C = X.new_empty((U.shape[1], X.shape[1]))
        self._check(lib().hzb_pod_project(self._h, int(U.shape[0]), int(U.shape[1]), int(X.shape[1]), _ptr(U),
                                          _ptr(X), _ptr(C)))
        return C

    def pod_expand(self, U, coef):
        """x0 = U coef (N x R) for CUDA complex128 U (N x k) and coef (k x R)."""
        if U.shape[1] != coef.shape[0] or not (U.is_contiguous() and coef.is_contiguous()):
            raise ValueError("U (N x k) and coef (k x R) must be contiguous with the same k")
        x0 = U.new_empty((U.shape[0], coef.shape[1]))
        self._check(lib().hzb_pod_expand(self._h, int(U.shape[0]), int(U.shape[1]), int(coef.shape[1]), _ptr(U),
                                         _ptr(coef), _ptr(x0)))
        return x0

    def pod_guess(self, U, y, scale: float):
        """x0 = U coef from the network's FP32 outputs y (R x 2k CUDA tensor), coef_j = scale (y_2j + i y_2j+1)."""
        import torch
        if not (y.dtype == torch.float32 and y.is_contiguous() and y.shape[1] == 2 * U.shape[1]):
            raise ValueError("y must be a contiguous R x 2k float32 CUDA tensor")
        x0 = U.new_empty((U.shape[0], y.shape[0]))
        self._check(lib().hzb_pod_guess(self._h, int(U.shape[0]), int(U.shape[1]), int(y.shape[0]), _ptr(U),
                                        _ptr(y), float(scale), _ptr(x0)))
        return x0

    PEAK_KINDS = ("ffma", "ffma2", "dfma", "mufu", "tf32_tcgen05")

    def measure_peak(self, kind: str) -> float:
        """Measured throughput of one pipe (hzb_measure_peak): TFLOP/s for the FMA and
        tensor-core kinds, T operations/s for the transcendental unit ("mufu")."""
        v = ctypes.c_double()
        self._check(lib().hzb_measure_peak(self._h, self.PEAK_KINDS.index(kind), ctypes.byref(v)))
        return v.value

    FP32_KERNELS = ("nbody32_kernel", "nbody32x2_kernel", "nbody32_sym_kernel", "nbody_tc_kernel", "nbody_tc5_kernel")

    def tuned_config(self, R: int = 1) -> dict:
        """The inter-body kernels this solver launches for R right-hand sides."""
        out = np.zeros(6, dtype=np.int32)
        self._check(lib().hzb_tuned_config(self._h, int(R), _ptr(out)))
        return {"fp32_kernel": self.FP32_KERNELS[out[0]], "fp32_tpt": int(out[1]), "fp32_split": int(out[2]),
                "fp64_kernel": "nbody64_sym_kernel" if out[3] else "nbody64_kernel",
                "fp64_tpt": int(out[4]), "fp64_split": int(out[5])}

    def save_scattering(self, path: str):
        """Write the per-shape modal matrices (A~_p, S_p) to `path`."""
        self._check(lib().hzb_save_scattering(self._h, os.fsencode(path)))

    def load_scattering(self, path: str):
        """Read matrices written by save_scattering instead of building them."""
        self._check(lib().hzb_load_scattering(self._h, os.fsencode(path)))

    def build_scattering_matrices(self):
        self._check(lib().hzb_build_scattering_matrices(self._h))

    def get_modal_block(self, body: int, p: int, which: int = 1, ng: int = None) -> np.ndarray:
        """which = 0: A~_p, which = 1: S_p (N_G x N_G complex)."""
        if ng is None:
            raise ValueError("pass ng (rings of the body's shape)")
        out = np.zeros((ng, ng), dtype=np.complex128)
        self._check(lib().hzb_get_modal_block(self._h, int(body), int(p), int(which), _ptr(out)))
        return out

    # ------------------------------------------------------------ operators
    def _io(self, a):
        dev = _is_dev(a)
        N = self.N
        if dev:
            check_device_vectors(N, self._opt.device, a)
            out = a.new_empty(a.shape)
        else:
            a = np.ascontiguousarray(a, dtype=np.complex128)
            if a.ndim not in (1, 2) or a.shape[0] != N:
                raise ValueError("expected an N or N x R complex array, N = %d; got shape %s" % (N, a.shape))
            out = np.empty_like(a)
        R = 1 if a.ndim == 1 else int(a.shape[1])
        return a, out, R, int(dev)

    def interbody(self, sigma, precision: int = HZB_PREC_FP64):
        a, out, R, dev = self._io(sigma)
        self._check(lib().hzb_interbody(self._h, R, _ptr(a), _ptr(out), dev, int(precision)))
        return out

    def interbody_bodies(self, sigma, body_begin: int, body_end: int, precision: int = HZB_PREC_FP64):
        """Rows of B sigma for the targets of bodies [body_begin, body_end) (sigma: all N rows)."""
        a, _, R, dev = self._io(sigma)
        offs = np.concatenate([[0], np.cumsum(self._body_n)]).astype(int)
        if not (0 <= body_begin < body_end <= len(self._body_n)):
            raise ValueError("body range out of bounds or empty")
        nr = int(offs[body_end] - offs[body_begin])
        shape = (nr,) if a.ndim == 1 else (nr, R)
        out = a.new_empty(shape) if dev else np.empty(shape, dtype=np.complex128)
        self._check(lib().hzb_interbody_bodies(self._h, R, _ptr(a), int(body_begin), int(body_end), _ptr(out), dev,
                                               int(precision)))
        return out

    def local_inverse(self, y, sigma=None, alpha: float = 0.0, beta: float = 1.0, precision: int = HZB_PREC_FP64):
        a, out, R, dev = self._io(y)
        sp = None
        if sigma is not None:
            if dev:
                check_device_vectors(self.N, self._opt.device, a, sigma)
                s2 = sigma
            else:
                s2 = np.ascontiguousarray(sigma, dtype=np.complex128)
                if s2.shape != a.shape:
                    raise ValueError("sigma must have the shape of y")
            sp = _ptr(s2)
        self._check(lib().hzb_local_inverse(self._h, R, _ptr(a), sp, float(alpha), float(beta), _ptr(out), dev,
                                            int(precision)))
        return out

    def local_inverse_noalloc(self, y, sigma=None, alpha: float = 0.0, beta: float = 1.0, out=None):
        """FP64 D^{-1} apply through hzb_local_inverse_noalloc: device tensors only; the
        library allocates nothing for this call (static scratch, see include/hzb.h).
        y, sigma and out are checked (contiguous complex128 CUDA tensors of shape N or
        N x R on the context's device, all of one shape) before their addresses reach
        the C call, which cannot check sizes itself."""
        if out is None:
            check_device_vectors(self.N, self._opt.device, y)
            out = y.new_empty(y.shape)
        check_device_vectors(self.N, self._opt.device, y, sigma, out)
        R = 1 if y.ndim == 1 else int(y.shape[1])
        sp = _ptr(sigma) if sigma is not None else None
        self._check(lib().hzb_local_inverse_noalloc(self._h, R, _ptr(y), sp, float(alpha), float(beta), _ptr(out)))
        return out

    def apply(self, sigma, precision: int = HZB_PREC_FP64):
        a, out, R, dev = self._io(sigma)
        self._check(lib().hzb_apply(self._h, R, _ptr(a), _ptr(out), dev, int(precision)))
        return out

    # ------------------------------------------------------------ solves
    def _stats(self, st: _Stats, status: int) -> Stats:
        return Stats(st.iterations, st.outer_iterations, bool(st.converged), st.rel_residual, st.t_solve_ms,
                     st.t_setup_ms, st.interbody_applies, st.t_nbody64_ms, st.t_nbody32_ms, st.n_nbody64,
                     st.n_nbody32, st.kernel_launches, st.t_nbodydf_ms, st.n_nbodydf, status)

    def solve_plane_waves(self, dirs, allow_noconv: bool = False) -> Stats:
        d = np.ascontiguousarray(np.atleast_2d(dirs), dtype=np.float64)
        st = _Stats()
        rc = lib().hzb_solve_plane_waves(self._h, int(d.shape[0]), _ptr(d), ctypes.byref(st))
        if rc != 0 and not (allow_noconv and rc == -4):
            self._check(rc)
        self._R = int(d.shape[0])
        return self._stats(st, rc)

    def plane_waves(self, dirs, device: bool = True):
        """v = exp(i k d.x) at the nodes (N x R) for unit directions dirs (R x 3), on the
        library's kernel: a CUDA tensor (device=True) or a numpy array."""
        d = np.ascontiguousarray(np.atleast_2d(dirs), dtype=np.float64)
        R = d.shape[0]
        if device:
            import torch
            v = torch.empty((self.N, R), dtype=torch.complex128, device="cuda:%d" % self._opt.device)
        else:
            v = np.empty((self.N, R), dtype=np.complex128)
        self._check(lib().hzb_incident_plane_waves(self._h, R, _ptr(d), _ptr(v), int(device)))
        return v

    def solve_data(self, v, x0=None, allow_noconv: bool = False) -> Stats:
        N = self.N
        if _is_dev(v):
            check_device_vectors(N, self._opt.device, v, x0 if _is_dev(x0) else None)
            a = v
        else:
            a = np.ascontiguousarray(v, dtype=np.complex128)
            if a.ndim not in (1, 2) or a.shape[0] != N:
                raise ValueError("expected v of shape (N,) or (N, R) with N = %d, got %s" % (N, a.shape))
        R = 1 if a.ndim == 1 else int(a.shape[1])
        xp = None
        if x0 is not None:
            if _is_dev(x0) != _is_dev(a):
                raise ValueError("v and x0 must both be host arrays or both CUDA tensors")
            if not _is_dev(x0):
                x0 = np.ascontiguousarray(x0, dtype=np.complex128)
                if x0.shape != a.shape:
                    raise ValueError("x0 must have the shape of v")
            xp = _ptr(x0)
        st = _Stats()
        rc = lib().hzb_solve_data(self._h, R, _ptr(a), xp, int(_is_dev(a)), ctypes.byref(st))
        if rc != 0 and not (allow_noconv and rc == -4):
            self._check(rc)
        self._R = R
        return self._stats(st, rc)

    # ------------------------------------------------------------ accelerated scheme
    def compress(self, eps: float, n_theta: int = 0, proxy_radius: float = 0.0):
        """Skeletons of every shape by the GPU's interpolative decomposition (Sec. 5);
        solves then run on the reduced system of Eq. (ip6)."""
        self._check(lib().hzb_compress(self._h, float(eps), int(n_theta), float(proxy_radius)))

    def set_skeleton(self, body: int, J, T):
        J = np.ascontiguousarray(J, dtype=np.int32)
        T = np.ascontiguousarray(T, dtype=np.complex128)
        self._check(lib().hzb_set_skeleton(self._h, int(body), int(J.size), _ptr(J), _ptr(T)))

    def get_skeleton(self, body: int):
        """(J ascending, T with rows in J's order) of the body's shape, or None."""
        k = ctypes.c_int()
        self._check(lib().hzb_get_skeleton(self._h, int(body), ctypes.byref(k), None, None))
        if k.value == 0:
            return None
        n = self._body_n[body]
        J = np.zeros(k.value, dtype=np.int32)
        T = np.zeros((k.value, n), dtype=np.complex128)
        self._check(lib().hzb_get_skeleton(self._h, int(body), ctypes.byref(k), _ptr(J), _ptr(T)))
        return J, T

    def get_skeleton_info(self, body: int):
        """(k, eps, rho) of the skeleton of the body's shape (eps = rho = 0: set by the caller)."""
        k, e, r = ctypes.c_int(), ctypes.c_double(), ctypes.c_double()
        self._check(lib().hzb_get_skeleton_info(self._h, int(body), ctypes.byref(k), ctypes.byref(e), ctypes.byref(r)))
        return k.value, e.value, r.value

    def get_skeleton_size(self, body: int) -> int:
        k = ctypes.c_int()
        self._check(lib().hzb_get_skeleton(self._h, int(body), ctypes.byref(k), None, None))
        return k.value

    def set_acceleration(self, on: bool):
        self._check(lib().hzb_set_acceleration(self._h, int(bool(on))))

    @property
    def reduced_size(self) -> int:
        n = ctypes.c_longlong()
        self._check(lib().hzb_reduced_size(self._h, ctypes.byref(n)))
        return n.value

    def apply_reduced(self, sig, precision: int = HZB_PREC_FP64):
        a = np.ascontiguousarray(sig, dtype=np.complex128)
        R = 1 if a.ndim == 1 else int(a.shape[1])
        out = np.zeros_like(a)
        self._check(lib().hzb_apply_reduced(self._h, R, _ptr(a), _ptr(out), int(precision)))
        return out

    def interp_decomp(self, Z, eps: float):
        """GPU interpolative decomposition of Z (rows x cols): (J in pivot order, T)."""
        Z = np.asarray(Z, dtype=np.complex128)
        rows, cols = Z.shape
        Zc = np.asfortranarray(Z)
        J = np.zeros(cols, dtype=np.int32)
        T = np.zeros((min(rows, cols), cols), dtype=np.complex128)
        k = ctypes.c_int()
        self._check(lib().hzb_interp_decomp(self._h, rows, cols, Zc.ctypes.data_as(ctypes.c_void_p), float(eps),
                                            ctypes.byref(k), _ptr(J), _ptr(T)))
        return J[:k.value].copy(), T[:k.value].copy()

    def get_density(self, out=None):
        R = getattr(self, "_R", 1)
        if out is None:
            out = np.zeros((self.N, R), dtype=np.complex128)
        elif _is_dev(out):
            check_device_vectors(self.N, self._opt.device, out)
            if out.numel() != self.N * R:
                raise ValueError("out must hold N x R = %d x %d values" % (self.N, R))
        elif not (isinstance(out, np.ndarray) and out.dtype == np.complex128 and out.flags.c_contiguous
                  and out.size == self.N * R):
            raise ValueError("out must be a C-contiguous complex128 array of N x R values")
        self._check(lib().hzb_get_density(self._h, _ptr(out), int(_is_dev(out))))
        return out

    def far_field(self, xhat) -> np.ndarray:
        x = np.ascontiguousarray(np.atleast_2d(xhat), dtype=np.float64)
        out = np.zeros((x.shape[0], getattr(self, "_R", 1)), dtype=np.complex128)
        self._check(lib().hzb_far_field(self._h, int(x.shape[0]), _ptr(x), _ptr(out)))
        return out

    def eval_field(self, pts) -> np.ndarray:
        x = np.ascontiguousarray(np.atleast_2d(pts), dtype=np.float64)
        out = np.zeros((x.shape[0], getattr(self, "_R", 1)), dtype=np.complex128)
        self._check(lib().hzb_eval_field(self._h, int(x.shape[0]), _ptr(x), _ptr(out)))
        return out


class Mlp:
    """The warm-start network of the C ABI (hzb_mlp_*): BF16 weights, FP32 activations
    and accumulation, Adam.  Batches are float32 arrays (numpy host or torch CUDA)."""

    def __init__(self, n_in: int, width: int, depth: int, n_out: int, seed: int = 1, device: int = 0,
                 stream=None):
        L = lib()
        self._sig()
        h = ctypes.c_void_p()
        rc = L.hzb_mlp_create(int(device), stream, int(n_in), int(width), int(depth), int(n_out),
                              ctypes.c_ulonglong(seed), ctypes.byref(h))
        if rc != 0:
            raise HzbError(rc, "hzb_mlp_create")
        self._h = h
        self.n_in, self.width, self.depth, self.n_out = n_in, width, depth, n_out

    @staticmethod
    def _sig():
        L = lib()
        i, p, f = ctypes.c_int, ctypes.c_void_p, ctypes.c_float
        for name, res, args in (
                ("hzb_mlp_create", i, [i, p, i, i, i, i, ctypes.c_ulonglong, ctypes.POINTER(p)]),
                ("hzb_mlp_destroy", i, [p]),
                ("hzb_mlp_last_error", ctypes.c_char_p, [p]),
                ("hzb_mlp_num_params", i, [p, ctypes.POINTER(ctypes.c_longlong)]),
                ("hzb_mlp_get_params", i, [p, p]),
                ("hzb_mlp_set_tensor_cores", i, [p, i]),
                ("hzb_mlp_set_params", i, [p, p]),
                ("hzb_mlp_forward", i, [p, i, p, p, i]),
                ("hzb_mlp_gradients", i, [p, i, p, p, ctypes.POINTER(f), p, i]),
                ("hzb_mlp_train_step", i, [p, i, p, p, f, ctypes.POINTER(f), i])):
            fn = getattr(L, name)
            fn.restype, fn.argtypes = res, args

    def _check(self, rc):
        if rc != 0:
            raise HzbError(rc, lib().hzb_mlp_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            lib().hzb_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def num_params(self) -> int:
        n = ctypes.c_longlong()
        self._check(lib().hzb_mlp_num_params(self._h, ctypes.byref(n)))
        return n.value

    def set_tensor_cores(self, on: bool):
        """Tensor-core (tcgen05 BF16) products for whole-tile layers (default on)."""
        self._check(lib().hzb_mlp_set_tensor_cores(self._h, int(bool(on))))

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.num_params, dtype=np.float32)
        self._check(lib().hzb_mlp_get_params(self._h, _ptr(out)))
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        self._check(lib().hzb_mlp_set_params(self._h, _ptr(p)))

    def layers(self, flat: np.ndarray):
        """Split a flat parameter vector into [(W, b)] per layer."""
        out, off = [], 0
        dims = [self.n_in] + [self.width] * self.depth + [self.n_out]
        for i, o in zip(dims[:-1], dims[1:]):
            W = flat[off:off + i * o].reshape(o, i); off += i * o
            b = flat[off:off + o]; off += o
            out.append((W, b))
        return out

    def forward(self, x):
        dev = _is_dev(x)
        if dev:
            y = x.new_empty((x.shape[0], self.n_out))
        else:
            x = np.ascontiguousarray(x, dtype=np.float32)
            y = np.zeros((x.shape[0], self.n_out), dtype=np.float32)
        self._check(lib().hzb_mlp_forward(self._h, int(x.shape[0]), _ptr(x), _ptr(y), int(dev)))
        return y

    def gradients(self, x, t):
        x = np.ascontiguousarray(x, dtype=np.float32)
        t = np.ascontiguousarray(t, dtype=np.float32)
        g = np.zeros(self.num_params, dtype=np.float32)
        loss = ctypes.c_float()
        self._check(lib().hzb_mlp_gradients(self._h, int(x.shape[0]), _ptr(x), _ptr(t), ctypes.byref(loss),
                                            _ptr(g), 0))
        return float(loss.value), g

    def train_step(self, x, t, lr: float) -> float:
        dev = _is_dev(x)
        if not dev:
            x = np.ascontiguousarray(x, dtype=np.float32)
            t = np.ascontiguousarray(t, dtype=np.float32)
        loss = ctypes.c_float()
        self._check(lib().hzb_mlp_train_step(self._h, int(x.shape[0]), _ptr(x), _ptr(t), float(lr),
                                             ctypes.byref(loss), int(dev)))
        return float(loss.value)
