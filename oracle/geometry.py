"""Oracle geometry: generating curves, composite Gauss-Legendre panels, the tensor
product surface rule and the near-panel sets.  FP64, numpy.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. 3.2: a body is the curve gamma(t) = (r(t), z(t)) swept about the z axis; the
curve is split into panels carrying p-point Gauss-Legendre rules and the circle
carries an N_F-point trapezoid rule; the surface rule is their tensor product
(Eq. (basicquad) with nodes x_(i,l) and weights w_(i,l) = w_i^GL |gamma'(t_i)| r_i 2pi/N_F).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Tuple

import numpy as np

from workloads import CURVE_SPLINE, OPEN_SHELL, SPHERE, SPHEROID, Body, ShapeSpec

# Near-panel radius in units of the panel's arclength: a panel b is "near" a target
# on the same curve when some node of b lies closer than NEAR_RHO * L_b.
NEAR_RHO = 1.0


def gauss_legendre(n: int) -> Tuple[np.ndarray, np.ndarray]:
    """n-point Gauss-Legendre rule on [-1, 1] (library routine)."""
    x, w = np.polynomial.legendre.leggauss(n)
    return x, w


# ----------------------------------------------------------------------------- curves

class Piece:
    """One smooth piece of a generating curve.

    eval(t)      -> (r, z, r', z')
    delta(t, h)  -> gamma(t + h) - gamma(t), formed with difference identities
                    (sin(a+h) - sin a = 2 cos(a + h/2) sin(h/2), ...) so that it
                    keeps full relative accuracy for tiny h.
    """

    def eval(self, t):
        raise NotImplementedError

    def delta(self, t, h):
        raise NotImplementedError


class _Ellipse(Piece):
    """(a sin t, c cos t): a sphere of radius a when c = a, else a spheroid."""

    def __init__(self, a: float, c: float):
        self.a, self.c = a, c

    def eval(self, t):
        return self.a * np.sin(t), self.c * np.cos(t), self.a * np.cos(t), -self.c * np.sin(t)

    def delta(self, t, h):
        s = 2.0 * np.sin(0.5 * h)
        return self.a * np.cos(t + 0.5 * h) * s, -self.c * np.sin(t + 0.5 * h) * s


class _Arc(Piece):
    """Arc of the given radius at polar angle phi = th0 + sign * t."""

    def __init__(self, radius: float, th0: float, sign: float):
        self.R, self.th0, self.sg = radius, th0, sign

    def eval(self, t):
        ph = self.th0 + self.sg * t
        R, sg = self.R, self.sg
        return R * np.sin(ph), R * np.cos(ph), sg * R * np.cos(ph), -sg * R * np.sin(ph)

    def delta(self, t, h):
        ph = self.th0 + self.sg * t
        dp = self.sg * h
        s = 2.0 * np.sin(0.5 * dp)
        return self.R * np.cos(ph + 0.5 * dp) * s, -self.R * np.sin(ph + 0.5 * dp) * s


class _Rim(Piece):
    """Semicircle of radius rho centred at center_radius * u, u = (sin th, cos th),
    from the outer point (s = 0) around the side of larger polar angle to the inner
    point (s = pi)."""

    def __init__(self, center_radius: float, rho: float, th: float):
        self.u = np.array([np.sin(th), np.cos(th)])
        self.e = np.array([np.cos(th), -np.sin(th)])
        self.c = center_radius * self.u
        self.rho = rho

    def eval(self, s):
        u, e, c, rho = self.u, self.e, self.c, self.rho
        cs, sn = np.cos(s), np.sin(s)
        r = c[0] + rho * (cs * u[0] + sn * e[0])
        z = c[1] + rho * (cs * u[1] + sn * e[1])
        dr = rho * (-sn * u[0] + cs * e[0])
        dz = rho * (-sn * u[1] + cs * e[1])
        return r, z, dr, dz

    def delta(self, s, h):
        u, e, rho = self.u, self.e, self.rho
        q = 2.0 * np.sin(0.5 * h)
        dc = -np.sin(s + 0.5 * h) * q         # cos(s+h) - cos s
        dsn = np.cos(s + 0.5 * h) * q         # sin(s+h) - sin s
        return rho * (dc * u[0] + dsn * e[0]), rho * (dc * u[1] + dsn * e[1])


class _CubicSegment(Piece):
    """One segment t in [t_k, t_{k+1}] of a spline generating curve: r and z are cubic
    polynomials in u = t - t_k with coefficients (c3, c2, c1, c0) (highest power first)."""

    def __init__(self, tk: float, cr, cz):
        self.tk = tk
        self.cr = np.asarray(cr, dtype=np.float64)
        self.cz = np.asarray(cz, dtype=np.float64)

    @staticmethod
    def _val(c, u):
        return ((c[0] * u + c[1]) * u + c[2]) * u + c[3]

    @staticmethod
    def _der(c, u):
        return (3.0 * c[0] * u + 2.0 * c[1]) * u + c[2]

    @staticmethod
    def _diff(c, u, h):
        # p(u + h) - p(u) = h (c1 + c2 (2u + h) + c3 (3u^2 + 3uh + h^2)), no cancellation
        return h * (c[2] + c[1] * (2.0 * u + h) + c[0] * (3.0 * u * u + 3.0 * u * h + h * h))

    def eval(self, t):
        u = t - self.tk
        return self._val(self.cr, u), self._val(self.cz, u), self._der(self.cr, u), self._der(self.cz, u)

    def delta(self, t, h):
        u = t - self.tk
        return self._diff(self.cr, u, h), self._diff(self.cz, u, h)


def spline_pieces(rz: np.ndarray) -> List[Tuple[Piece, float, float]]:
    """Spline generating curve through the points rz (n x 2, top pole first): parameter
    = cumulative chord length; r(t) natural (r'' = 0) and z(t) clamped (z' = 0) at both
    poles, so the surface of revolution closes smoothly on the axis.  The interpolating
    cubic splines come from scipy (library routine); one piece per segment."""
    from scipy.interpolate import CubicSpline
    rz = np.asarray(rz, dtype=np.float64).reshape(-1, 2)
    if rz.shape[0] < 3 or rz[0, 0] != 0.0 or rz[-1, 0] != 0.0 or not rz[0, 1] > rz[-1, 1]:
        raise ValueError("spline curve: >= 3 points from the top pole down to the bottom pole")
    t = np.concatenate([[0.0], np.cumsum(np.hypot(np.diff(rz[:, 0]), np.diff(rz[:, 1])))])
    sr = CubicSpline(t, rz[:, 0], bc_type=((2, 0.0), (2, 0.0)))
    sz = CubicSpline(t, rz[:, 1], bc_type=((1, 0.0), (1, 0.0)))
    return [(_CubicSegment(t[k], sr.c[:, k], sz.c[:, k]), float(t[k]), float(t[k + 1]))
            for k in range(t.size - 1)]


@dataclass
class Curve:
    pieces: List[Tuple[Piece, float, float]]      # (piece, t0, t1)
    panels: List[Tuple[int, float, float]]        # (piece, ta, tb) in order along the curve

    def eval(self, piece: int, t):
        return self.pieces[piece][0].eval(np.asarray(t, dtype=np.float64))

    def delta(self, piece: int, t, h):
        return self.pieces[piece][0].delta(np.asarray(t, dtype=np.float64), np.asarray(h, dtype=np.float64))


def shell_panel_split(n: int, L_out: float, L_rim: float, L_in: float) -> Tuple[int, int, int]:
    """Panels per piece of the open shell: proportional to arclength, at least two on
    the rim."""
    L = L_out + L_rim + L_in
    n_rim = max(2, int(round(n * L_rim / L)))
    rest = n - n_rim
    n_out = int(round(rest * L_out / (L_out + L_in)))
    return n_out, n_rim, rest - n_out


def shape_curve(shape: ShapeSpec) -> Curve:
    n = shape.n_panels
    if shape.kind == SPHERE:
        pieces = [(_Ellipse(shape.params[0], shape.params[0]), 0.0, np.pi)]
        counts = [n]
    elif shape.kind == SPHEROID:
        pieces = [(_Ellipse(shape.params[0], shape.params[1]), 0.0, np.pi)]
        counts = [n]
    elif shape.kind == OPEN_SHELL:
        r_out, r_in, half, rho = shape.params
        if abs(2.0 * rho - (r_out - r_in)) > 1e-12:
            raise ValueError("rim radius must be half the wall thickness")
        th = np.pi - half
        pieces = [(_Arc(r_out, 0.0, +1.0), 0.0, th),
                  (_Rim(0.5 * (r_out + r_in), rho, th), 0.0, np.pi),
                  (_Arc(r_in, th, -1.0), 0.0, th)]
        counts = list(shell_panel_split(n, r_out * th, np.pi * rho, r_in * th))
    elif shape.kind == CURVE_SPLINE:
        pieces = spline_pieces(shape.curve_points())
        if len(pieces) != n:
            raise ValueError("a spline curve has one panel per segment")
        counts = [1] * n
    else:
        raise ValueError("unknown shape kind %r" % shape.kind)
    panels = []
    for pi_, ((_, t0, t1), m) in enumerate(zip(pieces, counts)):
        edges = np.linspace(t0, t1, m + 1)
        for q in range(m):
            panels.append((pi_, float(edges[q]), float(edges[q + 1])))
    return Curve(pieces, panels)


# ----------------------------------------------------------------------- ring nodes

@dataclass
class Rings:
    """The discretised generating curve of one shape (N_G = n_panels * gl_order rings)."""
    shape: ShapeSpec
    curve: Curve
    t: np.ndarray          # parameter of each ring node
    piece: np.ndarray      # piece index of each ring node
    panel: np.ndarray      # panel index of each ring node
    r: np.ndarray
    z: np.ndarray
    speed: np.ndarray      # |gamma'(t)|
    nr: np.ndarray         # outward profile normal (-z', r') / |gamma'|
    nz: np.ndarray
    ds: np.ndarray         # w^GL |gamma'|  (arclength weight)
    panel_len: np.ndarray  # L_b = sum of ds over the panel

    @property
    def n(self) -> int:
        return int(self.t.size)

    def panel_nodes(self, b: int) -> np.ndarray:
        return np.nonzero(self.panel == b)[0]


def rings(shape: ShapeSpec) -> Rings:
    cv = shape_curve(shape)
    x, w = gauss_legendre(shape.gl_order)
    T, P, B, WT = [], [], [], []
    for b, (pc, ta, tb) in enumerate(cv.panels):
        h = 0.5 * (tb - ta)
        T.append(0.5 * (ta + tb) + h * x)
        WT.append(h * w)
        P.append(np.full(x.size, pc))
        B.append(np.full(x.size, b))
    t = np.concatenate(T)
    piece = np.concatenate(P)
    panel = np.concatenate(B)
    wt = np.concatenate(WT)
    r = np.empty_like(t); z = np.empty_like(t); dr = np.empty_like(t); dz = np.empty_like(t)
    for pc in range(len(cv.pieces)):
        m = piece == pc
        r[m], z[m], dr[m], dz[m] = cv.eval(pc, t[m])
    speed = np.hypot(dr, dz)
    ds = wt * speed
    panel_len = np.array([ds[panel == b].sum() for b in range(len(cv.panels))])
    return Rings(shape, cv, t, piece, panel, r, z, speed, -dz / speed, dr / speed, ds, panel_len)


def near_panels(rg: Rings, i: int) -> List[int]:
    """Panels treated by product integration for target ring i: its own panel, the
    panels adjacent along the curve, and any panel with a node closer to the target
    than NEAR_RHO times the panel's arclength (the reading of the paper's "small
    distance" entries, Sec. 3.1)."""
    bi = int(rg.panel[i])
    out = []
    for b in range(len(rg.curve.panels)):
        if abs(b - bi) <= 1:
            out.append(b)
            continue
        nodes = rg.panel_nodes(b)
        d = np.hypot(rg.r[nodes] - rg.r[i], rg.z[nodes] - rg.z[i]).min()
        if d < NEAR_RHO * rg.panel_len[b]:
            out.append(b)
    return out


# ---------------------------------------------------------------------- 3-D nodes

@dataclass
class SurfaceNodes:
    x: np.ndarray      # (N, 3)
    n: np.ndarray      # (N, 3) outward unit normals
    w: np.ndarray      # (N,) surface weights
    body: np.ndarray   # (N,) int32 body index
    offsets: np.ndarray  # (m+1,) start of each body's block


def body_nodes(body: Body, rg: Rings) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Nodes of one body, ring-major with the azimuth index fastest:
    x_(i,l) = c + Rot (r_i cos th_l, r_i sin th_l, z_i), th_l = 2 pi l / N_F."""
    nf = body.shape.n_modes
    th = 2.0 * np.pi * np.arange(nf) / nf
    ct, st = np.cos(th), np.sin(th)
    loc = np.stack([rg.r[:, None] * ct[None, :], rg.r[:, None] * st[None, :],
                    np.broadcast_to(rg.z[:, None], (rg.n, nf))], axis=-1).reshape(-1, 3)
    nrm = np.stack([rg.nr[:, None] * ct[None, :], rg.nr[:, None] * st[None, :],
                    np.broadcast_to(rg.nz[:, None], (rg.n, nf))], axis=-1).reshape(-1, 3)
    w = np.broadcast_to((rg.ds * rg.r * 2.0 * np.pi / nf)[:, None], (rg.n, nf)).reshape(-1)
    return loc @ body.rot.T + body.center, nrm @ body.rot.T, w.copy()


def surface_nodes(bodies: List[Body], ring_cache=None) -> SurfaceNodes:
    ring_cache = {} if ring_cache is None else ring_cache
    X, Nn, W, Bd, off = [], [], [], [], [0]
    for q, b in enumerate(bodies):
        if b.shape not in ring_cache:
            ring_cache[b.shape] = rings(b.shape)
        x, n, w = body_nodes(b, ring_cache[b.shape])
        X.append(x); Nn.append(n); W.append(w)
        Bd.append(np.full(w.size, q, dtype=np.int32))
        off.append(off[-1] + w.size)
    return SurfaceNodes(np.concatenate(X), np.concatenate(Nn), np.concatenate(W),
                        np.concatenate(Bd).astype(np.int32), np.array(off))
