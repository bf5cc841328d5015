"""Oracle per-mode Nystrom matrices and scattering matrices of one body shape.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. 3.2: with sigma(x) = sum_p sigma_p(r,z) e^{ip theta}, the surface BIE (Eq.
(intHelm2)) splits into one BIE per azimuthal mode on the generating curve
(Eq. (seqBIE)).  Written with unnormalised modal kernels,

    1/2 sigma_p(y) + int_gamma k_p(y, y') sigma_p(y') r' ds' = -v_p(y),
    k_p(y, y') = int_0^{2pi} K(x(y, 0), x(y', psi)) e^{i p psi} dpsi,

and its Nystrom discretisation on the ring nodes is the N_G x N_G matrix
A~_p = 1/2 I + K_p, where (Sec. 3.1, Eq. (nystromnaive) per mode)

  * far panel b:  K_p(i, j) = k_p(y_i, y_j) r_j ds_j                    (smooth rule)
  * near panel b: K_p(i, j) = int_{panel b} k_p(y_i, gamma(t)) L_j(t) r(t) |gamma'(t)| dt
                  (product integration against the panel's Lagrange basis L_j),

with "near" as in geometry.near_panels.  S_p = A~_p^{-1} (Eq. (singleinverse)).
The paper delegates the modal kernels and its singular corrections to its ref.
[2012_martinsson_axisymmetric]; the rules here are direct quadratures of the
definitions, converged to about 1e-14:

  * far pairs: trapezoid rule in psi, doubled until converged (orc_modes_trapezoid);
  * near panels: composite Gauss-Legendre in t on a mesh graded geometrically
    (ratio T_RATIO) toward the point t* of the panel nearest the target, and for
    every such t a composite Gauss-Legendre rule in psi graded toward psi = 0
    (orc_modes_graded).
"""
from __future__ import annotations

from typing import Dict, Optional

import numpy as np

from . import _native as nat
from .geometry import Rings, gauss_legendre, near_panels

GL_ORDER_T = 16
GL_ORDER_PSI = 16
T_RATIO = 0.3          # geometric grading ratio of the t-mesh toward t*
T_DEPTH = 1e-18        # the graded t-mesh stops at T_DEPTH times the side length
PSI_HMAX = 0.25        # widest psi interval
TRAP_TOL = 1e-14


def _modes_trapezoid(rg: Rings, i: int, js: np.ndarray, k: float, eta: float, M: int) -> np.ndarray:
    out = np.zeros((js.size, M + 1), dtype=np.complex128)
    if js.size == 0:
        return out
    md, _ = modes_trapezoid_at(rg.r[i], rg.r[js], rg.r[js] - rg.r[i], rg.z[js] - rg.z[i],
                               rg.nr[js], rg.nz[js], k, eta, M)
    return md


def modes_graded(r: float, rs, drs, dzs, nrs, nzs, k: float, eta: float, M: int,
                 ngl: int = GL_ORDER_PSI, hmax: float = PSI_HMAX) -> np.ndarray:
    """k_p(y, y'_s), p = 0..M, for a target ring of radius r and source rings s of
    radius rs whose profile points are offset by (drs, dzs) from the target's, with
    the psi-mesh graded toward psi = 0."""
    L = nat.lib()
    rs, drs, dzs, nrs, nzs = (nat.as_f64(np.atleast_1d(a)) for a in (rs, drs, dzs, nrs, nzs))
    x, w = gauss_legendre(ngl)
    x, w = nat.as_f64(x), nat.as_f64(w)
    buf = np.zeros(2 * rs.size * (M + 1))
    L.orc_modes_graded(float(r), int(rs.size), nat.dptr(rs), nat.dptr(drs), nat.dptr(dzs),
                       nat.dptr(nrs), nat.dptr(nzs), float(k), float(eta), int(M), float(hmax),
                       int(ngl), nat.dptr(x), nat.dptr(w), nat.dptr(buf))
    return buf.view(np.complex128).reshape(rs.size, M + 1)


def modes_trapezoid_at(r, rs, drs, dzs, nrs, nzs, k, eta, M, tol=TRAP_TOL):
    """k_p by the doubled trapezoid rule (also returns the number of samples used)."""
    L = nat.lib()
    rs, drs, dzs, nrs, nzs = (nat.as_f64(np.atleast_1d(a)) for a in (rs, drs, dzs, nrs, nzs))
    buf = np.zeros(2 * rs.size * (M + 1))
    used = np.zeros(rs.size, dtype=np.int32)
    L.orc_modes_trapezoid(float(r), int(rs.size), nat.dptr(rs), nat.dptr(drs), nat.dptr(dzs),
                          nat.dptr(nrs), nat.dptr(nzs), float(k), float(eta), int(M), float(tol),
                          nat.dptr(buf), nat.iptr(used))
    return buf.view(np.complex128).reshape(rs.size, M + 1), used


def _closest_parameter(rg: Rings, i: int, b: int) -> float:
    """Parameter on panel b of the curve point nearest ring node i (sampling, then
    golden-section refinement of |gamma(t) - y_i|^2)."""
    pc, ta, tb = rg.curve.panels[b]
    if int(rg.panel[i]) == b:
        return float(rg.t[i])

    def dist2(t):
        r, z, _, _ = rg.curve.eval(pc, t)
        return (r - rg.r[i]) ** 2 + (z - rg.z[i]) ** 2

    ts = np.linspace(ta, tb, 401)
    m = int(np.argmin(dist2(ts)))
    lo, hi = ts[max(m - 1, 0)], ts[min(m + 1, ts.size - 1)]
    g = 0.5 * (np.sqrt(5.0) - 1.0)
    a, c = lo, hi
    x1, x2 = c - g * (c - a), a + g * (c - a)
    f1, f2 = dist2(x1), dist2(x2)
    for _ in range(200):
        if c - a < 1e-15 * max(1.0, abs(tb - ta)):
            break
        if f1 < f2:
            c, x2, f2 = x2, x1, f1
            x1 = c - g * (c - a)
            f1 = dist2(x1)
        else:
            a, x1, f1 = x1, x2, f2
            x2 = a + g * (c - a)
            f2 = dist2(x2)
    return float(min(max(0.5 * (a + c), ta), tb))


def graded_mesh(H: float, ratio: float = T_RATIO, depth: float = T_DEPTH, ngl: int = GL_ORDER_T):
    """Composite Gauss-Legendre rule for the offsets h from t* over [0, H] (H of
    either sign), graded geometrically toward h = 0: intervals
    [ratio^(m+1), ratio^m] * H down to depth * H.  Returns (offsets, weights)."""
    if H == 0.0:
        return np.zeros(0), np.zeros(0)
    x, w = gauss_legendre(ngl)
    T, Wt = [], []
    hi = 1.0
    while hi > depth:
        lo = hi * ratio
        a, b = lo * H, hi * H
        c, h = 0.5 * (a + b), 0.5 * (b - a)
        T.append(c + h * x)
        Wt.append(abs(h) * w)
        hi = lo
    return np.concatenate(T), np.concatenate(Wt)


def lagrange_basis(nodes: np.ndarray, t: np.ndarray) -> np.ndarray:
    """L_j(t) = prod_{m != j} (t - t_m) / (t_j - t_m); returns (len(t), len(nodes))."""
    out = np.ones((t.size, nodes.size))
    for j in range(nodes.size):
        for m in range(nodes.size):
            if m != j:
                out[:, j] *= (t - nodes[m]) / (nodes[j] - nodes[m])
    return out


def near_panel_entries(rg: Rings, i: int, b: int, k: float, eta: float, M: int) -> np.ndarray:
    """(M+1, p) entries K_p(i, j), j on panel b, by product integration."""
    pc, ta, tb = rg.curve.panels[b]
    tstar = _closest_parameter(rg, i, b)
    H1, W1 = graded_mesh(ta - tstar)
    H2, W2 = graded_mesh(tb - tstar)
    h = np.concatenate([H1, H2])
    wt = np.concatenate([W1, W2])
    t = tstar + h
    r, z, dr, dz = rg.curve.eval(pc, t)
    sp = np.hypot(dr, dz)
    nr, nz = -dz / sp, dr / sp
    if int(rg.panel[i]) == b:
        # the target is the curve point at t*: offsets without cancellation
        offr, offz = rg.curve.delta(pc, tstar, h)
    else:
        offr, offz = r - rg.r[i], z - rg.z[i]
    modes = modes_graded(rg.r[i], r, offr, offz, nr, nz, k, eta, M)      # (S, M+1)
    cols = rg.panel_nodes(b)
    Lb = lagrange_basis(rg.t[cols], t)                                    # (S, p)
    return np.einsum("s,sj,sp->pj", wt * r * sp, Lb, modes)


def _modal_row(rg: Rings, i: int, k: float, eta: float, M: int) -> np.ndarray:
    """Row i of K_p for p = 0..M as (M+1, N_G): far panels by the trapezoid rule of
    C3 (Eq. (nystromnaive) per mode), near panels by product integration (C4)."""
    row = np.zeros((M + 1, rg.n), dtype=np.complex128)
    nb = near_panels(rg, i)
    far = np.nonzero(~np.isin(rg.panel, nb))[0]
    if far.size:
        md = _modes_trapezoid(rg, i, far, k, eta, M)
        row[:, far] = (md * (rg.r[far] * rg.ds[far])[:, None]).T
    for b in nb:
        row[:, rg.panel_nodes(b)] = near_panel_entries(rg, i, b, k, eta, M)
    return row


def modal_matrices(rg: Rings, k: float, eta: float, M: Optional[int] = None) -> np.ndarray:
    """K_p for p = 0..M as an (M+1, N_G, N_G) complex array (row i depends only on
    target ring i)."""
    if M is None:
        M = (rg.shape.n_modes - 1) // 2
    K = np.zeros((M + 1, rg.n, rg.n), dtype=np.complex128)
    for i in range(rg.n):
        K[:, i, :] = _modal_row(rg, i, k, eta, M)
    return K


def modal_system(rg: Rings, k: float, eta: float, M: Optional[int] = None) -> np.ndarray:
    """A~_p = 1/2 I + K_p, p = 0..M."""
    K = modal_matrices(rg, k, eta, M)
    K[:, np.arange(rg.n), np.arange(rg.n)] += 0.5
    return K


def scattering_matrices(A: np.ndarray) -> np.ndarray:
    """S_p = A~_p^{-1} (LU with partial pivoting, library routine)."""
    return np.linalg.inv(A)


_CACHE: Dict[tuple, np.ndarray] = {}


def cached_scattering(rg: Rings, k: float, eta: float) -> np.ndarray:
    key = (rg.shape, float(k), float(eta))
    if key not in _CACHE:
        _CACHE[key] = scattering_matrices(modal_system(rg, k, eta))
    return _CACHE[key]


def modal_rows(rg: Rings, rows, k: float, eta: float, M: Optional[int] = None) -> np.ndarray:
    """Rows i in `rows` of A~_p = 1/2 I + K_p for p = 0..M, as (M+1, len(rows), N_G):
    the rows modal_system builds (same per-row routine), computed only for the
    requested targets."""
    if M is None:
        M = (rg.shape.n_modes - 1) // 2
    rows = np.atleast_1d(rows)
    out = np.zeros((M + 1, rows.size, rg.n), dtype=np.complex128)
    for a, i in enumerate(rows):
        out[:, a, :] = _modal_row(rg, int(i), k, eta, M)
        out[:, a, int(i)] += 0.5
    return out
