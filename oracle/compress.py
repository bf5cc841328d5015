"""Oracle of the accelerated scheme: interpolative decomposition (ID) of each shape's
interactions with everything outside a proxy sphere, and the reduced system.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. 5 (Eqs. (ip0)-(ip6)): every off-diagonal block factors as
    A_pq = U_p A~_pq V_q^* + R_pq,      ||R_pq|| <= eps,
where an interpolative decomposition makes U_p(I_p, :) = V_p(I_p, :) = I_k for one
skeleton index set I_p, so A~_pq = A_pq(I_p, I_q) is a submatrix of B.  With
    sig~_p = V_p^* sig_p,   v~_p = V_p^* A_pp^{-1} v_p,   S_p = V_p^* A_pp^{-1} U_p
the preconditioned system becomes  sig~ + S B~ sig~ = -v~  (Eq. (ip6)).

The steps, in the paper's order:
  1. U_p, V_p from a local procedure independent of the other bodies: a basis of all
     fields the body radiates to, and receives from, the region outside a proxy
     sphere around it (the representation technique the first bullet after Eq. (ip6)
     names).  Outgoing: the combined-field potential of each node at proxy points,
     K(z, y_j) w_j.  Incoming: fields inside the sphere are fixed by single- and
     double-layer sources on it, so G(x_i, z) and dG/dn_z(x_i, z) at the nodes.
  2. The ID of the stacked matrix (one index set for both directions, as the second
     bullet after Eq. (ip6) has U and V share I_p): column-pivoted QR, a library
     primitive, Z P = Q R; the rank k counts |R_jj| > eps |R_11|; T = [I, R11^{-1} R12]
     in the original column order, so Z ~ Z(:, J) T with T(:, J) = I.
     Then V_p^* = T (outgoing: K(., y) W ~ K(., y_J) W_J T) and U_p = T^T (incoming:
     any incoming field f on the nodes satisfies f ~ T^T f(J)).
  3. S_p = T A_pp^{-1} T^T and v~_p = T A_pp^{-1} v_p with A_pp^{-1} applied through the
     azimuthal DFT and the scattering matrices (third bullet after Eq. (ip6)).
  4. GMRES on Eq. (ip6); B~ is the direct sum restricted to skeleton nodes.
  5. The density on all nodes (needed for fields; the paper stops at Eq. (ip6)):
     Eq. (ip1) with A_pq sig_q ~ U_p A~_pq sig~_q gives
         sig = D^{-1} (-v - U B~ sig~).

Readings where the paper is silent: the proxy surface is a sphere centred on the
body's centre, radius `rho` (default: midway between the body's bounding radius and
the nearest other body's bounding sphere, over all bodies of that shape), sampled by
`n_theta` Gauss-Legendre rings in cos(theta) times q N_F azimuths (q = 1: the body's own
azimuthal grid); the three blocks are each scaled to unit Frobenius norm before stacking,
so that the tolerance applies to the incoming and outgoing parts alike.  With q = 1 the
proxy sees the outgoing fields only at the body's azimuths; an open shell with N_F = 17
then keeps an error floor near 1e-6 that q = 3 removes (pinned below).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Dict, List

import numpy as np
import scipy.linalg as sla

from workloads import Workload

from . import _native as nat
from .geometry import Rings, gauss_legendre
from .operator import Problem
from .solvers import gmres


def proxy_sphere(n_modes: int, rho: float, n_theta: int, q: int = 1):
    """Points and outward unit normals of the proxy sphere in the body frame:
    rings at Gauss-Legendre nodes of cos(theta), q N_F azimuths 2 pi a / (q N_F) each,
    ring-major with the azimuth fastest (q = 1: the body's own azimuthal grid)."""
    ct, _ = gauss_legendre(n_theta)
    st = np.sqrt(1.0 - ct * ct)
    ph = 2.0 * np.pi * np.arange(q * n_modes) / (q * n_modes)
    u = np.stack([np.outer(st, np.cos(ph)), np.outer(st, np.sin(ph)),
                  np.outer(ct, np.ones(q * n_modes))], axis=-1).reshape(-1, 3)
    return rho * u, u


def shape_nodes(rg: Rings, n_modes: int):
    """Nodes, normals and weights of one body of this shape in its own frame."""
    th = 2.0 * np.pi * np.arange(n_modes) / n_modes
    ct, st = np.cos(th), np.sin(th)
    x = np.stack([rg.r[:, None] * ct, rg.r[:, None] * st,
                  np.broadcast_to(rg.z[:, None], (rg.n, n_modes))], axis=-1).reshape(-1, 3)
    n = np.stack([rg.nr[:, None] * ct, rg.nr[:, None] * st,
                  np.broadcast_to(rg.nz[:, None], (rg.n, n_modes))], axis=-1).reshape(-1, 3)
    w = np.broadcast_to((rg.ds * rg.r * 2.0 * np.pi / n_modes)[:, None], (rg.n, n_modes)).reshape(-1)
    return x, n, w.copy()


def proxy_matrix(x, n, w, z, nz, k: float, eta: float) -> np.ndarray:
    """[K(z, y_j) w_j ; G(x_i, z) ; dG/dn_z(x_i, z)], rows = proxy points, columns =
    body nodes, each block scaled to unit Frobenius norm.
    G(x, y) = e^{ik|x-y|} / (4 pi |x-y|); K(x, y) = dG/dn_y(x, y) - i eta G(x, y)."""
    d = z[:, None, :] - x[None, :, :]                       # z - y
    r = np.sqrt((d * d).sum(-1))
    g = np.exp(1j * k * r) / (4.0 * np.pi * r)
    dg = g * (1j * k - 1.0 / r) / r                         # G'(r) / r
    # dG/dn_y(z, y) = G'(r) n_y . (y - z) / r, and y - z = -d
    out = (dg * (-(n[None, :, :] * d).sum(-1)) - 1j * eta * g) * w[None, :]
    gin = g                                                  # G(x_i, z): symmetric in its arguments
    din = dg * (nz[:, None, :] * d).sum(-1)                  # dG/dn_z(x_i, z) = G'(r) n_z . (z - x) / r
    blocks = [out, gin, din]
    return np.vstack([b / np.linalg.norm(b) for b in blocks])


@dataclass
class ID:
    J: np.ndarray      # (k,) skeleton columns, in pivot order
    T: np.ndarray      # (k, n) with T[:, J] = I and Z ~ Z[:, J] T
    rank: int
    diag: np.ndarray   # |R_jj| of the pivoted QR


def interpolative_decomposition(Z: np.ndarray, eps: float, rank: int = None) -> ID:
    """Column ID from column-pivoted QR (library primitive): Z P = Q R, rank =
    #{j : |R_jj| > eps |R_11|} (or the given rank), T = [I, R11^{-1} R12] P^T."""
    _, R, piv = sla.qr(Z, mode="economic", pivoting=True)
    d = np.abs(np.diag(R))
    k = int((d > eps * d[0]).sum()) if rank is None else int(rank)
    n = Z.shape[1]
    T = np.zeros((k, n), dtype=np.complex128)
    T[:, piv[:k]] = np.eye(k)
    if k < n:
        T[:, piv[k:]] = sla.solve_triangular(R[:k, :k], R[:k, k:n])
    return ID(piv[:k].copy(), T, k, d)


def default_proxy_radius(wl: Workload, shape) -> float:
    """Midway between the shape's bounding radius and the nearest bounding sphere of
    another body, over all bodies of the shape."""
    rb = shape.bounding_radius()
    best = np.inf
    for p, bp in enumerate(wl.bodies):
        if bp.shape != shape:
            continue
        for q, bq in enumerate(wl.bodies):
            if q != p:
                best = min(best, np.linalg.norm(bq.center - bp.center) - bq.shape.bounding_radius())
    if not np.isfinite(best):
        return 1.5 * rb
    if best <= rb * 1.02:
        raise ValueError("bodies too close for a proxy sphere")
    return 0.5 * (rb + best)


class Compressed:
    """The reduced system (Eq. (ip6)) of a Problem."""

    def __init__(self, P: Problem, eps: float, n_theta: int = None, rho: Dict = None,
                 skeletons: Dict = None, q: int = 1):
        self.P = P
        self.eps = eps
        wl = P.wl
        self.ids: Dict = {}
        self.rho: Dict = {}
        for shp in wl.distinct_shapes():
            if skeletons is not None and shp in skeletons:
                J, T = skeletons[shp]
                self.ids[shp] = ID(np.asarray(J), np.asarray(T, dtype=np.complex128), len(J), None)
                continue
            rg = P.rings[shp]
            rho_s = (rho or {}).get(shp, default_proxy_radius(wl, shp))
            nt = n_theta if n_theta is not None else max(16, int(np.ceil(1.2 * rg.n)))
            x, n, w = shape_nodes(rg, shp.n_modes)
            z, nz = proxy_sphere(shp.n_modes, rho_s, nt, q)
            self.rho[shp] = rho_s
            self.ids[shp] = interpolative_decomposition(proxy_matrix(x, n, w, z, nz, P.k, P.eta), eps)
        # skeleton nodes in global numbering, body by body, in each shape's J order
        sl = P.body_slices()
        self.offsets = [0]
        glob = []
        for q, b in enumerate(wl.bodies):
            glob.append(sl[q].start + self.ids[b.shape].J)
            self.offsets.append(self.offsets[-1] + self.ids[b.shape].rank)
        self.glob = np.concatenate(glob).astype(np.int64)
        self.Nk = int(self.glob.size)
        self.S: Dict = {}
        for shp in wl.distinct_shapes():
            T = self.ids[shp].T
            self.S[shp] = T @ self._shape_inverse(shp, T.T)        # S_p = V_p^* A_pp^{-1} U_p

    def _shape_inverse(self, shp, X: np.ndarray) -> np.ndarray:
        """A_pp^{-1} X for a body of this shape (rotation- and translation-invariant),
        via the Problem's block-diagonal inverse on that body's block."""
        P = self.P
        q = next(i for i, b in enumerate(P.wl.bodies) if b.shape == shp)
        s = P.body_slices()[q]
        full = np.zeros((P.N, X.shape[1]), dtype=np.complex128)
        full[s] = X
        return P.local_inverse(full)[s]

    def body_blocks(self):
        for q, b in enumerate(self.P.wl.bodies):
            yield q, b, slice(self.offsets[q], self.offsets[q + 1]), self.P.body_slices()[q]

    def interbody(self, sig_t: np.ndarray) -> np.ndarray:
        """B~ sig~: the inter-body direct sum over skeleton nodes only."""
        nd = self.P.nodes
        g = self.glob
        sig2 = np.ascontiguousarray(np.asarray(sig_t, dtype=np.complex128).reshape(self.Nk, -1))
        R = sig2.shape[1]
        x = np.ascontiguousarray(nd.x[g]); n = np.ascontiguousarray(nd.n[g])
        w = np.ascontiguousarray(nd.w[g]); body = np.ascontiguousarray(nd.body[g]).astype(np.int32)
        tg = np.arange(self.Nk, dtype=np.int32)
        out = np.zeros(2 * self.Nk * R)
        nat.lib().orc_direct_sum(self.Nk, nat.dptr(nat.as_f64(x)), nat.dptr(nat.as_f64(n)),
                                 nat.dptr(nat.as_f64(w)), nat.iptr(body), R,
                                 nat.dptr(nat.as_c128_view(sig2)), self.P.k, self.P.eta,
                                 self.Nk, nat.iptr(tg), nat.dptr(out))
        return out.view(np.complex128).reshape(np.shape(sig_t))

    def local(self, y: np.ndarray) -> np.ndarray:
        """S y, block by block."""
        y2 = np.asarray(y, dtype=np.complex128).reshape(self.Nk, -1)
        out = np.zeros_like(y2)
        for q, b, st, _ in self.body_blocks():
            out[st] = self.S[b.shape] @ y2[st]
        return out.reshape(np.shape(y))

    def apply(self, sig_t: np.ndarray) -> np.ndarray:
        """sig~ + S B~ sig~ (left side of Eq. (ip6))."""
        return np.asarray(sig_t) + self.local(self.interbody(sig_t))

    def rhs(self, v: np.ndarray) -> np.ndarray:
        """-v~ with v~_p = V_p^* A_pp^{-1} v_p."""
        w = self.P.local_inverse(v).reshape(self.P.N, -1)
        out = np.zeros((self.Nk, w.shape[1]), dtype=np.complex128)
        for q, b, st, sf in self.body_blocks():
            out[st] = -(self.ids[b.shape].T @ w[sf])
        return out.reshape((self.Nk,) + np.shape(v)[1:])

    def density(self, sig_t: np.ndarray, v: np.ndarray) -> np.ndarray:
        """sig = D^{-1} (-v - U B~ sig~) on all nodes (Eq. (ip1) with Eq. (ip0))."""
        y = self.interbody(sig_t).reshape(self.Nk, -1)
        u = -np.asarray(v, dtype=np.complex128).reshape(self.P.N, -1).copy()
        for q, b, st, sf in self.body_blocks():
            u[sf] -= self.ids[b.shape].T.T @ y[st]
        return self.P.local_inverse(u).reshape(np.shape(v))

    def solve(self, v: np.ndarray, tol: float):
        """GMRES on Eq. (ip6), then the density on all nodes."""
        res = gmres(self.apply, self.rhs(v), tol)
        return self.density(res.x, v), res
