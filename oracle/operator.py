"""Oracle operator: inter-body direct sum B, block-diagonal inverse D^{-1} via the
azimuthal DFT and the scattering matrices, and the preconditioned apply.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. 4: A = D + B with D = diag(A_11, ..., A_mm); GMRES runs on
    sigma + D^{-1} B sigma = -D^{-1} v                                   (Eq. (precond))
with B's entries B(i, j) = K(x_i, x_j) w_j for nodes on different bodies
(Sec. 3.3, Eq. (nystromnaive)) and A_qq^{-1} = F^* A~^{-1} F (Eq. (singleinverse)),
applied per body as (1) a DFT over the azimuth of each ring, (2) one N_G x N_G
scattering matrix per Fourier mode, (3) the inverse DFT (Remark after Eq. (precond)).

Conventions: node order body-major, ring-major, azimuth fastest; the DFT is
    y^_p(i) = sum_l y(i, l) exp(-2 pi i p l / N_F),     p = -M..M, N_F = 2M + 1,
and its inverse carries 1/N_F.  S_{-p} = S_p.
"""
from __future__ import annotations

from typing import Dict, List

import numpy as np

from workloads import Workload

from . import _native as nat
from .geometry import Rings, SurfaceNodes, rings, surface_nodes
from .modal import cached_scattering


class Problem:
    """Discretised multibody problem built from a Workload (oracle side)."""

    def __init__(self, wl: Workload, scattering: Dict = None):
        self.wl = wl
        self.k, self.eta = float(wl.k), float(wl.eta)
        self.rings: Dict = {}
        self.nodes: SurfaceNodes = surface_nodes(wl.bodies, self.rings)
        self.N = int(self.nodes.w.size)
        self._S = {} if scattering is None else dict(scattering)

    def S(self, shape) -> np.ndarray:
        if shape not in self._S:
            self._S[shape] = cached_scattering(self.rings[shape], self.k, self.eta)
        return self._S[shape]

    def body_slices(self) -> List[slice]:
        o = self.nodes.offsets
        return [slice(int(o[q]), int(o[q + 1])) for q in range(len(self.wl.bodies))]

    # ------------------------------------------------------------------ B
    def interbody(self, sigma: np.ndarray, targets: np.ndarray = None) -> np.ndarray:
        """y = B sigma for sigma of shape (N,) or (N, R); optionally only the rows in
        `targets`."""
        sig = np.asarray(sigma, dtype=np.complex128)
        one = sig.ndim == 1
        sig2 = sig.reshape(self.N, -1)
        R = sig2.shape[1]
        tg = np.arange(self.N, dtype=np.int32) if targets is None else np.asarray(targets, np.int32)
        out = np.zeros(2 * tg.size * R)
        nd = self.nodes
        nat.lib().orc_direct_sum(self.N, nat.dptr(nat.as_f64(nd.x)), nat.dptr(nat.as_f64(nd.n)),
                                 nat.dptr(nat.as_f64(nd.w)), nat.iptr(np.ascontiguousarray(nd.body)),
                                 R, nat.dptr(nat.as_c128_view(sig2)), self.k, self.eta,
                                 int(tg.size), nat.iptr(np.ascontiguousarray(tg)), nat.dptr(out))
        y = out.view(np.complex128).reshape(tg.size, R)
        return y[:, 0] if one else y

    # ------------------------------------------------------------------ D^{-1}
    @staticmethod
    def dft_matrix(nf: int) -> np.ndarray:
        """F[p_index, l] = exp(-2 pi i p l / N_F) for p = -M..M (the definition)."""
        M = (nf - 1) // 2
        p = np.arange(-M, M + 1)
        return np.exp(-2j * np.pi * np.outer(p, np.arange(nf)) / nf)

    def local_inverse(self, y: np.ndarray) -> np.ndarray:
        """tau = D^{-1} y, per body F^{-1} diag(S_|p|) F."""
        y2 = np.asarray(y, dtype=np.complex128).reshape(self.N, -1)
        out = np.zeros_like(y2)
        for q, sl in enumerate(self.body_slices()):
            shp = self.wl.bodies[q].shape
            nf, ng = shp.n_modes, self.rings[shp].n
            M = (nf - 1) // 2
            S = self.S(shp)
            F = self.dft_matrix(nf)
            Finv = np.conj(F).T / nf
            yb = y2[sl].reshape(ng, nf, -1)                     # (ring, azimuth, rhs)
            yh = np.einsum("pl,ilr->pir", F, yb)                # (mode, ring, rhs)
            th = np.empty_like(yh)
            for pidx in range(nf):
                th[pidx] = S[abs(pidx - M)] @ yh[pidx]
            out[sl] = np.einsum("lp,pir->ilr", Finv, th).reshape(ng * nf, -1)
        return out.reshape(np.shape(y))

    def apply(self, sigma: np.ndarray) -> np.ndarray:
        """z = sigma + D^{-1} B sigma."""
        return np.asarray(sigma) + self.local_inverse(self.interbody(sigma))

    def rhs(self, v: np.ndarray) -> np.ndarray:
        """b = -D^{-1} v."""
        return -self.local_inverse(v)

    # ------------------------------------------------------------------ dense
    def dense_block_diagonal(self, q: int) -> np.ndarray:
        """A_qq as an n x n matrix: A((i,l),(j,m)) = (1/N_F) sum_p A~_p(i,j) e^{ip(th_l - th_m)}."""
        shp = self.wl.bodies[q].shape
        nf, ng = shp.n_modes, self.rings[shp].n
        M = (nf - 1) // 2
        A = np.linalg.inv(self.S(shp))                         # A~_p, p = 0..M
        F = self.dft_matrix(nf)
        Finv = np.conj(F).T / nf
        full = np.zeros((ng, nf, ng, nf), dtype=np.complex128)
        for pidx in range(nf):
            ap = A[abs(pidx - M)]
            full += np.einsum("l,ij,m->iljm", Finv[:, pidx], ap, F[pidx, :])
        return full.reshape(ng * nf, ng * nf)

    def dense_matrix(self) -> np.ndarray:
        """The full N x N Nystrom matrix A = D + B (Eq. (blocksystem))."""
        nd = self.nodes
        A = interaction_block(nd.x, nd.x, nd.n, nd.w, self.k, self.eta, same=True)
        for q, sl in enumerate(self.body_slices()):
            A[sl, sl] = self.dense_block_diagonal(q)
        return A


def interaction_block(xt: np.ndarray, xs: np.ndarray, ns: np.ndarray, ws: np.ndarray, k: float, eta: float,
                      same: bool = False) -> np.ndarray:
    """K(x_i, y_j) w_j for targets xt and sources (xs, ns, ws): the entries of B
    (Sec. 3.3, Eq. (nystromnaive)), K(x, y) = dphi/dn(y) - i eta phi.  same = True
    when targets and sources are one node set: the diagonal is then evaluated at
    distance 1 and the caller overwrites it."""
    d = xt[:, None, :] - xs[None, :, :]                       # x_i - y_j
    R = np.sqrt((d * d).sum(-1))
    if same:
        np.fill_diagonal(R, 1.0)
    phi = np.exp(1j * k * R) / (4.0 * np.pi * R)
    n_dot_ymx = -(ns[None, :, :] * d).sum(-1)
    K = phi * (1j * k - 1.0 / R) * n_dot_ymx / R - 1j * eta * phi
    return K * ws[None, :]


def problem(wl: Workload) -> Problem:
    return Problem(wl)


def ring_geometry(shape) -> Rings:
    return rings(shape)
