"""Oracle solvers: GMRES (Saad-Schultz, modified Gram-Schmidt, Givens rotations)
and a dense direct solve of the full Nystrom system.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. 4: GMRES on sigma + D^{-1} B sigma = -D^{-1} v (Eq. (precond)); the paper
stops at a residual of 1e-9 and states neither restart nor orthogonalisation; the
reading used here is a zero initial guess (unless x0 is given), modified
Gram-Schmidt, restart m (None = no restart), and the stopping test
||b - A x|| <= tol ||b|| on the preconditioned system.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, List, Optional

import numpy as np


@dataclass
class GmresResult:
    x: np.ndarray
    iterations: int
    converged: bool
    residuals: List[float] = field(default_factory=list)   # relative residual estimates


def gmres(apply: Callable[[np.ndarray], np.ndarray], b: np.ndarray, tol: float,
          maxit: int = 500, restart: Optional[int] = None, x0: Optional[np.ndarray] = None
          ) -> GmresResult:
    b = np.asarray(b, dtype=np.complex128)
    n = b.size
    x = np.zeros(n, dtype=np.complex128) if x0 is None else np.array(x0, dtype=np.complex128)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return GmresResult(x, 0, True, [0.0])
    m = maxit if restart is None else restart
    hist: List[float] = []
    it = 0
    first = True
    while True:
        r = b.copy() if (first and x0 is None) else b - apply(x)
        first = False
        beta = np.linalg.norm(r)
        hist.append(beta / bnorm)
        if beta <= tol * bnorm:
            return GmresResult(x, it, True, hist)
        if it >= maxit:
            return GmresResult(x, it, False, hist)
        V = np.zeros((m + 1, n), dtype=np.complex128)
        H = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m, dtype=np.complex128)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        V[0] = r / beta
        g[0] = beta
        j_done = 0
        for j in range(m):
            w = apply(V[j])
            for i in range(j + 1):                      # modified Gram-Schmidt
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):                          # previous rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + np.conj(cs[i]) * H[i + 1, j]
                H[i, j] = t
            a, c = H[j, j], H[j + 1, j]                 # rotation zeroing H[j+1, j]
            den = np.sqrt(abs(a) ** 2 + abs(c) ** 2)
            cs[j] = np.conj(a) / den if den else 1.0
            sn[j] = np.conj(c) / den if den else 0.0
            H[j, j] = cs[j] * a + sn[j] * c
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            j_done = j + 1
            hist.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) <= tol * bnorm or it >= maxit or H[j, j] == 0.0:
                break
        y = np.linalg.solve(np.triu(H[:j_done, :j_done]), g[:j_done])
        x = x + V[:j_done].T @ y


def dense_solve(A: np.ndarray, v: np.ndarray) -> np.ndarray:
    """sigma with A sigma = -v (LU with partial pivoting, library routine)."""
    return np.linalg.solve(A, -np.asarray(v, dtype=np.complex128))
