"""Body-partitioned solve of the preconditioned system (Sec. 4, Eq. (precond)) on
several ranks, one GPU per rank.

The operator z = sigma + D^{-1} B sigma splits by bodies: D is block diagonal (one
block per body, Sec. 3.2), and the rows of B sigma that belong to the bodies of a
rank need every source but only that rank's targets (Sec. 3.3, Eq. (nystromnaive)).
So each rank owns a contiguous range of bodies (their nodes, their densities, their
rows of the Krylov basis), and one GMRES iteration has exactly two exchange steps:

  * all-gather of sigma (every rank's owned rows) before the inter-body sum;
  * all-reduce (sum) of the Gram-Schmidt dot products and of the norms, per Arnoldi
    step; the Hessenberg matrix, its Givens rotations and the least-squares update are
    then identical on every rank (replicated, not communicated).

The bodies are split into contiguous ranges that balance the inter-body pair work
sum_q n_q (N - n_q) of the owned targets (D^{-1} is a small part of an apply).

The rank-local pieces are supplied by a `LocalOperator`: `LibraryOperator` runs them
in the library's CUDA kernels (the inter-body sum of the owned bodies' targets
through hzb_interbody_bodies, D^{-1} through hzb_local_inverse); tests supply an
oracle-backed one on CPU ranks.  The Krylov vector algebra of this driver (dot
products, axpy) runs in the array library of the vectors it is given (torch on the
GPU, numpy on CPU ranks).  The exchange uses torch.distributed (NCCL between GPUs,
gloo on CPU), launched one process per GPU by torchrun.
"""
from __future__ import annotations

import abc
from typing import List, Sequence, Tuple

import numpy as np


def partition_bodies(sizes: Sequence[int], world: int) -> List[Tuple[int, int]]:
    """Contiguous body ranges [begin, end) for `world` ranks that balance the pair work
    w_q = n_q (N - n_q) of the owned targets: the largest rank share is minimised over
    all contiguous splits (binary search on the share, greedy check).  Ranks beyond the
    body count get empty ranges."""
    sizes = [int(n) for n in sizes]
    N = sum(sizes)
    w = [n * (N - n) for n in sizes]
    m = len(w)
    if world < 1:
        raise ValueError("world must be >= 1")

    def split(cap):
        out, b = [], 0
        while b < m:
            e, s = b, 0
            while e < m and (s + w[e] <= cap or e == b):
                s += w[e]
                e += 1
            out.append((b, e))
            b = e
        return out

    lo, hi = max(w) if w else 0, sum(w)
    while lo < hi:
        mid = (lo + hi) // 2
        if len(split(mid)) <= world:
            hi = mid
        else:
            lo = mid + 1
    parts = split(lo) if m else []
    while len(parts) < world:
        parts.append((m, m))
    return parts


def row_ranges(sizes: Sequence[int], parts: Sequence[Tuple[int, int]]) -> List[Tuple[int, int]]:
    """Node rows [r0, r1) of each rank's body range (bodies are numbered in node order)."""
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(int)
    return [(int(offs[b]), int(offs[e])) for b, e in parts]


class RankFailure(RuntimeError):
    """A collective of the partitioned solve failed: a peer rank left (raised, exited or
    was killed between steps) or the process group's timeout ran out.  Raised on every
    surviving rank at its next exchange, so no rank waits forever on a dead peer; the
    solve cannot continue without that rank's bodies."""


class Exchange:
    """The two collectives of the partitioned solve, on torch.distributed.  A failed
    collective (a peer gone, or the group's timeout: pass a short `timeout` to
    init_process_group to bound the wait) surfaces as RankFailure naming the step."""

    def __init__(self, dist, rows: Sequence[Tuple[int, int]]):
        self.dist = dist
        self.rows = list(rows)
        self.rank = dist.get_rank()
        self.world = dist.get_world_size()

    def _collective(self, what, fn, *args):
        try:
            fn(*args)
        except Exception as e:          # the backend's error type differs (gloo, NCCL)
            raise RankFailure("%s failed on rank %d of %d: %s" % (what, self.rank, self.world, e)) from e

    def allgather_rows(self, local):
        """Full N x R array from every rank's owned rows (rank order = row order).  The
        collective moves equal-size blocks, so each rank's rows are padded to the largest
        share and the padding is dropped after the gather."""
        import torch
        is_np = isinstance(local, np.ndarray)
        t = torch.from_numpy(np.ascontiguousarray(local)) if is_np else local.contiguous()
        R = t.shape[1]
        counts = [r1 - r0 for r0, r1 in self.rows]
        mx = max(counts)
        send = t.new_zeros((mx, R))
        send[: t.shape[0]] = t
        parts = [t.new_zeros((mx, R)) for _ in counts]
        if t.is_complex():                    # the collectives move real views of the complex data
            self._collective("all-gather of sigma", self.dist.all_gather, [torch.view_as_real(p) for p in parts],
                             torch.view_as_real(send))
        else:
            self._collective("all-gather of sigma", self.dist.all_gather, parts, send)
        full = torch.cat([p[:n] for p, n in zip(parts, counts)], 0)
        return full.numpy() if is_np else full

    def allreduce_sum(self, a):
        """Sum over ranks of a small array (dot products, norms), in place for torch."""
        import torch
        is_np = isinstance(a, np.ndarray)
        t = torch.from_numpy(np.ascontiguousarray(a)) if is_np else a
        if t.is_complex():
            self._collective("all-reduce of dot products", self.dist.all_reduce, torch.view_as_real(t))
        else:
            self._collective("all-reduce of dot products", self.dist.all_reduce, t)
        return t.numpy() if is_np else t


class LocalOperator(abc.ABC):
    """Rank-local pieces of Eq. (precond): `rows` = (r0, r1) owned node rows;
    apply_local(sigma_full) = rows r0:r1 of sigma + D^{-1} B sigma;
    rhs_local(v_local) = rows r0:r1 of -D^{-1} v (v given on the owned rows only,
    which suffices because D^{-1} is block diagonal)."""
    rows: Tuple[int, int]

    @abc.abstractmethod
    def apply_local(self, sigma_full):
        ...

    @abc.abstractmethod
    def rhs_local(self, v_local):
        ...


def _vdot_cols(a, b):
    """Per-column inner products sum_i conj(a_i) b_i of N x R arrays (numpy or torch)."""
    return (a.conj() * b).sum(0)


def gmres_distributed(op: LocalOperator, ex: Exchange, b_local, tol: float, maxit: int = 500):
    """GMRES on the owned rows (Sec. 4): zero initial guess, classical Gram-Schmidt
    applied twice (CGS2) with the dot products all-reduced, Givens rotations and the
    residual estimate replicated on every rank, stop on the preconditioned relative
    residual per right-hand side.  b_local: n_local x R.  Returns (x_local, iterations,
    converged, final relative residual estimates)."""
    is_np = isinstance(b_local, np.ndarray)
    lib = np if is_np else __import__("torch")
    R = b_local.shape[1]

    def host(v):
        return np.asarray(v) if is_np else v.detach().cpu().numpy()

    def dev(v, like):
        return v if is_np else lib.as_tensor(v, dtype=like.dtype, device=like.device)

    bn = np.sqrt(np.maximum(host(ex.allreduce_sum(_vdot_cols(b_local, b_local))).real, 0.0))
    if not np.all(np.isfinite(bn)):
        raise FloatingPointError("non-finite right-hand side")
    m = maxit
    V = [b_local / dev(np.where(bn > 0, bn, 1.0), b_local)]
    H = np.zeros((m + 1, m, R), dtype=np.complex128)
    cs = np.zeros((m, R), dtype=np.complex128)
    sn = np.zeros((m, R), dtype=np.complex128)
    g = np.zeros((m + 1, R), dtype=np.complex128)
    g[0] = bn
    active = bn > 0
    jdone = np.zeros(R, dtype=int)
    rel = np.where(bn > 0, 1.0, 0.0)
    for j in range(m):
        if not active.any():
            break
        w = op.apply_local(ex.allgather_rows(V[j]))
        h = np.zeros((j + 1, R), dtype=np.complex128)
        for _ in range(2):                                       # CGS2
            Vj = lib.stack(V[: j + 1], 0)                         # (j+1) x n x R
            c = host(ex.allreduce_sum((Vj.conj() * w[None]).sum(1)))
            w = w - (Vj * dev(c, w)[:, None, :]).sum(0)
            h += c
        hn = np.sqrt(np.maximum(host(ex.allreduce_sum(_vdot_cols(w, w))).real, 0.0))
        if not np.all(np.isfinite(hn)) or not np.all(np.isfinite(h)):
            raise FloatingPointError("non-finite Arnoldi vector")
        H[: j + 1, j] = h
        H[j + 1, j] = hn
        for i in range(j):                                       # previous rotations
            t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
            H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + np.conj(cs[i]) * H[i + 1, j]
            H[i, j] = t
        a, b = H[j, j].copy(), H[j + 1, j].copy()
        den = np.sqrt(np.abs(a) ** 2 + np.abs(b) ** 2)
        cs[j] = np.where(den > 0, np.conj(a) / np.where(den > 0, den, 1), 1.0)
        sn[j] = np.where(den > 0, np.conj(b) / np.where(den > 0, den, 1), 0.0)
        H[j, j] = cs[j] * a + sn[j] * b
        H[j + 1, j] = 0.0
        g[j + 1] = np.where(active, -np.conj(sn[j]) * g[j], g[j + 1])
        g[j] = np.where(active, cs[j] * g[j], g[j])
        rel = np.where(active, np.abs(g[j + 1]) / np.where(bn > 0, bn, 1), rel)
        jdone = np.where(active, j + 1, jdone)
        active = active & (rel > tol) & (hn > 1e-300)
        # a converged right-hand side is frozen: its next basis vectors are zero
        V.append(w * dev(np.where(active, 1.0 / np.where(hn > 0, hn, 1.0), 0.0), w))
    x = b_local * 0
    for r in range(R):                                           # per right-hand side: y = H^{-1} g
        n = int(jdone[r])
        if n == 0:
            continue
        y = np.linalg.solve(np.triu(H[:n, :n, r]), g[:n, r])
        for i in range(n):
            x[:, r] = x[:, r] + V[i][:, r] * dev(np.asarray(y[i]), b_local)
    return x, int(jdone.max()), bool(np.all(rel <= tol)), rel


class LibraryOperator(LocalOperator):
    """Rank-local operator on the library's kernels: a Solver holding every body (the
    geometry is replicated; each rank builds the scattering matrices of all shapes) of
    which this rank owns bodies [b0, b1).  Vectors are torch CUDA tensors."""

    def __init__(self, solver, body_range: Tuple[int, int], rows: Tuple[int, int], precision: int = 0):
        self.s = solver
        self.b0, self.b1 = body_range
        self.rows = rows
        self.precision = precision

    def _full(self, local):
        import torch
        full = torch.zeros((self.s.N, local.shape[1]), dtype=local.dtype, device=local.device)
        full[self.rows[0]:self.rows[1]] = local
        return full

    def apply_local(self, sigma_full):
        r0, r1 = self.rows
        y = self.s.interbody_bodies(sigma_full, self.b0, self.b1, precision=self.precision)
        tau = self.s.local_inverse(self._full(y), precision=self.precision)
        return sigma_full[r0:r1] + tau[r0:r1]

    def rhs_local(self, v_local):
        r0, r1 = self.rows
        return -self.s.local_inverse(self._full(v_local))[r0:r1]


def solve_partitioned(op: LocalOperator, ex: Exchange, v_local, tol: float, maxit: int = 500):
    """sigma (owned rows) of Eq. (precond) for data v (owned rows, n_local x R)."""
    return gmres_distributed(op, ex, op.rhs_local(v_local), tol, maxit)
