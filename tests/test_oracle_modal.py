"""Pins of the oracle's modal kernels and per-mode matrices (Sec. 3.2).

  * trapezoid modal sums against scipy's adaptive Gauss-Kronrod quadrature;
  * the graded rule against the trapezoid rule (two independent quadratures);
  * the Laplace single-layer modal kernel against its closed form through the
    Legendre function Q_{p-1/2} (toroidal harmonic, hypergeometric series);
  * the per-mode matrices against the exact eigenvalues of the combined-field
    operator on a sphere (spherical harmonics), which checks the near-panel
    product integration, the weights, the normal and the coupling sign together.
"""
import numpy as np
import pytest
from scipy import integrate, special

import oracle._native as nat
import workloads as W
from oracle import fields, rings
from oracle.modal import modal_rows, modal_system, modes_graded, modes_trapezoid_at


def _quad_mode(r, rs, dr, dz, nr, nz, k, eta, p):
    out = np.zeros(2)
    L = nat.lib()

    def f(psi, part):
        L.orc_kernel_ring(r, rs, dr, dz, nr, nz, psi, k, eta, nat.dptr(out))
        v = (out[0] + 1j * out[1]) * np.exp(1j * p * psi)
        return v.real if part == 0 else v.imag
    kw = dict(epsabs=1e-14, epsrel=1e-14, limit=400)
    return integrate.quad(f, 0, 2 * np.pi, args=(0,), **kw)[0] + \
        1j * integrate.quad(f, 0, 2 * np.pi, args=(1,), **kw)[0]


@pytest.mark.parametrize("case", [(0.7, 0.9, 0.3, 0.6, 0.8, 3.0, 3.0),
                                  (1.2, 0.4, -0.5, -0.28, 0.96, 6.0, -6.0),
                                  (0.05, 0.3, 0.9, 1.0, 0.0, 2.0, 2.0)])
def test_trapezoid_matches_library_quadrature(case):
    r, rs, dz, nr, nz, k, eta = case
    M = 12
    md, _ = modes_trapezoid_at(r, rs, rs - r, dz, nr, nz, k, eta, M)
    scale = np.abs(md).max()
    for p in (0, 1, 5, 12):
        q = _quad_mode(r, rs, rs - r, dz, nr, nz, k, eta, p)
        assert abs(md[0, p] - q) < 1e-13 * scale


@pytest.mark.parametrize("d,tol", [(0.5, 2e-13), (1e-2, 2e-13), (1e-4, 1e-12)])
def test_graded_matches_trapezoid(d, tol):
    """Nearly touching rings need ~1e5 trapezoid samples, whose summation rounding
    sets the looser tolerance of the last case."""
    r, nr, nz, k, eta = 0.7, 0.6, 0.8, 3.0, 3.0
    M = 20
    dr, dz = 0.6 * d, -0.8 * d
    md, _ = modes_trapezoid_at(r, r + dr, dr, dz, nr, nz, k, eta, M)
    mg = modes_graded(r, r + dr, dr, dz, nr, nz, k, eta, M)
    assert np.abs(md - mg).max() < tol * np.abs(md).max()


def test_laplace_single_layer_closed_form():
    # k = 0 and zero normal: K = -i eta / (4 pi R); its modal kernel is
    # -i eta / (4 pi) * 2 Q_{p-1/2}(chi) / sqrt(r r'),  chi = (r^2 + r'^2 + dz^2) / (2 r r').
    r, rs, dz, eta = 0.7, 0.9, 0.3, 1.0
    M = 12
    md, _ = modes_trapezoid_at(r, rs, rs - r, dz, 0.0, 0.0, 0.0, eta, M)
    chi = (r * r + rs * rs + dz * dz) / (2 * r * rs)
    for p in range(M + 1):
        Q = (np.sqrt(np.pi) * special.gamma(p + 0.5) / (special.gamma(p + 1) * (2 * chi) ** (p + 0.5))
             * special.hyp2f1((2 * p + 3) / 4, (2 * p + 1) / 4, p + 1, 1 / chi ** 2))
        closed = -1j * eta / (4 * np.pi) * 2 * Q / np.sqrt(r * rs)
        assert abs(md[0, p] - closed) < 1e-14 * abs(md[0, 0])


@pytest.mark.parametrize("k,eta", [(2.0, 2.0), (2.0, -2.0), (0.5, 1.0)])
def test_sphere_eigenvalues(k, eta):
    """A~_m applied to P_n^m(cos t) sampled at the ring nodes is lambda_n P_n^m."""
    a = 1.0
    rg = rings(W.ShapeSpec(W.SPHERE, (a,), 8, 10, 13))
    A = modal_system(rg, k, eta)
    ct = np.cos(rg.t)
    for m in (0, 1, 2, 5):
        for n in (m, m + 1, m + 2):
            P = special.lpmv(m, n, ct)
            lam = fields.sphere_eigenvalue(n, a, k, eta)
            err = np.abs(A[m] @ P - lam * P).max() / np.abs(lam * P).max()
            assert err < 1e-11, (m, n, err)


def test_modal_rows_pinned_by_sphere_eigenvalues():
    """modal_rows on its own (the checker of the full-size setup tests): its rows of
    A~_m, applied to P_n^m(cos t) at the ring nodes, give lambda_n P_n^m at those rows,
    the exact sphere eigenvalue; a dropped 1/2 I, a wrong near-panel set or a wrong
    weight moves the result by far more than the tolerance."""
    a, k, eta = 1.0, 2.0, 2.0
    rg = rings(W.ShapeSpec(W.SPHERE, (a,), 8, 10, 13))
    rows = np.array([0, 9, 33, 79])
    Ar = modal_rows(rg, rows, k, eta)
    ct = np.cos(rg.t)
    for m in (0, 2, 6):
        for n in (m, m + 1):
            P = special.lpmv(m, n, ct)
            lam = fields.sphere_eigenvalue(n, a, k, eta)
            err = np.abs(Ar[m] @ P - lam * P[rows]).max() / np.abs(lam * P).max()
            assert err < 1e-11, (m, n, err)


@pytest.mark.parametrize("spec", [W.ShapeSpec(W.SPHEROID, (1.0, 2.0), 4, 6, 9),
                                  W.ShapeSpec(W.OPEN_SHELL, (1.0, 0.8, np.pi / 3, 0.1), 6, 5, 9)])
def test_modal_rows_equal_modal_system_rows(spec):
    """The requested rows of modal_system, with the 1/2 on the diagonal, for a
    spheroid and an open shell (where the near-panel set crosses the rim)."""
    k, eta = 3.0, 3.0
    rg = rings(spec)
    A = modal_system(rg, k, eta)
    rows = np.array([0, rg.n // 3, rg.n - 1])
    Ar = modal_rows(rg, rows, k, eta)
    assert Ar.shape == (A.shape[0], rows.size, rg.n)
    assert np.abs(Ar - A[:, rows, :]).max() <= 1e-15 * np.abs(A).max()
