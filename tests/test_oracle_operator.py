"""Pins of the oracle's operator pieces (Sec. 3.3, Sec. 4)."""
import numpy as np
from scipy import special

import workloads as W
from oracle import Problem


def _h0(x):
    return special.spherical_jn(0, x) + 1j * special.spherical_yn(0, x)


def test_direct_sum_uniform_density_closed_form():
    """sigma = 1 on a sphere radiates i k a^2 h_0(k r)[k j_0'(ka) - i eta j_0(ka)]
    outside it (addition theorem, n = 0 term); the inter-body sum evaluates the
    other sphere's field at each node."""
    a, k, eta = 1.0, 2.0, 1.5
    wl = W.two_spheres(n_panels=8, gl_order=10, n_modes=41, k=k, eta=eta, sep=1.5)
    P = Problem(wl)
    y = P.interbody(np.ones(P.N, dtype=complex))
    other = np.where(P.nodes.body == 0, 1, 0)
    centers = np.array([b.center for b in wl.bodies])
    r = np.linalg.norm(P.nodes.x - centers[other], axis=1)
    exact = 1j * k * a * a * _h0(k * r) * (k * special.spherical_jn(0, k * a, derivative=True)
                                           - 1j * eta * special.spherical_jn(0, k * a))
    assert np.abs(y - exact).max() < 1e-10 * np.abs(exact).max()


def test_direct_sum_excludes_own_body_and_is_linear():
    wl = W.tiny_two_spheres()
    P = Problem(wl)
    rng = np.random.default_rng(1)
    s1 = rng.standard_normal(P.N) + 1j * rng.standard_normal(P.N)
    s2 = rng.standard_normal(P.N) + 1j * rng.standard_normal(P.N)
    y = P.interbody(np.stack([s1, s2], 1))
    assert np.allclose(y[:, 0], P.interbody(s1), rtol=0, atol=1e-14 * np.abs(y).max())
    # own-body sources do not contribute
    s3 = s1.copy()
    s3[P.nodes.body == 0] = 0.0
    y3 = P.interbody(s3)
    assert np.abs(y3[P.nodes.body == 1]).max() == 0.0


def test_dft_definition_matches_library_fft():
    nf = 9
    F = Problem.dft_matrix(nf)
    rng = np.random.default_rng(2)
    y = rng.standard_normal(nf) + 1j * rng.standard_normal(nf)
    ref = np.fft.fft(y)                      # index p mod nf
    M = (nf - 1) // 2
    got = F @ y
    for pidx in range(nf):
        assert abs(got[pidx] - ref[(pidx - M) % nf]) < 1e-13
    assert np.allclose(np.conj(F).T @ (F @ y) / nf, y, atol=1e-14)


def test_local_inverse_inverts_block_diagonal():
    wl = W.tiny_two_spheres()
    P = Problem(wl)
    rng = np.random.default_rng(3)
    s = rng.standard_normal(P.N) + 1j * rng.standard_normal(P.N)
    Dq = [P.dense_block_diagonal(q) for q in range(2)]
    Ds = np.concatenate([Dq[q] @ s[sl] for q, sl in enumerate(P.body_slices())])
    assert np.abs(P.local_inverse(Ds) - s).max() < 1e-12 * np.abs(s).max()


def test_dense_matrix_consistent_with_apply():
    wl = W.tiny_two_spheres()
    P = Problem(wl)
    A = P.dense_matrix()
    rng = np.random.default_rng(4)
    s = rng.standard_normal(P.N) + 1j * rng.standard_normal(P.N)
    lhs = P.local_inverse(A @ s)                        # D^{-1} A s = s + D^{-1} B s
    assert np.abs(lhs - P.apply(s)).max() < 1e-11 * np.abs(s).max()
