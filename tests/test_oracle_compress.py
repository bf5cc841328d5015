"""Pins of the oracle's accelerated scheme (Sec. 5, Eqs. (ip0)-(ip6)) against what
the mathematics fixes, independently of the proxy construction where it matters:

  * the ID of an exactly low-rank matrix recovers its rank and reproduces it;
  * with eps = 0 on a full-rank proxy matrix every node is a skeleton node, and the
    reduced system's solution is the uncompressed one (the scheme reduces to Eq.
    (precond));
  * Eq. (ip0): each off-diagonal block of the dense Nystrom matrix (brute force) is
    reproduced by U_p A_pq(I_p, I_q) V_q^* to about eps;
  * the compressed solve matches the uncompressed dense solve to about eps, and the
    identity V_p^* sig_p = sig~_p holds for the recovered density;
  * Green's identity: interior point sources' boundary data gives back their field
    outside, through the compressed solve.
"""
import numpy as np
import pytest

import workloads as W
from oracle import Problem, dense_solve, fields
from oracle.compress import Compressed, interpolative_decomposition


@pytest.fixture(scope="module")
def wl():
    # 3 spheroids (0.5, 0.5, 1) of 6 x 8 x 21 = 1,008 nodes, spacing 4, k = 2
    return W.separated_spheroids(spacing=4.0, n_panels=6, gl_order=8, n_modes=21)


@pytest.fixture(scope="module")
def P(wl):
    return Problem(wl)


@pytest.fixture(scope="module")
def dense(P):
    return P.dense_matrix()


def test_id_of_exactly_low_rank_matrix():
    rng = np.random.default_rng(11)
    r = 12
    A = rng.standard_normal((60, r)) + 1j * rng.standard_normal((60, r))
    B = rng.standard_normal((r, 80)) + 1j * rng.standard_normal((r, 80))
    Z = A @ B
    idd = interpolative_decomposition(Z, 1e-12)
    assert idd.rank == r
    assert np.allclose(idd.T[:, idd.J], np.eye(r), atol=0)
    assert np.linalg.norm(Z - Z[:, idd.J] @ idd.T) < 1e-12 * np.linalg.norm(Z)
    # full column rank with eps = 0: every column is kept and T is the identity
    Zf = rng.standard_normal((50, 30)) + 1j * rng.standard_normal((50, 30))
    f = interpolative_decomposition(Zf, 0.0)
    assert f.rank == 30 and sorted(f.J) == list(range(30))
    assert np.array_equal(f.T[:, f.J], np.eye(30)) and np.count_nonzero(f.T) == 30


def test_full_skeleton_reduces_to_uncompressed(P, dense):
    C = Compressed(P, 0.0)
    for shp, idd in C.ids.items():
        assert idd.rank == shp.n_nodes
    v = fields.plane_wave(P.nodes.x, P.wl.directions, P.k)[:, 0]
    sig, res = C.solve(v, 1e-13)
    assert res.converged
    ref = dense_solve(dense, v)
    assert np.linalg.norm(sig - ref) < 1e-11 * np.linalg.norm(ref)


@pytest.mark.parametrize("eps", [1e-6, 1e-10])
def test_off_diagonal_blocks_factor_to_eps(P, dense, eps):
    C = Compressed(P, eps)
    sl = P.body_slices()
    shp = P.wl.bodies[0].shape
    assert C.ids[shp].rank < 0.75 * shp.n_nodes
    T = C.ids[shp].T
    J = C.ids[shp].J
    for p in range(len(sl)):
        for q in range(len(sl)):
            if p == q:
                continue
            A = dense[sl[p], sl[q]]
            approx = T.T @ A[np.ix_(J, J)] @ T
            assert np.linalg.norm(A - approx) < eps * np.linalg.norm(A)


def test_compressed_solve_matches_uncompressed(P, dense):
    eps = 1e-10
    C = Compressed(P, eps)
    v = fields.plane_wave(P.nodes.x, P.wl.directions, P.k)[:, 0]
    sig, res = C.solve(v, 1e-13)
    assert res.converged
    ref = dense_solve(dense, v)
    assert np.linalg.norm(sig - ref) < 10 * eps * np.linalg.norm(ref)
    # V_p^* sig_p = sig~_p for the recovered density
    for q, b, st, sf in C.body_blocks():
        t = C.ids[b.shape].T @ sig[sf]
        assert np.linalg.norm(t - res.x[st]) < 1e-11 * np.linalg.norm(res.x[st])
    # far field from the recovered density
    xh = W.uniform_directions(12, 7)
    uf = fields.far_field(P.nodes, sig, P.k, P.eta, xh)
    ur = fields.far_field(P.nodes, ref, P.k, P.eta, xh)
    assert np.abs(uf - ur).max() < 10 * eps * np.abs(ur).max()


def test_green_identity_through_compressed_solve(wl, P):
    C = Compressed(P, 1e-10)
    src = W.point_sources(wl, 5)
    tg = W.exterior_targets(wl, 10, 6)
    v = -fields.point_source_field(P.nodes.x, src, wl.k)
    sig, res = C.solve(v, 1e-13)
    assert res.converged
    u = fields.field(P.nodes, sig, wl.k, wl.eta, tg)
    ue = fields.point_source_field(tg, src, wl.k)
    assert np.abs(u - ue).max() < 1e-8 * np.abs(ue).max()


def test_fourier_route_to_the_id(P):
    """Reading P21 (the GPU's route to the ID), checked on the mathematics alone: the
    proxy matrix M is block-circulant in the azimuth (each block is (1/N_F) F^* diag(M^_p) F
    with M^_p = M^_{-p}); truncating a pivoted QR of every M^_p at 0.3 eps |M|_col and
    stacking the rows R_p[s, i] e^{-2 pi i p l / N_F} / sqrt(N_F) gives Z with |Zx| ~ |Mx|
    for all x, so the ID of Z reproduces M to about eps."""
    import scipy.linalg as sla
    from oracle.compress import default_proxy_radius, proxy_matrix, proxy_sphere, shape_nodes
    shp = P.wl.bodies[0].shape
    rg = P.rings[shp]
    nf, ng = shp.n_modes, rg.n
    nt = max(16, int(np.ceil(1.2 * ng)))
    x, n, w = shape_nodes(rg, nf)
    z, nz = proxy_sphere(nf, default_proxy_radius(P.wl, shp), nt)
    M = proxy_matrix(x, n, w, z, nz, P.k, P.eta)                    # (3 nt nf) x (ng nf)
    # rows (b, r, a), columns (i, l): M[(b, r, a), (i, l)] = f_{b r i}(a - l)
    f = M.reshape(3, nt, nf, ng, nf)[:, :, :, :, 0]                  # l = 0: f(a)
    Mh = np.fft.fft(f, axis=2)                                       # sum_a f(a) e^{-2 pi i p a / nf}
    Mh = np.moveaxis(Mh, 2, 0).reshape(nf, 3 * nt, ng)               # mode index p mod nf
    for p in range(1, (nf - 1) // 2 + 1):
        assert np.allclose(Mh[p], Mh[nf - p], atol=1e-12 * np.abs(Mh).max())
    colmax = np.sqrt((np.abs(M) ** 2).sum(0).max())
    eps = 1e-8
    rows = []
    l = np.arange(nf)
    for p in range(nf):
        _, R, piv = sla.qr(Mh[p], mode="economic", pivoting=True)
        trail = np.array([np.linalg.norm(R[s:, s:], axis=0).max() for s in range(R.shape[0])] + [0.0])
        r = int(np.argmax(trail <= 0.3 * eps * colmax))
        Zp = np.zeros((r, ng), dtype=complex)
        Zp[:, piv] = R[:r]
        ph = np.exp(-2j * np.pi * p * l / nf) / np.sqrt(nf)
        rows.append((Zp[:, :, None] * ph[None, None, :]).reshape(r, ng * nf))
    Z = np.vstack(rows)
    assert Z.shape[0] < 0.8 * M.shape[1]
    g = np.random.default_rng(2)
    X = g.standard_normal((M.shape[1], 6)) + 1j * g.standard_normal((M.shape[1], 6))
    nm, nzx = np.linalg.norm(M @ X, axis=0), np.linalg.norm(Z @ X, axis=0)
    assert np.abs(nm - nzx).max() < 1e-3 * eps * colmax * np.linalg.norm(X, axis=0).max()
    from oracle.compress import interpolative_decomposition
    idd = interpolative_decomposition(Z, eps)
    err = np.linalg.norm(M - M[:, idd.J] @ idd.T, 2)
    assert err < 3 * eps * np.linalg.norm(M, 2)


@pytest.mark.parametrize("kind,q", [("sphere", 1), ("shell", 3), ("spline", 1)])
def test_factorisation_for_other_shape_kinds(kind, q):
    """Eq. (ip0) on the dense blocks for the other generating curves: a sphere, an open
    shell (whose cavity lies inside the proxy sphere with the body) and a spline pear.
    The shell at N_F = 17 needs the proxy sampled at 3 N_F azimuths (q = 3): at N_F
    azimuths its off-diagonal blocks keep an error floor near 1e-6."""
    import math
    if kind == "sphere":
        shp = W.ShapeSpec(W.SPHERE, (0.8,), 5, 8, 17)
    elif kind == "shell":
        shp = W.ShapeSpec(W.OPEN_SHELL, (1.0, 0.8, math.radians(60.0), 0.1), 12, 6, 17)
    else:
        pts = W.pear_curve(7)
        shp = W.ShapeSpec(W.CURVE_SPLINE, pts, 6, 8, 17)
    rot = [W.rotation_taking_z_to(a) for a in ([0.3, 0.2, 1.0], [1.0, -0.4, 0.2], [-0.2, 1.0, 0.5])]
    cen = [np.array([0.0, 0.0, 0.0]), np.array([4.2, 0.5, -0.3]), np.array([1.5, 3.9, 0.8])]
    wl = W.Workload(kind, [W.Body(shp, c, r) for c, r in zip(cen, rot)], 2.0, 2.0, np.array([[0.0, 0.0, 1.0]]))
    P = Problem(wl)
    D = P.dense_matrix()
    sl = P.body_slices()

    def worst(C):
        idd = C.ids[shp]
        w = 0.0
        for p in range(3):
            for r in range(3):
                if p != r:
                    A = D[sl[p], sl[r]]
                    w = max(w, np.linalg.norm(A - idd.T.T @ A[np.ix_(idd.J, idd.J)] @ idd.T) / np.linalg.norm(A))
        return idd.rank, w

    eps = 1e-9
    rank, err = worst(Compressed(P, eps, q=q))
    assert rank < shp.n_nodes and err < eps, (kind, rank, err)
    if kind == "shell":
        assert worst(Compressed(P, eps, q=1))[1] > 100 * eps     # the floor that q = 3 removes


def test_fourier_route_with_offset_proxy_rings():
    """The route of reading P21 with the proxy sampled at 3 N_F azimuths (q = 3): the
    points fall in three classes of N_F azimuths offset by 0, +1/3 and +2/3 (= -1/3 of the
    next) of the azimuthal step, each class block-circulant; M^_{-p} and M^_p then have the
    same Gram matrix (the +-1/3 classes trade places), so one pivoted QR per |p| still
    gives Z with |Zx| ~ |Mx|, and the ID of Z meets eps on the open shell where q = 1 does
    not."""
    import math
    import scipy.linalg as sla
    from oracle.compress import default_proxy_radius, interpolative_decomposition, proxy_matrix, proxy_sphere, \
        shape_nodes
    shp = W.ShapeSpec(W.OPEN_SHELL, (1.0, 0.8, math.radians(60.0), 0.1), 12, 6, 17)
    rot = [W.rotation_taking_z_to(a) for a in ([0.3, 0.2, 1.0], [1.0, -0.4, 0.2], [-0.2, 1.0, 0.5])]
    cen = [np.array([0.0, 0.0, 0.0]), np.array([4.2, 0.5, -0.3]), np.array([1.5, 3.9, 0.8])]
    wl = W.Workload("shell", [W.Body(shp, c, r) for c, r in zip(cen, rot)], 2.0, 2.0, np.array([[0.0, 0.0, 1.0]]))
    P = Problem(wl)
    rg = P.rings[shp]
    nf, ng, q = shp.n_modes, rg.n, 3
    nt = max(16, int(np.ceil(1.2 * ng)))
    x, n, w = shape_nodes(rg, nf)
    z, nz = proxy_sphere(nf, default_proxy_radius(wl, shp), nt, q)
    M = proxy_matrix(x, n, w, z, nz, P.k, P.eta)                       # rows (blk, r, b), b < q nf
    f = M.reshape(3, nt, q * nf, ng, nf)[:, :, :, :, 0]                # node azimuth l = 0
    f = f.reshape(3, nt, nf, q, ng)                                     # b = q a + t
    Mh = np.fft.fft(f, axis=2)                                          # DFT over a, per class t
    Mh = np.moveaxis(Mh, 2, 0).reshape(nf, 3 * nt * q, ng)
    for p in range(1, (nf - 1) // 2 + 1):                              # same Gram matrix for +-p
        G1, G2 = Mh[p].conj().T @ Mh[p], Mh[nf - p].conj().T @ Mh[nf - p]
        assert np.abs(G1 - G2).max() < 1e-11 * np.abs(G1).max()
    colmax = np.sqrt((np.abs(M) ** 2).sum(0).max())
    eps = 1e-9
    l = np.arange(nf)
    rows = []
    for p in range(nf):
        pp = p if p <= (nf - 1) // 2 else nf - p                         # one QR per |p|
        _, R, piv = sla.qr(Mh[pp], mode="economic", pivoting=True)
        trail = np.array([np.linalg.norm(R[s:, s:], axis=0).max() for s in range(R.shape[0])] + [0.0])
        r = int(np.argmax(trail <= 0.3 * eps * colmax))
        Zp = np.zeros((r, ng), dtype=complex)
        Zp[:, piv] = R[:r]
        ph = np.exp(-2j * np.pi * p * l / nf) / np.sqrt(nf)
        rows.append((Zp[:, :, None] * ph[None, None, :]).reshape(r, ng * nf))
    Z = np.vstack(rows)
    g = np.random.default_rng(3)
    X = g.standard_normal((M.shape[1], 6)) + 1j * g.standard_normal((M.shape[1], 6))
    nm, nzx = np.linalg.norm(M @ X, axis=0), np.linalg.norm(Z @ X, axis=0)
    assert np.abs(nm - nzx).max() < 1e-3 * eps * colmax * np.linalg.norm(X, axis=0).max()
    idd = interpolative_decomposition(Z, eps)
    D = P.dense_matrix()
    sl = P.body_slices()
    for a in range(3):
        for b in range(3):
            if a != b:
                A = D[sl[a], sl[b]]
                assert np.linalg.norm(A - idd.T.T @ A[np.ix_(idd.J, idd.J)] @ idd.T) < eps * np.linalg.norm(A)
