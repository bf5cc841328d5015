"""The seeded synthetic workloads against the configurations they stand for: body counts
and kinds, sizes, grids, discretisations, node counts, wavenumbers, incident directions,
seeding, and (48-body workload) the surface gaps, measured here by a surface sampler of
this test's own, independent of the generator's."""
import math

import numpy as np
import pytest
from scipy.spatial import cKDTree

import workloads as W


def _surface_points(body, n_t=48, n_phi=48):
    """Points on the body's surface from its generating curve (analytic pieces), in world
    coordinates."""
    s = body.shape
    t = np.linspace(0.0, 1.0, n_t)
    if s.kind == W.SPHERE:
        th = math.pi * t
        r, z = s.params[0] * np.sin(th), s.params[0] * np.cos(th)
    elif s.kind == W.SPHEROID:
        th = math.pi * t
        r, z = s.params[0] * np.sin(th), s.params[1] * np.cos(th)
    else:
        ro, ri, half, rim = s.params
        th_rim = math.pi - half
        th = th_rim * t
        mid = 0.5 * (ro + ri)
        ang = th_rim + math.pi * t                       # rim semicircle, bulging outward
        rr = np.concatenate([ro * np.sin(th), mid * math.sin(th_rim) + rim * np.sin(ang), ri * np.sin(th)])
        zz = np.concatenate([ro * np.cos(th), mid * math.cos(th_rim) + rim * np.cos(ang), ri * np.cos(th)])
        r, z = rr, zz
    ph = 2.0 * math.pi * np.arange(n_phi) / n_phi
    local = np.stack([np.outer(r, np.cos(ph)), np.outer(r, np.sin(ph)), np.outer(z, np.ones(n_phi))], -1)
    return local.reshape(-1, 3) @ np.asarray(body.rot).T + np.asarray(body.center)


def test_two_spheres_is_the_two_sphere_configuration():
    wl = W.two_spheres()
    assert len(wl.bodies) == 2 and wl.n_nodes == 8200
    assert wl.k == 2.0 and wl.eta == 2.0
    for b, x in zip(wl.bodies, (-1.5, 1.5)):
        assert b.shape.kind == W.SPHERE and b.shape.params[0] == 1.0
        assert (b.shape.n_panels, b.shape.gl_order, b.shape.n_modes) == (10, 10, 41)
        assert np.allclose(b.center, [x, 0.0, 0.0])
    assert np.allclose(wl.directions, [[0.0, 0.0, 1.0]])


def test_spheroids8_is_the_eight_spheroid_configuration():
    wl = W.spheroids8()
    assert len(wl.bodies) == 8 and wl.n_nodes == 258560 and wl.k == 4.0 and wl.n_rhs == 1
    cen = np.array([b.center for b in wl.bodies])
    assert np.allclose(np.sort(np.unique(np.round(cen, 9))), [-2.5, 2.5])   # a 2 x 2 x 2 grid of spacing 5
    assert len({tuple(np.round(c, 9)) for c in cen}) == 8
    axes = []
    for b in wl.bodies:
        assert b.shape.kind == W.SPHEROID and tuple(b.shape.params) == (1.0, 2.0)
        assert (b.shape.n_panels, b.shape.gl_order, b.shape.n_modes) == (20, 16, 101)
        R = np.asarray(b.rot)
        assert np.allclose(R.T @ R, np.eye(3), atol=1e-12) and np.linalg.det(R) > 0
        axes.append(R[:, 2])
    assert len({tuple(np.round(a, 6)) for a in axes}) == 8             # seeded, distinct axes
    w2 = W.spheroids8()
    assert all(np.array_equal(a.rot, b.rot) for a, b in zip(wl.bodies, w2.bodies))


def test_mixed27_is_the_27_body_configuration():
    wl = W.mixed27()
    assert len(wl.bodies) == 27 and wl.k == 4.0 and wl.n_rhs == 64 and wl.n_nodes == 750368
    cen = np.array([b.center for b in wl.bodies])
    vals = np.sort(np.unique(np.round(cen, 9)))
    assert np.allclose(vals, [-5.0, 0.0, 5.0])                         # a 3 x 3 x 3 grid of spacing 5
    kinds = [b.shape.kind for b in wl.bodies]
    assert set(kinds) == {W.SPHERE, W.SPHEROID} and 5 <= kinds.count(W.SPHERE) <= 22
    for b in wl.bodies:
        s = b.shape
        if s.kind == W.SPHERE:
            assert 0.5 <= s.params[0] <= 1.5
        else:
            assert s.params[0] == 1.0 and 1.0 <= s.params[1] <= 2.0
        assert 12 <= s.n_panels <= 24 and s.gl_order == 16
        assert s.n_modes % 2 == 1 and 61 <= s.n_modes <= 121
    assert len({b.shape.n_nodes for b in wl.bodies}) > 5                # uneven sizes
    assert np.allclose(np.linalg.norm(wl.directions, axis=1), 1.0)


def test_mixed48_is_the_48_body_configuration_with_unit_gaps():
    wl = W.mixed48()
    assert len(wl.bodies) == 48 and wl.k == 6.0 and wl.n_rhs == 16 and wl.n_nodes == 2230272
    kinds = [b.shape.kind for b in wl.bodies]
    assert kinds.count(W.SPHERE) == kinds.count(W.SPHEROID) == kinds.count(W.OPEN_SHELL) == 16
    for b in wl.bodies:
        assert (b.shape.n_panels, b.shape.gl_order, b.shape.n_modes) == (24, 16, 121)
        if b.shape.kind == W.OPEN_SHELL:
            ro, ri, half, rim = b.shape.params
            assert (ro, ri, rim) == (1.0, 0.8, 0.1) and abs(half - math.pi / 3) < 1e-15
    # centres: the 4 x 4 x 3 grid of spacing 4.5 about the origin, jittered by at most 0.5 per axis
    grid = np.array([[4.5 * (i - 1.5), 4.5 * (j - 1.5), 4.5 * (l - 1.0)]
                     for i in range(4) for j in range(4) for l in range(3)])
    cen = np.array([b.center for b in wl.bodies])
    assert np.abs(cen - grid).max() <= 0.5
    # surface gaps >= 1, measured on this test's own surface samples (spacing ~0.07 on the
    # largest body, so a sampled distance is at most ~0.05 above the true one)
    pts = [_surface_points(b) for b in wl.bodies]
    trees = [cKDTree(p) for p in pts]
    rad = [b.shape.bounding_radius() for b in wl.bodies]
    worst = np.inf
    for a in range(48):
        for b in range(a + 1, 48):
            if np.linalg.norm(cen[a] - cen[b]) - rad[a] - rad[b] > 1.5:
                continue
            d, _ = trees[b].query(pts[a], k=1)
            worst = min(worst, d.min())
    assert worst >= 0.95, worst


@pytest.mark.parametrize("n", [1, 64, 4096])
def test_uniform_directions_are_seeded_unit_vectors(n):
    d = W.uniform_directions(n, 20140602)
    assert d.shape == (n, 3) and np.allclose(np.linalg.norm(d, axis=1), 1.0)
    assert np.array_equal(d, W.uniform_directions(n, 20140602))
    if n >= 4096:
        assert np.abs(d.mean(0)).max() < 0.05                            # uniform on the sphere
        assert abs(np.mean(d[:, 2] ** 2) - 1.0 / 3.0) < 0.02
