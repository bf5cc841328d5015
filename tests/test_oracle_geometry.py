"""Pins of the oracle's geometry against closed forms (Sec. 3.2 tensor-product rule)."""
import numpy as np
import pytest

import workloads as W
from oracle import gauss_legendre, near_panels, rings, surface_nodes
from oracle.geometry import shell_panel_split


@pytest.mark.parametrize("n", [4, 10, 16])
def test_gauss_legendre_exact_to_degree_2n_minus_1(n):
    x, w = gauss_legendre(n)
    for deg in range(2 * n):
        exact = 0.0 if deg % 2 else 2.0 / (deg + 1)
        assert abs((w * x ** deg).sum() - exact) < 1e-14
    # and not exact one degree higher
    deg = 2 * n
    assert abs((w * x ** deg).sum() - 2.0 / (deg + 1)) > 1e-11


def _integrals(shape):
    body = W.Body(shape, np.array([0.3, -0.2, 0.5]), W.rotation_taking_z_to([1.0, 2.0, 0.5]))
    nd = surface_nodes([body])
    area = nd.w.sum()
    nsum = (nd.n * nd.w[:, None]).sum(0)
    vol = ((nd.x - body.center) * nd.n * nd.w[:, None]).sum() / 3.0
    return area, nsum, vol


def test_sphere_area_volume():
    a = 1.3
    area, nsum, vol = _integrals(W.ShapeSpec(W.SPHERE, (a,), 8, 10, 17))
    assert abs(area - 4 * np.pi * a * a) < 1e-12
    assert np.abs(nsum).max() < 1e-12
    assert abs(vol - 4 * np.pi * a ** 3 / 3) < 1e-12      # outward normals


def test_prolate_spheroid_area_volume():
    a, c = 1.0, 2.0
    area, nsum, vol = _integrals(W.ShapeSpec(W.SPHEROID, (a, c), 12, 12, 21))
    e = np.sqrt(1 - a * a / (c * c))
    exact = 2 * np.pi * a * a * (1 + c / (a * e) * np.arcsin(e))
    assert abs(area - exact) < 1e-11
    assert np.abs(nsum).max() < 1e-11
    assert abs(vol - 4 * np.pi * a * a * c / 3) < 1e-11


def test_open_shell_area_volume():
    Ro, Ri, half, rho = 1.0, 0.8, np.pi / 3, 0.1
    area, nsum, vol = _integrals(W.ShapeSpec(W.OPEN_SHELL, (Ro, Ri, half, rho), 24, 12, 21))
    th = np.pi - half
    cr = 0.5 * (Ro + Ri) * np.sin(th)
    er = np.cos(th)
    caps = 2 * np.pi * (Ro ** 2 + Ri ** 2) * (1 - np.cos(th))
    rim = 2 * np.pi * (np.pi * rho * cr + 2 * rho * rho * er)           # Pappus
    assert abs(area - (caps + rim)) < 1e-11
    assert np.abs(nsum).max() < 1e-11
    v_sector = 2 * np.pi / 3 * (Ro ** 3 - Ri ** 3) * (1 - np.cos(th))
    v_rim = 2 * np.pi * (cr + 4 * rho / (3 * np.pi) * er) * (np.pi * rho * rho / 2)   # Pappus
    assert abs(vol - (v_sector + v_rim)) < 1e-11


def test_shell_panel_split_is_proportional_with_two_on_rim():
    th = 2 * np.pi / 3
    assert shell_panel_split(24, th, 0.1 * np.pi, 0.8 * th) == (12, 2, 10)
    assert shell_panel_split(9, th, 0.1 * np.pi, 0.8 * th)[1] == 2


def test_node_layout_ring_major_azimuth_fastest():
    shape = W.ShapeSpec(W.SPHERE, (1.0,), 3, 4, 7)
    nd = surface_nodes([W.Body(shape, np.zeros(3), np.eye(3))])
    rg = rings(shape)
    x = nd.x.reshape(rg.n, 7, 3)
    assert np.allclose(x[:, 0, 1], 0.0)                      # theta_0 = 0 on the body x axis
    assert np.allclose(x[:, :, 2], rg.z[:, None])
    th = np.arctan2(x[2, :, 1], x[2, :, 0]) % (2 * np.pi)
    assert np.allclose(th, 2 * np.pi * np.arange(7) / 7)


def test_near_sets_contain_self_and_neighbours():
    rg = rings(W.ShapeSpec(W.SPHERE, (1.0,), 10, 10, 41))
    for i in range(rg.n):
        nb = near_panels(rg, i)
        b = int(rg.panel[i])
        assert b in nb
        for a in (b - 1, b + 1):
            if 0 <= a < 10:
                assert a in nb
        # on a uniformly paneled sphere the next-but-one panel is beyond one panel length
        assert all(abs(q - b) <= 1 for q in nb)


def test_rotation_takes_ez_to_axis():
    rng = np.random.default_rng(0)
    for a in list(rng.standard_normal((20, 3))) + [np.array([0, 0, -1.0]), np.array([0, 0, 1.0])]:
        R = W.rotation_taking_z_to(a)
        assert np.allclose(R.T @ R, np.eye(3), atol=1e-14)
        assert abs(np.linalg.det(R) - 1) < 1e-14
        assert np.allclose(R[:, 2], a / np.linalg.norm(a), atol=1e-14)


def _sphere_points(n):
    th = np.linspace(0.0, np.pi, n)
    rz = np.stack([np.sin(th), np.cos(th)], axis=1)
    rz[0, 0] = rz[-1, 0] = 0.0
    return rz


def test_spline_curve_interpolates_with_pole_conditions():
    """The spline pieces pass through the points, r'' = 0 and z' = 0 at both poles, and
    value, first and second derivative are continuous at the joints."""
    from oracle.geometry import spline_pieces
    rz = np.asarray(W.pear_curve(11)).reshape(-1, 2)
    pcs = spline_pieces(rz)
    for k, (pc, t0, t1) in enumerate(pcs):
        r0, z0, _, _ = pc.eval(np.array(t0))
        r1, z1, _, _ = pc.eval(np.array(t1))
        assert abs(r0 - rz[k, 0]) < 1e-14 and abs(z0 - rz[k, 1]) < 1e-14
        assert abs(r1 - rz[k + 1, 0]) < 1e-13 and abs(z1 - rz[k + 1, 1]) < 1e-13
    first, last = pcs[0][0], pcs[-1][0]
    assert abs(first.cr[1]) < 1e-14 and abs(first.cz[2]) < 1e-14          # r''(0) = 0, z'(0) = 0
    u = pcs[-1][2] - pcs[-1][1]
    assert abs(6 * last.cr[0] * u + 2 * last.cr[1]) < 1e-12              # r''(end) = 0
    assert abs(3 * last.cz[0] * u * u + 2 * last.cz[1] * u + last.cz[2]) < 1e-12   # z'(end) = 0
    for (a, _, ta1), (b, tb0, _) in zip(pcs[:-1], pcs[1:]):
        ea, eb = a.eval(np.array(ta1)), b.eval(np.array(tb0))
        assert np.allclose(ea, eb, atol=1e-12)
        # second derivatives r'' and z'' agree at the joint
        ua = ta1 - a.tk
        assert abs((6 * a.cr[0] * ua + 2 * a.cr[1]) - 2 * b.cr[1]) < 1e-10
        assert abs((6 * a.cz[0] * ua + 2 * a.cz[1]) - 2 * b.cz[1]) < 1e-10


def test_spline_surface_rule_integrates_its_own_area():
    """The tensor rule on the spline body integrates the area of that surface of
    revolution, 2 pi int r |gamma'| dt, computed independently by adaptive quadrature
    of scipy's spline objects."""
    from scipy.integrate import quad
    from scipy.interpolate import CubicSpline
    rz = np.asarray(W.pear_curve(13)).reshape(-1, 2)
    t = np.concatenate([[0.0], np.cumsum(np.hypot(np.diff(rz[:, 0]), np.diff(rz[:, 1])))])
    sr = CubicSpline(t, rz[:, 0], bc_type=((2, 0.0), (2, 0.0)))
    sz = CubicSpline(t, rz[:, 1], bc_type=((1, 0.0), (1, 0.0)))
    f = lambda x: 2 * np.pi * sr(x) * np.hypot(sr(x, 1), sz(x, 1))
    exact = sum(quad(f, t[k], t[k + 1], epsabs=0.0, epsrel=1e-13, limit=200)[0] for k in range(t.size - 1))
    shape = W.ShapeSpec(W.CURVE_SPLINE, tuple(rz.reshape(-1)), 12, 10, 9)
    area, nsum, _ = _integrals(shape)
    assert abs(area - exact) < 1e-12 * exact
    assert np.abs(nsum).max() < 1e-12


def test_spline_through_sphere_points_converges_to_the_sphere():
    """Spline curves through points of the unit circle give surfaces whose area tends to
    4 pi at the interpolation order (error / 16 when the point spacing halves)."""
    errs = []
    for n in (17, 33, 65):
        shape = W.ShapeSpec(W.CURVE_SPLINE, tuple(_sphere_points(n).reshape(-1)), n - 1, 8, 9)
        area, _, vol = _integrals(shape)
        errs.append(abs(area - 4 * np.pi))
        assert abs(vol - 4 * np.pi / 3) < 1e-3
    assert errs[1] < errs[0] / 8 and errs[2] < errs[1] / 8
