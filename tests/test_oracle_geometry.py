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
