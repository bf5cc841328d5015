"""GPU parity of the setup (Sec. 3.2): surface rule, per-mode matrices A~_p and
scattering matrices S_p, against the oracle on the same shapes."""
import numpy as np
import pytest

import workloads as W
from tests._common import gpu_solver, rel_l2, require_gpu

pytestmark = pytest.mark.gpu

SHAPES = {
    "sphere": W.ShapeSpec(W.SPHERE, (1.0,), 6, 8, 13),
    "spheroid": W.ShapeSpec(W.SPHEROID, (1.0, 2.0), 7, 8, 15),
    "shell": W.ShapeSpec(W.OPEN_SHELL, (1.0, 0.8, np.pi / 3, 0.1), 9, 8, 13),
    "spline": W.ShapeSpec(W.CURVE_SPLINE, W.pear_curve(11), 10, 8, 13),
}


def _single(shape, k=2.0, eta=2.0, rot=None):
    rot = np.eye(3) if rot is None else rot
    return W.Workload("one", [W.Body(shape, np.array([0.2, -0.1, 0.3]), rot)], k, eta, np.array([[0, 0, 1.0]]))


@pytest.mark.parametrize("name", list(SHAPES))
def test_surface_rule_matches_oracle(name):
    require_gpu()
    from oracle import surface_nodes
    wl = _single(SHAPES[name], rot=W.rotation_taking_z_to([0.3, -0.4, 0.8]))
    s = gpu_solver(wl)
    x, n, w = s.get_nodes()
    nd = surface_nodes(wl.bodies)
    assert np.abs(x - nd.x).max() < 1e-13
    assert np.abs(n - nd.n).max() < 1e-13
    assert np.abs(w - nd.w).max() < 1e-14


@pytest.mark.parametrize("name", list(SHAPES))
@pytest.mark.parametrize("k,eta", [(2.0, 2.0), (4.0, -4.0)])
def test_modal_and_scattering_matrices_match_oracle(name, k, eta):
    require_gpu()
    from oracle import rings
    from oracle.modal import modal_system
    shape = SHAPES[name]
    s = gpu_solver(_single(shape, k, eta))
    rg = rings(shape)
    A = modal_system(rg, k, eta)
    S = np.linalg.inv(A)
    M = (shape.n_modes - 1) // 2
    for p in range(M + 1):
        Ag = s.get_modal_block(0, p, 0, rg.n)
        Sg = s.get_modal_block(0, p, 1, rg.n)
        assert np.abs(Ag - A[p]).max() < 1e-11 * np.abs(A[p]).max(), p
        assert rel_l2(Sg, S[p]) < 1e-11, p


def test_sphere_eigenvalues_on_device():
    """A~_m P_n^m = lambda_n P_n^m for the GPU's own matrices (closed form)."""
    require_gpu()
    from scipy import special
    from oracle import fields, rings
    shape = W.ShapeSpec(W.SPHERE, (1.0,), 8, 10, 13)
    k, eta = 2.0, 2.0
    s = gpu_solver(_single(shape, k, eta))
    rg = rings(shape)
    ct = np.cos(rg.t)
    for m in (0, 2, 5):
        A = s.get_modal_block(0, m, 0, rg.n)
        for n in (m, m + 1, m + 2):
            P = special.lpmv(m, n, ct)
            lam = fields.sphere_eigenvalue(n, 1.0, k, eta)
            assert np.abs(A @ P - lam * P).max() < 1e-11 * np.abs(lam * P).max()


def test_repeated_shapes_share_matrices():
    require_gpu()
    wl = W.two_spheres(n_panels=4, gl_order=6, n_modes=9)
    s = gpu_solver(wl)
    a = s.get_modal_block(0, 3, 1, 24)
    b = s.get_modal_block(1, 3, 1, 24)
    assert np.array_equal(a, b)
