"""Edge cases of the hot path through the C ABI: the smallest discretisation (one panel
of two Gauss-Legendre nodes, N_F = 3), many bodies whose node count is below one
warp and one source tile (every kernel's ragged paths), every inter-body engine
against the oracle there; empty requests and out-of-range engine selectors are
refused with HZB_EINVAL."""
import numpy as np
import pytest

import workloads as W
from tests._common import gpu_solver, rand_c, rel_l2, require_gpu

pytestmark = pytest.mark.gpu


def _tiny_many(n_bodies=5):
    """n_bodies spheres of 1 panel x 2 GL nodes x 3 azimuthal nodes (6 nodes each) and
    one spheroid of 2 x 3 x 5 (30 nodes), on a line with gap > 1."""
    sph = W.ShapeSpec(W.SPHERE, (0.5,), 1, 2, 3)
    spd = W.ShapeSpec(W.SPHEROID, (0.4, 0.8), 2, 3, 5)
    bodies = [W.Body(sph, np.array([2.2 * q, 0.1 * q, -0.05 * q]), np.eye(3)) for q in range(n_bodies)]
    bodies.append(W.Body(spd, np.array([-2.5, 0.3, 0.2]), W.rotation_taking_z_to([0.2, 1.0, 0.1])))
    return W.Workload("tiny_many", bodies, 2.0, 2.0, np.array([[0.0, 0.0, 1.0]]))


@pytest.fixture(scope="module")
def tiny():
    require_gpu()
    from oracle import Problem
    wl = _tiny_many()
    return gpu_solver(wl), Problem(wl)


@pytest.mark.parametrize("engine", [0, 1])
@pytest.mark.parametrize("R", [1, 3, 6, 20])
def test_fp64_and_double_float_engines_on_tiny_bodies(tiny, R, engine):
    s, P = tiny
    sig = rand_c((P.N, R), 191 + R)
    ref = P.interbody(sig)
    s.set_fp64_interbody_engine(engine)
    try:
        y64 = s.interbody(sig)
        ydf = s.interbody(sig, precision=2)
    finally:
        s.set_fp64_interbody_engine(-1)
    scale = np.abs(ref).max()
    assert np.abs(y64 - ref).max() < 1e-12 * scale
    assert np.abs(ydf - ref).max() < 1e-12 * scale


@pytest.mark.parametrize("engine", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("R", [1, 5, 17])
def test_fp32_engines_on_tiny_bodies(tiny, R, engine):
    s, P = tiny
    sig = rand_c((P.N, R), 201 + R)
    ref = P.interbody(sig)
    s.set_interbody_engine(engine)
    try:
        got = s.interbody(sig, precision=1)
    finally:
        s.set_interbody_engine(-1)
    assert rel_l2(got, ref) < 5e-6


@pytest.mark.parametrize("R", [5, 17])
def test_single_term_tf32_engine_on_tiny_bodies(tiny, R):
    """Engine 7: tcgen05 with TF32 products and no hi/lo split; its own bar, set by the
    2^-11 rounding of both factors (measured ~3e-4 on the eight spheroids)."""
    s, P = tiny
    sig = rand_c((P.N, R), 211 + R)
    ref = P.interbody(sig)
    s.set_interbody_engine(7)
    try:
        got = s.interbody(sig, precision=1)
    finally:
        s.set_interbody_engine(-1)
    assert rel_l2(got, ref) < 2e-3


def test_solve_on_tiny_bodies(tiny):
    s, P = tiny
    from oracle import fields, gmres
    wl = _tiny_many()
    st = s.solve_plane_waves(wl.directions)
    v = fields.plane_wave(P.nodes.x, wl.directions, wl.k)[:, 0]
    ref = gmres(P.apply, P.rhs(v), 1e-13).x
    assert st.converged
    assert rel_l2(s.get_density()[:, 0], ref) < 1e-10


def test_empty_requests_and_bad_selectors_are_refused(tiny):
    from paper_1406_0236_gb300 import HzbError
    s, P = tiny
    for call in (lambda: s.interbody(np.zeros((P.N, 0), complex)),
                 lambda: s.apply(np.zeros((P.N, 0), complex)),
                 lambda: s.solve_plane_waves(np.zeros((0, 3))),
                 lambda: s.set_interbody_engine(8),
                 lambda: s.set_interbody_engine(-2),
                 lambda: s.set_fp64_interbody_engine(3),
                 lambda: s.set_modal_engine(3)):
        with pytest.raises(HzbError) as e:
            call()
        assert e.value.status == -1
    s.solve_plane_waves([[0.0, 0.0, 1.0]])
    with pytest.raises(HzbError) as e:
        s.far_field(np.zeros((0, 3)))
    assert e.value.status == -1
