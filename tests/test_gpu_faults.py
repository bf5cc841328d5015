"""Failure detection through the C ABI, with every fault made on the host (no GPU
fault, trap or hang): HZB_ENAN from NaN data, a NaN guess and an injected NaN right-hand
side; HZB_ENOMEM from injected allocation failures; HZB_EINVAL from intersecting or
nested bodies, a non-finite centre and an injected invalid node; HZB_ETIMEOUT from the
tcgen05 inter-body kernel's bounded-wait exit, entered through a flag the host sets
before the launch (the kernel leaves before issuing any MMA).  After each one the
context (or a new one) still solves correctly."""
import numpy as np
import pytest

import workloads as W
from tests._common import gpu_solver, rand_c, rel_l2, require_gpu

pytestmark = pytest.mark.gpu

ENOMEM, EINVAL, ENAN, ETIMEOUT = -2, -1, -5, -6


def _err():
    from paper_1406_0236_gb300 import HzbError
    return HzbError


def _plane_wave_data(s, wl):
    x, _, _ = s.get_nodes()
    return np.exp(1j * wl.k * (x @ wl.directions.T))


@pytest.mark.parametrize("precision", [0, 1])
def test_nan_in_data_and_guess_gives_enan(precision):
    require_gpu()
    wl = W.tiny_two_spheres()
    s = gpu_solver(wl, precision=precision, tol=1e-10)
    v = _plane_wave_data(s, wl)
    ok = s.solve_data(v)
    assert ok.converged
    ref = s.get_density().copy()
    bad = v.copy()
    bad[7, 0] = np.nan
    with pytest.raises(_err()) as e:
        s.solve_data(bad)
    assert e.value.status == ENAN
    x0 = np.zeros_like(v)
    x0[3, 0] = np.inf
    with pytest.raises(_err()) as e:
        s.solve_data(v, x0=x0)
    assert e.value.status == ENAN
    s.solve_data(v)                                  # the context still solves
    assert rel_l2(s.get_density(), ref) < 1e-8


def test_injected_nan_rhs(monkeypatch):
    require_gpu()
    monkeypatch.setenv("HZB_FAULT", "nan")
    wl = W.tiny_two_spheres()
    s = gpu_solver(wl, precision=0, tol=1e-12)
    with pytest.raises(_err()) as e:
        s.solve_plane_waves(wl.directions)
    assert e.value.status == ENAN
    st = s.solve_plane_waves(wl.directions)          # one-shot: the next solve is clean
    assert st.converged
    monkeypatch.delenv("HZB_FAULT")
    s2 = gpu_solver(wl, precision=0, tol=1e-12)
    s2.solve_plane_waves(wl.directions)
    assert rel_l2(s.get_density(), s2.get_density()) < 1e-12


def test_injected_allocation_failure(monkeypatch):
    require_gpu()
    from paper_1406_0236_gb300 import Options, Solver
    monkeypatch.setenv("HZB_FAULT", "alloc")
    wl = W.tiny_two_spheres()
    s = Solver.from_workload(wl, Options(precision=0))
    with pytest.raises(_err()) as e:
        s.build_scattering_matrices()
    assert e.value.status == ENOMEM
    s.close()
    monkeypatch.delenv("HZB_FAULT")
    s2 = gpu_solver(wl)                              # a new context allocates normally
    assert s2.solve_plane_waves(wl.directions).converged


def test_injected_invalid_node(monkeypatch):
    require_gpu()
    from paper_1406_0236_gb300 import Options, Solver
    monkeypatch.setenv("HZB_FAULT", "geom")
    wl = W.tiny_two_spheres()
    s = Solver.from_workload(wl, Options(precision=0, gmres_tol=1e-12))
    with pytest.raises(_err()) as e:
        s.build_scattering_matrices()
    assert e.value.status == EINVAL and "invalid" in str(e.value)
    s.build_scattering_matrices()                    # one-shot: regenerated nodes are valid
    assert s.solve_plane_waves(wl.directions).converged


@pytest.mark.parametrize("case", ["intersecting", "nested", "shell_wall"])
def test_overlapping_bodies_are_refused(case):
    require_gpu()
    from paper_1406_0236_gb300 import Options, Solver
    ball = W.ShapeSpec(W.SPHERE, (1.0,), 4, 6, 9)
    small = W.ShapeSpec(W.SPHERE, (0.3,), 4, 6, 9)
    shell = W.ShapeSpec(W.OPEN_SHELL, (1.0, 0.8, np.pi / 3, 0.1), 6, 5, 9)
    if case == "intersecting":
        bodies = [W.Body(ball, np.zeros(3), np.eye(3)), W.Body(ball, np.array([1.5, 0.2, 0.0]), np.eye(3))]
    elif case == "nested":
        bodies = [W.Body(ball, np.zeros(3), np.eye(3)), W.Body(small, np.array([0.2, 0.1, -0.3]), np.eye(3))]
    else:       # a small sphere cut by the wall of a shell (wall between radii 0.8 and 1)
        bodies = [W.Body(shell, np.zeros(3), np.eye(3)), W.Body(small, np.array([0.0, 0.0, 0.9]), np.eye(3))]
    wl = W.Workload("overlap", bodies, 1.0, 1.0, np.array([[0, 0, 1.0]]))
    s = Solver.from_workload(wl, Options(precision=0))
    with pytest.raises(_err()) as e:
        s.build_scattering_matrices()
    assert e.value.status == EINVAL and "overlap" in str(e.value)


def test_body_inside_a_shell_cavity_is_accepted():
    """A sphere in the cavity of an open shell (fluid) does not touch the wall."""
    require_gpu()
    shell = W.ShapeSpec(W.OPEN_SHELL, (1.0, 0.8, np.pi / 3, 0.1), 6, 5, 9)
    small = W.ShapeSpec(W.SPHERE, (0.3,), 4, 6, 9)
    bodies = [W.Body(shell, np.zeros(3), np.eye(3)), W.Body(small, np.zeros(3), np.eye(3))]
    wl = W.Workload("cavity", bodies, 1.0, 1.0, np.array([[0, 0, 1.0]]))
    s = gpu_solver(wl, tol=1e-10)
    assert s.solve_plane_waves(wl.directions).converged


def test_non_finite_centre_is_refused():
    require_gpu()
    from paper_1406_0236_gb300 import Options, Solver
    s = Solver(1.0, 1.0, Options())
    with pytest.raises(_err()) as e:
        s.add_body(W.SPHERE, (1.0,), 4, 6, 9, np.array([np.nan, 0.0, 0.0]), np.eye(3))
    assert e.value.status == EINVAL


def test_tcgen05_timeout_exit_reports_etimeout(monkeypatch):
    require_gpu()
    monkeypatch.setenv("HZB_FAULT", "timeout")
    wl = W.tiny_two_spheres()
    s = gpu_solver(wl)
    s.set_interbody_engine(5)
    sig = rand_c((s.N, 16), 61)
    with pytest.raises(_err()) as e:
        s.interbody(sig, precision=1)
    assert e.value.status == ETIMEOUT
    y = s.interbody(sig, precision=1)              # flag cleared: the context still works
    monkeypatch.delenv("HZB_FAULT")
    ref = gpu_solver(wl).interbody(sig, precision=0)
    assert rel_l2(y, ref) < 5e-6
