"""Saving and loading the per-shape modal matrices (Sec. 3.2: the precomputation
depends only on the shape and the wavenumber): a context that loads them solves like
one that built them, also with the bodies moved; mismatched files are refused."""
import numpy as np
import pytest

import workloads as W
from tests._common import gpu_solver, rel_l2, require_gpu

pytestmark = pytest.mark.gpu


def _moved(wl, shift):
    bodies = [W.Body(b.shape, b.center + np.asarray(shift) * (q + 1), b.rot) for q, b in enumerate(wl.bodies)]
    return W.Workload(wl.name + "_moved", bodies, wl.k, wl.eta, wl.directions)


def test_load_equals_build(tmp_path):
    require_gpu()
    from paper_1406_0236_gb300 import Options, Solver
    wl = W.tiny_two_spheres()
    built = gpu_solver(wl)
    path = str(tmp_path / "scat.bin")
    built.save_scattering(path)
    loaded = Solver.from_workload(wl, Options(precision=0, gmres_tol=1e-12))
    loaded.load_scattering(path)
    for body, b in enumerate(wl.bodies):
        ng = b.shape.n_panels * b.shape.gl_order
        for p in (0, 3):
            for which in (0, 1):
                assert np.array_equal(built.get_modal_block(body, p, which, ng),
                                      loaded.get_modal_block(body, p, which, ng)), (body, p, which)
    built.solve_plane_waves(wl.directions)
    loaded.solve_plane_waves(wl.directions)
    assert rel_l2(loaded.get_density(), built.get_density()) < 1e-13


def test_load_with_moved_bodies(tmp_path):
    """The matrices of a shape serve any placement: load them into moved bodies and
    compare with a build for the moved geometry."""
    require_gpu()
    from paper_1406_0236_gb300 import Options, Solver
    wl = W.tiny_two_spheres()
    path = str(tmp_path / "scat.bin")
    gpu_solver(wl).save_scattering(path)
    mv = _moved(wl, [0.3, -0.2, 0.5])
    fresh = gpu_solver(mv)
    loaded = Solver.from_workload(mv, Options(precision=0, gmres_tol=1e-12))
    loaded.load_scattering(path)
    fresh.solve_plane_waves(mv.directions)
    loaded.solve_plane_waves(mv.directions)
    assert rel_l2(loaded.get_density(), fresh.get_density()) < 1e-12


def test_load_refuses_mismatch(tmp_path):
    require_gpu()
    from paper_1406_0236_gb300 import HzbError, Options, Solver
    wl = W.tiny_two_spheres()
    path = str(tmp_path / "scat.bin")
    s = gpu_solver(wl)
    s.save_scattering(path)
    with pytest.raises(HzbError):                         # already built
        s.load_scattering(path)
    other_k = W.Workload("k", wl.bodies, wl.k * 1.5, wl.eta, wl.directions)
    t = Solver.from_workload(other_k, Options(precision=0))
    with pytest.raises(HzbError):                         # other wavenumber
        t.load_scattering(path)
    bad = tmp_path / "bad.bin"
    bad.write_bytes(b"not a file of this library")
    u = Solver.from_workload(wl, Options(precision=0))
    with pytest.raises(HzbError):
        u.load_scattering(str(bad))
    u.load_scattering(path)                               # a refused load left the context usable


def test_skeletons_saved_and_restored(tmp_path):
    """The accelerated scheme's skeletons travel with the matrices: a loaded context
    solves the reduced system like the compressing one; moved so close that the saved
    proxy sphere no longer separates the bodies, the skeletons are left out and the
    direct solve runs."""
    require_gpu()
    from paper_1406_0236_gb300 import Options, Solver
    wl = W.separated_spheroids(spacing=4.0, n_panels=6, gl_order=8, n_modes=21)
    s = gpu_solver(wl, precision=0, tol=1e-12)
    s.compress(1e-10)
    path = str(tmp_path / "scat_skel.bin")
    s.save_scattering(path)
    s.solve_plane_waves(wl.directions)
    ref = s.get_density().copy()
    loaded = Solver.from_workload(wl, Options(precision=0, gmres_tol=1e-12))
    loaded.load_scattering(path)
    assert loaded.reduced_size == s.reduced_size
    J0, T0 = s.get_skeleton(0)
    J1, T1 = loaded.get_skeleton(0)
    assert np.array_equal(J0, J1) and np.array_equal(T0, T1)
    loaded.solve_plane_waves(wl.directions)
    assert rel_l2(loaded.get_density(), ref) < 1e-13
    # bodies pushed together: the proxy sphere of the file would cut a neighbour
    close = [W.Body(b.shape, b.center * 0.55, b.rot) for b in wl.bodies]
    cw = W.Workload("close", close, wl.k, wl.eta, wl.directions)
    t = Solver.from_workload(cw, Options(precision=0, gmres_tol=1e-12))
    t.load_scattering(path)
    assert t.reduced_size == 0 and t.get_skeleton(0) is None
    t.solve_plane_waves(cw.directions)
    fresh = gpu_solver(cw, precision=0, tol=1e-12)
    fresh.solve_plane_waves(cw.directions)
    assert rel_l2(t.get_density(), fresh.get_density()) < 1e-12


def test_saved_skeletons_carry_eps_and_caller_skeletons_their_arrangement(tmp_path):
    """Version-4 files: a computed skeleton is restored with the tolerance it was computed
    for; a skeleton the caller set is restored only into the arrangement it was set for."""
    require_gpu()
    from paper_1406_0236_gb300 import Options, Solver
    wl = W.separated_spheroids(spacing=4.0, n_panels=6, gl_order=8, n_modes=21)
    s = gpu_solver(wl, precision=0, tol=1e-12)
    s.compress(1e-9)
    k, eps, rho = s.get_skeleton_info(0)
    assert k > 0 and eps == 1e-9 and rho > 0
    path = str(tmp_path / "computed.bin")
    s.save_scattering(path)
    t = Solver.from_workload(wl, Options(precision=0, gmres_tol=1e-12))
    t.load_scattering(path)
    assert t.get_skeleton_info(0) == (k, 1e-9, rho)
    # the caller's skeleton (the computed one, given back by hand)
    J, T = s.get_skeleton(0)
    u = gpu_solver(wl, precision=0, tol=1e-12)
    u.set_skeleton(0, J, T)
    assert u.get_skeleton_info(0) == (J.size, 0.0, 0.0)
    path2 = str(tmp_path / "caller.bin")
    u.save_scattering(path2)
    same = Solver.from_workload(wl, Options(precision=0, gmres_tol=1e-12))
    same.load_scattering(path2)
    assert same.get_skeleton_size(0) == J.size
    moved = [W.Body(b.shape, b.center + np.array([0.0, 0.0, 0.5]), b.rot) for b in wl.bodies]
    mw = W.Workload("moved", moved, wl.k, wl.eta, wl.directions)
    other = Solver.from_workload(mw, Options(precision=0, gmres_tol=1e-12))
    other.load_scattering(path2)
    assert other.get_skeleton_size(0) == 0 and other.reduced_size == 0
