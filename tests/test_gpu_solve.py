"""GPU solves (Sec. 4 GMRES on Eq. (precond)) against the oracle and physics:
FP64 path <= 1e-10 and mixed path <= 1e-7 relative l2 in density and far field;
Green's identity (Sec. 6 accuracy protocol); Mie series; multi-RHS batches; the
stored oracle far field; error statuses of the C ABI."""
import os

import numpy as np
import pytest

import workloads as W
from tests._common import gpu_solver, rel_l2, require_gpu

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "two_spheres_8200_farfield.txt")


@pytest.fixture(scope="module")
def two_spheres_ref():
    """Oracle reference of the two-sphere 8,200-unknown workload (GMRES to 1e-13)."""
    require_gpu()
    from oracle import Problem, fields, gmres
    wl = W.two_spheres()
    P = Problem(wl)
    v = fields.plane_wave(P.nodes.x, wl.directions, wl.k)[:, 0]
    res = gmres(P.apply, P.rhs(v), 1e-13)
    assert res.converged
    return wl, P, res.x


def test_fp64_solve_matches_oracle(two_spheres_ref):
    from oracle import fields
    wl, P, sig_ref = two_spheres_ref
    s = gpu_solver(wl, precision=0, tol=1e-12)
    st = s.solve_plane_waves(wl.directions)
    assert st.converged and st.rel_residual <= 1e-12
    sig = s.get_density()[:, 0]
    assert rel_l2(sig, sig_ref) <= 1e-10
    xh = W.uniform_directions(12, 5)
    ff = s.far_field(xh)[:, 0]
    assert rel_l2(ff, fields.far_field(P.nodes, sig_ref, wl.k, wl.eta, xh)) <= 1e-10
    gold = np.loadtxt(GOLDEN)
    ffg = s.far_field(gold[:, :3])[:, 0]
    assert rel_l2(ffg, gold[:, 3] + 1j * gold[:, 4]) <= 1e-10


def test_mixed_solve_matches_oracle(two_spheres_ref):
    from oracle import fields
    wl, P, sig_ref = two_spheres_ref
    s = gpu_solver(wl, precision=1, tol=1e-9)
    st = s.solve_plane_waves(wl.directions)
    assert st.converged and st.outer_iterations >= 1
    sig = s.get_density()[:, 0]
    assert rel_l2(sig, sig_ref) <= 1e-7
    xh = W.uniform_directions(12, 6)
    assert rel_l2(s.far_field(xh)[:, 0], fields.far_field(P.nodes, sig_ref, wl.k, wl.eta, xh)) <= 1e-7


def test_green_identity_on_device():
    require_gpu()
    from oracle import fields
    wl = W.two_spheres()
    s = gpu_solver(wl, tol=1e-12)
    x, _, _ = s.get_nodes()
    src = W.point_sources(wl, 5)
    tg = W.exterior_targets(wl, 10, 6)
    v = -fields.point_source_field(x, src, wl.k)
    st = s.solve_data(v)
    assert st.converged
    u = s.eval_field(tg)[:, 0]
    ue = fields.point_source_field(tg, src, wl.k)
    assert np.abs(u - ue).max() / np.abs(ue).max() < 1e-10


def test_green_identity_spline_bodies_on_device():
    """Green's identity (the paper's accuracy test) on two pear-shaped spline bodies and a
    sphere: interior point sources' data are reproduced outside."""
    require_gpu()
    from oracle import fields
    pear = W.ShapeSpec(W.CURVE_SPLINE, W.pear_curve(21), 20, 10, 31)
    ball = W.ShapeSpec(W.SPHERE, (0.7,), 8, 10, 31)
    bodies = [W.Body(pear, np.array([-1.6, 0.0, 0.0]), W.rotation_taking_z_to([0.3, 0.2, 1.0])),
              W.Body(pear, np.array([1.7, 0.2, 0.1]), W.rotation_taking_z_to([-0.5, 1.0, 0.2])),
              W.Body(ball, np.array([0.0, 2.2, -0.3]), np.eye(3))]
    wl = W.Workload("pears", bodies, 2.0, 2.0, np.array([[0, 0, 1.0]]))
    s = gpu_solver(wl, tol=1e-12)
    x, _, _ = s.get_nodes()
    src = np.array([[-1.6, 0.05, 0.1], [1.7, 0.15, 0.05], [0.1, 2.2, -0.3]])
    tg = W.exterior_targets(wl, 10, 6)
    v = -fields.point_source_field(x, src, wl.k)
    st = s.solve_data(v)
    assert st.converged
    u = s.eval_field(tg)[:, 0]
    ue = fields.point_source_field(tg, src, wl.k)
    assert np.abs(u - ue).max() / np.abs(ue).max() < 1e-8


def test_mie_single_sphere_on_device():
    require_gpu()
    from oracle import fields
    sh = W.ShapeSpec(W.SPHERE, (1.0,), 8, 10, 25)
    wl = W.Workload("sphere", [W.Body(sh, np.zeros(3), np.eye(3))], 2.0, 2.0, np.array([[0, 0, 1.0]]))
    s = gpu_solver(wl, tol=1e-12)
    s.solve_plane_waves(wl.directions)
    xh = W.uniform_directions(16, 3)
    mie = fields.mie_far_field(1.0, 2.0, xh[:, 2])
    assert np.abs(s.far_field(xh)[:, 0] - mie).max() < 1e-11 * np.abs(mie).max()


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_rhs_equal_single_solves(precision):
    require_gpu()
    wl = W.two_spheres(n_panels=6, gl_order=8, n_modes=21)
    dirs = W.uniform_directions(5, 9)
    s = gpu_solver(wl, precision=precision, tol=1e-11)
    st = s.solve_plane_waves(dirs)
    assert st.converged
    batch = s.get_density()
    for r in (0, 3):
        s1 = gpu_solver(wl, precision=precision, tol=1e-11)
        s1.solve_plane_waves(dirs[r:r + 1])
        assert rel_l2(batch[:, r], s1.get_density()[:, 0]) < (1e-10 if precision == 0 else 1e-8)


def test_restarted_gmres_and_initial_guess():
    require_gpu()
    wl = W.two_spheres(n_panels=6, gl_order=8, n_modes=21)
    s = gpu_solver(wl, tol=1e-12)
    s.solve_plane_waves(wl.directions)
    ref = s.get_density()
    s2 = gpu_solver(wl, tol=1e-12, restart=3, maxit=300)
    st = s2.solve_plane_waves(wl.directions)
    assert st.converged
    assert rel_l2(s2.get_density(), ref) < 1e-10
    x, _, _ = s.get_nodes()
    from oracle import fields
    v = fields.plane_wave(x, wl.directions, wl.k)
    st3 = s.solve_data(v, x0=ref)          # exact start: converges at once
    assert st3.converged and st3.iterations <= 1


def test_mixed_refinement_from_a_guess():
    """Mixed precision from a guess: the first correction solves with the FP32 operator's
    residual and aims at the absolute level inner_tol |b|, so a guess 1e-3 off needs fewer
    inner iterations than a zero start; a guess whose FP32 residual is already below that
    level skips the FP32 step (no inner iteration) and keeps its accuracy; both end at the
    zero-start answer."""
    require_gpu()
    from oracle import fields
    wl = W.two_spheres(n_panels=6, gl_order=8, n_modes=21)
    s = gpu_solver(wl, precision=1, tol=1e-10, inner_tol=1e-5)
    x, _, _ = s.get_nodes()
    v = fields.plane_wave(x, wl.directions, wl.k)
    st0 = s.solve_data(v)
    assert st0.converged
    ref = s.get_density().copy()
    g = np.random.default_rng(3)
    noise = g.standard_normal(ref.shape) + 1j * g.standard_normal(ref.shape)
    x0 = ref + 1e-3 * np.linalg.norm(ref) / np.linalg.norm(noise) * noise
    st1 = s.solve_data(v, x0=x0)
    assert st1.converged and st1.iterations < st0.iterations
    assert rel_l2(s.get_density(), ref) < 1e-8
    st2 = s.solve_data(v, x0=ref)
    assert st2.converged and st2.iterations == 0
    assert rel_l2(s.get_density(), ref) < 1e-12


def test_mixed_solve_with_single_term_tf32_inner_sums():
    """Inner FP32 solves on the single-term TF32 tensor-core engine (7) at R = 16: the
    double-float refinement residual brings the densities to the mixed bar against the
    FP64 solve."""
    require_gpu()
    wl = W.two_spheres(n_panels=6, gl_order=8, n_modes=21)
    dirs = W.uniform_directions(16, 31)
    s = gpu_solver(wl, tol=1e-12)
    s.solve_plane_waves(dirs)
    ref = s.get_density().copy()
    m = gpu_solver(wl, precision=1, tol=1e-8, residual=2)
    m.set_interbody_engine(7)
    st = m.solve_plane_waves(dirs)
    assert st.converged
    got = m.get_density()
    for r in range(16):
        assert rel_l2(got[:, r], ref[:, r]) < 1e-7


def test_error_statuses():
    require_gpu()
    from paper_1406_0236_gb300 import HzbError, Solver
    s = Solver(2.0, 2.0)
    with pytest.raises(HzbError) as e:
        s.add_body(W.SPHERE, (1.0,), 4, 6, 8, np.zeros(3), np.eye(3))     # even N_F
    assert e.value.status == -1
    with pytest.raises(HzbError) as e:
        s.build_scattering_matrices()                                      # no bodies
    assert e.value.status == -7
    with pytest.raises(HzbError) as e:
        s.add_body(W.SPHERE, (1.0,), 4, 6, 9, np.zeros(3), 2 * np.eye(3))   # not a rotation
    assert e.value.status == -1
    s.add_body(W.SPHERE, (1.0,), 4, 6, 9, np.zeros(3), np.eye(3))
    with pytest.raises(HzbError) as e:
        s.solve_plane_waves([[0, 0, 1.0]])                                 # not built
    assert e.value.status == -7
    s.build_scattering_matrices()
    with pytest.raises(HzbError) as e:
        s.solve_plane_waves([[0, 0, 2.0]])                                 # not a unit vector
    assert e.value.status == -1
    with pytest.raises(HzbError) as e:
        s.far_field([[0, 0, 1.0]])                                         # no solve yet
    assert e.value.status == -7
    st = s.solve_plane_waves([[0, 0, 1.0]])
    assert st.converged


def test_nonconvergence_is_reported():
    require_gpu()
    from paper_1406_0236_gb300 import HzbError
    wl = W.two_spheres(n_panels=6, gl_order=8, n_modes=21)
    s = gpu_solver(wl, tol=1e-14, maxit=2)
    with pytest.raises(HzbError) as e:
        s.solve_plane_waves(wl.directions)
    assert e.value.status == -4
    st = s.solve_plane_waves(wl.directions, allow_noconv=True)
    assert not st.converged and st.iterations == 2


def test_mixed_a_priori_stop_meets_1e7(two_spheres_ref):
    """verify_final = 0 stops after one FP64 residual on the refinement bound; the
    density must still meet 1e-7 against the oracle."""
    wl, P, sig_ref = two_spheres_ref
    from paper_1406_0236_gb300 import Options, Solver
    s = Solver.from_workload(wl, Options(precision=1, gmres_tol=1e-8, verify_final=0))
    s.build_scattering_matrices()
    st = s.solve_plane_waves(wl.directions)
    assert st.converged
    assert rel_l2(s.get_density()[:, 0], sig_ref) <= 1e-7


def test_autotuned_launch_shapes_keep_results():
    require_gpu()
    from oracle import Problem
    from tests._common import rand_c
    wl = W.two_spheres(n_panels=6, gl_order=8, n_modes=21)
    s = gpu_solver(wl)
    P = Problem(wl)
    sig = rand_c((P.N, 2), 5)
    ref = P.interbody(sig)
    best = s.autotune(2, 3)
    assert best[0] > 0 and best[1] > 0
    assert np.abs(s.interbody(sig) - ref).max() < 1e-12 * np.abs(ref).max()
    assert rel_l2(s.interbody(sig, precision=1), ref) < 2e-6


@pytest.mark.parametrize("precision", [0, 1])
def test_graph_replay_and_chunked_steps_match_plain_gmres(precision):
    """Arnoldi steps captured as CUDA graphs (on a non-default stream) and issued in
    chunks without host synchronisation give the same densities as the plain loop."""
    require_gpu()
    import torch
    wl = W.two_spheres(n_panels=6, gl_order=8, n_modes=21)
    dirs = W.uniform_directions(3, 17)
    plain = gpu_solver(wl, precision=precision, tol=1e-11)
    plain.set_execution(1, 0)
    st0 = plain.solve_plane_waves(dirs)
    ref = plain.get_density()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        from paper_1406_0236_gb300 import Options, Solver
        s = Solver.from_workload(wl, Options(precision=precision, gmres_tol=1e-11), stream=stream.cuda_stream)
        s.build_scattering_matrices()
        s.set_execution(3, 1)
        for _ in range(2):                      # second solve replays the captured graphs
            st = s.solve_plane_waves(dirs)
            assert st.converged and st.iterations == st0.iterations
            got = s.get_density()
            assert rel_l2(got, ref) < (1e-12 if precision == 0 else 1e-9)
        s.close()                           # before its stream goes away
    torch.cuda.synchronize()


def test_mixed_with_double_float_residual(two_spheres_ref):
    """Refinement residual in double-float: the density still reaches the FP64 bar."""
    wl, P, sig_ref = two_spheres_ref
    from paper_1406_0236_gb300 import Options, Solver
    s = Solver.from_workload(wl, Options(precision=1, gmres_tol=1e-11, residual=2))
    s.build_scattering_matrices()
    st = s.solve_plane_waves(wl.directions)
    assert st.converged and st.n_nbodydf >= 1 and st.n_nbody64 == 0
    assert rel_l2(s.get_density()[:, 0], sig_ref) <= 1e-10


def test_mixed_batch_on_tensor_cores(two_spheres_ref):
    """20 right-hand sides: the inner FP32 applies take the tensor-core inter-body path
    and the FP32 modal GEMM on tensor cores; the refined densities meet the FP64 bar."""
    from oracle import fields, gmres
    wl, P, _ = two_spheres_ref
    dirs = W.uniform_directions(20, 77)
    s = gpu_solver(wl, precision=1, tol=1e-11)
    st = s.solve_plane_waves(dirs)
    assert st.converged
    got = s.get_density()
    for r in (0, 13):
        v = fields.plane_wave(P.nodes.x, dirs[r:r + 1], wl.k)[:, 0]
        ref = gmres(P.apply, P.rhs(v), 1e-13).x
        assert rel_l2(got[:, r], ref) <= 1e-9
