"""GPU parity of the hot-path operators: inter-body sum B (Sec. 3.3), block-diagonal
inverse D^{-1} (Remark after Eq. (precond)) and the preconditioned apply, in FP64
and FP32, against the oracle on the same seeded inputs."""
import numpy as np
import pytest

import workloads as W
from tests._common import gpu_solver, oracle_problem, rand_c, rel_l2, require_gpu

pytestmark = pytest.mark.gpu


def _mixed_pair():
    sph = W.ShapeSpec(W.SPHEROID, (1.0, 2.0), 5, 7, 11)
    shell = W.ShapeSpec(W.OPEN_SHELL, (1.0, 0.8, np.pi / 3, 0.1), 9, 6, 9)
    ball = W.ShapeSpec(W.SPHERE, (0.7,), 3, 5, 7)
    bodies = [W.Body(sph, np.array([-2.0, 0.2, 0.0]), W.rotation_taking_z_to([0.3, 1.0, 0.2])),
              W.Body(shell, np.array([1.7, -0.1, 0.3]), W.rotation_taking_z_to([-1.0, 0.2, 0.4])),
              W.Body(ball, np.array([0.1, 2.4, -0.5]), np.eye(3)),
              W.Body(sph, np.array([0.0, -2.6, 1.0]), W.rotation_taking_z_to([0.0, 0.0, -1.0]))]
    return W.Workload("mixed4", bodies, 3.0, 3.0, np.array([[0, 0, 1.0]]))


CASES = {"two_spheres_tiny": lambda: W.tiny_two_spheres(), "mixed4": _mixed_pair}


@pytest.fixture(scope="module", params=list(CASES))
def pair(request):
    require_gpu()
    from oracle import Problem
    wl = CASES[request.param]()
    return gpu_solver(wl), Problem(wl)


@pytest.mark.parametrize("R", [1, 3, 9])
def test_interbody_fp64(pair, R):
    s, P = pair
    sig = rand_c((P.N, R), 11 + R)
    got = s.interbody(sig)
    ref = P.interbody(sig)
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("engine", [0, 1])
@pytest.mark.parametrize("R", [1, 2, 5])
def test_interbody_fp64_engines(pair, R, engine):
    """One-directional (0) and pair-symmetric (1) FP64 kernels, each forced; R = 5
    takes two right-hand-side chunks of the symmetric kernel, the second ragged."""
    s, P = pair
    sig = rand_c((P.N, R), 161 + R)
    ref = P.interbody(sig)
    s.set_fp64_interbody_engine(engine)
    try:
        got = s.interbody(sig)
    finally:
        s.set_fp64_interbody_engine(-1)
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("R", [1, 5])
def test_interbody_fp32(pair, R):
    s, P = pair
    sig = rand_c((P.N, R), 21 + R)
    got = s.interbody(sig, precision=1)
    ref = P.interbody(sig)
    assert rel_l2(got, ref) < 2e-6


@pytest.mark.parametrize("engine", [2, 3, 4])
@pytest.mark.parametrize("R", [1, 2, 5, 9])
def test_interbody_fp32_kernel_variants(pair, R, engine):
    """Scalar (2), packed-pair f32x2 (3) and pair-symmetric packed (4) FP32 CUDA-core
    kernels, each forced, over ragged source tiles (odd node counts) and ragged
    right-hand-side chunks (R = 5, 9)."""
    s, P = pair
    sig = rand_c((P.N, R), 151 + R)
    ref = P.interbody(sig)
    s.set_interbody_engine(engine)
    try:
        got = s.interbody(sig, precision=1)
    finally:
        s.set_interbody_engine(-1)
    assert rel_l2(got, ref) < 2e-6


@pytest.mark.parametrize("engine", [1, 2])
@pytest.mark.parametrize("R", [1, 3, 24])
def test_local_inverse_tensor_cores(pair, R, engine):
    """FP32 modal GEMM on the tensor cores (TF32 with a three-term split): mma.sync (1)
    and tcgen05 fed by TMA (2)."""
    s, P = pair
    y = rand_c((P.N, R), 131 + R)
    ref = P.local_inverse(y)
    s.set_modal_engine(engine)
    try:
        got = s.local_inverse(y, precision=1)
    finally:
        s.set_modal_engine(-1)
    assert rel_l2(got, ref) < 1e-5


@pytest.mark.parametrize("R", [1, 4, 24])
def test_local_inverse(pair, R):
    s, P = pair
    y = rand_c((P.N, R), 31 + R)
    sig = rand_c((P.N, R), 41 + R)
    ref = 0.5 * sig - 2.0 * P.local_inverse(y)
    got = s.local_inverse(y, sig, alpha=0.5, beta=-2.0)
    assert rel_l2(got, ref) < 1e-11
    got32 = s.local_inverse(y, sig, alpha=0.5, beta=-2.0, precision=1)
    assert rel_l2(got32, ref) < 1e-5
    # double-float DFTs and mode GEMMs on the FP32 pipe: the FP64 bar
    gotdf = s.local_inverse(y, sig, alpha=0.5, beta=-2.0, precision=2)
    assert rel_l2(gotdf, ref) < 1e-11
    assert np.abs(gotdf - ref).max() < 1e-11 * np.abs(ref).max()


def test_apply_fp64(pair):
    s, P = pair
    sig = rand_c((P.N, 2), 51)
    assert rel_l2(s.apply(sig), P.apply(sig)) < 1e-11
    # the refinement residual's operator: inter-body sum and D^{-1} in double-float
    assert rel_l2(s.apply(sig, precision=2), P.apply(sig)) < 1e-11


def test_device_tensors_round_trip(pair):
    import torch
    s, P = pair
    sig = rand_c((P.N, 2), 61)
    t = torch.from_numpy(sig).cuda()
    s.set_stream(torch.cuda.current_stream().cuda_stream)
    out = s.apply(t)
    torch.cuda.synchronize()
    assert rel_l2(out.cpu().numpy(), P.apply(sig)) < 1e-11


def test_spheroids_258560_sampled_rows():
    """Full-size eight-spheroid workload in the benchmark's launch configuration:
    B sigma on 96 seeded target rows (FP64 and FP32) against the oracle's rows."""
    require_gpu()
    from oracle import Problem
    wl = W.spheroids8()
    s = gpu_solver(wl)
    P = Problem(wl)
    assert s.N == 258560 == P.N
    sig = rand_c((P.N, 1), 71)
    rows = np.sort(np.random.default_rng(72).choice(P.N, 96, replace=False)).astype(np.int32)
    ref = P.interbody(sig, targets=rows)
    y64 = s.interbody(sig)
    assert np.abs(y64[rows] - ref).max() < 1e-11 * np.abs(ref).max()
    # FP32: the phase k r carries the relative error of r (~2 ulp after the hardware
    # reciprocal square root) times k r <= 4 x 14 here, ~1e-5 per term at most.
    for engine in (2, 3, 4):
        s.set_interbody_engine(engine)
        y32 = s.interbody(sig, precision=1)
        assert rel_l2(y32[rows], ref) < 3e-5, engine
    # tensor-core contraction, 16 right-hand sides: 258,560 sources per target
    sig16 = rand_c((P.N, 16), 73)
    ref16 = P.interbody(sig16, targets=rows)
    for engine in (1, 5, 6):             # mma.sync, tcgen05, tcgen05 warp-specialised
        s.set_interbody_engine(engine)
        ytc = s.interbody(sig16, precision=1)
        assert rel_l2(ytc[rows], ref16) < 3e-5, engine
    s.set_interbody_engine(7)            # single-term TF32 products: its own bar
    ytc = s.interbody(sig16, precision=1)
    assert rel_l2(ytc[rows], ref16) < 1e-3
    s.set_interbody_engine(-1)


@pytest.mark.parametrize("engine", [0, 1, 2])
@pytest.mark.parametrize("R", [1, 3, 9, 17, 40])
def test_interbody_double_float(pair, R, engine):
    """Double-float (two FP32 numbers) inter-body sum: FP64-class accuracy; the
    one-directional (0; right-hand sides in chunks of 1, 4, 8, 16 and 32, the last with
    two 256-thread CTAs per target block, ragged chunks at R = 17 and 40), the
    pair-symmetric lean (1) and the pair-symmetric normalised (2) kernel."""
    s, P = pair
    sig = rand_c((P.N, R), 81 + R)
    s.set_fp64_interbody_engine(engine)
    try:
        got = s.interbody(sig, precision=2)
    finally:
        s.set_fp64_interbody_engine(-1)
    ref = P.interbody(sig)
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()


def test_spheroids_258560_double_float_rows():
    """At full size, in the launch the benchmark's refinement residual uses (R = 1,
    pair-symmetric lean double-float): the FP64 kernel's bar, 1e-12 of max |y|."""
    require_gpu()
    from oracle import Problem
    wl = W.spheroids8()
    s = gpu_solver(wl)
    P = Problem(wl)
    sig = rand_c((P.N, 1), 91)
    rows = np.sort(np.random.default_rng(92).choice(P.N, 256, replace=False)).astype(np.int32)
    ref = P.interbody(sig, targets=rows)
    assert s.tuned_config(1)["fp64_kernel"] == "nbody64_sym_kernel"
    ydf = s.interbody(sig, precision=2)
    assert np.abs(ydf[rows] - ref).max() < 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("R", [1, 5, 16, 40])
def test_interbody_tensor_cores(pair, R):
    """FP32 inter-body sum with the contraction on the tensor cores (TF32, 3-term split)."""
    s, P = pair
    sig = rand_c((P.N, R), 141 + R)
    ref = P.interbody(sig)
    s.set_interbody_engine(1)
    try:
        got = s.interbody(sig, precision=1)
    finally:
        s.set_interbody_engine(-1)
    assert rel_l2(got, ref) < 5e-6


@pytest.mark.parametrize("engine", [5, 6])
@pytest.mark.parametrize("R", [1, 5, 16, 40])
def test_interbody_tcgen05(pair, R, engine):
    """FP32 inter-body sum with the contraction on tcgen05 tensor cores (TF32 three-term
    split, accumulators in tensor memory drained into FP32 sums every 32 sources): the
    per-CTA form (5) and the warp-specialised pipeline (6)."""
    s, P = pair
    sig = rand_c((P.N, R), 171 + R)
    ref = P.interbody(sig)
    s.set_interbody_engine(engine)
    try:
        got = s.interbody(sig, precision=1)
    finally:
        s.set_interbody_engine(-1)
    assert rel_l2(got, ref) < 5e-6
