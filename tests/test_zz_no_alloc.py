"""hzb_local_inverse_noalloc: the D^{-1} apply for callers that cannot allocate
device memory when they call (inside CUDA stream capture, or with a memory budget
fixed at start-up).  Its output must equal hzb_local_inverse's and the oracle's
D^{-1}, within the tolerance of the other D^{-1} tests, on two calls in a row (the
static scratch is reused) and with the accelerated scheme on; sizes beyond its
16 MiB scratch are rejected.  The file name makes pytest
collect it last."""
import numpy as np
import pytest

import workloads as W
from tests._common import gpu_solver, rand_c, rel_l2, require_gpu

pytestmark = pytest.mark.gpu


def _mixed_shapes():
    sph = W.ShapeSpec(W.SPHEROID, (1.0, 2.0), 5, 7, 11)
    ball = W.ShapeSpec(W.SPHERE, (0.7,), 3, 5, 7)
    bodies = [W.Body(sph, np.array([-2.0, 0.2, 0.0]), W.rotation_taking_z_to([0.3, 1.0, 0.2])),
              W.Body(ball, np.array([0.1, 2.4, -0.5]), np.eye(3)),
              W.Body(sph, np.array([0.0, -2.6, 1.0]), W.rotation_taking_z_to([0.0, 0.0, -1.0]))]
    return W.Workload("mixed3", bodies, 3.0, 3.0, np.array([[0, 0, 1.0]]))


def _oracle_local_inverse(wl, y):
    from oracle import Problem
    P = Problem(wl)
    return np.stack([P.local_inverse(y[:, r]) for r in range(y.shape[1])], axis=1)


@pytest.mark.parametrize("R", [1, 3])
def test_noalloc_local_inverse_matches_allocating_entry_point(R):
    require_gpu()
    import torch
    wl = _mixed_shapes()
    s = gpu_solver(wl)
    N = s.N
    for call in range(2):                                   # two calls in a row
        yh = rand_c((N, R), 100 + 10 * call + R)
        sh = rand_c((N, R), 200 + 10 * call + R)
        y = torch.from_numpy(yh).cuda()
        sig = torch.from_numpy(sh).cuda()
        ref = s.local_inverse(y, sig, alpha=0.5, beta=-2.0)
        got = s.local_inverse_noalloc(y, sig, alpha=0.5, beta=-2.0)
        torch.cuda.synchronize()
        assert rel_l2(got.cpu().numpy(), ref.cpu().numpy()) < 1e-11
        # against the oracle's D^{-1} (independent FP64 CPU code)
        orc = 0.5 * sh - 2.0 * _oracle_local_inverse(wl, yh)
        assert rel_l2(got.cpu().numpy(), orc) < 1e-11
        ref2 = s.local_inverse(y)
        got2 = s.local_inverse_noalloc(y)
        torch.cuda.synchronize()
        assert rel_l2(got2.cpu().numpy(), ref2.cpu().numpy()) < 1e-11
        assert rel_l2(got2.cpu().numpy(), _oracle_local_inverse(wl, yh)) < 1e-11


def test_noalloc_applies_the_direct_inverse_with_the_acceleration_on():
    """After hzb_compress both D^{-1} entry points still apply the direct block inverse."""
    require_gpu()
    import torch
    wl = W.separated_spheroids()
    s = gpu_solver(wl)
    s.compress(1e-8)
    assert s.reduced_size > 0
    yh = rand_c((s.N, 2), 77)
    y = torch.from_numpy(yh).cuda()
    got = s.local_inverse_noalloc(y)
    ref = s.local_inverse(y)
    torch.cuda.synchronize()
    assert rel_l2(got.cpu().numpy(), ref.cpu().numpy()) < 1e-11
    assert rel_l2(got.cpu().numpy(), _oracle_local_inverse(wl, yh)) < 1e-11


def test_noalloc_rejects_sizes_beyond_its_scratch():
    require_gpu()
    import torch
    from paper_1406_0236_gb300 import HzbError
    s = gpu_solver(W.tiny_two_spheres())
    R = 1200                                   # panel 5 x 24 x 4R complex > 524,288
    y = torch.zeros((s.N, R), dtype=torch.complex128, device="cuda")
    with pytest.raises(HzbError) as e:
        s.local_inverse_noalloc(y)
    assert e.value.status == -1 and "scratch" in str(e.value)
