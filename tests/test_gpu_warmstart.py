"""Learned warm start (no counterpart in the paper): the MLP's forward pass and
gradients on the GPU against the FP64 oracle network (same BF16-rounded weights),
training reduces the loss, and the trained guess cuts GMRES iterations on held-out
directions without changing the converged density."""
import numpy as np
import pytest

import workloads as W
from tests._common import gpu_solver, rel_l2, require_gpu

pytestmark = pytest.mark.gpu


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even), as float64."""
    b = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def test_mlp_forward_and_gradients_match_oracle():
    require_gpu()
    from oracle import mlp as omlp
    from paper_1406_0236_gb300 import Mlp
    net = Mlp(3, 48, 3, 10, seed=5)
    p = net.get_params()
    layers = net.layers(p)
    # the GPU multiplies with BF16 weights (biases stay FP32)
    ref_params = [(bf16_round(W), b.astype(np.float64)) for W, b in layers]
    rng = np.random.default_rng(3)
    x = rng.standard_normal((37, 3)).astype(np.float32)
    t = rng.standard_normal((37, 10)).astype(np.float32)
    y = net.forward(x)
    y_ref, _ = omlp.forward(ref_params, x.astype(np.float64))
    assert rel_l2(y, y_ref) < 1e-5
    loss, g = net.gradients(x, t)
    L_ref, g_ref = omlp.gradients(ref_params, x.astype(np.float64), t.astype(np.float64))
    assert abs(loss - L_ref) < 1e-5 * L_ref
    for (gW, gb), (rW, rb) in zip(net.layers(g), g_ref):
        assert rel_l2(gW, rW) < 2e-4
        assert rel_l2(gb, rb) < 2e-4


def test_training_reduces_loss():
    require_gpu()
    from paper_1406_0236_gb300 import Mlp
    net = Mlp(3, 64, 2, 8, seed=2)
    rng = np.random.default_rng(0)
    x = rng.standard_normal((256, 3)).astype(np.float32)
    t = np.stack([np.sin(x[:, 0] + q * x[:, 1]) for q in range(8)], 1).astype(np.float32)
    l0 = net.train_step(x, t, 1e-3)
    for _ in range(300):
        l1 = net.train_step(x, t, 3e-3)
    assert l1 < 0.1 * l0


def test_warm_start_cuts_iterations_and_keeps_the_answer():
    require_gpu()
    import torch
    from paper_1406_0236_gb300.warm_start import WarmStart, iterations_with_and_without, plane_wave_data
    wl = W.two_spheres(n_panels=6, gl_order=8, n_modes=21)
    s = gpu_solver(wl, precision=0, tol=1e-11)
    train = W.uniform_directions(512, 41)
    held = W.uniform_directions(16, 42)
    ws = WarmStart(s, n_pod=48, width=128, depth=3, seed=3)
    ws.fit(train, epochs=150, batch=128, lr=2e-3)
    s.set_options(gmres_tol=1e-7)
    it0, it1 = iterations_with_and_without(s, ws, held, wl.k, 1e-7)
    assert it1.mean() < it0.mean()
    # same converged density with or without the guess
    s.set_options(gmres_tol=1e-12)
    x, _, _ = s.get_nodes()
    v = plane_wave_data(x, held[:1], wl.k)
    s.solve_data(v)
    a = s.get_density().copy()
    s.solve_data(v, x0=ws.guess(held[:1]))
    b = s.get_density()
    assert rel_l2(b, a) < 1e-10
