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
    it0, it1 = iterations_with_and_without(s, ws, held, 1e-7)
    assert it1.mean() < it0.mean()
    # same converged density with or without the guess
    s.set_options(gmres_tol=1e-12)
    v = plane_wave_data(s, held[:1])
    s.solve_data(v)
    a = s.get_density().copy()
    s.solve_data(v, x0=ws.guess(held[:1]))
    b = s.get_density()
    assert rel_l2(b, a) < 1e-10


def test_pod_basis_orthonormal_and_captures_a_low_rank_snapshot_matrix():
    """hzb_pod_basis on X = A B of rank 12 (N = 1000, T = 300): U^H U = I, and the
    basis of 12 columns reproduces X to the FP32 level of its products."""
    require_gpu()
    import torch
    s = gpu_solver(W.tiny_two_spheres())
    g = np.random.default_rng(5)
    A = g.standard_normal((1000, 12)) + 1j * g.standard_normal((1000, 12))
    Bm = g.standard_normal((12, 300)) + 1j * g.standard_normal((12, 300))
    X = A @ Bm
    Xd = torch.from_numpy(X).cuda()
    U = s.pod_basis(Xd, 12, power_steps=2).cpu().numpy()
    assert np.abs(U.conj().T @ U - np.eye(12)).max() < 1e-12
    assert np.linalg.norm(X - U @ (U.conj().T @ X)) < 1e-5 * np.linalg.norm(X)
    C = s.pod_project(torch.from_numpy(U).cuda(), Xd).cpu().numpy()
    assert rel_l2(C, U.conj().T @ X) < 1e-6


def test_pod_guess_equals_host_expansion_of_the_network_output():
    """x0 = U c with c from the network's FP32 outputs (hzb_pod_guess) against numpy's
    U @ c on the same outputs, and against the oracle network's outputs."""
    require_gpu()
    import torch
    from oracle import mlp as omlp
    from paper_1406_0236_gb300 import Mlp
    s = gpu_solver(W.tiny_two_spheres())
    k, R = 16, 5
    g = np.random.default_rng(8)
    U = np.linalg.qr(g.standard_normal((s.N, k)) + 1j * g.standard_normal((s.N, k)))[0]
    net = Mlp(3, 32, 2, 2 * k, seed=4)
    dirs = W.uniform_directions(R, 9).astype(np.float32)
    y = net.forward(torch.from_numpy(dirs).cuda())
    x0 = s.pod_guess(torch.from_numpy(np.ascontiguousarray(U)).cuda(), y, 2.5).cpu().numpy()
    yh = y.cpu().numpy().astype(np.float64)
    c = 2.5 * (yh[:, 0::2] + 1j * yh[:, 1::2]).T
    assert rel_l2(x0, U @ c) < 1e-6
    ref_params = [(bf16_round(Wl), b.astype(np.float64)) for Wl, b in net.layers(net.get_params())]
    yo, _ = omlp.forward(ref_params, dirs.astype(np.float64))
    co = 2.5 * (yo[:, 0::2] + 1j * yo[:, 1::2]).T
    assert rel_l2(x0, U @ co) < 1e-4


def test_mlp_tensor_core_products_match_oracle_with_bf16_operands():
    """Width 512, batch 256: the hidden and output layers' products run on tcgen05 with
    BF16 operands (layer input and back-propagated gradient rounded to BF16, FP32
    accumulation); the oracle network with the same operands rounded (the first layer,
    3 inputs, stays in FP32 on the CUDA cores) gives the same outputs and gradients."""
    require_gpu()
    from oracle import mlp as omlp
    from paper_1406_0236_gb300 import Mlp
    net = Mlp(3, 512, 3, 512, seed=6)
    layers = net.layers(net.get_params())
    ref_params = [(bf16_round(W), b.astype(np.float64)) for W, b in layers]

    def operand(l, kind, a):
        return bf16_round(a) if l >= 1 else a

    rng = np.random.default_rng(4)
    x = rng.standard_normal((256, 3)).astype(np.float32)
    t = rng.standard_normal((256, 512)).astype(np.float32)
    y = net.forward(x)
    y_ref, _ = omlp.forward(ref_params, x.astype(np.float64), operand)
    # an operand whose FP32 (GPU) and FP64 (oracle) values straddle a BF16 rounding
    # boundary rounds to neighbouring values (2^-8 apart): ~1e-4 after four layers
    assert rel_l2(y, y_ref) < 1e-3
    loss, g = net.gradients(x, t)
    L_ref, g_ref = omlp.gradients(ref_params, x.astype(np.float64), t.astype(np.float64), operand)
    assert abs(loss - L_ref) < 1e-3 * L_ref
    for (gW, gb), (rW, rb) in zip(net.layers(g), g_ref):
        assert rel_l2(gW, rW) < 1e-3
        assert rel_l2(gb, rb) < 1e-3
    # the CUDA-core path (FP32 layer inputs) agrees to the BF16 rounding of the operands
    net.set_tensor_cores(False)
    y32 = net.forward(x)
    assert rel_l2(y, y32) < 2e-2
