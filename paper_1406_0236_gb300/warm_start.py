"""Learned warm start for GMRES: incident direction -> density, through a POD basis.

1. Training densities: the library solves the plane-wave problems of the training
   directions (batched right-hand sides, FP64 accuracy via mixed refinement).
2. POD basis: an orthonormal basis of the dominant n_pod-dimensional left singular
   subspace of the N x T snapshot matrix, by the randomized range finder of Halko,
   Martinsson and Tropp with two power steps (hzb_pod_basis: complex products in FP32,
   Gram-Schmidt twice in FP64); the coefficients c = U^H x by hzb_pod_project.
3. Network: hzb_mlp (BF16 weights, FP32 accumulation, hand-written CUDA kernels)
   maps the direction (3 numbers) to the n_pod complex POD coefficients (2 n_pod
   real outputs, scaled to unit RMS), trained with Adam on the MSE loss.
4. Guess: x0 = U c(d) (hzb_pod_guess on the network's outputs), passed to
   hzb_solve_data; the zero-guess solve is the fallback (a guess never changes the
   converged answer, only the iterations).
5. The held-out batches run once more through the accelerated scheme (Sec. 5):
   hzb_compress, then the reduced system, the guess restricted to the skeleton.

Run the full protocol (two unit spheres, 8,200 unknowns; 4,096 training and 512
held-out directions; 4 hidden layers of 512, 256 POD modes):

    python -m paper_1406_0236_gb300.warm_start
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


class WarmStart:
    def __init__(self, solver, n_pod: int = 256, width: int = 512, depth: int = 4, seed: int = 1):
        import torch

        from .binding import Mlp
        self.torch = torch
        self.s = solver
        self.n_pod, self.width, self.depth = n_pod, width, depth
        self.mlp = Mlp(3, width, depth, 2 * n_pod, seed=seed, stream=torch.cuda.current_stream().cuda_stream)
        self.U = None
        self.scale = 1.0
        self.losses = []

    # -------------------------------------------------------------- data
    def training_densities(self, dirs: np.ndarray, batch: int = 64):
        """Densities (N x T complex128, device) of the plane waves `dirs` (T x 3)."""
        torch = self.torch
        N = self.s.N
        X = torch.empty((N, dirs.shape[0]), dtype=torch.complex128, device="cuda")
        for a in range(0, dirs.shape[0], batch):
            d = dirs[a:a + batch]
            self.s.solve_plane_waves(d)
            out = torch.empty((N, d.shape[0]), dtype=torch.complex128, device="cuda")
            self.s.get_density(out)
            X[:, a:a + d.shape[0]] = out
        return X

    def pod_basis(self, X, power_steps: int = 2, seed: int = 7):
        """Orthonormal basis of the dominant n_pod-dimensional subspace of the snapshots X
        (N x T): randomized range finder with power steps, on the library's kernels
        (hzb_pod_basis)."""
        return self.s.pod_basis(X, self.n_pod, power_steps=power_steps, seed=seed)

    def fit(self, dirs: np.ndarray, X=None, epochs: int = 400, batch: int = 256, lr: float = 1e-3,
            lr_final: float = 2e-5):
        torch = self.torch
        if X is None:
            X = self.training_densities(dirs)
        t0 = time.time()
        self.U = self.pod_basis(X)
        C = self.s.pod_project(self.U, X)                               # n_pod x T coefficients
        # T x 2 n_pod targets: row t = (Re c_0, Im c_0, Re c_1, Im c_1, ...) of sample t
        T = torch.stack([C.real, C.imag], dim=-1).permute(1, 0, 2).reshape(X.shape[1], 2 * self.n_pod).contiguous()
        torch.cuda.synchronize()
        self.t_pod = time.time() - t0
        self.scale = float(T.pow(2).mean().sqrt())
        Tn = (T / self.scale).float().contiguous()
        D = torch.from_numpy(np.ascontiguousarray(dirs, dtype=np.float32)).cuda()
        n = D.shape[0]
        t0 = time.time()
        g = torch.Generator(device="cuda").manual_seed(11)
        steps = epochs * max(1, n // batch)
        q = 0
        for ep in range(epochs):
            perm = torch.randperm(n, device="cuda", generator=g)
            for a in range(0, n - batch + 1, batch):
                idx = perm[a:a + batch]
                rate = lr * (lr_final / lr) ** (q / max(steps - 1, 1))      # geometric decay
                loss = self.mlp.train_step(D[idx].contiguous(), Tn[idx].contiguous(), rate)
                q += 1
            self.losses.append(loss)
        torch.cuda.synchronize()
        self.t_train = time.time() - t0
        self.train_steps = q
        return self

    def guess(self, dirs: np.ndarray):
        """x0 = U c(d) for directions (R x 3): N x R complex128 device tensor (network
        forward pass and POD expansion on the library's kernels)."""
        torch = self.torch
        D = torch.from_numpy(np.ascontiguousarray(dirs, dtype=np.float32)).cuda()
        y = self.mlp.forward(D)                                         # R x 2 n_pod, FP32
        return self.s.pod_guess(self.U, y.contiguous(), self.scale)


def plane_wave_data(s, dirs):
    """v = exp(i k d . x) at the nodes (N x R complex128, device), by the library."""
    return s.plane_waves(dirs, device=True)


def iterations_with_and_without(s, ws: WarmStart, dirs, tol: float):
    """Per-direction GMRES iterations to the relative residual tol, zero guess vs warm start."""
    it0, it1 = [], []
    for r in range(dirs.shape[0]):
        v = plane_wave_data(s, dirs[r:r + 1])
        st0 = s.solve_data(v)
        x0 = ws.guess(dirs[r:r + 1])
        st1 = s.solve_data(v, x0=x0)
        it0.append(st0.iterations)
        it1.append(st1.iterations)
    return np.array(it0), np.array(it1)


def main():
    import torch

    import workloads as W
    from .binding import Options, Solver

    wl = W.two_spheres()
    s = Solver.from_workload(wl, Options(precision=1, gmres_tol=1e-11, verify_final=1),
                             stream=torch.cuda.current_stream().cuda_stream)
    s.build_scattering_matrices()
    train = W.uniform_directions(4096, 20140602)
    held = W.uniform_directions(512, 20140603)
    t0 = time.time()
    ws = WarmStart(s)
    X = ws.training_densities(train)
    t_data = time.time() - t0
    t0 = time.time()
    ws.fit(train, X)
    torch.cuda.synchronize()
    t_fit = time.time() - t0
    # iterations to 1e-7 on the held-out directions: FP64 path, zero guess vs warm start
    s.set_options(precision=0, gmres_tol=1e-7)
    it0, it1 = iterations_with_and_without(s, ws, held, 1e-7)
    # density error of the bare guess (reference: mixed refinement to 1e-11)
    s.set_options(precision=1, gmres_tol=1e-11, verify_final=1)
    Xh = ws.training_densities(held)
    G = ws.guess(held)
    gerr = (torch.linalg.vector_norm(G - Xh, dim=0) / torch.linalg.vector_norm(Xh, dim=0)).cpu().numpy()
    # held-out throughput, batches of 64 right-hand sides, residual 1e-8 (density error checked):
    # FP64 GPU path from zero against mixed precision + warm start
    x, _, _ = s.get_nodes()

    def timed(prec, warm, residual=0):
        s.set_options(precision=prec, gmres_tol=1e-8, verify_final=1 if prec == 0 else 0, residual=residual)
        out = torch.empty_like(Xh)
        torch.cuda.synchronize()
        t0 = time.time()
        its = []
        for a in range(0, held.shape[0], 64):
            d = held[a:a + 64]
            v = plane_wave_data(s, d)
            st = s.solve_data(v, x0=ws.guess(d) if warm else None)
            its.append(st.iterations)
            part = torch.empty((out.shape[0], d.shape[0]), dtype=out.dtype, device=out.device)
            s.get_density(part)
            out[:, a:a + d.shape[0]] = part
        torch.cuda.synchronize()
        dt = time.time() - t0
        err = float((torch.linalg.vector_norm(out - Xh, dim=0) / torch.linalg.vector_norm(Xh, dim=0)).max())
        return held.shape[0] / dt, its, err

    r64, it64, e64 = timed(0, False)
    rmw, itmw, emw = timed(1, True)
    rm0, itm0, em0 = timed(1, False)
    rdw, itdw, edw = timed(1, True, residual=2)         # double-float refinement residual
    rd0, itd0, ed0 = timed(1, False, residual=2)
    # the accelerated scheme (Sec. 5): reduced system over skeleton nodes, warm start
    # restricted to it, density recovered on all nodes
    t0 = time.time()
    s.compress(1e-8)
    t_comp = time.time() - t0
    n_red = s.reduced_size
    raw, itaw, eaw = timed(1, True)
    ra0, ita0, ea0 = timed(1, False)
    s.set_acceleration(False)
    print(json.dumps({
        "workload": "two_spheres_8200", "train": 4096, "held_out": 512, "pod_modes": ws.n_pod,
        "mlp": "3 -> 4 x 512 GELU -> 512", "t_training_solves_s": t_data, "t_fit_s": t_fit,
        "t_pod_s": ws.t_pod, "t_train_s": ws.t_train, "train_steps": ws.train_steps,
        "final_loss": ws.losses[-1],
        "gmres_iterations_to_1e-7": {"zero_guess_mean": float(it0.mean()), "warm_mean": float(it1.mean()),
                                     "zero_guess_max": int(it0.max()), "warm_max": int(it1.max())},
        "guess_rel_err_median": float(np.median(gerr)), "guess_rel_err_max": float(gerr.max()),
        "held_out_solves_per_s": {"fp64_gpu_zero_guess": r64, "mixed_plus_mlp": rmw, "mixed_zero_guess": rm0,
                                  "mixed_df_plus_mlp": rdw, "mixed_df_zero_guess": rd0},
        "held_out_density_err_max": {"fp64_gpu_zero_guess": e64, "mixed_plus_mlp": emw, "mixed_zero_guess": em0,
                                     "mixed_df_plus_mlp": edw, "mixed_df_zero_guess": ed0},
        "batch_iterations": {"fp64_gpu_zero_guess": it64, "mixed_plus_mlp": itmw, "mixed_zero_guess": itm0,
                             "mixed_df_plus_mlp": itdw, "mixed_df_zero_guess": itd0},
        "accelerated": {"eps": 1e-8, "compress_s": t_comp, "reduced_unknowns": n_red,
                        "held_out_solves_per_s": {"mixed_plus_mlp": raw, "mixed_zero_guess": ra0},
                        "held_out_density_err_max": {"mixed_plus_mlp": eaw, "mixed_zero_guess": ea0},
                        "batch_iterations": {"mixed_plus_mlp": itaw, "mixed_zero_guess": ita0}},
    }))


if __name__ == "__main__":
    main()
