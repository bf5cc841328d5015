"""Pin of the oracle MLP's reverse-mode gradients against central finite differences."""
import numpy as np

from oracle import mlp


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    sizes = [3, 7, 6, 4]
    params = [(rng.standard_normal((o, i)) / np.sqrt(i), 0.1 * rng.standard_normal(o))
              for i, o in zip(sizes[:-1], sizes[1:])]
    x = rng.standard_normal((5, 3))
    t = rng.standard_normal((5, 4))
    L, grads = mlp.gradients(params, x, t)
    assert abs(L - mlp.loss(params, x, t)) < 1e-14
    h = 1e-6
    for l, (W, b) in enumerate(params):
        for arr, g in ((W, grads[l][0]), (b, grads[l][1])):
            for idx in list(np.ndindex(arr.shape))[:12]:
                old = arr[idx]
                arr[idx] = old + h
                lp = mlp.loss(params, x, t)
                arr[idx] = old - h
                lm = mlp.loss(params, x, t)
                arr[idx] = old
                fd = (lp - lm) / (2 * h)
                assert abs(fd - g[idx]) < 1e-7 * max(1.0, abs(fd)), (l, idx, fd, g[idx])


def test_gelu_closed_values():
    # GELU(0) = 0, GELU(a) -> a for large a, GELU(-a) -> 0; derivative at 0 is 1/2
    assert mlp.gelu(np.array(0.0)) == 0.0
    assert abs(mlp.gelu(np.array(8.0)) - 8.0) < 1e-12
    assert abs(mlp.gelu(np.array(-8.0))) < 1e-12
    assert abs(mlp.gelu_grad(np.array(0.0)) - 0.5) < 1e-15
