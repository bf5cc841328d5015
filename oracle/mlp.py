"""Oracle of the learned warm start's network: forward pass, loss and gradients of
a plain multilayer perceptron in FP64 (numpy).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The network maps an incident direction (3 numbers) through `depth` hidden layers
of `width` units with the GELU activation, GELU(a) = a Phi(a) (Phi the standard
normal distribution function), to `out` outputs (POD coefficients of the density,
real and imaginary parts interleaved).  Loss: mean over the batch of the squared
error summed over outputs,  L = (1/B) sum_b sum_o (y_bo - t_bo)^2.
Layer l: a_l = h_{l-1} W_l^T + b_l,  h_l = GELU(a_l) for hidden layers, y = a_last.
Gradients by the chain rule (reverse mode), checked in tests against central finite
differences.
"""
from __future__ import annotations

from typing import List, Tuple

import numpy as np
from scipy import special


def gelu(a):
    return a * 0.5 * (1.0 + special.erf(a / np.sqrt(2.0)))


def gelu_grad(a):
    phi = np.exp(-0.5 * a * a) / np.sqrt(2.0 * np.pi)
    return 0.5 * (1.0 + special.erf(a / np.sqrt(2.0))) + a * phi


def _keep(l, kind, a):
    return a


def forward(params: List[Tuple[np.ndarray, np.ndarray]], x: np.ndarray, operand=_keep):
    """params: [(W_l (out_l x in_l), b_l (out_l))]; returns (y, cache).  `operand(l,
    "h", h)` gives the layer input as it enters the product (identity by default; a
    caller emulating reduced-precision operands passes a rounding)."""
    h = np.asarray(x, dtype=np.float64)
    cache = []
    for l, (W, b) in enumerate(params):
        a = operand(l, "h", h) @ W.T + b
        cache.append((h, a))
        h = gelu(a) if l < len(params) - 1 else a
    return h, cache


def loss(params, x, t) -> float:
    y, _ = forward(params, x)
    return float(((y - t) ** 2).sum() / x.shape[0])


def gradients(params, x, t, operand=_keep):
    """(loss, [(dW_l, db_l)]); `operand` as in forward, also applied (kind "g") to the
    back-propagated gradient where it enters the two products of a layer."""
    y, cache = forward(params, x, operand)
    B = x.shape[0]
    g = 2.0 * (y - t) / B                                   # dL/dy
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        h_in, a = cache[l]
        if l < len(params) - 1:
            g = g * gelu_grad(a)                            # through the activation
        W, _ = params[l]
        gp = operand(l, "g", g)
        grads[l] = (gp.T @ operand(l, "h", h_in), g.sum(axis=0))
        g = gp @ W                                          # to the layer input
    return float(((y - t) ** 2).sum() / B), grads
