"""FP64 reference of the warm-start network: periodic 3-D convolutions with
3x3x3 kernels, bias and ReLU, forward and backward.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The network is not in the paper; it is the learned warm start of the
Krylov solve (a prediction of the next step's displacement increment).
Layout: activations are channels-last arrays [N3, N2, N1, C]; a layer's
weights are W[o, co, ci] for the 27 offsets o = (dz, dy, dx) in {-1,0,1}^3
enumerated with dx fastest (o = 9 (dz+1) + 3 (dy+1) + (dx+1)); bias b[co].
    y[x, co] = b[co] + sum_o sum_ci W[o, co, ci] * in[(x + o) mod N, ci]
"""
from __future__ import annotations

import numpy as np

OFFSETS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def shifted(a: np.ndarray, off) -> np.ndarray:
    """a[(x + off) mod N] over the three spatial axes of a channels-last array."""
    dz, dy, dx = off
    return np.roll(a, shift=(-dz, -dy, -dx), axis=(0, 1, 2))


def conv_forward(x: np.ndarray, W: np.ndarray, b: np.ndarray) -> np.ndarray:
    y = np.broadcast_to(b, x.shape[:3] + (W.shape[1],)).astype(np.float64).copy()
    for o, off in enumerate(OFFSETS):
        y += np.einsum("zyxi,ci->zyxc", shifted(x, off), W[o], optimize=True)
    return y


def conv_backward(x: np.ndarray, W: np.ndarray, dy: np.ndarray):
    """Gradients of sum(dy * conv_forward(x, W, b)) w.r.t. x, W, b."""
    dx = np.zeros_like(x, dtype=np.float64)
    dW = np.zeros_like(W, dtype=np.float64)
    for o, off in enumerate(OFFSETS):
        xs = shifted(x, off)
        dW[o] = np.einsum("zyxc,zyxi->ci", dy, xs, optimize=True)
        # y[x] depends on in[x + off]: scatter back with the opposite shift
        dx += shifted(np.einsum("zyxc,ci->zyxi", dy, W[o], optimize=True), tuple(-v for v in off))
    db = dy.sum(axis=(0, 1, 2))
    return dx, dW, db


def net_forward(x: np.ndarray, params):
    """params: list of (W, b); ReLU after every layer but the last.  Returns the
    output and the list of layer inputs / pre-activations kept for backward."""
    cache = []
    h = x
    for i, (W, b) in enumerate(params):
        z = conv_forward(h, W, b)
        cache.append((h, z))
        h = np.maximum(z, 0.0) if i < len(params) - 1 else z
    return h, cache


def net_backward(params, cache, dout: np.ndarray):
    grads = [None] * len(params)
    g = dout
    for i in range(len(params) - 1, -1, -1):
        h, z = cache[i]
        if i < len(params) - 1:
            g = g * (z > 0.0)
        dx, dW, db = conv_backward(h, params[i][0], g)
        grads[i] = (dW, db)
        g = dx
    return grads, g


def masked_mse(pred: np.ndarray, target: np.ndarray, free: np.ndarray):
    """Mean squared error over the entries where `free` (bool, shape of pred) is
    set -- the free DOFs of a training pair -- and its gradient w.r.t. pred."""
    diff = (pred - target) * free
    n = max(int(free.sum()), 1)
    return float((diff ** 2).sum() / n), 2.0 * diff / n
