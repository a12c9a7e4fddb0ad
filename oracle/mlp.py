"""FP64 reference of the force surrogate network (test infrastructure only).

A multilayer perceptron 4 -> 64 -> 64 -> 64 -> 6 with tanh hidden units and a linear output,
trained on the mean squared error with Adam. Parameter layout (flat): for each layer W (out x in,
row-major) then b (out). The GPU kernels compute with the weights rounded to bfloat16 and FP32
accumulation; `bf16` rounds an array the same way so both sides can be fed the same weights.
"""
from __future__ import annotations

import numpy as np

SIZES = (4, 64, 64, 64, 6)


def n_params(sizes=SIZES):
    return sum(sizes[k + 1] * sizes[k] + sizes[k + 1] for k in range(len(sizes) - 1))


def unpack(p, sizes=SIZES):
    out, o = [], 0
    for k in range(len(sizes) - 1):
        ni, no = sizes[k], sizes[k + 1]
        W = p[o:o + no * ni].reshape(no, ni)
        o += no * ni
        b = p[o:o + no]
        o += no
        out.append((W, b))
    return out


def init(seed=0, sizes=SIZES):
    """Glorot-uniform weights, zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for k in range(len(sizes) - 1):
        ni, no = sizes[k], sizes[k + 1]
        lim = np.sqrt(6.0 / (ni + no))
        parts.append(rng.uniform(-lim, lim, size=no * ni))
        parts.append(np.zeros(no))
    return np.concatenate(parts)


def bf16(a):
    """Round to bfloat16 (round to nearest, ties to even) through the float32 bit pattern."""
    f = np.asarray(a, np.float32).copy()
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(p, x, sizes=SIZES):
    h = np.asarray(x, np.float64)
    layers = unpack(np.asarray(p, np.float64), sizes)
    acts = [h]
    for k, (W, b) in enumerate(layers):
        z = h @ W.T + b
        h = np.tanh(z) if k < len(layers) - 1 else z
        acts.append(h)
    return h, acts


def loss_grad(p, x, t, sizes=SIZES):
    """Mean squared error over samples and outputs, and its gradient (backpropagation)."""
    y, acts = forward(p, x, sizes)
    n, m = y.shape
    r = y - np.asarray(t, np.float64)
    loss = float(np.sum(r * r) / (n * m))
    layers = unpack(np.asarray(p, np.float64), sizes)
    delta = 2.0 * r / (n * m)
    grads = []
    for k in range(len(layers) - 1, -1, -1):
        W, b = layers[k]
        h_in = acts[k]
        grads.append((delta.T @ h_in, delta.sum(0)))
        if k > 0:
            delta = (delta @ W) * (1.0 - acts[k] ** 2)
    flat = []
    for dW, db in reversed(grads):
        flat.append(dW.reshape(-1))
        flat.append(db)
    return loss, np.concatenate(flat)


def adam(p, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
