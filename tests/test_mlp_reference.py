"""Pins of the FP64 reference network: backpropagation against central finite differences, the
bfloat16 rounding against exact cases, and Adam's first step (sign step of size lr)."""
import numpy as np

from oracle import mlp


def test_param_count():
    assert mlp.n_params() == 4 * 64 + 64 + 64 * 64 + 64 + 64 * 64 + 64 + 6 * 64 + 6 == 9030


def test_backprop_matches_finite_differences():
    rng = np.random.default_rng(1)
    p = mlp.init(3) + 0.05 * rng.standard_normal(mlp.n_params())
    x = rng.standard_normal((17, 4))
    t = rng.standard_normal((17, 6))
    _, g = mlp.loss_grad(p, x, t)
    idx = rng.choice(mlp.n_params(), 60, replace=False)
    h = 1e-6
    for k in idx:
        e = np.zeros_like(p)
        e[k] = h
        fd = (mlp.loss_grad(p + e, x, t)[0] - mlp.loss_grad(p - e, x, t)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1e-3, abs(g[k])) + 1e-10, (k, fd, g[k])


def test_bf16_rounding():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7, 1.0 + 3 * 2 ** -8, -3.140625, 0.0])
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: even mantissa -> 1; 1 + 3*2^-8 rounds up to 1 + 2^-6
    assert np.array_equal(mlp.bf16(vals), [1.0, 1.0, 1.0 + 2 ** -7, 1.0 + 2 ** -6, -3.140625, 0.0])


def test_adam_first_step_is_a_sign_step():
    p = np.array([0.5, -0.2, 0.0])
    g = np.array([3.0, -0.01, 1e-3])
    q, m, v = mlp.adam(p, g, np.zeros(3), np.zeros(3), 1, lr=1e-2, eps=0.0)
    assert np.allclose(q, p - 1e-2 * np.sign(g))
