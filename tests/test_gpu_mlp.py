"""The surrogate network's GPU kernels against the FP64 reference (oracle/mlp.py) fed the same
bfloat16-rounded weights: forward within 1e-4 relative, gradients within 1e-3 relative (FP32
accumulation, block partial sums), one Adam step, and that training lowers the loss."""
import numpy as np
import pytest

from oracle import mlp as ref

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def net():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1902_10432_gb300 import cbl

    return cbl.MLP()


def _data(n, seed):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((n, 4))
    t = np.stack([np.sin(x[:, 0]) * x[:, 1], np.cos(x[:, 2]), x[:, 3] ** 2 - 1, x[:, 0] * x[:, 2],
                  np.tanh(x[:, 1] + x[:, 3]), 0.1 * x.sum(1)], 1)
    return x, t


def test_forward_matches_reference(net):
    import torch

    p = ref.init(5)
    net.set_params(p)
    pb = ref.bf16(p)
    x, _ = _data(1000, 1)
    y = net.forward(torch.tensor(x, dtype=torch.float32, device="cuda")).cpu().numpy()
    yr, _ = ref.forward(pb, x.astype(np.float32).astype(np.float64))
    assert np.abs(y - yr).max() <= 1e-4 * max(1.0, np.abs(yr).max())


@pytest.mark.parametrize("n", [1, 63, 64, 1000, 4097])
def test_gradient_matches_reference(net, n):
    import torch

    p = ref.init(7) + 0.02 * np.random.default_rng(0).standard_normal(ref.n_params())
    net.set_params(p)
    net.zero_grad()
    x, t = _data(n, 2)
    xt = torch.tensor(x, dtype=torch.float32, device="cuda")
    tt = torch.tensor(t, dtype=torch.float32, device="cuda")
    loss = net.grad(xt, tt)
    g = net.read_grad()
    lr_, gr = ref.loss_grad(ref.bf16(p), x.astype(np.float32).astype(np.float64), t.astype(np.float32).astype(np.float64))
    assert abs(loss - lr_) <= 1e-4 * lr_
    assert np.abs(g - gr).max() <= 1e-3 * np.abs(gr).max()


def test_adam_step_matches_reference(net):
    import torch

    p = ref.init(9)
    net.set_params(p)
    net.zero_grad()
    x, t = _data(256, 3)
    net.grad(torch.tensor(x, dtype=torch.float32, device="cuda"), torch.tensor(t, dtype=torch.float32, device="cuda"))
    g = net.read_grad().astype(np.float64)
    net.adam_step(lr=1e-3)
    q = net.params()
    qr, _, _ = ref.adam(p.astype(np.float32).astype(np.float64), g, np.zeros_like(g), np.zeros_like(g), 1, lr=1e-3)
    assert np.abs(q - qr).max() <= 1e-6
    assert np.abs(net.read_grad()).max() == 0.0  # cleared


def test_training_lowers_the_loss(net):
    import torch

    net.set_params(ref.init(11))
    x, t = _data(4096, 4)
    xt = torch.tensor(x, dtype=torch.float32, device="cuda")
    tt = torch.tensor(t, dtype=torch.float32, device="cuda")
    net.zero_grad()
    first = net.grad(xt, tt)
    net.zero_grad()
    for _ in range(400):
        net.grad(xt, tt, want_loss=False)
        net.adam_step(lr=3e-3)
    last = net.grad(xt, tt)
    assert last < 0.2 * first
