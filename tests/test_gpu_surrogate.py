"""The learned surrogate's advance on the device, and the hybrid advance against the plain method.

Not part of the paper's method: between full lattice-Boltzmann force evaluations the bodies move
under a network's pair forces (the window), with the fluid frozen.

* The window on the device (cbl_mlp_advance: pair features, the network with its weights in shared
  memory, translation and rotation of every body, all steps in one launch) against the same window
  computed on the host from the same network.
* A reduced packing (96^3, 30 spheres R U[9, 13], drops of 0.2 of the pair's solid volume at the
  25 pairs closer than 5 cells; dense enough that the drops hold: in a sparser packing the vapour
  takes up the small drops within a few hundred steps, and each body's tile overlaps at most 20
  others, within the neighbour-list capacity) advanced by the hybrid method (K-step LBM bursts that also correct the bodies, W-step surrogate windows) and by
  the plain method over the same number of steps, on the same GPU: the time-to-solution gain and
  the surrogate's force error at the corrections are measured and printed, and the test asserts
  the gain. The network is trained in the test on a small set of force-gap sweeps of held
  two-sphere bridges, so its error is large (the target of 2 % is not reached by this surrogate;
  the value is stated, not hidden).
"""
import math
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


def _random_surrogate(seed=0):
    from paper_1902_10432_gb300 import cbl, surrogate

    net = cbl.MLP()
    net.set_params(surrogate._glorot(seed))
    xm = np.array([1.0, 0.5, 1.0, 0.1])
    xs = np.array([0.8, 0.3, 0.2, 0.05])
    ym = np.array([0.01, -0.02, 0.3, 0.001, 0.002, -0.001])
    ys = np.array([0.05, 0.05, 0.4, 0.01, 0.01, 0.01])
    return surrogate.Surrogate(net, xm, xs, ym, ys, np.array([-1.0, -1.0, 0.5, 0.0]), np.array([4.0, 1.0, 2.0, 0.5]))


def test_device_window_matches_host_window():
    from paper_1902_10432_gb300 import surrogate

    sur = _random_surrogate()
    rng = np.random.default_rng(2)
    dims = (96, 80, 112)
    nb = 6
    X = rng.uniform(0, 1, (nb, 3)) * np.array(dims)
    R = rng.uniform(8, 14, nb)
    # place pairs within a few cells of contact
    for a, b in ((0, 1), (2, 3), (4, 5)):
        e = rng.normal(size=3)
        e /= np.linalg.norm(e)
        X[b] = (X[a] + e * (R[a] + R[b] + rng.uniform(1, 5))) % np.array(dims)
    pairs = [(0, 1), (2, 3), (4, 5), (1, 2)]
    VL = {p: float(rng.uniform(200, 800)) for p in pairs}
    V = rng.normal(scale=1e-3, size=(nb, 3))
    W = rng.normal(scale=1e-4, size=(nb, 3))
    M = 4.0 * 4.0 / 3.0 * math.pi * R ** 3
    Iinv = 1.0 / (0.4 * M * R * R)
    bias = rng.normal(scale=1e-3, size=(nb, 3))
    steps = 25
    Xh, Vh, Wh = surrogate.advance_host(sur, X, V, W, M, Iinv, R, pairs, VL, 45.0, dims, bias, steps)
    Xd, Vd, Wd = surrogate.advance_device(sur, X, V, W, M, Iinv, R, pairs, VL, 45.0, dims, bias, steps)
    dX = np.abs(((Xd - Xh) + np.array(dims) / 2) % np.array(dims) - np.array(dims) / 2).max()
    disp = np.abs(((Xh - X) + np.array(dims) / 2) % np.array(dims) - np.array(dims) / 2).max()
    assert disp > 1e-3  # the window moved the bodies
    # the same network and features; the device standardises the features in FP32 after forming them
    # in FP64, the host in FP64: agreement to FP32 rounding of the network's inputs
    assert dX < 1e-5 * disp + 1e-9, (dX, disp)
    assert np.abs(Vd - Vh).max() < 1e-5 * np.abs(Vh).max()
    assert np.abs(Wd - Wh).max() < 1e-5 * np.abs(Wh).max()


def test_hybrid_advance_gain_and_stated_error():
    import torch

    from paper_1902_10432_gb300 import cbl, surrogate, workloads

    ws = workloads.batch64(seed=11, n=12, gap=(3.0, 7.0), fixed=True)
    X, Y, inst = surrogate.generate(ws, equil=300, hold=100, avg=50, records=12, dgap=-0.1)
    assert len(X) > 50
    sur, tr = surrogate.train(X, Y, inst, iters=1200)
    w, pairs, VL = workloads.packing(seed=0, n_spheres=30, L=96, Rmin=9.0, Rmax=13.0, rho_s=200.0, bridge_gap=5.0,
                                     liquid_fraction=0.2)
    assert len(pairs) >= 20
    R = [b["radius"] for b in w.bodies]
    dims = (w.nx, w.ny, w.nz)
    hyb = cbl.Sim(w.nx, w.ny, w.nz, **w.params)
    workloads.build(hyb, w)
    hyb.step(500)
    torch.cuda.synchronize()
    rho = torch.empty((w.nz, w.ny, w.nx), dtype=torch.float64, device="cuda")
    hyb.fields_device(rho)
    Xb = hyb.bodies()["X"]
    states = [(p, surrogate.pair_frame(Xb[p[0]], Xb[p[1]], dims)[1] - R[p[0]] - R[p[1]],
               *surrogate.bridge_state(rho, Xb[p[0]], Xb[p[1]], R[p[0]], R[p[1]], dims)) for p in pairs]
    print("bridges after equilibration (pair, gap, volume, intact):", states)
    assert hyb.info()["device_error"] == 0
    assert sum(1 for s in states if s[3]) >= len(pairs) // 2
    res = surrogate.hybrid_run(hyb, sur, R, pairs, VL, w.meta["theta_deg"], dims, windows=3, K=100, W=300)
    hyb.close()
    plain = cbl.Sim(w.nx, w.ny, w.nz, **w.params)
    workloads.build(plain, w)
    plain.step(500)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain.step(res["steps"])
    plain.total_mass()
    plain_s = time.perf_counter() - t0
    gain = plain_s / res["wall_seconds"]
    print("surrogate hybrid vs plain, %d steps: time-to-solution gain %.2f; force error at the corrections: "
          "median %s, p95 %s over %d bodies; held-out network error: median %s" % (
              res["steps"], gain, res["force_rel_err_median"], res["force_rel_err_p95"], res["n_rel"],
              tr["heldout_force_rel_err_median"]))
    assert gain > 1.2, gain
    assert res["n_rel"] > 0
    assert res["force_err_over_2piRsigma_median"] is not None and np.isfinite(res["force_err_over_2piRsigma_median"])
