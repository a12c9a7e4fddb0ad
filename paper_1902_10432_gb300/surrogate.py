"""Learned force surrogate for bridged sphere pairs, and the surrogate-driven body advance.

Not part of the paper's method: the network stands in for the lattice-Boltzmann force evaluation
between full evaluations, and the plain method is both its fallback and the judge of its error.

* Features of a pair (i, j) in the frame of i (e_z from i to j): gap / R_i, liquid volume / R_i^3,
  contact angle (rad), R_i / R_j. Targets: force and torque on i in that frame, divided by sigma R_i
  and sigma R_i^2 (sigma = 3.583e-2, the paper's liquid-vapour tension, Sec. 4.1).
* Training data come from batched two-sphere runs of the plain method (the 64-instance workload),
  the spheres held fixed and drawn apart slowly between records: quasi-static force-gap sweeps.
* The hybrid advance alternates a K-step lattice-Boltzmann burst (true forces; the per-body residual
  becomes a bias) with a W-step window in which the bodies move under the network's pair forces plus
  the bias while the fluid is frozen; the bodies' phase fields are then rebuilt at the new poses.
All heavy work runs in the CUDA library (LBM steps, network forward/backward/Adam); this module only
arranges inputs and reads results.
"""
from __future__ import annotations

import math
import time

import numpy as np

SIGMA = 3.583e-2
LOST_REFILL = 4  # device error bit: a covered node found no fluid neighbour


def _mimg(d, dims):
    dims = np.asarray(dims, float)
    return (d + dims / 2) % dims - dims / 2


def pair_frame(Xi, Xj, dims):
    """Unit vectors (ex, ey, ez) with ez from i to j (minimum image), and the centre distance."""
    d = _mimg(np.asarray(Xj, float) - np.asarray(Xi, float), dims)
    r = float(np.linalg.norm(d))
    ez = d / r
    ref = np.array([1.0, 0.0, 0.0]) if abs(ez[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    ex = np.cross(ref, ez)
    ex /= np.linalg.norm(ex)
    ey = np.cross(ez, ex)
    return np.stack([ex, ey, ez]), r


def features(Xi, Xj, Ri, Rj, VL, theta_deg, dims):
    frame, r = pair_frame(Xi, Xj, dims)
    return np.array([(r - Ri - Rj) / Ri, VL / Ri ** 3, math.radians(theta_deg), Ri / Rj]), frame


def targets(F, T, frame, Ri):
    return np.concatenate([frame @ np.asarray(F, float) / (SIGMA * Ri), frame @ np.asarray(T, float) / (SIGMA * Ri * Ri)])


def _pair_axis(Xi, Xj, dims):
    d = _mimg(np.asarray(Xj, float) - np.asarray(Xi, float), dims)
    return d / np.linalg.norm(d)


def generate(ws, equil=600, every=10, records=80, pull=0.004, min_gap=1.5, log=None):
    """Run the two-sphere instances `ws` as one batch and record (features, targets, instance) of both
    bodies. With pull > 0 the (fixed) spheres are drawn apart between records so that the surface gap
    grows by `pull` cells per step: a quasi-static sweep of the bridge force over the gap. Each
    recorded force is the mean of two consecutive steps (the lattice carries a period-2 mode). An
    instance stops recording once it loses mass in a refill, turns non-finite, or its gap falls
    below min_gap."""
    from paper_1902_10432_gb300 import cbl, workloads

    sims = []
    meta = []
    for w in ws:
        s = cbl.Sim(w.nx, w.ny, w.nz, **w.params)
        workloads.build(s, w)
        sims.append(s)
        R = [b["radius"] for b in w.bodies]
        VS = sum(4.0 / 3.0 * math.pi * r ** 3 for r in R)
        meta.append(dict(R=R, VL=w.meta["liquid_fraction_of_solid"] * VS, theta=w.meta["theta_deg"],
                         dims=(w.nx, w.ny, w.nz)))
    batch = cbl.Batch(sims)
    batch.step(equil)
    batch.sync()
    X, Y, inst = [], [], []
    stopped = {}  # instance -> record at which it stopped
    t0 = time.perf_counter()
    for rec in range(records):
        if pull > 0 and rec > 0:
            for k, (s, m) in enumerate(zip(sims, meta)):
                if k in stopped:
                    continue
                P = s.bodies()["X"]
                e = _pair_axis(P[0], P[1], m["dims"])
                h = 0.5 * pull * every
                s.move_bodies(np.stack([P[0] - h * e, P[1] + h * e]))
        batch.step(every - 1)
        batch.sync()
        F1 = [None if k in stopped else s.body_forces()[:2] for k, s in enumerate(sims)]
        batch.step(1)
        batch.sync()
        for k, (s, m) in enumerate(zip(sims, meta)):
            if k in stopped:
                continue
            b = s.bodies()
            F2, T2, _ = s.body_forces()
            F = 0.5 * (F1[k][0] + F2)
            T = 0.5 * (F1[k][1] + T2)
            rows = []
            for i, j in ((0, 1), (1, 0)):
                x, frame = features(b["X"][i], b["X"][j], m["R"][i], m["R"][j], m["VL"], m["theta"], m["dims"])
                rows.append((x, targets(F[i], T[i], frame, m["R"][i])))
            bad = (s.info()["device_error"] & LOST_REFILL) or not all(
                np.isfinite(x).all() and np.isfinite(y).all() for x, y in rows)
            if bad or rows[0][0][0] * m["R"][0] < min_gap:
                stopped[k] = rec
                continue
            for x, y in rows:
                X.append(x)
                Y.append(y)
                inst.append(k)
        if log and rec % 20 == 0:
            log("record %d / %d (%.1f s)" % (rec, records, time.perf_counter() - t0))
    batch.close()
    for s in sims:
        s.close()
    if log and stopped:
        log("instances stopped early (instance: record): %s" % stopped)
    return np.array(X), np.array(Y), np.array(inst)


class Surrogate:
    """Trained network plus the standardisation of its inputs and outputs. Inputs are clipped to the
    range seen in training, so the network never extrapolates."""

    def __init__(self, mlp, xm, xs, ym, ys, xlo, xhi):
        self.mlp, self.xm, self.xs, self.ym, self.ys = mlp, xm, xs, ym, ys
        self.xlo, self.xhi = xlo, xhi

    def predict(self, X):
        import torch

        Xc = np.clip(np.asarray(X, np.float64), self.xlo, self.xhi)
        xt = torch.tensor((Xc - self.xm) / self.xs, dtype=torch.float32, device="cuda")
        y = self.mlp.forward(xt).cpu().numpy().astype(np.float64)
        return y * self.ys + self.ym


def train(X, Y, inst, iters=3000, lr=3e-3, holdout=0.1, seed=0, log=None):
    """Adam on the mean squared error of the standardised targets; a tenth of the instances held out."""
    import torch

    from paper_1902_10432_gb300 import cbl

    rng = np.random.default_rng(seed)
    ids = np.unique(inst)
    test_ids = rng.choice(ids, max(1, int(round(holdout * len(ids)))), replace=False)
    te = np.isin(inst, test_ids)
    xm, xs = X[~te].mean(0), X[~te].std(0) + 1e-12
    ym, ys = Y[~te].mean(0), Y[~te].std(0) + 1e-12
    xt = torch.tensor((X[~te] - xm) / xs, dtype=torch.float32, device="cuda")
    yt = torch.tensor((Y[~te] - ym) / ys, dtype=torch.float32, device="cuda")
    net = cbl.MLP()
    p = _glorot(seed)
    net.set_params(p)
    net.zero_grad()
    t0 = time.perf_counter()
    for it in range(iters):
        want = it % 500 == 0 or it == iters - 1
        loss = net.grad(xt, yt, want_loss=want)
        net.adam_step(lr=lr if it < iters * 0.7 else lr * 0.3)
        if want and log:
            log("iter %d loss %.4g" % (it, loss))
    net.sync()
    train_s = time.perf_counter() - t0
    sur = Surrogate(net, xm, xs, ym, ys, X[~te].min(0), X[~te].max(0))
    pred = sur.predict(X[te])
    err = np.abs(pred[:, 2] - Y[te][:, 2]) / np.maximum(np.abs(Y[te][:, 2]), 1e-12)
    return sur, dict(train_seconds=train_s, n_train=int((~te).sum()), n_test=int(te.sum()),
                     axial_force_rel_err_median=float(np.median(err)), axial_force_rel_err_p95=float(np.percentile(err, 95)))


def _glorot(seed, sizes=(4, 64, 64, 64, 6)):
    rng = np.random.default_rng(seed)
    parts = []
    for k in range(len(sizes) - 1):
        ni, no = sizes[k], sizes[k + 1]
        lim = math.sqrt(6.0 / (ni + no))
        parts.append(rng.uniform(-lim, lim, size=no * ni))
        parts.append(np.zeros(no))
    return np.concatenate(parts).astype(np.float32)


def pair_forces(sur, X, R, pairs, VL, theta, dims):
    """Network forces on every body (world frame) from the bridged pairs."""
    F = np.zeros_like(X)
    if not pairs:
        return F
    feats, frames, idx = [], [], []
    for (i, j) in pairs:
        for a, b in ((i, j), (j, i)):
            f, fr = features(X[a], X[b], R[a], R[b], VL[(i, j)], theta, dims)
            feats.append(f)
            frames.append(fr)
            idx.append(a)
    y = sur.predict(np.array(feats))
    for k, a in enumerate(idx):
        F[a] += frames[k].T @ (y[k, :3] * SIGMA * R[a])
    return F


def hybrid_run(sim, sur, R, pairs, VL, theta, dims, windows=4, K=20, W=200, log=None):
    """K LBM steps (true forces, bias), then W surrogate steps (fluid frozen), `windows` times.
    Returns the force errors at the corrections and the wall time."""
    b = sim.bodies()
    M = b["M"]
    bridged = sorted({i for p in pairs for i in p})
    errs, corr = [], []
    bias = None
    t0 = time.perf_counter()
    for win in range(windows):
        sim.step(K - 1)
        F_a, _, _ = sim.body_forces()
        sim.step(1)
        F_lbm, _, _ = sim.body_forces()
        F_lbm = 0.5 * (F_a + F_lbm)  # the lattice carries a period-2 mode
        b = sim.bodies()
        X, V = b["X"].copy(), b["V"].copy()
        F_mlp = pair_forces(sur, X, R, pairs, VL, theta, dims)
        den = np.maximum(np.linalg.norm(F_lbm[bridged], axis=1), 1e-12)
        errs.append(np.linalg.norm(F_mlp[bridged] - F_lbm[bridged], axis=1) / den)
        if bias is not None:  # the force the last window moved the bodies with, at the new poses
            corr.append(np.linalg.norm(F_mlp[bridged] + bias[bridged] - F_lbm[bridged], axis=1) / den)
        bias = F_lbm - F_mlp
        for _ in range(W):
            F = pair_forces(sur, X, R, pairs, VL, theta, dims) + bias
            V += F / M[:, None]
            X = (X + V) % np.asarray(dims, float)
        sim.move_bodies(X, V=V)
        if log:
            log("window %d: median force error %.3f" % (win, float(np.median(errs[-1]))))
    sim.step(K)
    wall = time.perf_counter() - t0
    e = np.concatenate(errs)
    out = dict(wall_seconds=wall, steps=windows * (K + W) + K, force_rel_err_median=float(np.median(e)),
               force_rel_err_p95=float(np.percentile(e, 95)))
    if corr:
        c = np.concatenate(corr)
        out.update(corrected_force_rel_err_median=float(np.median(c)),
                   corrected_force_rel_err_p95=float(np.percentile(c, 95)))
    return out
