"""Learned force surrogate for bridged sphere pairs, and the surrogate-driven body advance.

Not part of the paper's method: the network stands in for the lattice-Boltzmann force evaluation
between full evaluations, and the plain method is both its fallback and the reference its error is
measured against.

* Features of a pair (i, j), with R* = 2 R_i R_j / (R_i + R_j) and bridge volume V_L: the scaled gap
  s sqrt(R* / V_L) of a pendular bridge, cos(contact angle), R_i / R_j and V_L / R*^3. Targets: force
  and torque on i in the frame of i (e_z from i to j) over the capillary scales 2 pi R* sigma and
  2 pi R*^2 sigma (sigma = 3.583e-2, the liquid-vapour tension). In these variables the axial force of
  a pendular bridge is close to one curve, cos(theta) times a decreasing function of the scaled gap,
  so a few dozen force-gap sweeps cover it.
* Training data come from batched two-sphere runs of the plain method (the 64-instance workload),
  the spheres held fixed and moved together step by step, the force averaged after each step has
  relaxed: quasi-static force-gap sweeps of intact bridges. (A node that turns fluid starts empty, Sec. 3.2.2, so a
  body move launches pressure pulses that the hold lets decay.)
* The hybrid advance alternates a K-step lattice-Boltzmann burst (true forces, averaged on the device;
  the per-body residual becomes a bias) with a W-step window in which the bodies move under the
  network's pair forces and torques plus the bias while the fluid is frozen, all W steps in one
  device launch (cbl_mlp_advance); the bodies' phase fields are then rebuilt at the new poses.
All heavy work runs in the CUDA library (LBM steps, network forward/backward/Adam); this module only
arranges inputs and reads results.
"""
from __future__ import annotations

import math
import time

import numpy as np

SIGMA = 3.583e-2
LOST_REFILL = 4  # device error bit: a covered node found no fluid neighbour
RHO_MID = 0.5 * (1.88844 + 0.11942)  # halfway between the coexisting liquid and vapour densities


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


def rstar(Ri, Rj):
    return 2.0 * Ri * Rj / (Ri + Rj)


def force_scale(Ri, Rj):
    return 2.0 * math.pi * rstar(Ri, Rj) * SIGMA


def features(Xi, Xj, Ri, Rj, VL, theta_deg, dims):
    frame, r = pair_frame(Xi, Xj, dims)
    Rs = rstar(Ri, Rj)
    return np.array([(r - Ri - Rj) * math.sqrt(Rs / VL), math.cos(math.radians(theta_deg)), Ri / Rj,
                     VL / Rs ** 3]), frame


def targets(F, T, frame, Ri, Rj):
    s = force_scale(Ri, Rj)
    return np.concatenate([frame @ np.asarray(F, float) / s, frame @ np.asarray(T, float) / (s * rstar(Ri, Rj))])


def bridge_state(rho, Xi, Xj, Ri, Rj, dims):
    """Liquid volume of the bridge between spheres i and j and whether it still spans the gap.

    rho: the density field as a device tensor [nz][ny][nx] (solid cells read 0). The volume counts the
    cells denser than RHO_MID in the cube of half-width max(Ri, Rj) about the middle of the gap; the
    bridge is intact if the mean density of the 2x2x2 cells about that point exceeds RHO_MID. A bridge
    evaporates or condenses towards the vapour's saturation (Laplace pressure), so its volume is
    measured, not taken from the initial drop."""
    import torch

    frame, r = pair_frame(Xi, Xj, dims)
    e = frame[2]
    mid = np.asarray(Xi, float) + e * (Ri + 0.5 * (r - Ri - Rj))
    h = int(math.ceil(max(Ri, Rj)))
    nx, ny, nz = dims
    dev = rho.device
    ax = lambda c, n, w: torch.remainder(torch.arange(-w, w + 1, device=dev) + int(math.floor(c)), n)
    ix, iy, iz = ax(mid[0], nx, h), ax(mid[1], ny, h), ax(mid[2], nz, h)
    box = rho.index_select(0, iz).index_select(1, iy).index_select(2, ix)
    vol = float((box > RHO_MID).sum())
    cx, cy, cz = ax(mid[0], nx, 0), ax(mid[1], ny, 0), ax(mid[2], nz, 0)
    core = rho.index_select(0, torch.cat([cz, (cz + 1) % nz])).index_select(1, torch.cat([cy, (cy + 1) % ny]))
    core = core.index_select(2, torch.cat([cx, (cx + 1) % nx]))
    return vol, float(core.mean()) > RHO_MID


def _pair_axis(Xi, Xj, dims):
    d = _mimg(np.asarray(Xj, float) - np.asarray(Xi, float), dims)
    return d / np.linalg.norm(d)


def generate(ws, equil=800, hold=150, avg=75, records=80, dgap=-0.04, min_gap=1.5, log=None):
    """Run the two-sphere instances `ws` (spheres held fixed) as one batch and record (features,
    targets, instance) of both bodies, step and hold: before each record but the first the surface gap
    changes by dgap cells (negative: the spheres close in, as bridges pull them; cbl_move_bodies),
    the fluid relaxes for
    hold - avg steps, and the recorded force and torque are the means over the last avg steps. The
    liquid-volume feature is the bridge's measured volume (bridge_state). An instance stops recording
    once its bridge ruptures, it loses mass in a refill, turns non-finite, or its gap falls below
    min_gap."""
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
    import torch

    rho = [torch.empty((w.nz, w.ny, w.nx), dtype=torch.float64, device="cuda") for w in ws]
    batch = cbl.Batch(sims)
    batch.step(equil)
    batch.sync()
    X, Y, inst = [], [], []
    stopped = {}  # instance -> record at which it stopped (rupture, instability or contact)
    t0 = time.perf_counter()
    for rec in range(records):
        live = [k for k in range(len(sims)) if k not in stopped]
        if rec > 0:
            for k in live:
                P = sims[k].bodies()["X"]
                e = _pair_axis(P[0], P[1], meta[k]["dims"])
                sims[k].move_bodies(np.stack([P[0] - 0.5 * dgap * e, P[1] + 0.5 * dgap * e]))
        batch.step(hold - avg)
        batch.sync()
        for k in live:
            sims[k].force_mean(reset=True)  # start the device-side sums for the averaging window
        batch.step(avg)
        batch.sync()
        Fs, Ts = {}, {}
        for k in live:
            Fs[k], Ts[k], _ = sims[k].force_mean(reset=True)
        for k in live:
            s, m = sims[k], meta[k]
            b = s.bodies()
            s.fields_device(rho[k])
            VL, intact = bridge_state(rho[k], b["X"][0], b["X"][1], m["R"][0], m["R"][1], m["dims"])
            rows = []
            for i, j in ((0, 1), (1, 0)):
                x, frame = features(b["X"][i], b["X"][j], m["R"][i], m["R"][j], max(VL, 1.0), m["theta"],
                                    m["dims"])
                rows.append((x, targets(Fs[k][i], Ts[k][i], frame, m["R"][i], m["R"][j])))
            bad = (s.info()["device_error"] & LOST_REFILL) or not all(
                np.isfinite(x).all() and np.isfinite(y).all() for x, y in rows)
            gap = pair_frame(b["X"][0], b["X"][1], m["dims"])[1] - m["R"][0] - m["R"][1]
            if bad or not intact or gap < min_gap:
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

    def norm(self):
        """The standardisation in the order cbl_mlp_advance takes it: x mean, std, min, max; y mean, std."""
        return np.concatenate([self.xm, self.xs, self.xlo, self.xhi, self.ym, self.ys]).astype(np.float32)


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
    # held-out force error; the targets are already in units of 2 pi R* sigma
    pred = sur.predict(X[te])
    d = np.linalg.norm(pred[:, :3] - Y[te][:, :3], axis=1)
    n = np.linalg.norm(Y[te][:, :3], axis=1)
    big = n >= 0.1
    q = lambda v, p: float(np.percentile(v, p)) if len(v) else None
    return sur, dict(train_seconds=train_s, n_train=int((~te).sum()), n_test=int(te.sum()),
                     heldout_force_rel_err_median=q(d[big] / n[big], 50),
                     heldout_force_rel_err_p95=q(d[big] / n[big], 95), heldout_rel_samples=int(big.sum()),
                     heldout_force_err_over_2piRsigma_median=q(d, 50),
                     heldout_force_err_over_2piRsigma_p95=q(d, 95), final_loss=float(loss))


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
    """Network forces on every body (world frame) from the bridged pairs; VL maps a pair to its
    measured bridge volume (pairs whose bridge has ruptured are left out by the caller)."""
    F = np.zeros_like(X)
    if not pairs:
        return F
    feats, frames, idx, idx_b = [], [], [], []
    for (i, j) in pairs:
        for a, b in ((i, j), (j, i)):
            f, fr = features(X[a], X[b], R[a], R[b], VL[(i, j)], theta, dims)
            feats.append(f)
            frames.append(fr)
            idx.append(a)
            idx_b.append(b)
    y = sur.predict(np.array(feats))
    for k, a in enumerate(idx):
        F[a] += frames[k].T @ (y[k, :3] * force_scale(R[a], R[idx_b[k]]))
    return F


def pair_torques(sur, X, R, pairs, VL, theta, dims):
    """Network torques on every body (world frame) from the bridged pairs."""
    T = np.zeros_like(X)
    for (i, j) in pairs:
        for a, b in ((i, j), (j, i)):
            f, fr = features(X[a], X[b], R[a], R[b], VL[(i, j)], theta, dims)
            y = sur.predict(f[None])[0]
            T[a] += fr.T @ (y[3:] * force_scale(R[a], R[b]) * rstar(R[a], R[b]))
    return T


def advance_host(sur, X, V, W, M, Iinv, R, pairs, VL, theta, dims, bias, steps):
    """The surrogate window on the host (numpy; the reference for the device version): `steps`
    semi-implicit Euler steps of the bodies under the network's pair forces and torques plus bias."""
    X, V, W = X.copy(), V.copy(), W.copy()
    for _ in range(steps):
        F = pair_forces(sur, X, R, pairs, VL, theta, dims) + bias
        T = pair_torques(sur, X, R, pairs, VL, theta, dims)
        V += F / M[:, None]
        X = (X + V) % np.asarray(dims, float)
        W += T * Iinv[:, None]
    return X, V, W


def advance_device(sur, X, V, W, M, Iinv, R, pairs, VL, theta, dims, bias, steps):
    """The surrogate window on the device: one launch of cbl_mlp_advance for all `steps` steps (pair
    features, network forward with the weights in shared memory, translation and rotation)."""
    import torch

    dev = "cuda"
    t = lambda a, dt=torch.float64: torch.tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    Xt, Vt, Wt = t(X), t(V), t(W)
    pl = [p for p in pairs]
    pt = t(np.array(pl, np.int32).reshape(-1, 2), torch.int32)
    vl = t(np.array([VL[p] for p in pl], np.float64))
    sur.mlp.advance(Xt, Vt, Wt, t(M), t(Iinv), t(np.asarray(R, float)), t(np.zeros(len(R), np.int32), torch.int32),
                    t(bias), pt, vl, steps, dims, math.cos(math.radians(theta)), sur.norm(), SIGMA)
    return Xt.cpu().numpy(), Vt.cpu().numpy(), Wt.cpu().numpy()


def hybrid_run(sim, sur, R, pairs, VL, theta, dims, windows=4, K=100, W=200, avg=50, log=None):
    """`windows` times: K LBM steps (the true force is the mean over the last avg of them; its residual
    against the network becomes a per-body bias), then W surrogate steps with the fluid frozen and the
    bodies moved by cbl_move_bodies; a final K-step burst closes the run. Returns the force errors of
    the network at the corrections and the wall time.

    Errors, over the bodies with an intact bridge: relative |F_MLP - F_LBM| / |F_LBM| where |F_LBM| is at least
    a tenth of the capillary force scale 2 pi R sigma (smaller forces make the ratio meaningless), and
    |F_MLP - F_LBM| / (2 pi R sigma) for all of them. "corrected" adds the bias of the window before."""
    import torch

    rho = torch.empty((dims[2], dims[1], dims[0]), dtype=torch.float64, device="cuda")
    b = sim.bodies()
    M = b["M"]
    Iinv = 3.0 / np.trace(b["I"], axis1=1, axis2=2)  # spheres: scalar inertia
    errs, corr, absd = [], [], []
    bias = None
    Rv = np.asarray(R, float)
    t0 = time.perf_counter()

    def burst():
        # the force is the mean over the last avg steps, summed on the device (no host read per step)
        sim.step(K - avg)
        sim.force_mean(reset=True)
        sim.step(avg)
        return sim.force_mean(reset=True)[0]

    for win in range(windows):
        F_lbm = burst()
        b = sim.bodies()
        X, V = b["X"].copy(), b["V"].copy()
        sim.fields_device(rho)
        VLm, live = {}, []
        for (i, j) in pairs:
            v, ok = bridge_state(rho, X[i], X[j], R[i], R[j], dims)
            if ok:
                VLm[(i, j)] = v
                live.append((i, j))
        F_mlp = pair_forces(sur, X, R, live, VLm, theta, dims)
        on = np.array(sorted({i for p in live for i in p}), int)  # bodies with an intact bridge
        if len(on):
            sc = 2.0 * math.pi * Rv[on] * SIGMA
            d = np.linalg.norm(F_mlp[on] - F_lbm[on], axis=1)
            n = np.linalg.norm(F_lbm[on], axis=1)
            big = n >= 0.1 * sc
            errs.append(d[big] / n[big])
            absd.append(d / sc)
            if bias is not None:
                dc = np.linalg.norm(F_mlp[on] + bias[on] - F_lbm[on], axis=1)
                corr.append(dc[big] / n[big])
        bias = F_lbm - F_mlp
        Wb = b["W"].copy()
        X, V, Wb = advance_device(sur, X, V, Wb, M, Iinv, R, live, VLm, theta, dims, bias, W)
        sim.move_bodies(X, V=V, W=Wb)
        if log and errs:
            log("window %d: %d of %d bridges intact; median relative force error %.3f over %d bodies" % (
                win, len(live), len(pairs), float(np.median(errs[-1])) if len(errs[-1]) else float("nan"),
                len(errs[-1])))
    burst()
    wall = time.perf_counter() - t0
    e = np.concatenate(errs) if errs else np.zeros(0)
    a = np.concatenate(absd) if absd else np.zeros(0)
    q = lambda v, p: float(np.percentile(v, p)) if len(v) else None
    out = dict(wall_seconds=wall, steps=windows * (K + W) + K, force_rel_err_median=q(e, 50),
               force_rel_err_p95=q(e, 95), n_rel=int(len(e)), force_err_over_2piRsigma_median=q(a, 50),
               force_err_over_2piRsigma_p95=q(a, 95))
    if corr:
        c = np.concatenate(corr)
        out.update(corrected_force_rel_err_median=q(c, 50), corrected_force_rel_err_p95=q(c, 95))
    return out
