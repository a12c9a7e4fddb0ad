"""The plate experiments of Sec. 4.2 on the GPU, through the C ABI.

  static_force : a bridge between fixed plates, the force on a plate after equilibration, to compare
                 with F_c = pi sigma R (cylindrical) and F_p = 2 sigma L (planar) of Sec. 2.1.
  plate_motion : heavy free plates released at rest, the decrease of their distance h(t) over the
                 first part of the motion, in the paper's units h / R and t / t_c, t_c = sqrt(m / sigma)
                 with m the mass of one plate (Eq. plate_motion_rescaled).

Forces are averaged over consecutive steps: with tau = 1 the lattice carries an undamped period-2
mode left by the sharp initial interfaces, under which the per-step force on a wall alternates about
its mean. The mode cancels in the average (and in the motion, which integrates the force).
"""
from __future__ import annotations

import math

import numpy as np

from . import cbl, workloads

SIGMA = 3.583e-2  # liquid-vapour tension from the Laplace law (Sec. 4.1), the value used for forces


def make(w: workloads.Workload, q: int = None) -> cbl.Sim:
    """The workload on the GPU (its own velocity set unless `q` is given; D3Q19 by default)."""
    params = dict(w.params)
    if q is not None:
        params["q"] = q
    s = cbl.Sim(w.nx, w.ny, w.nz, **params)
    for k, v in w.meta.get("options", {}).items():
        s.set_option(k, v)
    workloads.build(s, w)
    return s


def mean_force(sim: cbl.Sim, n: int = 200, body: int = 0) -> np.ndarray:
    """Force on `body` averaged over the next n steps (the steps are taken)."""
    acc = np.zeros(3)
    for _ in range(n):
        sim.step(1)
        acc += sim.body_forces()[0][body]
    return acc / n


def static_force(w: workloads.Workload, steps: int = 8000, avg: int = 200, q: int = None) -> dict:
    """Mean z-force on the lower plate (towards the upper one) over the last `avg` of `steps` steps,
    and the density field at the end; the workload's plates should be fixed."""
    s = make(w, q)
    try:
        s.step(steps - avg)
        F = mean_force(s, avg)
        rho = s.fields()[0]
        err = s.info()["device_error"]
    finally:
        s.close()
    return dict(F=float(F[2]), F_vec=F, rho=rho, device_error=err)


def plate_motion(w: workloads.Workload, t_end: int = 0, tc_end: float = 0.15, samples: int = 20, equil: int = 3000,
                 q: int = None) -> dict:
    """Distance decrease of two free plates (bodies 0 and 1, normal z) over t_end steps.

    The plates are held while the fluid relaxes for `equil` steps from its sharp initial state, then
    released at rest and the clock starts (as for the particles of Sec. 4.3.2). The run ends at t_end steps, or at t = tc_end * t_c when t_end is 0. Returns t,
    t / t_c, (h0 - h) / R, the plate mass m, t_c and the mean force of the last 2 steps of each
    sample."""
    s = make(w, q)
    try:
        b = s.bodies()
        X0 = b["X"].copy()
        m = float(b["M"][0])
        d0 = X0[1, 2] - X0[0, 2]
        if equil:
            s.set_fixed([True, True])
            s.step(equil)
            s.set_fixed([False, False])
        R = w.meta["R"]
        tc = math.sqrt(m / SIGMA)
        if not t_end:
            t_end = int(round(tc_end * tc))
        ts = np.linspace(0, t_end, samples + 1)[1:].astype(int)
        dh, Fm, t = [], [], 0
        for tt in ts:
            s.step(int(tt) - t - 2)
            Fm.append(float(mean_force(s, 2)[2]))
            t = int(tt)
            X = s.bodies()["X"]
            dh.append((d0 - (X[1, 2] - X[0, 2])) / R)
        out = dict(t=ts.astype(float), t_over_tc=ts / tc, dh_over_R=np.array(dh), F=np.array(Fm), m=m, t_c=tc,
                   W=s.bodies()["W"].copy(), device_error=s.info()["device_error"])
    finally:
        s.close()
    return out


def fit_t2(t_over_tc: np.ndarray, dh_over_R: np.ndarray) -> tuple:
    """Least-squares k of (h0 - h) / R = k (t / t_c)^2 through the origin, and the log-log slope of
    (h0 - h) against t over the samples (2 for uniformly accelerated plates)."""
    x = np.asarray(t_over_tc, float) ** 2
    y = np.asarray(dh_over_R, float)
    k = float((x * y).sum() / (x * x).sum())
    slope = float(np.polyfit(np.log(t_over_tc), np.log(np.maximum(y, 1e-300)), 1)[0])
    return k, slope


def _pair_gaps(X, R, dims):
    """Surface distances |X_i - X_j| - 2R of every pair (minimum image)."""
    L = np.asarray(dims, float)
    out = []
    for i in range(len(X)):
        for j in range(i + 1, len(X)):
            d = X[j] - X[i]
            d -= L * np.round(d / L)
            out.append(float(np.linalg.norm(d)) - 2.0 * R)
    return out


def phi_gap(sim: cbl.Sim, w: workloads.Workload) -> float:
    """Closest distance of the phi = 1/2 surfaces of a pair on the z axis (bodies 0 below, 1 above),
    read along the line of centres: the surface distance as the phase fields see it, which the
    kinetics can change without moving the rigid-body centres."""
    X = sim.bodies()["X"]
    i, j = int(round(X[0, 0])), int(round(X[0, 1]))
    p0 = sim.phi(0)[:, j, i]
    p1 = sim.phi(1)[:, j, i]
    z0, z1 = int(round(X[0, 2])), int(round(X[1, 2]))

    def crossing(p, a, b, step):
        for z in range(a, b, step):
            if (p[z] - 0.5) * (p[z + step] - 0.5) <= 0 and p[z] != p[z + step]:
                return z + step * (p[z] - 0.5) / (p[z] - p[z + step])
        return float("nan")

    return crossing(p1, z1, z0, -1) - crossing(p0, z0, z1, 1)


def particle_dynamics(w: workloads.Workload, hold: int = 15000, t_end: int = 8000, every: int = 50,
                      q: int = None, phi_every: int = 0) -> dict:
    """Spheres joined by a capillary bridge (Sec. 4.3): the particles are held for `hold` steps while
    the liquid settles, then released at t = 0 (Sec. 4.3.2); the surface distance of every pair is
    sampled every `every` steps up to t_end. Returns t, the pair distances h (samples x pairs), their
    mean, its rate of change (central differences) and the bodies' final state; for a pair with
    phi_every > 0, also the phase-field surface distance (phi_gap) every phi_every steps."""
    s = make(w, q)
    try:
        nb = len(w.bodies)
        R = float(w.bodies[0]["radius"])
        dims = (w.nx, w.ny, w.nz)
        if hold:
            s.set_fixed([True] * nb)
            s.step(hold)
            s.set_fixed([False] * nb)
        ts, hs = [0], [_pair_gaps(s.bodies()["X"], R, dims)]
        tp, hp = [], []
        if phi_every and nb == 2:
            tp.append(0)
            hp.append(phi_gap(s, w))
        t = 0
        while t < t_end:
            s.step(every)
            t += every
            ts.append(t)
            hs.append(_pair_gaps(s.bodies()["X"], R, dims))
            if phi_every and nb == 2 and t % phi_every == 0:
                tp.append(t)
                hp.append(phi_gap(s, w))
        b = s.bodies()
        try:
            mass = s.total_mass()
        except cbl.CblError:  # not finite: reported as NaN, the caller checks
            mass = float("nan")
        out = dict(t=np.array(ts, float), h=np.array(hs), X=b["X"].copy(), V=b["V"].copy(),
                   device_error=s.info()["device_error"], fluid_mass=mass, t_phi=np.array(tp, float),
                   h_phi=np.array(hp))
    finally:
        s.close()
    hm = out["h"].mean(axis=1)
    out["h_mean"] = hm
    out["h_dot"] = np.gradient(hm, out["t"])
    return out


def contact_time(t: np.ndarray, h: np.ndarray, h_dot: np.ndarray, frac: float = 0.1) -> float:
    """The time the approach stops: the first sample after the fastest approach (minimum of h_dot)
    where |h_dot| has fallen below `frac` of its peak (the steep drop of the velocity to zero that
    marks contact, Sec. 4.3.2); inf if it never does."""
    k = int(np.argmin(h_dot))
    peak = -h_dot[k]
    if peak <= 0:
        return math.inf
    after = np.nonzero(-h_dot[k:] < frac * peak)[0]
    return float(t[k + after[0]]) if len(after) else math.inf


def _plates_summary() -> dict:
    out = {}
    for kind in ("cylinder", "planar"):
        w = workloads.plate_bridge(kind, fixed=True)
        F = static_force(w)["F"]
        L = w.meta["R"] if kind == "cylinder" else w.meta["depth"]
        Fth = math.pi * SIGMA * L if kind == "cylinder" else 2.0 * SIGMA * L
        r = plate_motion(workloads.plate_bridge(kind))
        k, slope = fit_t2(r["t_over_tc"], r["dh_over_R"])
        out[kind] = dict(F=F, F_over_theory=F / Fth, k=k, k_theory=math.pi if kind == "cylinder" else 2.0,
                         loglog_slope=slope, t_end_over_tc=float(r["t_over_tc"][-1]))
    return out


def _particles_summary() -> dict:
    out = {}
    for n in (2, 3, 4):
        for c in (0.2, 0.3, 0.5):
            w = workloads.cluster(n, c)
            r = particle_dynamics(w, hold=15000 if n < 4 else 10000, t_end=6000)
            k = int(np.argmin(r["h_dot"]))
            out["%d_particles_c%.1f" % (n, c)] = dict(
                contact_t=contact_time(r["t"], r["h_mean"], r["h_dot"]), peak_approach=float(-r["h_dot"][k]),
                peak_t=float(r["t"][k]), min_h=float(r["h_mean"].min()),
                h_dot_at_200=float(r["h_dot"][4]), device_error=int(r["device_error"]))
    return out


if __name__ == "__main__":
    import json
    import sys

    what = sys.argv[1] if len(sys.argv) > 1 else "plates"
    if what not in ("plates", "particles"):
        raise SystemExit("usage: python -m paper_1902_10432_gb300.experiments [plates|particles]")
    print(json.dumps(_plates_summary() if what == "plates" else _particles_summary(), indent=1))
