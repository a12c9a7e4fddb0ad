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


def make(w: workloads.Workload, q: int = 19) -> cbl.Sim:
    s = cbl.Sim(w.nx, w.ny, w.nz, q=q, **w.params)
    workloads.build(s, w)
    return s


def mean_force(sim: cbl.Sim, n: int = 200, body: int = 0) -> np.ndarray:
    """Force on `body` averaged over the next n steps (the steps are taken)."""
    acc = np.zeros(3)
    for _ in range(n):
        sim.step(1)
        acc += sim.body_forces()[0][body]
    return acc / n


def static_force(w: workloads.Workload, steps: int = 8000, avg: int = 200, q: int = 19) -> dict:
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
                 q: int = 19) -> dict:
    """Distance decrease of two free plates (bodies 0 and 1, normal z) over t_end steps.

    The fluid first relaxes for `equil` steps from its sharp initial state; the plates are then put
    back at their initial positions at rest (they drift by less than 0.02 cells meanwhile) and the
    clock starts. The run ends at t_end steps, or at t = tc_end * t_c when t_end is 0. Returns t,
    t / t_c, (h0 - h) / R, the plate mass m, t_c and the mean force of the last 2 steps of each
    sample."""
    s = make(w, q)
    try:
        b = s.bodies()
        X0 = b["X"].copy()
        m = float(b["M"][0])
        d0 = X0[1, 2] - X0[0, 2]
        if equil:
            s.step(equil)
            s.move_bodies(X0, V=np.zeros((2, 3)), W=np.zeros((2, 3)))
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
