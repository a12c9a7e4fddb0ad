"""Helpers shared by the GPU parity tests: build one workload on the CUDA path and on the oracle."""
import numpy as np

import oracle
from paper_1902_10432_gb300 import cbl, workloads


def make_pair(w, options=None, **override):
    """The workload on the CUDA path (execution options, e.g. tile_tail, applied before the bodies are
    added) and on the oracle."""
    params = dict(w.params)
    params.update(override)
    g = cbl.Sim(w.nx, w.ny, w.nz, **params)
    for k, v in (options or {}).items():
        g.set_option(k, v)
    workloads.build(g, w)
    o = oracle.Oracle(w.nx, w.ny, w.nz, **{k: v for k, v in params.items() if k != "prec"})
    workloads.build(o, w)
    return g, o


def rel_linf(a, b, mask=None):
    a = np.asarray(a)
    b = np.asarray(b)
    if mask is not None:
        a, b = a[mask], b[mask]
    scale = np.abs(b).max()
    return float(np.abs(a - b).max() / scale) if scale > 0 else float(np.abs(a - b).max())


def compare(g, o):
    """Relative L-infinity errors of density, each velocity component (fluid cells where both sides
    agree on the flag), per-body force and torque; plus the number of disagreeing flags."""
    sg, og = g.flags()
    so, oo = o.flags()
    fluid = (sg == 0) & (so == 0)
    rg, vg, pg = g.fields()
    ro, vo, po = o.fields()
    out = dict(flag_mismatch=int((sg != so).sum() + ((sg == 1) & (og != oo)).sum()),
               rho=rel_linf(rg, ro, fluid),
               vel=max(rel_linf(vg[..., a], vo[..., a], fluid) for a in range(3)),
               # the same over the velocity vector (for set-ups where a component is zero up to
               # round-off by symmetry, whose per-component relative error is noise over noise)
               vel_vec=rel_linf(vg[fluid], vo[fluid]),
               phi_fluid=float(np.abs(pg - po).max()))
    if o.nbodies:
        Fg, Tg, Pg = g.body_forces()
        Fo, To, Po = o.body_forces()
        out["force"] = rel_linf(Fg, Fo)
        out["torque"] = float(np.abs(Tg - To).max() / max(np.abs(To).max(), np.abs(Fo).max() * 10))
        out["parts"] = rel_linf(Pg, Po)
        bg, bo = g.bodies(), o.bodies()
        out["X"] = float(np.abs(bg["X"] - bo["X"]).max())
        out["V"] = float(np.abs(bg["V"] - bo["V"]).max())
        out["M"] = rel_linf(bg["M"], bo["M"])
    return out
