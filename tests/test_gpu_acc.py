"""The accumulating bulk pass (lbm_variant 2: the collision also sums the next step's density from
the populations it stores, so each step pulls the populations once) against the split pass
(lbm_variant 0) and against the FP64 oracle, through the C ABI.

The density of a cell is the same sum of the same stored values (Sec. 3.2.1, the pull of Eq.
lb_streaming), added in another order: the regions' interior cells in the collision kernel, the
regions' edge cells from a partial sum plus the sources outside the region, the cells near a solid
from the populations (the tile pass). So the two passes agree to the rounding of that sum: FP64 at
round-off, FP32 within a few float ulps per step, binary16 storage within its storage rounding.
Ragged lattices (sides that are not multiples of the 32 x 8 / 32 x 16 regions, sides smaller than a
region, region depths that do not divide nz, one-plane regions) cover the region edges; free bodies
cover the cells whose neighbourhood changes every step; moves and checkpoint loads cover the
whole-lattice density pass that restarts the accumulation.
"""
import os
import tempfile

import numpy as np
import pytest

from paper_1902_10432_gb300 import cbl, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    import torch

    __graft_entry__.build()
    assert torch.cuda.is_available()


def _sim(nx, ny, nz, prec, variant, ty=8, sz=0, **kw):
    s = cbl.Sim(nx, ny, nz, prec=prec, **kw)
    s.set_option("lbm_variant", variant)
    if variant == 2:
        s.set_option("acc_ty", ty)
        s.set_option("acc_sz", sz)
    return s


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


TOL = {"fp64": 1e-13, "fp32": 2e-5, "fp16dev": 2e-2}


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16dev"])
@pytest.mark.parametrize("dims,ty,sz", [((37, 29, 23), 8, 0), ((37, 29, 23), 16, 5), ((4, 5, 6), 8, 0),
                                         ((70, 33, 17), 8, 1), ((64, 48, 40), 16, 7), ((64, 32, 40), 8, 40)])
def test_no_bodies_against_split(prec, dims, ty, sz):
    nx, ny, nz = dims
    rng = np.random.default_rng(nx * 131 + nz)
    rho = 0.12 + 1.77 * (rng.random((nz, ny, nx)) > 0.55)
    u = 0.02 * rng.standard_normal((nz, ny, nx, 3))
    a = _sim(nx, ny, nz, prec, 0)
    b = _sim(nx, ny, nz, prec, 2, ty, sz)
    for s in (a, b):
        s.init_fluid_fields(rho, u)
        s.step(12)
    ra, va, _ = a.fields()
    rb, vb, _ = b.fields()
    assert _rel(rb, ra) < TOL[prec], (_rel(rb, ra), prec)
    assert _rel(vb, va) < 20 * TOL[prec], (_rel(vb, va), prec)
    # the mass is the sum of the stored populations: equal up to their rounding
    assert abs(b.total_mass() - a.total_mass()) < {"fp64": 1e-12, "fp32": 1e-6, "fp16dev": 1e-3}[prec] * a.total_mass()
    assert b.info()["device_error"] == 0


def test_no_bodies_fp64_against_oracle():
    import oracle

    nx, ny, nz = 45, 19, 26
    rng = np.random.default_rng(7)
    rho = 0.12 + 1.77 * (rng.random((nz, ny, nx)) > 0.5)
    u = 0.02 * rng.standard_normal((nz, ny, nx, 3))
    g = _sim(nx, ny, nz, "fp64", 2, 8, 4)
    o = oracle.Oracle(nx, ny, nz)
    g.init_fluid_fields(rho, u)
    o.init_fluid_fields(rho, u)
    g.step(20)
    o.step(20)
    rg, vg, _ = g.fields()
    ro, vo, _ = o.fields()
    assert _rel(rg, ro) < 1e-12 and _rel(vg, vo) < 1e-11
    assert abs(g.total_mass() - o.total_mass()) < 1e-12 * o.total_mass()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
@pytest.mark.parametrize("ty", [8, 16])
def test_free_spheres_against_split(prec, tol, ty):
    # free, light spheres: cells covered and uncovered, the boundary list changing every step
    w = workloads.small_spheres(prec=prec, mobility=2e-3)
    sims = []
    for variant in (0, 2):
        s = _sim(w.nx, w.ny, w.nz, prec, variant, ty, 6, **{k: v for k, v in w.params.items() if k != "prec"})
        workloads.build(s, w)
        s.step(100)
        sims.append(s)
    a, b = sims
    sa, _ = a.flags()
    sb, _ = b.flags()
    assert (sa != sb).sum() == 0
    ra, va, _ = a.fields()
    rb, vb, _ = b.fields()
    assert _rel(rb, ra) <= tol and _rel(vb, va) <= 10 * tol
    assert np.abs(a.bodies()["X"] - b.bodies()["X"]).max() < 1e-6
    assert a.info()["device_error"] == 0 and b.info()["device_error"] == 0


def test_free_spheres_fp64_against_oracle():
    from _pair import compare, make_pair

    w = workloads.small_spheres(prec="fp64", mobility=2e-3)
    g, o = make_pair(w, options={"lbm_variant": 2, "acc_ty": 8, "acc_sz": 9})
    for _ in range(3):
        g.step(40)
        o.step(40)
        e = compare(g, o)
        assert e["flag_mismatch"] == 0, e
        assert e["rho"] < 1e-12 and e["vel_vec"] < 1e-11 and e["force"] < 1e-10 and e["X"] < 1e-10, e
    assert g.info()["device_error"] == 0


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_move_and_load_restart_the_accumulation(prec):
    # a move of the bodies and a checkpoint load change flags and populations between steps: psi of
    # the next step then comes from a whole-lattice density pass, as in the split pass
    w = workloads.small_spheres(prec=prec, mobility=2e-3)
    kw = {k: v for k, v in w.params.items() if k != "prec"}
    sims = []
    with tempfile.TemporaryDirectory() as d:
        for variant in (0, 2):
            s = _sim(w.nx, w.ny, w.nz, prec, variant, 8, 0, **kw)
            workloads.build(s, w)
            s.step(30)
            X = s.bodies()["X"].copy()
            X[0, 2] -= 0.4
            s.move_bodies(X)
            s.step(30)
            path = os.path.join(d, "v%d.ckpt" % variant)
            s.save(path)
            s.step(15)
            # a fresh context with the same set-up resumes from the checkpoint
            r = _sim(w.nx, w.ny, w.nz, prec, variant, 8, 0, **kw)
            for b in w.bodies:
                bk = dict(b)
                r.add_body(bk.pop("shape"), **bk)
            r.load(path)
            r.step(25)
            sims.append(r)
    a, b = sims
    tol = TOL[prec] if prec == "fp64" else 1e-5
    ra, va, _ = a.fields()
    rb, vb, _ = b.fields()
    assert _rel(rb, ra) <= 10 * tol and _rel(vb, va) <= 100 * tol
    assert abs(b.total_mass() - a.total_mass()) < (1e-12 if prec == "fp64" else 1e-7) * a.total_mass()


def test_option_switch_mid_run():
    # switching between the passes between steps keeps the state: split, accumulating, split
    w = workloads.small_spheres(prec="fp64", mobility=2e-3)
    a = _sim(w.nx, w.ny, w.nz, "fp64", 0, **{k: v for k, v in w.params.items() if k != "prec"})
    b = _sim(w.nx, w.ny, w.nz, "fp64", 0, **{k: v for k, v in w.params.items() if k != "prec"})
    for s in (a, b):
        workloads.build(s, w)
    a.step(60)
    b.step(20)
    b.set_option("lbm_variant", 2)
    b.step(20)
    b.set_option("acc_ty", 16)
    b.step(10)
    b.set_option("lbm_variant", 0)
    b.step(10)
    ra, _, _ = a.fields()
    rb, _, _ = b.fields()
    assert _rel(rb, ra) < 1e-12
