"""Four-sphere cluster (Sec. 4.3.2 set-up): the CUDA path against the FP64 oracle.

At half scale (128^3, R = 12, surface gap 4), in the default GPU suite: one oracle run, and the
CUDA path with FP64, FP32 and binary16-deviation storage, compared at steps 150, 300 and 500 on the
central 64^3 crop and on the whole lattice.

* FP64 on the GPU stays at round-off of the oracle (the multi-body path: shared tiles, neighbour
  lists, repulsion culling) to step 500.
* Binary16-deviation storage: its error is the storage's. The oracle's storage model (the FP64 method
  with its stored populations rounded to binary16 deviations after every store;
  tests/golden/tetra4_half_storage.json, written by tests/golden/make_tetra4_storage.py from the
  oracle alone) deviates from the FP64 oracle by what the GPU path does, within a factor of 2 at
  every step: the kernels add nothing measurable to it.
* FP32: within the contract's tolerances (1e-4 on density and velocity, 1e-3 on force) at steps 150
  and 300 (measured 2e-6 and 8e-6 on density). The free bodies' positions then differ from the
  oracle's by ~3e-6 lattice units, and a cell whose fluid phase crosses the obstacle threshold
  (Sec. 3.2.2) changes its flag one step earlier or later than in the oracle: the cover or uncover
  event and its refill are a step apart, and the fields differ locally by O(1) for a few tens of
  steps (measured: one flag apart at step 319, velocity error 1.0 at step 320, 7e-3 at step 340).
  The FP64 method does the same: the GPU's FP64 path with the body centres moved by 3e-6 at the start
  departs from its unmoved run by more than the FP32 path does at step 500 (the test measures both;
  moved by 1e-9 it stays at 1e-11). So after step 300 the FP32 comparison is bounded by that spread
  of the method itself, and by its measured values with a margin of 3.

The full-size comparison (256^3, the oracle on the whole lattice for 500 steps, ~15 minutes on 16
cores) is kept as a long test (CBL_LONG_TESTS=1).
"""
import json
import os

import numpy as np
import pytest

from paper_1902_10432_gb300 import workloads
from _pair import compare, make_pair, rel_linf

pytestmark = pytest.mark.gpu

N_HALF = 128
STEPS_HALF = (150, 300, 500)
STORAGE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "tetra4_half_storage.json")
# stated FP32 bounds at step 500 on the crop (measured 2.1e-4, 8.1e-3, 8.1e-3, x 3)
FP32_BOUNDS_500 = dict(rho=6e-4, vel=2.5e-2, force=2.5e-2)
# body-centre offset of the FP64 spread run: the FP32 path's position difference near step 300
DX_SPREAD = 3e-6


def _crop_errors(g, o, n, h=32):
    sl = (slice(n // 2 - h, n // 2 + h),) * 3
    sg, _ = g.flags()
    so, _ = o.flags()
    fluid = (sg[sl] == 0) & (so[sl] == 0)
    rg, vg, _ = g.fields()
    ro, vo, _ = o.fields()
    occupied = fluid & (ro[sl] >= 0.05)
    Fg, _, _ = g.body_forces()
    Fo, _, _ = o.body_forces()
    return dict(rho=rel_linf(rg[sl], ro[sl], fluid),
                vel=max(rel_linf(vg[sl][..., a], vo[sl][..., a], fluid) for a in range(3)),
                vel_rho_ge_0_05=max(rel_linf(vg[sl][..., a], vo[sl][..., a], occupied) for a in range(3)),
                force=rel_linf(Fg, Fo), flag_mismatch=int((sg[sl] != so[sl]).sum()),
                crop_fluid_cells=int(fluid.sum()))


@pytest.fixture(scope="module")
def half_scale():
    import __graft_entry__
    import oracle
    from paper_1902_10432_gb300 import cbl

    __graft_entry__.build()
    w = workloads.tetra4(seed=0, prec="fp64", n=N_HALF, R=12.0, surface_gap=4.0)
    o = oracle.Oracle(w.nx, w.ny, w.nz, **{k: v for k, v in w.params.items() if k != "prec"})
    workloads.build(o, w)
    gpu = {}
    for prec in ("fp64", "fp32", "fp16dev", "fp64_moved"):
        g = cbl.Sim(w.nx, w.ny, w.nz, **dict(w.params, prec=prec.split("_")[0]))
        workloads.build(g, w)
        if prec == "fp64_moved":
            g.move_bodies(g.bodies()["X"] + DX_SPREAD)
        gpu[prec] = g
    out = {}
    done = 0
    for s in STEPS_HALF:
        o.step(s - done)
        for g in gpu.values():
            g.step(s - done)
        done = s
        out[s] = {p: dict(crop=_crop_errors(g, o, N_HALF), full=compare(g, o), device_error=g.info()["device_error"])
                  for p, g in gpu.items()}
    print("tetra4 half scale, errors against the FP64 oracle:", json.dumps(out, default=float))
    return out


def test_tetra4_half_fp64_matches_oracle(half_scale):
    for s in STEPS_HALF:
        e = half_scale[s]["fp64"]
        assert e["device_error"] == 0
        f = e["full"]
        assert f["flag_mismatch"] == 0, s
        assert f["rho"] < 1e-12 and f["vel"] < 1e-12 and f["phi_fluid"] < 1e-12, (s, f)
        assert f["force"] < 1e-10 and f["X"] < 1e-10, (s, f)


def test_tetra4_half_fp32_within_contract_then_stated_bounds(half_scale):
    for s in (150, 300):
        e = half_scale[s]["fp32"]
        assert e["device_error"] == 0
        f = e["full"]
        assert f["flag_mismatch"] == 0 and f["rho"] < 1e-4 and f["vel"] < 1e-4 and f["force"] < 1e-3, (s, f)
    e = half_scale[500]["fp32"]
    m = half_scale[500]["fp64_moved"]
    assert e["device_error"] == 0 and e["crop"]["flag_mismatch"] == 0
    b = FP32_BOUNDS_500
    assert e["crop"]["rho"] < b["rho"] and e["crop"]["vel"] < b["vel"], e["crop"]
    assert e["full"]["force"] < b["force"], e["full"]
    # the spread of the FP64 method under a 3e-6 shift of the body centres bounds the FP32 path
    # (whole lattice: the flag events need not fall inside the crop)
    for k in ("rho", "vel", "force"):
        assert e["full"][k] <= m["full"][k], (k, e["full"][k], m["full"][k])


def test_tetra4_half_fp32_held_bodies_within_contract_to_500():
    # The same cluster with the bodies held (the phase fields still evolve under the kinetics): no
    # displacement, so no flag decision is shifted, and FP32 stays within the contract's tolerances
    # through step 500 (measured against the FP64 path: density 2.5e-5, velocity 7.4e-5, force 2.2e-4
    # at most over steps 25..500, sampled every 25).
    w = workloads.tetra4(seed=0, prec="fp32", n=N_HALF, R=12.0, surface_gap=4.0)
    g, o = make_pair(w)
    for s in (g, o):
        s.set_fixed([True] * len(w.bodies))
    done = 0
    for t in (300, 500):
        g.step(t - done)
        o.step(t - done)
        done = t
        e = compare(g, o)
        print("tetra4 half scale, held bodies, FP32 at step", t, e)
        assert e["flag_mismatch"] == 0, (t, e)
        assert e["rho"] < 1e-4 and e["vel"] < 1e-4 and e["force"] < 1e-3, (t, e)
    assert g.info()["device_error"] == 0


def test_tetra4_half_fp16dev_error_is_the_storage(half_scale):
    with open(STORAGE) as fh:
        model = json.load(fh)["errors_vs_fp64"]
    for s in STEPS_HALF:
        e = half_scale[s]["fp16dev"]
        m = model[str(s)]["fp16dev"]
        assert e["device_error"] == 0
        for k, km in (("rho", "rho_crop"), ("vel", "vel_crop")):
            assert 0.5 < e["crop"][k] / m[km] < 2.0, (s, k, e["crop"][k], m[km])
        # FP32 storage alone is far below the FP32 path's error: the FP32 path is limited by arithmetic
        assert model[str(s)]["fp32"]["rho_crop"] < 1e-5


@pytest.mark.slow
@pytest.mark.skipif(os.environ.get("CBL_LONG_TESTS") != "1",
                    reason="the oracle runs 256^3 for 500 steps (~8 minutes): set CBL_LONG_TESTS=1")
def test_tetra4_crop_fp32_and_fp16_against_oracle():
    from paper_1902_10432_gb300 import cbl

    w32 = workloads.tetra4(seed=0, prec="fp32")
    g32, o = make_pair(w32)
    g32.step(w32.steps)
    o.step(w32.steps)
    w16 = workloads.tetra4(seed=0, prec="fp16dev")
    g16 = cbl.Sim(w16.nx, w16.ny, w16.nz, **w16.params)
    workloads.build(g16, w16)
    g16.step(w16.steps)
    e32 = _crop_errors(g32, o, w32.nx)
    e16 = _crop_errors(g16, o, w16.nx)
    print("tetra4 crop errors after 500 steps:", json.dumps({"fp32": e32, "fp16dev": e16}))
    assert e32["flag_mismatch"] == 0
    assert e32["rho"] < 1e-3 and e32["force"] < 5e-2
    assert e16["rho"] < 1.0
