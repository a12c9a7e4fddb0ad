"""Four-sphere cluster. The multi-body path against the FP64 oracle at round-off (FP64 on both sides),
and the 256^3 crop errors of FP32 and binary16-deviation storage after 500 steps.

In this configuration the FP32 and binary16 differences from FP64 grow with time (measured: FP32
about 1e-6 at step 50, 2e-5 at 150, 1e-3 to 1e-2 at 500, while FP64 on the GPU stays at 1e-15 of the
oracle): the flow amplifies rounding, most where cells are nearly empty (a node that turns fluid
starts with density zero, Sec. 3.2.2) and the velocity m / rho is ill-conditioned. The crop test
states the errors; the FP64 test pins the implementation."""
import json
import os

import pytest

from paper_1902_10432_gb300 import workloads
from _pair import compare, make_pair, rel_linf

pytestmark = pytest.mark.gpu


@pytest.mark.slow
def test_tetra4_small_fp64_matches_oracle():
    # the cluster at half scale (128^3, R = 12, surface gap 4): four free bodies with shared tiles,
    # neighbour lists and repulsion culling, 300 steps
    w = workloads.tetra4(seed=0, prec="fp64", n=128, R=12.0, surface_gap=4.0)
    g, o = make_pair(w)
    g.step(300)
    o.step(300)
    e = compare(g, o)
    assert e["flag_mismatch"] == 0
    assert e["rho"] < 1e-12 and e["vel"] < 1e-12 and e["phi_fluid"] < 1e-12
    assert e["force"] < 1e-10 and e["X"] < 1e-10


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
    # stated errors (see the module docstring), bounded at a few times the measured values
    assert e32["flag_mismatch"] == 0
    assert e32["rho"] < 1e-3 and e32["force"] < 5e-2
    assert e16["rho"] < 1.0
