"""Particles joined by a capillary bridge (Sec. 4.3) on the GPU.

* Hold and release (the particles are held while the liquid settles, t = 0 is the release,
  Sec. 4.3.2) against the FP64 oracle at round-off.
* Two, three and four spheres around a central drop at reduced scale (R = 12, gap 8, c = 0.5, the
  paper's tau = 1.1 and D3Q27): the particles are pulled together and stop at contact without
  passing through each other, the triangle stays equilateral and the tetrahedron regular
  (Sec. 4.3.2: the force on each particle is the same).
"""
import numpy as np
import pytest

from paper_1902_10432_gb300 import experiments as ex
from paper_1902_10432_gb300 import workloads
from _pair import compare, make_pair

pytestmark = pytest.mark.gpu


def test_hold_and_release_fp64_match_oracle():
    w = workloads.small_spheres(prec="fp64")
    g, o = make_pair(w)
    X0 = g.bodies()["X"].copy()
    for s in (g, o):
        s.set_fixed([True, True])
        s.step(120)
    bg = g.bodies()
    assert (bg["X"] == X0).all() and (bg["V"] == 0).all()  # held: no motion
    assert np.abs(g.body_forces()[0]).max() > 0  # while the forces act
    for s in (g, o):
        s.set_fixed([False, False])
        s.step(150)
    e = compare(g, o)
    assert e["flag_mismatch"] == 0
    assert e["rho"] < 1e-10 and e["vel"] < 1e-8 and e["force"] < 1e-9 and e["X"] < 1e-10
    assert np.abs(g.bodies()["X"] - X0).max() > 0.02  # released: it moves
    assert g.info()["device_error"] == 0


@pytest.mark.parametrize("n", [2, 3, 4])
def test_spheres_pulled_together_stop_at_contact(n):
    w = workloads.cluster(n, 0.5, R=12.0, h0=8.0, margin=10)
    r = ex.particle_dynamics(w, hold=3000, t_end=1500, every=20)
    assert r["device_error"] == 0 and np.isfinite(r["fluid_mass"])
    h, hm, hd = r["h"], r["h_mean"], r["h_dot"]
    tc = ex.contact_time(r["t"], hm, hd)
    print("n = %d: contact at t = %s, min h = %.2f, peak approach %.2e" % (n, tc, hm.min(), -hd.min()))
    assert hm[0] == pytest.approx(8.0, abs=1e-3)  # centres from the phase fields
    assert tc < 1500 and hm.min() < 3.0  # pulled into contact within the window
    assert h.min() > -1.0  # and stopped there: the repulsion holds the surfaces apart
    before = hm > 5.0
    spread = (h.max(axis=1) - h.min(axis=1))[before]
    if n == 3:
        assert spread.max() < 0.02 * 8.0  # equilateral on a square lattice, up to its anisotropy
    if n == 4:
        # the regular tetrahedron keeps the lattice's symmetry (up to FP32 rounding order)
        assert spread.max() < 1e-3
