"""The plate experiments of Sec. 4.2 on the GPU.

* Free plates (cylindrical and planar bridge) against the FP64 oracle at round-off: moving box
  bodies, and plates that span the periodic axis (turning held to that axis).
* Static force at 90 degree wetting against F_c = pi sigma R and F_p = 2 sigma L (Sec. 2.1), and,
  off 90 degrees, the planar force against tension plus measured Laplace pressure.
* Heavy free plates (rho_S / rho_L = 1.72e4, Delta x / R = 0.05) against the rescaled early-time
  motion (h0 - h) / R = 2 (t / t_c)^2 (planar, L = R) and pi (t / t_c)^2 (cylindrical),
  Eq. plate_motion_rescaled.
"""
import math

import numpy as np
import pytest

from oracle import analysis as an
from paper_1902_10432_gb300 import experiments as ex
from paper_1902_10432_gb300 import workloads
from _pair import compare, make_pair

pytestmark = pytest.mark.gpu
SIGMA = ex.SIGMA


@pytest.mark.parametrize("kind,ratio", [("cylinder", 1.0), ("planar", 2.0)])
def test_free_plates_fp64_match_oracle(kind, ratio):
    # reduced set-up (R = 8, gap 8, plates 24 wide) with light plates, which the initial transient of
    # the sharp interfaces pushes apart by 0.7 (cylinder: the tiles recentre) and 0.5 (planar) cells
    # in the 300 steps
    w = workloads.plate_bridge(kind, prec="fp64", R=8, h0=8, width=24, margin=8, below=6, density_ratio=ratio)
    g, o = make_pair(w)
    g.step(300)
    o.step(300)
    e = compare(g, o)
    assert e["flag_mismatch"] == 0
    # the planar set-up is invariant along y, so v_y is round-off on both sides: velocity error
    # over the vector
    assert e["rho"] < 1e-10 and e["vel_vec"] < 1e-8 and e["phi_fluid"] < 1e-10
    assert e["force"] < 1e-9 and e["X"] < 1e-10
    bg, bo = g.bodies(), o.bodies()
    assert abs(bg["X"][0, 2] - w.bodies[0]["center"][2]) > 0.4  # the plates did move
    # the set-ups are mirror symmetric, so the turns are round-off on both sides (~1e-18)
    assert e["torque"] < 1e-9 and np.abs(bg["W"] - bo["W"]).max() < 1e-14
    if kind == "planar":  # spans y: no turn about x or z, on both sides exactly
        assert (bg["W"][:, [0, 2]] == 0).all() and (bo["W"][:, [0, 2]] == 0).all()
    assert g.info()["device_error"] == 0


@pytest.mark.parametrize("kind", ["cylinder", "planar"])
def test_static_plate_force_at_90_degrees(kind):
    w = workloads.plate_bridge(kind, fixed=True)
    r = ex.static_force(w)
    assert r["device_error"] == 0
    if kind == "cylinder":
        Fth = an.plate_force_cylinder(SIGMA, w.meta["R"])
    else:
        Fth = an.plate_force_planar(SIGMA, w.meta["depth"])
    assert abs(r["F"] / Fth - 1) < 0.06, r["F"] / Fth
    assert abs(r["F_vec"][0]) < 1e-3 * r["F"] and abs(r["F_vec"][1]) < 1e-3 * r["F"]


@pytest.mark.parametrize("varrho", [0.66, 0.74])
def test_planar_force_off_90_degrees_is_tension_plus_laplace_pressure(varrho):
    # a curved meniscus adds the Laplace pressure over the wetted area: F = 2 sigma L sin(theta)
    # - dp W L with cos(theta) = -dp h / (2 sigma) (Eq. young_laplace for a planar meniscus of
    # contact angle theta on both plates), dp and the liquid width W measured from the density
    w = workloads.plate_bridge("planar", fixed=True, varrho=varrho)
    r = ex.static_force(w)
    rho = r["rho"]
    h, L = w.meta["h0"], w.meta["depth"]
    z1, z2 = (b["center"][2] for b in w.bodies)
    zc, ic = int(round((z1 + z2) / 2)), w.nx // 2
    rl = rho[zc - 2:zc + 3, :, ic - 2:ic + 2].mean()
    rv = rho[zc - 2:zc + 3, :, 2:6].mean()
    dp = float(an.eos_pressure(np.array([rl]))[0] - an.eos_pressure(np.array([rv]))[0])
    prof = rho[zc, 0, :]
    thr = 0.5 * (workloads.RHO_L + workloads.RHO_V)
    xs = [i + (thr - prof[i]) / (prof[i + 1] - prof[i]) for i in range(w.nx - 1)
          if (prof[i] - thr) * (prof[i + 1] - thr) < 0]
    W = xs[-1] - xs[0]
    cos_t = -dp * h / (2 * SIGMA)
    assert 0.02 < abs(cos_t) < 0.2  # the meniscus is curved (about 84 to 96 degrees)
    pred = 2 * SIGMA * L * math.sqrt(1 - cos_t ** 2) - dp * W * L
    assert abs(r["F"] / pred - 1) < 0.05, (r["F"], pred)


@pytest.mark.parametrize("kind,coef", [("cylinder", math.pi), ("planar", 2.0)])
def test_free_heavy_plates_follow_the_rescaled_motion(kind, coef):
    w = workloads.plate_bridge(kind)
    res = ex.plate_motion(w, tc_end=0.15)
    assert res["device_error"] == 0
    t, dh = res["t_over_tc"], res["dh_over_R"]
    k, slope = ex.fit_t2(t, dh)
    print("%s: (h0 - h)/R = %.4f (t/t_c)^2 (theory %.4f), log-log slope %.3f" % (kind, k, coef, slope))
    # the theory of Eq. plate_motion_rescaled, via the oracle's closed forms with L = R
    R, m, tc = w.meta["R"], res["m"], res["t_c"]
    gap = an.plate_gap_cylinder if kind == "cylinder" else an.plate_gap_planar
    theory = (w.meta["h0"] - gap(w.meta["h0"], SIGMA, R, m, t * tc)) / R
    assert np.allclose(theory, coef * t ** 2)
    # early times: within 10 % of the theory, uniformly accelerated
    assert abs(k / coef - 1) < 0.10
    assert abs(slope - 2.0) < 0.1
    assert np.abs(dh - theory).max() < 0.10 * theory[-1]
    if kind == "planar":
        assert (res["W"][:, [0, 2]] == 0).all()


def test_plates48_60_degrees_against_toroidal_estimate():
    # The 48^3 two-plate bridge at 60 degrees (plates 12 apart, a cylinder of r = 10 seeded, FP64):
    # after equilibration the force on a plate against the toroidal (circular-meridian) estimate of
    # a bridge between parallel plates (the force of Sec. 2.1 with the Laplace pressure of Eq.
    # young_laplace: F = pi sigma a (1 + a / r1), r1 = h / (2 cos theta)) for the seeded volume
    # pi 10^2 12 (F = 1.91), within the 10 % that the approximation itself is good to. Printed beside
    # it: the neck radius a measured at mid-gap (the area of the liquid cross-section at the
    # mid-density surface) and the toroidal force for that neck at 60 degrees. The bridge loses about
    # a third of its liquid to the vapour (its Laplace pressure is above the vapour's) and its neck
    # narrows to ~7.7; the measured force then corresponds, in the toroidal picture, to a contact
    # angle well below 60 degrees in this geometry, so the agreement at the seeded volume is partly
    # a compensation of the two.
    w = workloads.plates48(prec="fp64")
    r = ex.static_force(w, steps=6000, avg=200)
    assert r["device_error"] == 0
    mid = 0.5 * (workloads.RHO_L + workloads.RHO_V)
    rho = r["rho"]
    V = float((rho[18:30] > mid).sum())  # fluid layers between the half-way walls 17.5 and 29.5
    neck = min(math.sqrt(float((rho[z] > mid).sum()) / math.pi) for z in range(22, 26))
    h, th = 12.0, math.radians(60.0)
    _, r1, Fseed = an.toroidal_bridge(SIGMA, th, h, math.pi * 100.0 * h)
    Fneck = math.pi * SIGMA * neck * (1.0 + neck / r1)
    print("plates48 60 deg: F = %.4f; toroidal: seeded volume %.4f, measured neck %.2f -> %.4f; liquid cells in "
          "the gap %.0f" % (r["F"], Fseed, neck, Fneck, V))
    assert abs(r["F"] / Fseed - 1) < 0.10, (r["F"], Fseed)
    assert abs(r["F_vec"][0]) < 1e-6 * r["F"] and abs(r["F_vec"][1]) < 1e-6 * r["F"]
