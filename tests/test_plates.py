"""Plate set-ups on the oracle (Sec. 2.1, Sec. 4.2): the 90 degree calibration reproduces the planar
plate force of Eq. plate_force_planar, and a plate that spans the periodic lattice turns only about
the axis it spans; held bodies stay in place and start from rest when released. No GPU."""
import math
import os
import sys

import numpy as np

import oracle
from oracle import analysis as an
from paper_1902_10432_gb300 import workloads

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
import make_wetting_90 as cal  # noqa: E402

SIGMA = 3.583e-2


def test_planar_plate_force_at_90_degrees():
    # at the calibrated varrho_B the meniscus is flat (what the calibration fixes) and then the force
    # on a plate is the tension of the two liquid-vapour interfaces, F_p = 2 sigma L with L the
    # periodic bridge length (Eq. plate_force_planar), within 5 % (the Laplace-law sigma, Sec. 4.1)
    v = workloads.varrho_90()
    assert 0.6 < v < 0.8
    o, zc, ic = cal.planar_bridge(v)
    assert abs(cal.laplace_pressure(o, zc, ic)) < 2e-6  # |cos theta| < 3e-4 through Eq. young_laplace
    F = 0.0
    for _ in range(100):
        o.step(1)
        F += o.body_forces()[0][0, 2] / 100
    Fp = an.plate_force_planar(SIGMA, cal.NY)
    assert abs(F / Fp - 1) < 0.05, F / Fp
    # the plates are pulled together: the lower plate towards +z, the upper one towards -z
    assert F > 0 and o.body_forces()[0][1, 2] < 0


def _one_plate(ny, half_y):
    o = oracle.Oracle(24, ny, 20, q=19, tau=1.0, G=-5.0)
    o.add_body("box", (11.5, (ny - 1) / 2.0, 8.0), half=(6.0, half_y, 3.3), wetting_rho=0.9, mass_density=50.0)
    z, y, x = np.mgrid[0:20, 0:ny, 0:24]
    # an off-centre drop on the plate's upper face, so that the plate feels a torque about x and y
    mask = ((x - 14) ** 2 + (y - ny / 3.0) ** 2 + (z - 12) ** 2 <= 9).astype(np.uint8)
    o.init_fluid(workloads.RHO_L, workloads.RHO_V, mask)
    o.step(40)
    return o.bodies()["W"][0], o.body_forces()[1][0]


def test_plate_spanning_the_periodic_axis_turns_only_about_it():
    # a plate of half extent 5 + 3.6 in y on 8 cells spans y (support 2 (8.6 + 2.5) >= 8): it is
    # infinite along y and may turn only about y; a plate that does not span y turns freely
    W, T = _one_plate(8, 8.6)
    assert W[0] == 0.0 and W[2] == 0.0
    assert abs(W[1]) > 0 and abs(T[0]) > 0  # the torque about x is there, the turn is held
    W2, _ = _one_plate(24, 4.0)
    assert abs(W2[0]) > 0 and abs(W2[1]) > 0


def test_plate_bridge_workloads():
    for kind in ("cylinder", "planar"):
        w = workloads.plate_bridge(kind)
        z1, z2 = (b["center"][2] for b in w.bodies)
        assert z2 - z1 == w.meta["h0"] + w.meta["layers"]
        assert all(b["mass_density"] == 1.72e4 * workloads.RHO_L and not b["fixed"] for b in w.bodies)
        zs = np.nonzero(w.mask.any(axis=(1, 2)))[0]
        assert zs[0] == z1 + 2 and zs[-1] == z2 - 2  # the liquid fills the gap between the solid layers
        if kind == "planar":
            assert w.ny == w.meta["R"] and w.bodies[0]["half"][1] > w.ny / 2.0  # L = R, plates span y
            assert (w.mask == w.mask[:, :1, :]).all()
        else:
            area = w.mask[int(z1 + 5)].sum()
            assert abs(area / (math.pi * w.meta["R"] ** 2) - 1) < 0.02


def test_held_bodies_stay_and_released_bodies_start_from_rest():
    # Sec. 4.3.2: the particles are held while the liquid settles; t = 0 is the release
    w = workloads.small_spheres(prec="fp64", nx=32, ny=32, nz=48, R=6.0, gap=2.0, f=0.3)
    o = oracle.Oracle(w.nx, w.ny, w.nz, **{k: v for k, v in w.params.items() if k != "prec"})
    workloads.build(o, w)
    X0 = o.bodies()["X"].copy()
    o.set_fixed([True, True])
    o.step(40)
    b = o.bodies()
    assert (b["X"] == X0).all() and (b["V"] == 0).all() and (b["W"] == 0).all()
    F = o.body_forces()[0]
    assert np.abs(F).max() > 0  # the bridge pulls while they are held
    o.set_fixed([False, False])
    o.step(1)
    b1 = o.bodies()
    # one semi-implicit Euler step from rest: V = F / M, X = X0 + V
    F1 = o.body_forces()[0]
    assert np.allclose(b1["V"], F1 / b1["M"][:, None], rtol=1e-12, atol=0)
    assert np.allclose(b1["X"] - X0, b1["V"], rtol=1e-9, atol=1e-15)
