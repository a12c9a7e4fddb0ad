"""Closed forms of Sec. 2 and App. A/B that the oracle's analysis helpers restate."""
import math

import pytest

from oracle import analysis as an


def test_sphere_bridge_limits():
    # Sec. 2.2: spherical bridge at (c = 0.75, Theta = 0) and cylindrical bridge at
    # (c = 0.2, Theta = 0) are the two ideal limits for spheres in contact.
    assert abs(an.theta_spherical(0.75)) < 1e-7  # acos near 1: sqrt(eps) limited
    assert abs(an.theta_cylindrical(0.2)) < 1e-7


@pytest.mark.parametrize("c", [0.02, 0.05, 0.1, 0.15, 0.19])
def test_cylindrical_bridge_root_is_physical(c):
    # App. B: the +pi/3 phase picks the root chi_c in [0, 1] of the cubic; Theta_c decreases
    # monotonically to 0 at c = 0.2 and the spherical solution lies above it.
    th = an.theta_cylindrical(c)
    assert 0 < th < math.pi / 2
    assert an.theta_spherical(c) > th
    assert an.theta_cylindrical(c + 0.005) < th


def test_plate_forces_and_motion():
    s, R = 3.583e-2, 20.0
    assert an.plate_force_cylinder(s, R) == pytest.approx(math.pi * s * R)
    assert an.plate_force_planar(s, R) == pytest.approx(2 * s * R)
    # App. A: at h = h0 the volume-constrained force is the cylinder force
    assert an.plate_force_volume(s, R, 12.0, 12.0) == pytest.approx(an.plate_force_cylinder(s, R))
    # Eq. plate_motion_rescaled: with t_c = sqrt(m / sigma) and L = R
    m, h0 = 1e5, 24.0
    tc = math.sqrt(m / s)
    t = 0.3 * tc
    assert an.plate_gap_planar(h0, s, R, m, t) / R == pytest.approx(h0 / R - 2 * (t / tc) ** 2)
    assert an.plate_gap_cylinder(h0, s, R, m, t) / R == pytest.approx(h0 / R - math.pi * (t / tc) ** 2)


def test_toroidal_bridge_limits_and_volume():
    # the toroidal approximation of a plate bridge (Sec. 2.1 force on a plate, Eq. young_laplace):
    # continuous into the 90-degree cylinder (Eq. plate_force), and its volume of revolution is the
    # one a voxel count of the shape gives
    s, h, V = 3.583e-2, 12.0, math.pi * 100.0 * 12.0
    a90, r90, F90 = an.toroidal_bridge(s, math.pi / 2, h, V)
    assert a90 == pytest.approx(10.0) and F90 == pytest.approx(an.plate_force_cylinder(s, 10.0))
    a, r1, F = an.toroidal_bridge(s, math.radians(89.99), h, V)
    assert F == pytest.approx(F90, rel=1e-3) and a == pytest.approx(10.0, rel=1e-3)
    a, r1, F = an.toroidal_bridge(s, math.radians(60.0), h, V)
    assert r1 == pytest.approx(12.0)
    assert F > F90  # a concave bridge pulls harder than the cylinder of the same volume
    import numpy as np

    n = 400  # voxel count of the revolved meridian r(z) = a + r1 - sqrt(r1^2 - z^2)
    z = (np.arange(n) + 0.5) / n * h - h / 2
    xy = (np.arange(2 * n) + 0.5) / (2 * n) * 60.0 - 30.0
    X, Y = np.meshgrid(xy, xy, indexing="ij")
    R2 = X * X + Y * Y
    cnt = sum(int((R2 <= (a + r1 - math.sqrt(r1 * r1 - zz * zz)) ** 2).sum()) for zz in z)
    vox = cnt * (h / n) * (60.0 / (2 * n)) ** 2
    assert vox == pytest.approx(V, rel=2e-3)
