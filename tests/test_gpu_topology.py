"""Bridge topology between two spheres in contact (Sec. 2.2): below the cylindrical solution
Theta_c(c) one radius of curvature of the bridge is negative (concave: the liquid surface is
narrowest at the contact plane), between the cylindrical and the spherical solutions the bridge is
convex (widest at the contact plane). Two held spheres of R = 24 whose phase fields overlap by two
cells (so that their solid cells touch), relaxed for 6000 steps from a central drop of liquid
fraction c = V_L / (V_L + V_S); the outer liquid-vapour surface is located to a fraction of a cell
along the diameter of each slice, and the sign of its curvature along the axis is read from a
parabola fitted over the slices near the contact plane."""
import math

import numpy as np
import pytest

from oracle import analysis as an
from paper_1902_10432_gb300 import cbl, workloads

pytestmark = pytest.mark.gpu


def _outer_surface(rho, solid, z, xc):
    # the outermost mid-density crossings left and right of the axis, interpolated linearly
    thr = 0.5 * (workloads.RHO_L + workloads.RHO_V)
    row = rho[z]
    nx = len(row)
    right = [x + (thr - row[x]) / (row[x + 1] - row[x]) for x in range(int(xc) + 1, nx - 1) if row[x] > thr >= row[x + 1]]
    left = [x + (row[x] - thr) / (row[x] - row[x + 1]) for x in range(0, int(xc)) if row[x] <= thr < row[x + 1]]
    if not right or not left or solid[z, int(right[-1])]:
        return None
    return 0.5 * ((right[-1] - xc) + (xc - left[0] - 1.0))


@pytest.mark.parametrize("c,theta", [(0.05, 30.0), (0.1, 20.0), (0.15, 45.0), (0.2, 50.0)])
def test_bridge_shape_follows_the_topology_map(c, theta):
    th_c, th_s = math.degrees(an.theta_cylindrical(c)), math.degrees(an.theta_spherical(c))
    concave = theta < th_c
    assert theta < th_s  # the spheres stay in contact: not a separating spherical bridge
    w = workloads.small_spheres(prec="fp32", nx=96, ny=96, nz=128, R=24.0, gap=-2.0, theta=theta, f=c / (1.0 - c),
                                mpf=0)
    s = cbl.Sim(w.nx, w.ny, w.nz, **w.params)
    workloads.build(s, w)
    s.set_fixed([True, True])
    s.step(6000)
    assert s.info()["device_error"] == 0
    j = w.ny // 2
    rho = s.fields()[0][:, j, :]
    solid = s.flags()[0][:, j, :]
    zm, xc = w.nz // 2, (w.nx - 1) / 2.0  # contact plane and axis
    pts = [(z - zm, _outer_surface(rho, solid, z, xc)) for z in range(zm - 8, zm + 9)]
    pts = [(dz, r) for dz, r in pts if r is not None]
    assert len(pts) >= 5  # the bridge spans the contact plane
    dz = np.array([p[0] for p in pts], float)
    r = np.array([p[1] for p in pts])
    b = np.polyfit(dz ** 2, r, 1)[0]  # r = a + b dz^2
    print("c %.2f theta %.0f (Theta_c %.1f, Theta_s %.1f): neck radius %.2f, curvature coefficient %+.4f (%s)" % (
        c, theta, th_c, th_s, r[np.argmin(np.abs(dz))], b, "concave" if concave else "convex"))
    if concave:
        assert b > 0
    else:
        assert b < 0
