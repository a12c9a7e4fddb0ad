"""Write paper_1902_10432_gb300/data/wetting_table.json (the calibration table the
package reads): contact angle Theta vs wetting parameter varrho_B.

The paper sets wetting through varrho_B (Sec. 3.2.3: solid nodes act as fluid of that density;
varrho = 2 in the parameter table of Sec. 3.3) and relates the contact angle to the interface
tensions by Young's law (Sec. 2.1.1). This script calibrates the map with the FP64 oracle only:
a cylindrical (2D) sessile drop on a flat wall, D3Q19, tau = 1, G = -5, equilibrated, and the
angle read from a circle fitted to the rho = (rho_l + rho_v)/2 contour:
cos(Theta) = (z_wall - z_centre) / R_fit. Run: python tests/golden/make_wetting_table.py
"""
import json
import math
import os
import sys

import numpy as np

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "..", ".."))
import oracle  # noqa: E402

RHO_L, RHO_V = 1.88844, 0.11942
NX, NZ = 128, 56
R0 = 20.0
STEPS = 8000


def contour_points(r, thr, zmin):
    pts = []
    nz, nx = r.shape
    for z in range(zmin, nz - 1):
        for x in range(nx - 1):
            a = r[z, x]
            for dz, dx in ((0, 1), (1, 0)):
                b = r[z + dz, x + dx]
                if (a - thr) * (b - thr) < 0:
                    s = (thr - a) / (b - a)
                    pts.append((x + s * dx, z + s * dz))
    return np.array(pts)


def fit_circle(p):
    # algebraic (Kasa) fit: x^2 + z^2 + D x + E z + F = 0
    A = np.c_[p[:, 0], p[:, 1], np.ones(len(p))]
    b = -(p[:, 0] ** 2 + p[:, 1] ** 2)
    D, E, F = np.linalg.lstsq(A, b, rcond=None)[0]
    xc, zc = -D / 2, -E / 2
    return xc, zc, math.sqrt(xc * xc + zc * zc - F)


def measure(varrho, steps=STEPS):
    o = oracle.Oracle(NX, 1, NZ, q=19, tau=1.0, G=-5.0)
    # wall: solid layers z = 2, 3, 4 spanning x (periodic); half-way wall plane at z = 4.5
    o.add_body("box", ((NX - 1) / 2, 0.0, 3.0), half=(1e3, 1e3, 3.3), wetting_rho=varrho, fixed=True)
    z, x = np.mgrid[0:NZ, 0:NX]
    zw = 4.5
    mask = ((x - NX / 2) ** 2 + (z - zw) ** 2 <= R0 * R0) & (z > zw)
    o.init_fluid(RHO_L, RHO_V, mask.reshape(NZ, 1, NX))
    o.step(steps)
    r, _, _ = o.fields()
    r = r[:, 0, :]
    pts = contour_points(r, 0.5 * (RHO_L + RHO_V), int(zw + 4))
    xc, zc, R = fit_circle(pts)
    c = max(-1.0, min(1.0, (zw - zc) / R))
    return math.degrees(math.acos(c)), R


def main():
    rhos = [0.2, 0.4, 0.6, 0.8, 1.0, 1.2, 1.4, 1.6, 1.8]
    out = {"description": "contact angle (deg) of a 2D sessile drop vs wetting parameter, FP64 oracle, "
                          "D3Q19, tau=1, G=-5, rho0=1, %d steps" % STEPS,
           "varrho": [], "theta_deg": [], "radius": []}
    for v in rhos:
        th, R = measure(v)
        print("varrho %.2f  theta %.2f deg  R %.2f" % (v, th, R), flush=True)
        out["varrho"].append(v)
        out["theta_deg"].append(round(th, 3))
        out["radius"].append(round(R, 3))
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))),
                        "paper_1902_10432_gb300", "data", "wetting_table.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
