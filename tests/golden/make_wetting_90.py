"""Write paper_1902_10432_gb300/data/wetting_90.json (the calibration table the
package reads): the wetting parameter varrho_B of a 90 degree contact angle.

At 90 degrees the liquid-vapour interfaces of a planar bridge between parallel plates are flat
(Sec. 2.1: the plate-force derivation assumes 90 degree wetting so that the solid-liquid terms
drop out), so the Laplace pressure inside the bridge vanishes (Eq. young_laplace with infinite
radius). This script finds varrho_B where the bulk pressure of the liquid at mid-gap (Eq. pressure)
equals that of the vapour, by secant steps on the FP64 oracle only: D3Q19, tau = 1, G = -5, two
fixed plates of three solid layers spanning a periodic 4-cell y extent (a 2D planar bridge), gap
20, liquid width 32. Run: python tests/golden/make_wetting_90.py

The sessile-drop table (wetting_table.json) places 90 degrees at varrho ~ 0.739; in the plate
geometry that value leaves a concave meniscus of about 86.6 degrees, which matters for the plate
force at the few-percent level (dF/F ~ 2 R cos(theta) / h), hence this direct calibration.
"""
import json
import os
import sys

import numpy as np

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "..", ".."))
import oracle  # noqa: E402
from oracle import analysis as an  # noqa: E402

RHO_L, RHO_V = 1.88844, 0.11942
PLATE_PAD = 1.8  # phi = 1/2 surface lies this far outside the solid layers (eta = 5)
STEPS = 4000
NX, NY, NZ, WIDTH, GAP, LAYERS = 64, 4, 40, 32, 20, 3


def planar_bridge(varrho, steps=STEPS):
    """The oracle after `steps` steps and the mid-gap indices (z, x) of the bridge centre."""
    z1 = 6 + (LAYERS - 1) / 2.0
    z2 = z1 + LAYERS + GAP
    cx = (NX - 1) / 2.0
    half = (24.0 + PLATE_PAD, NY / 2.0 + 2 * PLATE_PAD, LAYERS / 2.0 + PLATE_PAD)
    o = oracle.Oracle(NX, NY, NZ, q=19, tau=1.0, G=-5.0)
    for zz in (z1, z2):
        o.add_body("box", (cx, (NY - 1) / 2.0, zz), half=half, wetting_rho=varrho, fixed=True)
    z, y, x = np.mgrid[0:NZ, 0:NY, 0:NX]
    lo, hi = int(z1 + LAYERS / 2.0 + 0.5), int(z2 - LAYERS / 2.0 - 0.5)
    o.init_fluid(RHO_L, RHO_V, ((np.abs(x - cx) <= WIDTH / 2) & (z >= lo) & (z <= hi)).astype(np.uint8))
    o.step(steps)
    return o, int(round((z1 + z2) / 2)), int(round(cx))


def laplace_pressure(o, zc, ic):
    """p(liquid at the bridge centre) - p(vapour beside it), Eq. pressure on cell averages."""
    r = o.fields()[0]
    rl = r[zc - 2:zc + 3, :, ic - 2:ic + 2].mean()
    rv = r[zc - 2:zc + 3, :, 1:4].mean()
    return float(an.eos_pressure(np.array([rl]))[0] - an.eos_pressure(np.array([rv]))[0])


def main():
    samples = []

    def dp_of(v):
        dp = laplace_pressure(*planar_bridge(v))
        samples.append((round(v, 6), dp))
        print("varrho %.5f  dp %+.4e" % (v, dp), flush=True)
        return dp

    a, b = 0.70, 0.72
    fa, fb = dp_of(a), dp_of(b)
    for _ in range(6):
        c = b - fb * (b - a) / (fb - fa)
        fc = dp_of(c)
        a, fa, b, fb = b, fb, c, fc
        if abs(b - a) < 2e-4:
            break
    out = {"description": "varrho_B with a flat planar meniscus (zero Laplace pressure, 90 degree wetting), "
                          "FP64 oracle, D3Q19, tau=1, G=-5, rho0=1, plates gap %d, %d steps" % (GAP, STEPS),
           "varrho_90": round(b, 5), "samples": samples}
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))),
                        "paper_1902_10432_gb300", "data", "wetting_90.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
