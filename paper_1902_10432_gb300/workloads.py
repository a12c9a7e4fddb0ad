"""Seeded synthetic workloads (inputs only: geometry, parameters, liquid masks).

This module holds no arithmetic of the method; both the CUDA path and the CPU oracle are fed from
it. The paper generates every workload from geometry and parameters (Sec. 4.2 plates, Sec. 4.3
spheres), so these generators stand in for its set-ups at the sizes of the benchmark configs:

  plates48   : 48^3, two fixed 32x32x3 plates 12 cells apart, cylindrical bridge r = 10, 60 deg,
               FP64, tau = 1 (Sec. 4.2 geometry at a small size).
  spheres2   : 128x128x256, two free spheres R = 20, surface gap 4, liquid fraction and contact
               angle from a seed (Sec. 4.3.1 at R = 20).
  tetra4     : 256^3, four spheres R = 24 in a jittered tetrahedron (Sec. 4.3.2).
  small_*    : reduced versions used by the parity tests.

A body's shape is the phi = 1/2 surface. Contact angles are turned into the wetting parameter
varrho_B through the table tests/golden/wetting_table.json (written by the FP64 oracle from
sessile-drop runs).
"""
from __future__ import annotations

import json
import math
import os
from dataclasses import dataclass, field

import numpy as np

RHO_L, RHO_V = 1.88844, 0.11942  # flat-interface coexistence of G = -5, psi = 1 - exp(-rho)
_ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WETTING_TABLE = os.path.join(_ROOT, "tests", "golden", "wetting_table.json")

# Solid cells are those with fluid phase below 0.05, i.e. deeper than this below the phi = 1/2
# surface for eta = 5 ((eta/pi) asin(0.9) = 1.7822): plates are enlarged by it so that the
# configured number of cell layers is solid.
_PLATE_PAD = 1.8


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    nz: int
    params: dict
    bodies: list
    mask: np.ndarray  # uint8 (nz, ny, nx), 1 = liquid
    rho_l: float = RHO_L
    rho_v: float = RHO_V
    steps: int = 500
    meta: dict = field(default_factory=dict)

    @property
    def ncells(self):
        return self.nx * self.ny * self.nz


def varrho_for_angle(theta_deg: float) -> float:
    """Wetting parameter for a contact angle, by monotone linear interpolation of the table."""
    with open(WETTING_TABLE) as f:
        t = json.load(f)
    th = np.asarray(t["theta_deg"], float)
    vr = np.asarray(t["varrho"], float)
    order = np.argsort(th)
    th, vr = th[order], vr[order]
    if not (th[0] <= theta_deg <= th[-1]):
        raise ValueError("contact angle %.1f outside the calibrated range [%.1f, %.1f]" % (theta_deg, th[0], th[-1]))
    return float(np.interp(theta_deg, th, vr))


def _sphere_body(center, R, rho_s, varrho, fixed=False):
    return dict(shape="sphere", center=tuple(float(c) for c in center), radius=float(R), mass_density=rho_s,
                wetting_rho=varrho, fixed=fixed)


def _bridge_mask(nx, ny, nz, centers, R, volume, around):
    """Liquid cells: outside every sphere and within radius r of `around`; r by bisection so that
    the count is round(volume)."""
    z, y, x = np.mgrid[0:nz, 0:ny, 0:nx].astype(np.float32)

    def mind(a, c, n):
        d = np.abs(a - c)
        return np.minimum(d, n - d)

    outside = np.ones((nz, ny, nx), bool)
    for c in centers:
        d2 = mind(x, c[0], nx) ** 2 + mind(y, c[1], ny) ** 2 + mind(z, c[2], nz) ** 2
        outside &= d2 > R * R
    dc2 = mind(x, around[0], nx) ** 2 + mind(y, around[1], ny) ** 2 + mind(z, around[2], nz) ** 2
    target = int(round(volume))
    lo, hi = 0.0, float(max(nx, ny, nz))
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if np.count_nonzero(outside & (dc2 <= mid * mid)) < target:
            lo = mid
        else:
            hi = mid
    return (outside & (dc2 <= hi * hi)).astype(np.uint8), hi


def plates48(theta_deg=60.0, prec="fp64", n=48, gap=12, r_bridge=10.0, layers=3, width=32, tau=1.0):
    """Two fixed parallel plates (normal z) joined by a cylindrical bridge (Sec. 4.2 set-up)."""
    c = (n - 1) / 2.0
    z1 = 15 + (layers - 1) / 2.0          # solid layers z = 15..17
    z2 = z1 + layers + gap                # solid layers z = 30..32
    half = (width / 2.0 + _PLATE_PAD, width / 2.0 + _PLATE_PAD, layers / 2.0 + _PLATE_PAD)
    varrho = varrho_for_angle(theta_deg)
    bodies = [dict(shape="box", center=(c, c, z1), half=half, mass_density=4.0, wetting_rho=varrho, fixed=True),
              dict(shape="box", center=(c, c, z2), half=half, mass_density=4.0, wetting_rho=varrho, fixed=True)]
    z, y, x = np.mgrid[0:n, 0:n, 0:n]
    lo, hi = int(z1 + layers / 2.0 + 0.5), int(z2 - layers / 2.0 - 0.5)
    mask = (((x - c) ** 2 + (y - c) ** 2 <= r_bridge ** 2) & (z >= lo) & (z <= hi)).astype(np.uint8)
    params = dict(tau=tau, G=-5.0, rho0=1.0, prec=prec, mpf_kinetics=0)
    return Workload("plates48", n, n, n, params, bodies, mask, steps=500,
                    meta=dict(theta_deg=theta_deg, varrho=varrho, gap=gap, r_bridge=r_bridge))


def spheres2(seed=0, prec="fp32", nx=128, ny=128, nz=256, R=20.0, gap=4.0, mpf=1, rho_s=4.0):
    """Two free spheres on the z axis joined by a bridge; liquid fraction f ~ U[0.02, 0.2] of the
    solid volume and contact angle ~ U{30, 45, 60} deg from the seed (Sec. 4.3.1 at R = 20)."""
    rng = np.random.default_rng(seed)
    f = float(rng.uniform(0.02, 0.2))
    theta = float(rng.choice([30.0, 45.0, 60.0]))
    varrho = varrho_for_angle(theta)
    cx, cy, cz = nx / 2.0, ny / 2.0, nz / 2.0
    d = R + gap / 2.0
    centers = [(cx, cy, cz - d), (cx, cy, cz + d)]
    VS = 2 * 4.0 / 3.0 * math.pi * R ** 3
    mask, r = _bridge_mask(nx, ny, nz, centers, R, f * VS, (cx, cy, cz))
    bodies = [_sphere_body(c, R, rho_s, varrho) for c in centers]
    params = dict(tau=1.0, G=-5.0, rho0=1.0, prec=prec, mpf_kinetics=mpf)
    return Workload("spheres2", nx, ny, nz, params, bodies, mask, steps=500,
                    meta=dict(seed=seed, liquid_fraction_of_solid=f, c=f / (1 + f), theta_deg=theta,
                              varrho=varrho, bridge_radius=r))


def tetra4(seed=0, prec="fp32", n=256, R=24.0, f=0.05, theta=60.0, surface_gap=8.0, mpf=1, rho_s=4.0):
    """Four spheres in a tetrahedral cluster with integer jitter U{-2..2}^3 (Sec. 4.3.2 set-up)."""
    rng = np.random.default_rng(seed)
    varrho = varrho_for_angle(theta)
    a = 2 * R + surface_gap  # edge length
    verts = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], float) * (a / (2 * math.sqrt(2)))
    ctr = np.array([n / 2.0] * 3)
    centers = [tuple(ctr + v + rng.integers(-2, 3, size=3)) for v in verts]
    VS = 4 * 4.0 / 3.0 * math.pi * R ** 3
    mask, r = _bridge_mask(n, n, n, centers, R, f * VS, tuple(ctr))
    bodies = [_sphere_body(c, R, rho_s, varrho) for c in centers]
    params = dict(tau=1.0, G=-5.0, rho0=1.0, prec=prec, mpf_kinetics=mpf)
    return Workload("tetra4", n, n, n, params, bodies, mask, steps=500,
                    meta=dict(seed=seed, liquid_fraction_of_solid=f, theta_deg=theta, varrho=varrho))


def batch64(seed=0, n=64, prec="fp32", mpf=1, rho_s=4.0, gap=4.0):
    """Independent two-sphere bridges of uneven box size, liquid fraction and contact angle: box edges
    U{64..128} per axis, radius U[10, 24] clamped to fit the box (pair on the longest axis, surface gap
    4), liquid fraction U[0.01, 0.2] of the solid volume, contact angle U[30, 90] deg, all from one
    seed."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        L = [int(v) for v in rng.integers(64, 129, size=3)]
        R = float(rng.uniform(10.0, 24.0))
        f = float(rng.uniform(0.01, 0.2))
        theta = float(rng.uniform(30.0, 90.0))
        ax = int(np.argmax(L))
        others = [L[a] for a in range(3) if a != ax]
        R = min(R, (L[ax] - 4 - 2 * 4) / 4.0, (min(others) - 8) / 2.0)
        varrho = varrho_for_angle(theta)
        c = [v / 2.0 for v in L]
        centers = []
        for sgn in (-1, 1):
            p = list(c)
            p[ax] += sgn * (R + gap / 2.0)
            centers.append(tuple(p))
        VS = 2 * 4.0 / 3.0 * math.pi * R ** 3
        mask, r = _bridge_mask(L[0], L[1], L[2], centers, R, f * VS, tuple(c))
        bodies = [_sphere_body(p, R, rho_s, varrho) for p in centers]
        params = dict(tau=1.0, G=-5.0, rho0=1.0, prec=prec, mpf_kinetics=mpf)
        out.append(Workload("batch%02d" % k, L[0], L[1], L[2], params, bodies, mask, steps=500,
                            meta=dict(seed=seed, index=k, R=R, liquid_fraction_of_solid=f, theta_deg=theta,
                                      varrho=varrho)))
    return out


def small_spheres(seed=0, prec="fp64", nx=40, ny=36, nz=64, R=8.0, gap=3.0, mpf=1, rho_s=4.0,
                  theta=45.0, f=0.3, mobility=1e-5):
    """A reduced two-sphere bridge (the paper's mass density 4; the spheres move by cells within a
    few hundred steps)."""
    w = spheres2(seed=seed, prec=prec, nx=nx, ny=ny, nz=nz, R=R, gap=gap, mpf=mpf, rho_s=rho_s)
    varrho = varrho_for_angle(theta)
    for b in w.bodies:
        b["wetting_rho"] = varrho
    VS = 2 * 4.0 / 3.0 * math.pi * R ** 3
    centers = [b["center"] for b in w.bodies]
    w.mask, _ = _bridge_mask(nx, ny, nz, centers, R, f * VS, (nx / 2.0, ny / 2.0, nz / 2.0))
    w.params["mobility"] = mobility
    w.name = "small_spheres"
    w.meta.update(theta_deg=theta, varrho=varrho, liquid_fraction_of_solid=f)
    return w


def build(sim, w: Workload):
    """Add the workload's bodies to a simulation object (oracle or CUDA binding: both expose
    add_body / init_fluid with the same arguments) and initialise the fluid."""
    for b in w.bodies:
        kw = dict(b)
        shape = kw.pop("shape")
        sim.add_body(shape, **kw)
    sim.init_fluid(w.rho_l, w.rho_v, w.mask)
    return sim
