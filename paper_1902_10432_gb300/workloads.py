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
  cluster    : two, three or four spheres R = 30 around a central drop (Sec. 4.3 dynamics runs).
  plate_bridge: the plate experiments of Sec. 4.2 (cylindrical or planar bridge at 90 degrees, heavy
               free plates, R = 20).

A body's shape is the phi = 1/2 surface. Contact angles are turned into the wetting parameter
varrho_B through the table data/wetting_table.json (written by the FP64 oracle from
sessile-drop runs).
"""
from __future__ import annotations

import json
import math
import os
from dataclasses import dataclass, field

import numpy as np

RHO_L, RHO_V = 1.88844, 0.11942  # flat-interface coexistence of G = -5, psi = 1 - exp(-rho)
_DATA = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data")
WETTING_TABLE = os.path.join(_DATA, "wetting_table.json")
WETTING_90 = os.path.join(_DATA, "wetting_90.json")
PLATE_DENSITY_RATIO = 1.72e4  # rho_S / rho_L of the free plates (Sec. 4.2: slow, heavy plates)

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


def varrho_90() -> float:
    """Wetting parameter of a 90 degree contact angle: the value for which the meniscus of a planar
    bridge between plates is flat (zero Laplace pressure), from data/wetting_90.json (written
    by the FP64 oracle). The sessile-drop table places 90 degrees a few degrees off in the plate
    geometry, which the plate force is sensitive to."""
    with open(WETTING_90) as f:
        return float(json.load(f)["varrho_90"])


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


def _bridge_mask_radii(nx, ny, nz, centers, radii, volume, around, box=None):
    """Like _bridge_mask with one radius per sphere; optionally restricted to a local box
    (x0, x1, y0, y1, z0, z1) of periodic coordinates to keep large lattices cheap."""
    if box is None:
        box = (0, nx, 0, ny, 0, nz)
    x0, x1, y0, y1, z0, z1 = box
    zz, yy, xx = np.mgrid[z0:z1, y0:y1, x0:x1].astype(np.float32)

    def mind(a, c, n):
        d = np.abs(a - c) % n
        return np.minimum(d, n - d)

    outside = np.ones(zz.shape, bool)
    for c, R in zip(centers, radii):
        d2 = mind(xx, c[0], nx) ** 2 + mind(yy, c[1], ny) ** 2 + mind(zz, c[2], nz) ** 2
        outside &= d2 > R * R
    dc2 = mind(xx, around[0], nx) ** 2 + mind(yy, around[1], ny) ** 2 + mind(zz, around[2], nz) ** 2
    target = int(round(volume))
    lo, hi = 0.0, float(max(x1 - x0, y1 - y0, z1 - z0))
    for _ in range(50):
        mid = 0.5 * (lo + hi)
        if np.count_nonzero(outside & (dc2 <= mid * mid)) < target:
            lo = mid
        else:
            hi = mid
    local = (outside & (dc2 <= hi * hi))
    if box == (0, nx, 0, ny, 0, nz):
        return local.astype(np.uint8)
    return local, (zz.astype(np.int64) % nz, yy.astype(np.int64) % ny, xx.astype(np.int64) % nx)


def packing(seed=0, n_spheres=200, L=512, Rmin=12.0, Rmax=20.0, min_gap=2.0, liquid_fraction=0.1,
            bridge_gap=8.0, theta=45.0, prec="fp32", mpf=1, rho_s=4.0):
    """Many spheres in a periodic cube by random sequential addition (surface gaps >= min_gap), radii
    U[Rmin, Rmax]; a drop of liquid_fraction times the pair's solid volume (the two-sphere workload's
    definition) at the midpoint of every pair closer than bridge_gap (surface to surface). Returns the
    workload, the bridged pairs and their drop volumes."""
    rng = np.random.default_rng(seed)
    C, R = [], []
    tries = 0
    while len(C) < n_spheres and tries < 200000:
        tries += 1
        r = float(rng.uniform(Rmin, Rmax))
        c = rng.uniform(0, L, size=3)
        ok = True
        for cj, rj in zip(C, R):
            d = np.abs(c - cj)
            d = np.minimum(d, L - d)
            if np.sqrt((d * d).sum()) < r + rj + min_gap:
                ok = False
                break
        if ok:
            C.append(c)
            R.append(r)
    pairs = []
    for i in range(len(C)):
        for j in range(i + 1, len(C)):
            d = np.abs(C[i] - C[j])
            d = np.minimum(d, L - d)
            if np.sqrt((d * d).sum()) - R[i] - R[j] < bridge_gap:
                pairs.append((i, j))
    vols = {(i, j): liquid_fraction * 4.0 / 3.0 * math.pi * (R[i] ** 3 + R[j] ** 3) for (i, j) in pairs}
    mask = np.zeros((L, L, L), np.uint8)
    for (i, j) in pairs:
        vol = vols[(i, j)]
        d = C[j] - C[i]
        d = (d + L / 2) % L - L / 2
        mid = (C[i] + d / 2) % L
        h = int(max(R[i], R[j]) + 8)
        lo = np.floor(mid - h).astype(int)
        box = (lo[0], lo[0] + 2 * h, lo[1], lo[1] + 2 * h, lo[2], lo[2] + 2 * h)
        local, (zi, yi, xi) = _bridge_mask_radii(L, L, L, [tuple(C[i]), tuple(C[j])], [R[i], R[j]], vol,
                                                 tuple(mid), box=box)
        mask[zi[local], yi[local], xi[local]] = 1
    varrho = varrho_for_angle(theta)
    bodies = [_sphere_body(tuple(float(v) for v in c), r, rho_s, varrho) for c, r in zip(C, R)]
    params = dict(tau=1.0, G=-5.0, rho0=1.0, prec=prec, mpf_kinetics=mpf)
    w = Workload("packing", L, L, L, params, bodies, mask, steps=500,
                 meta=dict(seed=seed, n_spheres=len(C), theta_deg=theta, varrho=varrho, liquid_fraction=liquid_fraction))
    return w, pairs, vols


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


def plate_bridge(kind="cylinder", prec="fp32", R=20, h0=20, layers=3, width=64, depth=None, fixed=False,
                 density_ratio=PLATE_DENSITY_RATIO, varrho=None, margin=16, below=14):
    """Two parallel plates (normal z, gap h0) joined by a capillary bridge at 90 degree wetting, the
    set-ups of the plate experiments (Sec. 4.2, Sec. 2.1):

      kind="cylinder": a liquid cylinder of radius R between square plates of side `width`;
      kind="planar"  : a liquid slab of width 2R between plates of width `width` in x that span the
                       periodic y extent, which is the bridge length L (`depth`, default R: the
                       paper's L = R); the plates are infinite along y.

    The lattice spacing is 1, so R = 20 is the paper's Delta x / R = 0.05. Plates have mass density
    density_ratio * rho_L (1.72e4 in the paper: the plates move slowly against the fluid) and are
    free unless `fixed`. The lattice leaves `margin` cells of vapour beside the plates and `below`
    cells under the lower plate."""
    if kind not in ("cylinder", "planar"):
        raise ValueError("kind must be 'cylinder' or 'planar'")
    varrho = varrho_90() if varrho is None else float(varrho)
    nx = width + 2 * margin
    ny = nx if kind == "cylinder" else int(depth if depth is not None else R)
    nz = h0 + 2 * layers + 2 * below + 2
    z1 = below + (layers - 1) / 2.0
    z2 = z1 + layers + h0
    cx, cy = (nx - 1) / 2.0, (ny - 1) / 2.0
    hy = width / 2.0 + _PLATE_PAD if kind == "cylinder" else ny / 2.0 + 2 * _PLATE_PAD
    half = (width / 2.0 + _PLATE_PAD, hy, layers / 2.0 + _PLATE_PAD)
    rho_s = density_ratio * RHO_L
    bodies = [dict(shape="box", center=(cx, cy, zc), half=half, mass_density=rho_s, wetting_rho=varrho,
                   fixed=bool(fixed)) for zc in (z1, z2)]
    z, y, x = np.mgrid[0:nz, 0:ny, 0:nx]
    lo, hi = int(z1 + layers / 2.0 + 0.5), int(z2 - layers / 2.0 - 0.5)
    inside = ((x - cx) ** 2 + (y - cy) ** 2 <= R * R) if kind == "cylinder" else (np.abs(x - cx) <= R)
    mask = (inside & (z >= lo) & (z <= hi)).astype(np.uint8)
    params = dict(tau=1.0, G=-5.0, rho0=1.0, prec=prec, mpf_kinetics=0)
    return Workload("plates_" + kind, nx, ny, nz, params, bodies, mask, steps=500,
                    meta=dict(kind=kind, R=float(R), h0=float(h0), layers=layers, width=width,
                              depth=float(ny) if kind == "planar" else None, varrho=varrho,
                              density_ratio=density_ratio, fixed=bool(fixed)))


def cluster(n_particles=2, c=0.2, prec="fp32", R=30.0, h0=20.0, varrho=2.0, rho_s=4.0, mpf=1, margin=20,
            mobility=1e-5, e0=1.0, tau=1.1, q=27):
    """Two, three or four spheres of radius R with equal surface gaps h0 (a pair on the z axis, an
    equilateral triangle in the xy plane, a regular tetrahedron) and a drop of liquid at their centre
    whose volume gives the liquid volume fraction c = V_L / (V_L + V_S) (Sec. 4.3: R = 30, mass
    density 4, varrho_B = 2.0, c in {0.2, 0.3, 0.5}; the paper's parameter table: tau = 1.1, and its
    velocity set D3Q27). The lattice leaves `margin` cells of vapour
    around the spheres and the drop. The particles start free; the paper holds them while the
    liquid settles (see cbl_set_bodies_fixed)."""
    if n_particles not in (2, 3, 4):
        raise ValueError("2, 3 or 4 particles")
    if not 0.0 < c < 1.0:
        raise ValueError("liquid fraction c must be in (0, 1)")
    a = 2.0 * R + h0  # centre distance of neighbours
    if n_particles == 2:
        rel = np.array([[0, 0, -0.5], [0, 0, 0.5]]) * a
    elif n_particles == 3:
        rel = np.array([[math.cos(t), math.sin(t), 0.0] for t in (math.pi / 2 + k * 2 * math.pi / 3 for k in range(3))])
        rel *= a / math.sqrt(3.0)
    else:
        rel = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], float) * (a / (2 * math.sqrt(2.0)))
    VS = n_particles * 4.0 / 3.0 * math.pi * R ** 3
    VL = c / (1.0 - c) * VS
    r_drop = (3.0 * (VL + VS) / (4.0 * math.pi)) ** (1.0 / 3.0)  # bound on the drop's reach
    ext = np.maximum(np.abs(rel).max(axis=0) + R, r_drop) + margin
    dims = [int(2 * math.ceil(e / 2.0) * 2) for e in ext]  # even sides
    ctr = np.array(dims, float) / 2.0
    centers = [tuple(ctr + v) for v in rel]
    mask = _bridge_mask_radii(dims[0], dims[1], dims[2], centers, [R] * n_particles, VL, tuple(ctr))
    bodies = [_sphere_body(p, R, rho_s, varrho) for p in centers]
    # repulsion strength (not given in the paper): with e0 = 1e-3 spheres of R = 30 and mass density
    # 4 arriving at the speeds of these runs pass through each other (the summed potential of the
    # overlapping member points stays far below their kinetic energy); e0 = 1 stops them within
    # about a cell of contact
    params = dict(tau=tau, G=-5.0, rho0=1.0, prec=prec, mpf_kinetics=mpf, mobility=mobility, e0=e0, q=q)
    name = {2: "pair", 3: "triangle", 4: "tetrahedron"}[n_particles]
    return Workload("%s_c%.1f" % (name, c), dims[0], dims[1], dims[2], params, bodies, mask, steps=500,
                    meta=dict(n_particles=n_particles, c=c, R=R, h0=h0, varrho=varrho, rho_s=rho_s, mpf=mpf,
                              liquid_volume=VL, solid_volume=VS,
                              # the particles travel ~10 cells: room for the advection tail
                              options=dict(tile_tail=8.0)))


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


def batch64(seed=0, n=64, prec="fp32", mpf=1, rho_s=4.0, gap=4.0, fixed=False):
    """Independent two-sphere bridges of uneven box size, liquid fraction and contact angle: box edges
    U{64..128} per axis, radius U[10, 24] clamped to fit the box (pair on the longest axis, surface gap
    `gap`, or U[gap[0], gap[1]] per instance for a pair), liquid fraction U[0.01, 0.2] of the solid
    volume, contact angle U[30, 90] deg, all from one seed. `fixed` holds the spheres in place."""
    rng = np.random.default_rng(seed)
    out = []
    g_fixed = not isinstance(gap, (tuple, list))
    for k in range(n):
        L = [int(v) for v in rng.integers(64, 129, size=3)]
        Rs = [float(v) for v in rng.uniform(10.0, 24.0, size=2)]  # each sphere its own radius
        f = float(rng.uniform(0.01, 0.2))
        theta = float(rng.uniform(30.0, 90.0))
        g = float(gap) if g_fixed else float(rng.uniform(gap[0], gap[1]))
        ax = int(np.argmax(L))
        others = [L[a] for a in range(3) if a != ax]
        cap = min((L[ax] - g - 2 * 4) / 4.0, (min(others) - 8) / 2.0)
        Rs = [min(r, cap) for r in Rs]
        varrho = varrho_for_angle(theta)
        c = [v / 2.0 for v in L]
        # surface gap `gap` centred on the box centre along the longest axis
        centers = []
        p0 = list(c)
        p0[ax] -= g / 2.0 + Rs[0]
        p1 = list(c)
        p1[ax] += g / 2.0 + Rs[1]
        centers = [tuple(p0), tuple(p1)]
        VS = sum(4.0 / 3.0 * math.pi * r ** 3 for r in Rs)
        mask = _bridge_mask_radii(L[0], L[1], L[2], centers, Rs, f * VS, tuple(c))
        R = Rs[0]
        bodies = [_sphere_body(p, r, rho_s, varrho) for p, r in zip(centers, Rs)]
        for b in bodies:
            b["fixed"] = bool(fixed)
        params = dict(tau=1.0, G=-5.0, rho0=1.0, prec=prec, mpf_kinetics=mpf)
        out.append(Workload("batch%02d" % k, L[0], L[1], L[2], params, bodies, mask, steps=500,
                            meta=dict(seed=seed, index=k, R=R, liquid_fraction_of_solid=f, theta_deg=theta,
                                      varrho=varrho, gap=g, axis=ax)))
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
