"""The fused bulk pass (lbm_variant 1: density and collision in one pass over HBM, psi of each
plane and its one-cell ring in shared memory) against the split pass (lbm_variant 0: the density
kernel, then the collision kernel), through the C ABI.

Both compute the same terms in the same order (Sec. 3.2.1 streaming and collision, Sec. 3.2.3
Shan-Chen force), so where nothing is summed with atomics the populations agree bit for bit:
lattices without bodies and lattices whose bodies are held. With free bodies the FP64 force sums
are atomic (their order varies from run to run), so there the two are compared at round-off.
Ragged lattices (sides that are not multiples of the 32 x 4 / 32 x 8 block columns, sides
smaller than a block) and z extents that do not divide the lattice cover the block edges.
"""
import numpy as np
import pytest

from paper_1902_10432_gb300 import cbl, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    import torch

    __graft_entry__.build()
    assert torch.cuda.is_available()


def _sim(nx, ny, nz, prec, variant, ty=8, tz=0, **kw):
    s = cbl.Sim(nx, ny, nz, prec=prec, **kw)
    s.set_option("lbm_variant", variant)
    if variant == 1:
        s.set_option("fused_ty", ty)
        s.set_option("fused_tz", tz)
    return s


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16dev"])
@pytest.mark.parametrize("dims,ty,tz", [((37, 29, 23), 8, 0), ((37, 29, 23), 4, 5), ((4, 5, 6), 8, 0),
                                         ((70, 33, 17), 4, 1), ((64, 48, 40), 8, 7)])
def test_no_bodies_bitwise(prec, dims, ty, tz):
    nx, ny, nz = dims
    rng = np.random.default_rng(nx * 131 + nz)
    rho = 0.12 + 1.77 * (rng.random((nz, ny, nx)) > 0.55)
    u = 0.02 * rng.standard_normal((nz, ny, nx, 3))
    a = _sim(nx, ny, nz, prec, 0)
    b = _sim(nx, ny, nz, prec, 1, ty, tz)
    for s in (a, b):
        s.init_fluid_fields(rho, u)
        s.step(12)
    assert np.array_equal(a.populations(), b.populations())
    ra, va, _ = a.fields()
    rb, vb, _ = b.fields()
    assert np.array_equal(ra, rb) and np.array_equal(va, vb)
    assert a.total_mass() == b.total_mass() or abs(a.total_mass() - b.total_mass()) < 1e-13 * a.total_mass()


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16dev"])
@pytest.mark.parametrize("ty", [4, 8])
def test_held_plates_bitwise(prec, ty):
    # fixed plates: bounce-back, wetting, the cells next to a solid on the side branch with psi from
    # the tile pass; the forces do not feed back, so the populations are deterministic
    w = workloads.plates48(prec=prec)
    sims = []
    for variant in (0, 1):
        s = _sim(w.nx, w.ny, w.nz, prec, variant, ty, **{k: v for k, v in w.params.items() if k != "prec"})
        workloads.build(s, w)
        s.step(40)
        sims.append(s)
    a, b = sims
    assert np.array_equal(a.populations(), b.populations())
    Fa, Ta, _ = a.body_forces()
    Fb, Tb, _ = b.body_forces()
    assert np.abs(Fa - Fb).max() <= 1e-12 * np.abs(Fa).max()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_free_spheres_match(prec, tol):
    # free, light spheres: cells covered and uncovered, the boundary list changing every step
    w = workloads.small_spheres(prec=prec, mobility=2e-3)
    sims = []
    for variant in (0, 1):
        s = _sim(w.nx, w.ny, w.nz, prec, variant, 4, **{k: v for k, v in w.params.items() if k != "prec"})
        workloads.build(s, w)
        s.step(100)
        sims.append(s)
    a, b = sims
    sa, _ = a.flags()
    sb, _ = b.flags()
    assert (sa != sb).sum() == 0
    ra, va, _ = a.fields()
    rb, vb, _ = b.fields()
    assert np.abs(ra - rb).max() <= tol * np.abs(ra).max()
    assert np.abs(va - vb).max() <= 10 * tol * np.abs(va).max()
    Xa, Xb = a.bodies()["X"], b.bodies()["X"]
    assert np.abs(Xa - Xb).max() < 1e-6
    assert a.info()["device_error"] == 0 and b.info()["device_error"] == 0
