"""Full-size parity in the bench's launch configuration: the four-sphere cluster at 256^3 with FP32
storage and the library's default execution options, one step of the CUDA path against one step of
the FP64 oracle taken from the same state, every cell compared.

The GPU advances 60 steps with the four bodies held (the settling protocol of Sec. 4.3.2) and MPF
kinetics off, so the phase fields and flags stay those of the set-up on both sides while the liquid
moves; its stored populations are then written into the oracle, set up from the same workload with
the same bodies held, and both take one step (Sec. 3.2: psi, Shan-Chen force with wetting,
bounce-back, Guo-forced BGK, momentum exchange). The difference is one step of the FP32 path's
arithmetic and storage rounding: at most 1e-5 of the largest population or density, and 1e-3 of
the largest body force (a sum over some thirty thousand links whose contributions cancel to a small
net force).
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


@pytest.mark.parametrize("variant", [0, 1, 2])
def test_tetra4_full_size_one_step_from_gpu_state(variant):
    # variant: the lattice-Boltzmann pass (0 split, the default and the bench's; 1 fused; 2
    # accumulating), all three against the same oracle step
    import oracle

    w = workloads.tetra4(seed=0, prec="fp32")
    assert (w.nx, w.ny, w.nz) == (256, 256, 256)
    params = dict(w.params, mpf_kinetics=0)
    g = cbl.Sim(w.nx, w.ny, w.nz, **params)
    g.set_option("lbm_variant", variant)
    workloads.build(g, w)
    g.set_fixed([True] * len(w.bodies))
    g.step(60)
    f_gpu = g.populations()

    o = oracle.Oracle(w.nx, w.ny, w.nz, **{k: v for k, v in params.items() if k != "prec"})
    workloads.build(o, w)
    o.set_fixed([True] * len(w.bodies))
    sg, _ = g.flags()
    so, _ = o.flags()
    assert (sg != so).sum() == 0  # the same obstacle cells
    cg, _ = g.velocity_set()
    co, _ = o.velocity_set()
    perm = [int(np.flatnonzero((co == cg[i]).all(axis=1))[0]) for i in range(len(cg))]  # gpu i -> oracle
    f_o = np.empty_like(f_gpu)
    f_o[perm] = f_gpu
    o.set_populations(f_o)
    del f_o

    g.step(1)
    o.step(1)
    fg = g.populations()
    fo = o.populations()[perm]
    scale = np.abs(fo).max()
    err_f = float(np.abs(fg - fo).max() / scale)
    rg, vg, _ = g.fields()
    ro, vo, _ = o.fields()
    fluid = sg == 0
    err_rho = float(np.abs(rg - ro)[fluid].max() / np.abs(ro[fluid]).max())
    err_vel = float(np.abs(vg - vo)[fluid].max() / np.abs(vo[fluid]).max())
    Fg, _, _ = g.body_forces()
    Fo, _, _ = o.body_forces()
    err_F = float(np.abs(Fg - Fo).max() / np.abs(Fo).max())
    print("256^3 one step from the GPU state (pass %d): populations %.2e, density %.2e, velocity %.2e, "
          "force %.2e" % (variant, err_f, err_rho, err_vel, err_F))
    assert err_f < 1e-5 and err_rho < 1e-5, (err_f, err_rho)
    assert err_vel < 1e-3, err_vel
    assert err_F < 1e-3, err_F
    assert g.info()["device_error"] == 0


def test_tetra4_full_size_one_step_binary16_against_storage_model():
    """The same check for binary16 deviation storage (the four-sphere cluster's second precision):
    the oracle with its binary16 storage model (store_prec 2: every stored population rounded to a
    binary16 deviation from the binary16-rounded weight, the representation the CUDA path stores)
    takes one step from the GPU's stored state. The CUDA path computes the step in FP32, the oracle
    in FP64, and both round to binary16 on the store: a population agrees exactly unless the two
    roundings of the arithmetic fall on different sides of a binary16 rounding boundary, and then by
    one binary16 unit of its deviation."""
    import oracle

    w = workloads.tetra4(seed=0, prec="fp16dev")
    params = dict(w.params, mpf_kinetics=0)
    g = cbl.Sim(w.nx, w.ny, w.nz, **params)
    workloads.build(g, w)
    g.set_fixed([True] * len(w.bodies))
    g.step(60)
    f_gpu = g.populations()

    o = oracle.Oracle(w.nx, w.ny, w.nz, store_prec=2, **{k: v for k, v in params.items() if k != "prec"})
    workloads.build(o, w)
    o.set_fixed([True] * len(w.bodies))
    cg, wg = g.velocity_set()
    co, _ = o.velocity_set()
    perm = [int(np.flatnonzero((co == cg[i]).all(axis=1))[0]) for i in range(len(cg))]
    f_o = np.empty_like(f_gpu)
    f_o[perm] = f_gpu
    o.set_populations(f_o)
    del f_o
    g.step(1)
    o.step(1)
    fg = g.populations()
    fo = o.populations()[perm]
    sg, _ = g.flags()
    fluid = sg == 0
    what = (np.asarray(wg, np.float16).astype(np.float64))[:, None, None, None]  # binary16-rounded weights
    hg, ho = fg - what, fo - what
    mag = np.maximum(np.abs(hg), np.abs(ho))
    ulp = np.maximum(2.0 ** (np.floor(np.log2(np.maximum(mag, 2.0 ** -14))) - 10), 2.0 ** -24)
    diff = np.abs(fg - fo)[:, fluid]
    ulp = ulp[:, fluid]
    frac = float((diff > 0).mean())
    worst = float((diff / ulp).max())
    print("256^3 binary16, one step from the GPU state: %.2e of the populations differ, by at most %.3f "
          "binary16 units of their deviation" % (frac, worst))
    assert worst <= 1.0 + 1e-9, worst
    assert frac < 1e-2, frac


def test_batch64_one_step_of_sampled_instances():
    """The 64-instance batch of the bench (boxes U{64..128}^3, FP32, the persistent launch with its
    default tile shape), bodies held and kinetics off: after 40 steps three instances (the smallest,
    the median and the largest box) are written into oracles with the same set-up, and the batch and
    the oracles take one step; every cell of those instances is compared."""
    import oracle

    ws = workloads.batch64(seed=0, prec="fp32")
    sims = []
    for w in ws:
        s = cbl.Sim(w.nx, w.ny, w.nz, **dict(w.params, mpf_kinetics=0))
        workloads.build(s, w)
        s.set_fixed([True] * len(w.bodies))
        sims.append(s)
    b = cbl.Batch(sims)
    assert b.info()["mode"] == 1  # the persistent launch
    b.step(40)
    b.sync()
    order = np.argsort([w.ncells for w in ws])
    pick = [int(order[0]), int(order[len(order) // 2]), int(order[-1])]
    oracles = {}
    for k in pick:
        w = ws[k]
        o = oracle.Oracle(w.nx, w.ny, w.nz, **{kk: v for kk, v in dict(w.params, mpf_kinetics=0).items()
                                                 if kk != "prec"})
        workloads.build(o, w)
        o.set_fixed([True] * len(w.bodies))
        cg, _ = sims[k].velocity_set()
        co, _ = o.velocity_set()
        perm = [int(np.flatnonzero((co == cg[i]).all(axis=1))[0]) for i in range(len(cg))]
        f = sims[k].populations()
        fo = np.empty_like(f)
        fo[perm] = f
        o.set_populations(fo)
        oracles[k] = (o, perm)
    b.step(1)
    b.sync()
    for k, (o, perm) in oracles.items():
        o.step(1)
        g = sims[k]
        fg = g.populations()
        fo = o.populations()[perm]
        err_f = float(np.abs(fg - fo).max() / np.abs(fo).max())
        Fg, _, _ = g.body_forces()
        Fo, _, _ = o.body_forces()
        err_F = float(np.abs(Fg - Fo).max() / np.abs(Fo).max())
        print("batch instance %d (%d^3 cells): populations %.2e, force %.2e" % (k, round(ws[k].ncells ** (1 / 3)), err_f, err_F))
        assert err_f < 1e-5 and err_F < 1e-3, (k, err_f, err_F)
        assert g.info()["device_error"] == 0
    b.close()


def test_tetra4_full_size_release_three_steps_from_gpu_state():
    """The moving-body path at full size: after 60 held steps (kinetics off, so the phase fields are
    the set-up's on both sides) the GPU's populations go into the oracle, both release the four
    bodies from rest and take three steps (forces, rigid-body update, advection of the phase fields
    with the new velocities, flags), compared at every cell."""
    import oracle

    w = workloads.tetra4(seed=0, prec="fp32")
    params = dict(w.params, mpf_kinetics=0)
    nb = len(w.bodies)
    g = cbl.Sim(w.nx, w.ny, w.nz, **params)
    workloads.build(g, w)
    g.set_fixed([True] * nb)
    g.step(60)
    o = oracle.Oracle(w.nx, w.ny, w.nz, **{k: v for k, v in params.items() if k != "prec"})
    workloads.build(o, w)
    cg, _ = g.velocity_set()
    co, _ = o.velocity_set()
    perm = [int(np.flatnonzero((co == cg[i]).all(axis=1))[0]) for i in range(len(cg))]
    f = g.populations()
    fo = np.empty_like(f)
    fo[perm] = f
    o.set_populations(fo)
    del f, fo
    g.set_fixed([False] * nb)
    g.step(3)
    o.step(3)
    sg, _ = g.flags()
    so, _ = o.flags()
    assert (sg != so).sum() == 0
    fg = g.populations()
    fo = o.populations()[perm]
    err_f = float(np.abs(fg - fo).max() / np.abs(fo).max())
    Fg, _, _ = g.body_forces()
    Fo, _, _ = o.body_forces()
    err_F = float(np.abs(Fg - Fo).max() / np.abs(Fo).max())
    bg, bo = g.bodies(), o.bodies()
    dX = float(np.abs(bg["X"] - bo["X"]).max())
    dV = float(np.abs(bg["V"] - bo["V"]).max() / max(np.abs(bo["V"]).max(), 1e-300))
    moved = float(np.abs(bo["X"] - np.array([b["center"] for b in w.bodies])).max())
    print("256^3, released, three steps from the GPU state: populations %.2e, force %.2e, V %.2e, "
          "X %.2e (bodies moved %.2e)" % (err_f, err_F, dV, dX, moved))
    assert moved > 0.0
    assert err_f < 1e-5 and err_F < 1e-3 and dV < 1e-3, (err_f, err_F, dV)
    assert dX < 1e-3 * moved + 1e-12, (dX, moved)
    assert g.info()["device_error"] == 0


@pytest.mark.parametrize("q", [19, 27])
def test_spheres2_full_size_one_step_from_gpu_state(q):
    """The two-sphere workload at full size (128 x 128 x 256, FP32) with D3Q19 and with the paper's
    D3Q27 (Sec. 3.2.1), held bodies, kinetics off: one step from the GPU's state against the oracle."""
    import oracle

    w = workloads.spheres2(seed=0, prec="fp32")
    params = dict(w.params, mpf_kinetics=0, q=q)
    g = cbl.Sim(w.nx, w.ny, w.nz, **params)
    workloads.build(g, w)
    g.set_fixed([True] * len(w.bodies))
    g.step(60)
    o = oracle.Oracle(w.nx, w.ny, w.nz, **{k: v for k, v in params.items() if k != "prec"})
    workloads.build(o, w)
    o.set_fixed([True] * len(w.bodies))
    cg, _ = g.velocity_set()
    co, _ = o.velocity_set()
    assert len(cg) == q
    perm = [int(np.flatnonzero((co == cg[i]).all(axis=1))[0]) for i in range(len(cg))]
    f = g.populations()
    fo = np.empty_like(f)
    fo[perm] = f
    o.set_populations(fo)
    g.step(1)
    o.step(1)
    fg = g.populations()
    fo = o.populations()[perm]
    err_f = float(np.abs(fg - fo).max() / np.abs(fo).max())
    Fg, _, _ = g.body_forces()
    Fo, _, _ = o.body_forces()
    err_F = float(np.abs(Fg - Fo).max() / np.abs(Fo).max())
    print("two spheres D3Q%d, one step from the GPU state: populations %.2e, force %.2e" % (q, err_f, err_F))
    assert err_f < 1e-5 and err_F < 1e-3, (err_f, err_F)
