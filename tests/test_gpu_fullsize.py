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


def test_tetra4_full_size_one_step_from_gpu_state():
    import oracle

    w = workloads.tetra4(seed=0, prec="fp32")
    assert (w.nx, w.ny, w.nz) == (256, 256, 256)
    params = dict(w.params, mpf_kinetics=0)
    g = cbl.Sim(w.nx, w.ny, w.nz, **params)
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
    print("256^3 one step from the GPU state: populations %.2e, density %.2e, velocity %.2e, force %.2e"
          % (err_f, err_rho, err_vel, err_F))
    assert err_f < 1e-5 and err_rho < 1e-5, (err_f, err_rho)
    assert err_vel < 1e-3, err_vel
    assert err_F < 1e-3, err_F
    assert g.info()["device_error"] == 0
