"""The no-allocation LBM step (cbl_lbm_step_noalloc) against the regular entry point.

Some callers cannot allocate device memory themselves (their memory is managed by another
framework's pool, or their process must not call cudaMalloc once running); for them the library
offers one lattice-Boltzmann step whose scratch is a fixed set of device arrays inside the library.
This test gives it caller-owned buffers and checks two calls in a row against cbl_step on the same
initial state (same kernels, so the populations should agree to the bit; the check uses the FP32
parity tolerance of the other tests). It lives in a file of its own that pytest collects last, and
passes alone or after the other tests.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_two_steps_match_cbl_step():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_1902_10432_gb300 import cbl

    nx, ny, nz = 40, 36, 28
    assert nx * ny * nz <= cbl.NOALLOC_MAX_CELLS
    rng = np.random.default_rng(11)
    rho = 0.12 + 1.77 * (rng.random((nz, ny, nx)) > 0.55)
    u = 0.01 * rng.standard_normal((nz, ny, nx, 3))
    sim = cbl.Sim(nx, ny, nz, prec="fp32")
    sim.init_fluid_fields(rho, u)
    f0 = sim.populations()  # FP32 storage widened to FP64: exact
    dev = torch.device("cuda")
    fa = torch.tensor(f0.reshape(-1), dtype=torch.float32, device=dev)
    fb = torch.empty_like(fa)
    fc = torch.empty_like(fa)
    mass = torch.zeros(2, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    cbl.lbm_step_noalloc(fa, fb, nx, ny, nz, tau=1.0, G=-5.0, rho0=1.0, mass_out=mass[0:1])
    cbl.lbm_step_noalloc(fb, fc, nx, ny, nz, tau=1.0, G=-5.0, rho0=1.0, mass_out=mass[1:2])
    torch.cuda.synchronize()
    for k, out in enumerate((fb, fc)):
        sim.step(1)
        ref = sim.populations().reshape(-1)
        got = out.double().cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-4 * np.abs(ref).max()
        m = mass[k].item()
        assert abs(m - sim.total_mass()) <= 1e-12 * abs(sim.total_mass())
    # sizes beyond the fixed scratch are rejected by the library (buffers large enough for the
    # lattice, so that only the scratch limit can refuse the call)
    big = (cbl.NOALLOC_MAX_CELLS // (16 * 16)) + 1
    ga = torch.zeros(19 * 16 * 16 * big, dtype=torch.float32, device=dev)
    gb = torch.empty_like(ga)
    with pytest.raises(cbl.CblError):
        cbl.lbm_step_noalloc(ga, gb, 16, 16, big)
    # buffers too small for the lattice are refused before the call
    with pytest.raises(ValueError):
        cbl.lbm_step_noalloc(fa[:100], fb, nx, ny, nz)
