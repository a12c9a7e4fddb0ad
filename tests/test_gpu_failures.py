"""Failure paths of the C ABI, made on the host (nothing here faults, traps or hangs a GPU).

* A caller allocator that returns NULL: cbl_create frees what it took and returns CBL_ERR_OOM, and so
  does cbl_init_fluid when the bodies' arrays cannot be allocated.
* Non-finite or negative initial fields, centres, radii and velocities: CBL_ERR_ARG before any kernel
  runs, and the context stays usable.
* Populations that overflow the storage (a density of 1e39 stored in FP32 is Inf): the fluid mass is
  not finite and cbl_total_mass returns CBL_ERR_UNSTABLE; the steps before it complete (no device
  loop depends on a value).
* More overlapping body tiles than a neighbour list holds: device error bit 1 is set, read by
  cbl_info.
* A covered node whose mass has no fluid receiver (two plates closing on a liquid layer): device
  error bit 2.
"""
import ctypes
import math

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


def _params(n=16, prec=1):
    p = cbl.cbl_params()
    p.nx = p.ny = p.nz = n
    p.q, p.tau, p.G, p.rho0, p.prec = 19, 1.0, -5.0, 1.0, prec
    p.eta, p.mobility, p.sigma_sf, p.sigma_ss, p.e0, p.rc, p.nrep = 5.0, 1e-5, 3.583e-2, 1.79e-2, 1e-3, 3.0, 4
    p.solid_threshold, p.member_threshold = 0.05, 0.5
    return p


def _failing_allocator(k):
    """cbl_allocator that serves k allocations (from PyTorch's caching allocator), then returns NULL."""
    import torch

    state = {"n": 0, "live": set()}

    def _alloc(nbytes, user):
        if state["n"] >= k:
            return None
        state["n"] += 1
        ptr = torch.cuda.caching_allocator_alloc(int(nbytes))
        state["live"].add(ptr)
        return ptr

    def _free(ptr, user):
        state["live"].discard(ptr)
        torch.cuda.caching_allocator_delete(ptr)

    a = cbl.cbl_allocator(cbl.ALLOC_FN(_alloc), cbl.FREE_FN(_free), None)
    a._keep = (_alloc, _free)
    return a, state


@pytest.mark.parametrize("k", [0, 1, 4, 8])
def test_create_with_failing_allocator(k):
    lib = cbl.load()
    a, state = _failing_allocator(k)
    h = ctypes.c_void_p()
    st = lib.cbl_create(ctypes.byref(_params()), ctypes.byref(a), ctypes.byref(h))
    assert st == 3, st  # CBL_ERR_OOM
    assert b"allocation" in lib.cbl_last_error(None)
    assert not state["live"]  # everything it took was given back


def test_init_with_failing_allocator_after_create():
    lib = cbl.load()
    a, state = _failing_allocator(9)  # the lattice arrays fit, the bodies' arrays do not
    h = ctypes.c_void_p()
    assert lib.cbl_create(ctypes.byref(_params(24)), ctypes.byref(a), ctypes.byref(h)) == 0
    b = cbl.cbl_body()
    b.shape, b.center[:], b.radius, b.mass_density, b.wetting_rho = 0, (12.0, 12.0, 12.0), 4.0, 4.0, 1.0
    b.quat[:] = (1.0, 0.0, 0.0, 0.0)
    bid = ctypes.c_int()
    st = lib.cbl_add_body(h, ctypes.byref(b), ctypes.byref(bid))
    if st == 0:
        st = lib.cbl_init_fluid(h, 1.9, 0.12, None)
    assert st == 3, st
    assert lib.cbl_destroy(h) == 0
    assert not state["live"]


def test_non_finite_inputs_are_rejected():
    s = cbl.Sim(16, 16, 16, prec="fp32")
    rho = np.full((16, 16, 16), 0.5)
    for bad in (math.nan, math.inf, -1.0):
        r = rho.copy()
        r[3, 4, 5] = bad
        with pytest.raises(cbl.CblError) as e:
            s.init_fluid_fields(r)
        assert e.value.status == 1
    u = np.zeros((16, 16, 16, 3))
    u[1, 2, 3, 1] = math.nan
    with pytest.raises(cbl.CblError) as e:
        s.init_fluid_fields(rho, u)
    assert e.value.status == 1
    for kw in (dict(center=(math.nan, 8.0, 8.0), radius=3.0), dict(center=(8.0, 8.0, 8.0), radius=math.inf)):
        with pytest.raises(cbl.CblError) as e:
            s.add_body("sphere", mass_density=4.0, wetting_rho=1.0, **kw)
        assert e.value.status == 1
    # the context is still usable
    s.add_body("sphere", center=(8.0, 8.0, 8.0), radius=3.0, mass_density=4.0, wetting_rho=1.0)
    s.init_fluid_fields(rho)
    with pytest.raises(cbl.CblError) as e:
        s.set_body_velocities(V=np.array([[math.nan, 0.0, 0.0]]))
    assert e.value.status == 1
    with pytest.raises(cbl.CblError) as e:
        s.move_bodies(np.array([[8.0, math.inf, 8.0]]))
    assert e.value.status == 1
    s.step(5)
    assert np.isfinite(s.total_mass()) and s.info()["device_error"] == 0


def test_overflowing_populations_report_unstable():
    s = cbl.Sim(16, 16, 16, prec="fp32")
    rho = np.full((16, 16, 16), 0.5)
    rho[8, 8, 8] = 1e39  # finite in FP64, Inf once stored in FP32
    s.init_fluid_fields(rho)
    s.step(3)
    with pytest.raises(cbl.CblError) as e:
        s.total_mass()
    assert e.value.status == 6  # CBL_ERR_UNSTABLE


def test_neighbour_list_overflow_sets_device_error():
    # 40 spheres in a 96^3 box: some tiles overlap more than 24 others
    w, pairs, VL = workloads.packing(seed=0, n_spheres=40, L=96, Rmin=9.0, Rmax=13.0, rho_s=200.0, bridge_gap=5.0,
                                     liquid_fraction=0.2)
    s = cbl.Sim(w.nx, w.ny, w.nz, **w.params)
    workloads.build(s, w)
    assert s.info()["device_error"] & 2


def test_lost_refill_sets_device_error():
    # two plates spanning x and y with a liquid-filled gap of 8 cells; moving one onto the other
    # covers the gap's last fluid layer with no fluid node within sqrt(3) of it: its mass cannot be
    # handed on (Sec. 3.2.2), which device error bit 2 records
    n, nz = 32, 48
    s = cbl.Sim(n, n, nz, prec="fp64")
    half = (n / 2.0 + 2.0, n / 2.0 + 2.0, 1.5)
    c = (n - 1) / 2.0
    s.add_body("box", center=(c, c, 12.0), half=half, mass_density=4.0, wetting_rho=1.0, fixed=True)
    s.add_body("box", center=(c, c, 23.0), half=half, mass_density=4.0, wetting_rho=1.0, fixed=True)
    s.init_fluid(1.9, 0.12, np.ones((nz, n, n), np.uint8))
    s.step(2)
    assert s.info()["device_error"] == 0
    X = s.bodies()["X"].copy()
    X[1, 2] -= 8.0
    s.move_bodies(X)
    assert s.info()["device_error"] & 4
