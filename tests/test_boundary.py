"""The C-ABI library loads without a GPU and exports every function include/cbl.h declares;
host-side argument checks return CBL_ERR_ARG without touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1902_10432_gb300 import cbl

    return cbl.load()


def declared():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(cbl_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    from paper_1902_10432_gb300 import cbl

    assert set(names) <= set(cbl.SIGNATURES), set(names) - set(cbl.SIGNATURES)


def test_argument_errors_without_gpu(lib):
    from paper_1902_10432_gb300 import cbl

    h = ctypes.c_void_p()
    p = cbl.cbl_params()
    p.nx, p.ny, p.nz, p.q, p.tau, p.rho0, p.eta, p.rc, p.nrep = 2, 8, 8, 19, 1.0, 1.0, 5.0, 3.0, 4
    assert lib.cbl_create(ctypes.byref(p), None, ctypes.byref(h)) == 1  # CBL_ERR_ARG: side < 4
    assert b"lattice" in lib.cbl_last_error(None)
    p.nx, p.q = 8, 15
    assert lib.cbl_create(ctypes.byref(p), None, ctypes.byref(h)) == 7  # only D3Q19 and D3Q27
    p.q, p.tau = 19, 0.5
    assert lib.cbl_create(ctypes.byref(p), None, ctypes.byref(h)) == 1
    assert lib.cbl_create(None, None, ctypes.byref(h)) == 1
    assert lib.cbl_step(None, 1) == 1
    assert lib.cbl_destroy(None) == 0
    assert lib.cbl_save(None, b"/nonexistent/x") == 1
    assert lib.cbl_load(None, b"/nonexistent/x") == 1
    assert lib.cbl_set_bodies_fixed(None, None) == 1
