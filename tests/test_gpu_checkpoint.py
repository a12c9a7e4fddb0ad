"""Checkpoint and resume (cbl_save / cbl_load): a run saved after n steps and loaded into a fresh
context has the saved state bit for bit and continues as the uninterrupted run; a checkpoint of
another set-up is refused."""
import numpy as np
import pytest

from paper_1902_10432_gb300 import cbl, workloads

pytestmark = pytest.mark.gpu


def _state(s):
    rho, vel, phi = s.fields()
    solid, owner = s.flags()
    F, T, parts = s.body_forces()
    b = s.bodies()
    return dict(rho=rho, vel=vel, phi=phi, solid=solid, owner=owner, F=F, T=T, parts=parts, X=b["X"], V=b["V"],
                W=b["W"], Q=b["Q"], pops=s.populations(), mass=s.total_mass())


def _fresh(w):
    s = cbl.Sim(w.nx, w.ny, w.nz, **w.params)
    for b in w.bodies:
        kw = dict(b)
        s.add_body(kw.pop("shape"), **kw)
    return s


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-9), ("fp32", 1e-4), ("fp16dev", 1e-3)])
def test_resume_restores_the_state_and_continues(tmp_path, prec, tol):
    w = workloads.small_spheres(prec=prec)
    a = cbl.Sim(w.nx, w.ny, w.nz, **w.params)
    workloads.build(a, w)
    a.step(120)
    path = str(tmp_path / "run.ckpt")
    a.save(path)
    saved = _state(a)
    b = _fresh(w)
    b.load(path)
    loaded = _state(b)
    for k in saved:  # the restored state is the saved one, bit for bit
        assert np.array_equal(np.asarray(saved[k]), np.asarray(loaded[k])), k
    a.step(150)
    b.step(150)
    ref, got = _state(a), _state(b)
    # both runs continue alike; they can differ only by the order of the FP64 atomic sums (forces,
    # phase-field volumes), which is not fixed from one launch to the next
    assert np.array_equal(ref["solid"], got["solid"]) and np.array_equal(ref["owner"], got["owner"])
    for k in ("rho", "X", "F"):
        scale = max(np.abs(ref[k]).max(), 1e-30)
        assert np.abs(ref[k] - got[k]).max() <= tol * scale, k
    assert b.info()["device_error"] == 0


def test_checkpoint_of_another_setup_is_refused(tmp_path):
    w = workloads.small_spheres(prec="fp64")
    a = cbl.Sim(w.nx, w.ny, w.nz, **w.params)
    workloads.build(a, w)
    a.step(5)
    path = str(tmp_path / "run.ckpt")
    a.save(path)
    other = dict(w.params, tau=0.9)
    c = cbl.Sim(w.nx, w.ny, w.nz, **other)
    for bd in w.bodies:
        kw = dict(bd)
        c.add_body(kw.pop("shape"), **kw)
    with pytest.raises(cbl.CblError, match="ERR_ARG"):
        c.load(path)
    d = _fresh(w)
    d.init_fluid(w.rho_l, w.rho_v, w.mask)
    with pytest.raises(cbl.CblError, match="ERR_STATE"):
        d.load(path)
    e = cbl.Sim(w.nx, w.ny, w.nz, **w.params)  # no bodies added
    with pytest.raises(cbl.CblError, match="ERR_ARG"):
        e.load(path)
    with open(path, "r+b") as f:  # truncated
        f.truncate(1000)
    g = _fresh(w)
    with pytest.raises(cbl.CblError, match="ERR_ARG"):
        g.load(path)
