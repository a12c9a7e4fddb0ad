"""Batched execution and execution options: the same numbers as stepping each simulation alone."""
import numpy as np
import pytest

from paper_1902_10432_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


def _sim(w):
    from paper_1902_10432_gb300 import cbl

    s = cbl.Sim(w.nx, w.ny, w.nz, **w.params)
    workloads.build(s, w)
    return s


def test_batch_matches_individual_steps():
    from paper_1902_10432_gb300 import cbl

    ws = workloads.batch64(seed=3, n=3)
    alone = [_sim(w) for w in ws]
    grouped = [_sim(w) for w in ws]
    for s in alone:
        s.step(20)
    b = cbl.Batch(grouped)
    b.step(20)
    b.sync()
    for a, g in zip(alone, grouped):
        ra, va, pa = a.fields()
        rg, vg, pg = g.fields()
        # the per-body and per-phase FP64 sums are atomics: equal up to their addition order
        assert np.abs(ra - rg).max() <= 1e-12 * np.abs(ra).max()
        assert np.abs(va - vg).max() <= 1e-10 * max(np.abs(va).max(), 1e-30)
        assert np.abs(pa - pg).max() <= 1e-12
        Fa, _, _ = a.body_forces()
        Fg, _, _ = g.body_forces()
        assert np.allclose(Fa, Fg, rtol=1e-12, atol=1e-15)  # FP64 atomics may add in another order
    b.close()


@pytest.mark.parametrize("opts", [dict(lbm_block_x=64), dict(lbm_block_x=128), dict(lbm_variant=1)])
def test_execution_options_agree(opts):
    w = workloads.small_spheres(prec="fp32", mobility=2e-3)
    a, g = _sim(w), _sim(w)
    for k, v in opts.items():
        g.set_option(k, v)
    a.step(60)
    g.step(60)
    ra, va, _ = a.fields()
    rg, vg, _ = g.fields()
    if "lbm_variant" in opts:
        # another kernel: other rounding order
        assert np.abs(ra - rg).max() < 1e-5 * np.abs(ra).max()
    else:
        assert np.array_equal(ra, rg) and np.array_equal(va, vg)


def test_autotune_picks_a_candidate(tmp_path, monkeypatch):
    from paper_1902_10432_gb300 import autotune

    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "tune.json"))
    w = workloads.small_spheres(prec="fp32")
    s = _sim(w)
    choice, ms = autotune.tune(s, steps=3)
    assert choice in autotune.candidates("fp32") and len(ms) == len(autotune.candidates("fp32"))
    s2 = _sim(w)
    choice2, _ = autotune.tune(s2)  # from the cache
    assert choice2 == choice


def test_move_bodies_matches_fresh_setup_and_keeps_mass():
    from paper_1902_10432_gb300 import cbl

    w = workloads.small_spheres(prec="fp64")
    a = _sim(w)
    a.step(10)
    m0 = a.populations().sum()
    X = a.bodies()["X"]
    X1 = X + np.array([[0.6, -0.3, 1.4], [-0.2, 0.5, -1.1]])
    a.move_bodies(X1)
    assert abs(a.populations().sum() - m0) < 1e-12 * m0  # refill hands over what cover takes
    # a fresh simulation whose bodies start at the new centres has the same phase field and flags
    w2 = workloads.small_spheres(prec="fp64")
    for b, x in zip(w2.bodies, X1):
        b["center"] = tuple(x)
    f = _sim(w2)
    for k in range(2):
        assert np.abs(a.phi(k) - f.phi(k)).max() < 1e-12
    sa, oa = a.flags()
    sf, of = f.flags()
    assert np.array_equal(sa, sf) and np.array_equal(oa, of)
    a.step(5)  # the moved state steps cleanly
    assert a.info()["device_error"] == 0 and np.isfinite(a.total_mass())
