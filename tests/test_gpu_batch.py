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
