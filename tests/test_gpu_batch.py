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


def _batch_of(ws, mode=None, tile=None):
    from paper_1902_10432_gb300 import cbl

    sims = [_sim(w) for w in ws]
    b = cbl.Batch(sims)
    if mode is not None:
        b.set_option("mode", mode)
    if tile is not None:
        b.set_option("tile", tile)
    return sims, b


def test_persistent_batch_is_the_default_and_matches_branch_mode():
    # the persistent launch (psi and bulk collision of every instance in one kernel, work items from
    # a device queue, a grid barrier between the phases) against one fork/join branch per instance
    ws = workloads.batch64(seed=5, n=4)
    pa, ba = _batch_of(ws)
    assert ba.info()["mode"] == 1 and ba.info()["items"] > 0 and ba.info()["grid"] > 0
    pb, bb = _batch_of(ws, mode=0)
    for b in (ba, bb):
        b.step(30)
        b.sync()
    for a, g in zip(pa, pb):
        ra, va, _ = a.fields()
        rg, vg, _ = g.fields()
        assert np.abs(ra - rg).max() <= 1e-5 * np.abs(ra).max()  # FP32, forces summed in another order
        assert a.info()["device_error"] == 0
    ba.close()
    bb.close()


@pytest.mark.parametrize("tile", [0, 2, 3])
def test_persistent_tile_shapes_agree(tile):
    # every tile shape computes every cell once: the fields of a held-body batch (no force feedback)
    # agree bit for bit with the default tile
    ws = workloads.batch64(seed=6, n=3, fixed=True)
    pa, ba = _batch_of(ws)
    pb, bb = _batch_of(ws, tile=tile)
    for b in (ba, bb):
        b.step(12)
        b.sync()
    for a, g in zip(pa, pb):
        assert np.array_equal(a.populations(), g.populations())
    ba.close()
    bb.close()


def test_batched_instances_match_the_oracle():
    # FP64 instances of different sizes in one persistent batch, each against its own oracle run
    from _pair import compare

    import oracle

    ws = [workloads.small_spheres(seed=s, prec="fp64", nx=nx, ny=ny, nz=nz, mobility=2e-3)
          for s, (nx, ny, nz) in enumerate([(40, 36, 64), (36, 44, 56), (48, 40, 60)])]
    sims, b = _batch_of(ws)
    assert b.info()["mode"] == 1
    b.step(100)
    b.sync()
    for w, g in zip(ws, sims):
        o = oracle.Oracle(w.nx, w.ny, w.nz, **{k: v for k, v in w.params.items() if k != "prec"})
        workloads.build(o, w)
        o.step(100)
        e = compare(g, o)
        assert e["flag_mismatch"] == 0 and e["rho"] < 1e-10 and e["vel"] < 1e-8 and e["force"] < 1e-9, e
    b.close()


def test_persistent_barrier_timeout_is_reported_and_recoverable():
    # a barrier wait limit of 0 cycles makes every block but the last give up at once: the step's
    # results are not valid, cbl_batch_sync reports CBL_ERR_TIMEOUT, and with the limit restored the
    # batch steps normally again
    from paper_1902_10432_gb300 import cbl

    ws = workloads.batch64(seed=7, n=2)
    sims, b = _batch_of(ws)
    b.set_option("spin_limit", 0)
    b.step(1)
    with pytest.raises(cbl.CblError) as ei:
        b.sync()
    assert ei.value.status == 5  # CBL_ERR_TIMEOUT
    b.set_option("spin_limit", 4e9)
    b.step(3)
    b.sync()  # no error this time
    b.close()


def test_autotune_picks_a_batch_tile():
    from paper_1902_10432_gb300 import autotune

    ws = workloads.batch64(seed=8, n=3)
    sims, b = _batch_of(ws)
    tile, ms = autotune.tune_batch(b, steps=2)
    assert tile in autotune.BATCH_TILES and len(ms) == len(autotune.BATCH_TILES)
    assert b.info()["tile"] == tile
    b.close()
