"""D3Q27 (the velocity set the paper prints, Sec. 3.2.1) on the GPU against the oracle's D3Q27 mode."""
import numpy as np
import pytest

from paper_1902_10432_gb300 import workloads
from _pair import compare, make_pair

pytestmark = pytest.mark.gpu


def test_velocity_set_moments():
    from paper_1902_10432_gb300 import cbl

    for q in (19, 27):
        s = cbl.Sim(8, 8, 8, q=q, prec="fp64")
        c, w = s.velocity_set()
        assert c.shape == (q, 3) and np.isclose(w.sum(), 1.0)
        assert np.allclose(w @ c, 0.0)
        assert np.allclose(np.einsum("i,ia,ib->ab", w, c, c), np.eye(3) / 3.0)  # c_s^2 = 1/3
        assert np.allclose(np.einsum("i,ia,ib,ic->abc", w, c, c, c), 0.0)
        for i in range(1, q):  # opposite pairs: odd index, then its opposite
            j = i + 1 if i % 2 else i - 1
            assert (c[j] == -c[i]).all()
        s.close()


def test_plates_d3q27_fp64_matches_oracle():
    w = workloads.plates48(prec="fp64")
    g, o = make_pair(w, q=27)
    g.step(w.steps)
    o.step(w.steps)
    e = compare(g, o)
    assert e["flag_mismatch"] == 0
    assert e["rho"] < 1e-10 and e["vel"] < 1e-8
    assert e["force"] < 1e-9


def test_plates_d3q27_fp32():
    w = workloads.plates48(prec="fp32")
    g, o = make_pair(w, q=27)
    g.step(w.steps)
    o.step(w.steps)
    e = compare(g, o)
    assert e["flag_mismatch"] == 0
    assert e["rho"] < 1e-4 and e["vel"] < 1e-4
    assert e["force"] < 1e-3


def test_moving_spheres_d3q27_fp64_matches_oracle():
    w = workloads.small_spheres(prec="fp64")
    g, o = make_pair(w, q=27)
    g.step(200)
    o.step(200)
    e = compare(g, o)
    assert e["flag_mismatch"] == 0
    assert e["rho"] < 1e-9 and e["vel"] < 1e-8
    assert e["force"] < 1e-8 and e["X"] < 1e-10
