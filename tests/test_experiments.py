"""Host-side helpers of the experiments (no GPU): the t^2 fit of the plate motion, the contact-time
detector, periodic pair distances, and the geometry of the particle-cluster workloads."""
import itertools
import math

import numpy as np
import pytest

from paper_1902_10432_gb300 import workloads


def _experiments():
    # the module imports the CUDA binding lazily through cbl, which loads without a GPU
    from paper_1902_10432_gb300 import experiments
    return experiments


def test_fit_t2_recovers_a_uniform_acceleration():
    ex = _experiments()
    t = np.linspace(0.01, 0.15, 20)
    k, slope = ex.fit_t2(t, math.pi * t ** 2)  # Eq. plate_motion_rescaled, cylindrical
    assert k == pytest.approx(math.pi, rel=1e-12) and slope == pytest.approx(2.0, abs=1e-9)
    k, slope = ex.fit_t2(t, 2.0 * t ** 2 * (1 + 0.1 * t))  # slightly faster than uniform
    assert 2.0 < k < 2.04 and 2.0 < slope < 2.1


def test_contact_time_is_the_drop_of_the_approach_speed():
    ex = _experiments()
    t = np.arange(0, 3000, 10.0)
    # approach with constant acceleration until t = 2000, then held at contact
    h = np.where(t < 2000, 20.0 - 20.0 * (t / 2000.0) ** 2, 0.0)
    hd = np.gradient(h, t)
    tc = ex.contact_time(t, h, hd)
    assert 2000 <= tc <= 2020
    assert ex.contact_time(t, np.full_like(t, 5.0), np.zeros_like(t)) == math.inf  # never approaches


def test_pair_gaps_use_the_minimum_image():
    ex = _experiments()
    X = np.array([[1.0, 5.0, 5.0], [39.0, 5.0, 5.0], [20.0, 5.0, 5.0]])
    g = ex._pair_gaps(X, 0.5, (40, 10, 10))
    assert g == pytest.approx([2.0 - 1.0, 19.0 - 1.0, 19.0 - 1.0])


@pytest.mark.parametrize("n", [2, 3, 4])
def test_cluster_geometry(n):
    R, h0, c = 30.0, 20.0, 0.3
    w = workloads.cluster(n, c, R=R, h0=h0)
    C = np.array([b["center"] for b in w.bodies])
    assert len(C) == n and all(b["radius"] == R and b["wetting_rho"] == 2.0 for b in w.bodies)
    for i, j in itertools.combinations(range(n), 2):  # equal surface gaps h0
        assert np.linalg.norm(C[i] - C[j]) - 2 * R == pytest.approx(h0, abs=1e-9)
    # the drop sits at the centre and holds V_L = c / (1 - c) V_S (liquid fraction c, Sec. 2.2)
    VS = n * 4.0 / 3.0 * math.pi * R ** 3
    assert w.meta["liquid_volume"] == pytest.approx(c / (1 - c) * VS)
    assert abs(w.mask.sum() / w.meta["liquid_volume"] - 1) < 0.01
    z, y, x = np.nonzero(w.mask)
    assert np.allclose([x.mean(), y.mean(), z.mean()], C.mean(axis=0), atol=1.0)
    # the spheres and the drop stay inside the lattice with a margin (no periodic contact)
    dims = np.array([w.nx, w.ny, w.nz])
    assert (C.min(axis=0) - R >= 10).all() and (C.max(axis=0) + R <= dims - 10).all()
    assert w.params["tau"] == 1.1 and w.params["q"] == 27  # the paper's parameter table and lattice
