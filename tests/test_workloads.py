"""Seeded input generators: the shapes and invariants their docstrings promise (no GPU, no oracle)."""
import math

import numpy as np

from paper_1902_10432_gb300 import surrogate, workloads


def _min_image(d, L):
    d = np.asarray(d, float)
    return (d + L / 2.0) % L - L / 2.0


def test_packing_gaps_pairs_and_drop_volumes():
    w, pairs, vols = workloads.packing(seed=3, n_spheres=12, L=64, Rmin=5.0, Rmax=7.0, bridge_gap=6.0)
    C = [np.array(b["center"]) for b in w.bodies]
    R = [b["radius"] for b in w.bodies]
    assert len(C) == 12 and all(5.0 <= r <= 7.0 for r in R)
    for i in range(len(C)):
        for j in range(i + 1, len(C)):
            gap = np.linalg.norm(_min_image(C[j] - C[i], 64)) - R[i] - R[j]
            assert gap >= 2.0 - 1e-9  # random sequential addition keeps the minimum surface gap
            assert ((i, j) in pairs) == (gap < 6.0)
    for (i, j), v in vols.items():
        assert math.isclose(v, 0.1 * 4.0 / 3.0 * math.pi * (R[i] ** 3 + R[j] ** 3))
    # liquid cells are outside every sphere; each drop holds its volume unless drops overlap
    z, y, x = np.nonzero(w.mask)
    P = np.stack([x, y, z], 1).astype(float)
    for c, r in zip(C, R):
        assert (np.linalg.norm(_min_image(P - c, 64), axis=1) > r - 1e-9).all()
    assert w.mask.sum() <= sum(round(v) for v in vols.values())
    if len(pairs) == 1:
        assert w.mask.sum() == round(next(iter(vols.values())))


def test_batch64_radii_fit_and_gap():
    for w in workloads.batch64(seed=1, n=16):
        L = [w.nx, w.ny, w.nz]
        ax = int(np.argmax(L))
        c0, c1 = (np.array(b["center"]) for b in w.bodies)
        r0, r1 = (b["radius"] for b in w.bodies)
        assert math.isclose(abs(c1[ax] - c0[ax]) - r0 - r1, 4.0)
        others = [L[a] for a in range(3) if a != ax]
        assert max(r0, r1) <= (min(others) - 8) / 2.0 + 1e-12
        assert 30.0 <= w.meta["theta_deg"] <= 90.0


def test_pair_frame_and_targets_rotate_with_the_pair():
    # the frame is orthonormal, e_z points from i to j (minimum image), and the targets are the force
    # and torque in that frame over 2 pi R* sigma and 2 pi R*^2 sigma, R* = 2 Ri Rj / (Ri + Rj)
    frame, r = surrogate.pair_frame((60.0, 3.0, 5.0), (2.0, 3.0, 5.0), (64, 64, 64))
    assert math.isclose(r, 6.0)
    assert np.allclose(frame @ frame.T, np.eye(3))
    assert np.allclose(frame[2], [1.0, 0.0, 0.0])
    F, T = np.array([1.0, 2.0, 3.0]), np.array([0.5, -1.0, 0.25])
    y = surrogate.targets(F, T, frame, 2.0, 6.0)
    s = 2.0 * math.pi * 3.0 * surrogate.SIGMA
    assert np.allclose(frame.T @ y[:3] * s, F)
    assert np.allclose(frame.T @ y[3:] * s * 3.0, T)
    x, _ = surrogate.features((0.0, 0.0, 0.0), (0.0, 0.0, 10.0), 2.0, 6.0, 12.0, 60.0, (64, 64, 64))
    assert np.allclose(x, [2.0 * math.sqrt(3.0 / 12.0), 0.5, 1.0 / 3.0, 12.0 / 27.0])


def test_bridge_state_counts_liquid_and_detects_rupture():
    import torch

    # two spheres on the x axis of a periodic 40^3 box (centres across the boundary), surface gap 4,
    # a liquid cylinder of radius 3 spanning the gap
    n, R = 40, 6.0
    Xi, Xj = np.array([35.0, 20.0, 20.0]), np.array([51.0 - 40.0, 20.0, 20.0])
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    rho = np.full((n, n, n), 0.12)
    xs = (x - 35.0 + 20.0) % 40.0 - 20.0  # x relative to sphere i, minimum image
    cyl = (xs >= 6.0) & (xs <= 10.0) & ((y - 20.0) ** 2 + (z - 20.0) ** 2 <= 9.0)
    rho[cyl] = 1.9
    t = torch.tensor(rho)
    vol, intact = surrogate.bridge_state(t, Xi, Xj, R, R, (n, n, n))
    assert intact and vol == cyl.sum()
    rho[cyl & (xs >= 7.0) & (xs <= 9.0)] = 0.12  # cut the neck about the gap's middle
    vol2, intact2 = surrogate.bridge_state(torch.tensor(rho), Xi, Xj, R, R, (n, n, n))
    assert not intact2 and vol2 < vol
