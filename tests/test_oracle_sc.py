"""Pins of the oracle's Shan-Chen fluid against the paper's printed values (Sec. 3.3, Sec. 4.1).

Flat interface: bulk densities vs rho_L = 1.888 (parameter table) and the flat-interface
stability rule; planar tension from Eq. interface_tension vs the printed 3.297e-2; Laplace
law vs the printed 3.583e-2 (Sec. 4.1, D3Q27, tau = 1.1).
"""
import numpy as np
import pytest

import oracle
from oracle import analysis as an

RHO_L, RHO_V = 1.88844, 0.11942


def test_coexistence_rule_reproduces_paper_liquid_density():
    rl, rv = an.coexistence(G=-5.0, eps=0.0)
    assert abs(rl - 1.888) < 1e-3  # parameter table
    assert 0.10 < rv < 0.14
    # the classic rule (eps = 2) would not give the paper's value
    rl2, _ = an.coexistence(G=-5.0, eps=2.0, guess=(1.95, 0.18))
    assert abs(rl2 - 1.888) > 0.05


def _slab(q, tau, steps=12000):
    L = 64
    o = oracle.Oracle(1, 1, L, q=q, tau=tau)
    z = np.arange(L)
    o.init_fluid(RHO_L, RHO_V, ((z >= 16) & (z < 48)).reshape(L, 1, 1))
    o.step(steps)
    r, v, _ = o.fields()
    o.step(1)
    _, v1, _ = o.fields()
    return r[:, 0, 0], v, v1


@pytest.mark.parametrize("q,tau", [(19, 1.0), (27, 1.1)])
def test_flat_interface_bulk_densities_and_planar_tension(q, tau):
    r, v, v1 = _slab(q, tau)
    rl, rv = an.coexistence(G=-5.0, eps=0.0)
    assert abs(r[32] - 1.888) < 0.01 * 1.888          # paper's rho_L
    assert abs(r[32] - rl) < 1e-3 * rl                   # flat-interface rule
    assert abs(r[0] - rv) < 3e-3 * rv
    # equilibrium: no mean flow. The sharp initial step leaves the lattice's period-2
    # staggered mode (u alternating in space and time, always at equilibrium, so BGK cannot
    # damp it); it cancels between consecutive steps.
    assert np.abs(v + v1).max() < 1e-9
    sig = an.planar_tension(an.psi(r[0:33]))
    assert abs(sig - 3.297e-2) < 0.01 * 3.297e-2, sig  # Sec. 4.1 printed value


@pytest.mark.parametrize("q,tau,tol,tol_meas", [(27, 1.1, 0.02, 0.05), (19, 1.0, 0.03, 0.06)])
def test_laplace_law_cylindrical_droplets(q, tau, tol, tol_meas):
    # Sec. 4.1: cylindrical droplets, pressure difference from Eq. pressure vs 1/R; the paper's
    # fit (D3Q27, tau = 1.1) gives sigma = 3.583e-2. Fitted here against the nominal radii (within
    # 2 %) and against the radii measured from the liquid area (within 5 %); the D3Q19, tau = 1
    # fluid of the workloads is within 3 % of the same value with the nominal radii and 6 % with the
    # measured ones (its fits are printed: 3.50e-2 and 3.40e-2)
    n = 80
    nominal, measured, dps = [], [], []
    for R in (12, 16, 20):
        o = oracle.Oracle(n, 1, n, q=q, tau=tau)
        z, x = np.mgrid[0:n, 0:n]
        mask = (x - n / 2 + 0.5) ** 2 + (z - n / 2 + 0.5) ** 2 <= R * R
        o.init_fluid(RHO_L, RHO_V, mask.reshape(n, 1, n))
        o.step(3000)
        r, _, _ = o.fields()
        r = r[:, 0, :]
        c = slice(n // 2 - 2, n // 2 + 2)
        dp = an.eos_pressure(r[c, c]).mean() - an.eos_pressure(r[:4, :4]).mean()
        rl, rv = r[n // 2, n // 2], r[0, 0]
        nominal.append(1.0 / R)
        measured.append(1.0 / np.sqrt(((r - rv) / (rl - rv)).sum() / np.pi))
        dps.append(dp)
    s_nom = an.laplace_slope(nominal, dps)
    s_meas = an.laplace_slope(measured, dps)
    print("D3Q%d tau %.1f: Laplace sigma %.5f (nominal radii), %.5f (measured radii)" % (q, tau, s_nom, s_meas))
    assert abs(s_nom - 3.583e-2) < tol * 3.583e-2, s_nom
    assert abs(s_meas - 3.583e-2) < tol_meas * 3.583e-2, s_meas
    # linear in 1/R: each point within 4 % of the fitted line
    assert np.all(np.abs(np.array(dps) / (s_nom * np.array(nominal)) - 1) < 0.04)
