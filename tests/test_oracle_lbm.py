"""Pins of the oracle's lattice-Boltzmann part against closed forms, invariants and brute force.

Sec. 3.2.1 (velocity set, equilibrium, BGK, Guo forcing, streaming) and Sec. 3.2.2
(bounce-back, momentum exchange, mass correction).
"""

import numpy as np
import pytest

import oracle

RHO_L, RHO_V = 1.88844, 0.11942


@pytest.mark.parametrize("q", [19, 27])
def test_velocity_set_moments(q):
    # Isotropy of the weights: sum w = 1, sum w c = 0, sum w c_a c_b = c_s^2 delta_ab,
    # sum w c_a c_b c_c c_d = c_s^4 (dd + dd + dd) -- fixes the weights of Sec. 3.2.1 (Q27)
    # and of the D3Q19 reading.
    o = oracle.Oracle(2, 2, 2, q=q)
    c, w = o.velocity_set()
    assert c.shape == (q, 3)
    assert abs(w.sum() - 1) < 1e-15
    assert np.abs(w @ c).max() < 1e-15
    m2 = np.einsum("i,ia,ib->ab", w, c, c)
    assert np.abs(m2 - np.eye(3) / 3).max() < 1e-15
    m4 = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    d = np.eye(3)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d) + np.einsum("ad,bc->abcd", d, d)) / 9
    assert np.abs(m4 - iso).max() < 1e-15
    if q == 27:
        assert sorted(set(np.round(w * 216).astype(int))) == [1, 4, 16, 64]  # 1/216, 1/54, 2/27, 8/27


def test_static_uniform_is_fixed_point():
    # P1: uniform density at rest, no solids, with SC force: the state does not change.
    o = oracle.Oracle(6, 5, 4)
    o.init_fluid(1.3, 1.3)
    f0 = o.populations().copy()
    o.step(20)
    assert np.abs(o.populations() - f0).max() < 1e-14


@pytest.mark.parametrize("L", [32, 64])
def test_shear_wave_decay(L):
    # P2: u_x = A sin(2 pi z / L), G = 0: amplitude ~ exp(-nu k^2 t), nu = c_s^2 (tau - 1/2).
    # BGK's error in the decay rate is O(k^2): 2e-3 at L = 32, four times less at L = 64.
    tau = 0.8
    o = oracle.Oracle(2, 2, L, tau=tau, G=0.0)
    z = np.arange(L)[:, None, None] * np.ones((L, 2, 2))
    u = np.zeros((L, 2, 2, 3))
    u[..., 0] = 1e-3 * np.sin(2 * np.pi * z / L)
    o.init_fluid_fields(np.ones((L, 2, 2)), u)
    ts, amps = [], []
    span = L * L // 2
    for t in range(0, 2 * span + 1, span // 8):
        if t:
            o.step(span // 8)
        _, v, _ = o.fields()
        ts.append(o.t)
        amps.append(abs(np.fft.rfft(v[:, 0, 0, 0])[1]) * 2 / L)
    ts, amps = np.array(ts), np.array(amps)
    rate = -np.polyfit(ts[4:], np.log(amps[4:]), 1)[0]
    nu = (tau - 0.5) / 3
    k = 2 * np.pi / L
    rel = rate / (nu * k * k) - 1
    assert abs(rel) < (4e-3 if L == 32 else 1.2e-3), rel


def test_guo_force_momentum_exact():
    # P3: uniform force density f, G = 0, periodic: sum_i c_i f_i grows by exactly f per cell
    # per step (Eq. guo_forcing / Eq. fluid_velocity), and the reported velocity is the
    # half-step value (sum c f + f/2)/rho.
    fext = np.array([1e-5, -2e-5, 3e-5])
    o = oracle.Oracle(4, 3, 5, G=0.0, ext_force=tuple(fext))
    o.init_fluid(0.9, 0.9)
    N = 60
    p0, _ = o.total_momentum()
    o.step(7)
    p1, _ = o.total_momentum()
    assert np.allclose(p1 - p0, 7 * N * fext, rtol=1e-12, atol=0)
    _, v, _ = o.fields()
    # the 7th collision saw sum c f = 6 f after streaming, so rho v = 6 f + f/2
    assert np.allclose(v.reshape(-1, 3)[0] * 0.9, 6.5 * fext, rtol=1e-12)


def test_translation_invariance_bitwise():
    # P11: an integer translation of the initial state gives the translated result, bitwise.
    n = (10, 8, 12)
    rng = np.random.default_rng(3)
    rho = 0.2 + 1.6 * (rng.random((n[2], n[1], n[0])) > 0.5)
    a = oracle.Oracle(*n)
    a.add_body("sphere", (4.0, 3.0, 5.0), radius=2.6, wetting_rho=1.2, fixed=True)
    a.init_fluid_fields(rho)
    s = (3, 5, 7)  # shift in x, y, z
    b = oracle.Oracle(*n)
    b.add_body("sphere", (4.0 + s[0], 3.0 + s[1], 5.0 + s[2]), radius=2.6, wetting_rho=1.2, fixed=True)
    b.init_fluid_fields(np.roll(rho, (s[2], s[1], s[0]), axis=(0, 1, 2)))
    a.step(15)
    b.step(15)
    ra, va, _ = a.fields()
    rb, vb, _ = b.fields()
    assert np.array_equal(np.roll(ra, (s[2], s[1], s[0]), axis=(0, 1, 2)), rb)
    assert np.array_equal(np.roll(va, (s[2], s[1], s[0]), axis=(0, 1, 2)), vb)


def test_one_step_brute_force_bounce_back():
    # P12: 4^3 periodic box, one solid node, G = 0, random populations. One step computed here
    # by hand: pull, half-way bounce-back at the solid link, BGK towards f_eq, and the
    # momentum exchange -c_i (2 f*_opp + 0) on the resting body.
    o = oracle.Oracle(4, 4, 4, G=0.0, tau=0.9)
    o.add_body("sphere", (1.0, 2.0, 1.0), radius=2.0, wetting_rho=1.0, fixed=True)
    o.init_fluid(1.0, 1.0)
    solid, _ = o.flags()
    assert solid.sum() == 1 and solid[1, 2, 1] == 1
    c, w = o.velocity_set()
    Q = len(w)
    opp = [int(np.where((c == -c[i]).all(1))[0][0]) for i in range(Q)]
    rng = np.random.default_rng(0)
    f = 0.02 + 0.05 * rng.random((Q, 4, 4, 4))
    f[:, 1, 2, 1] = 0.0
    o.set_populations(f)
    o.step(1)
    exp = np.zeros_like(f)
    F = np.zeros(3)
    for z in range(4):
        for y in range(4):
            for x in range(4):
                if solid[z, y, x]:
                    continue
                fi = np.zeros(Q)
                for i in range(Q):
                    sx, sy, sz = (x - c[i, 0]) % 4, (y - c[i, 1]) % 4, (z - c[i, 2]) % 4
                    if i and solid[sz, sy, sx]:
                        fi[i] = f[opp[i], z, y, x]
                        F += -c[i] * 2 * f[opp[i], z, y, x]
                    else:
                        fi[i] = f[i, sz, sy, sx]
                rho = fi.sum()
                u = (c.T @ fi) / rho
                cu = c @ u
                feq = rho * w * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * u @ u)
                exp[:, z, y, x] = fi - (fi - feq) / 0.9
    got = o.populations()
    assert np.abs(got - exp).max() < 1e-15
    Fo, _, parts = o.body_forces()
    assert np.allclose(parts[0, 0, :3], F, rtol=1e-12, atol=1e-15)


def _plates(nx=48, q=19, wet=1.0, fixed=True, rho_s=4.0, gap_axis=2):
    o = oracle.Oracle(nx, nx, nx, q=q)
    c = (nx - 1) / 2.0
    o.add_body("box", (c, c, 16.0), half=(17.8, 17.8, 3.3), wetting_rho=wet, fixed=fixed, mass_density=rho_s)
    o.add_body("box", (c, c, 31.0), half=(17.8, 17.8, 3.3), wetting_rho=wet, fixed=fixed, mass_density=rho_s)
    z, y, x = np.mgrid[0:nx, 0:nx, 0:nx]
    mask = ((x - c) ** 2 + (y - c) ** 2 <= 100) & (z >= 18) & (z <= 29)
    o.init_fluid(RHO_L, RHO_V, mask)
    return o


def test_plate_geometry_and_mirror_symmetry():
    # P10: the two-plate bridge is mirror symmetric about the gap's mid-plane, so the force on
    # plate 1 is minus the force on plate 2, the torques vanish and the lateral components vanish.
    o = _plates()
    solid, owner = o.flags()
    assert solid.sum() == 2 * 32 * 32 * 3
    assert set(np.unique(np.nonzero(solid)[0])) == {15, 16, 17, 30, 31, 32}
    o.step(40)
    F, T, _ = o.body_forces()
    scale = np.abs(F).max()
    assert scale > 0.1
    assert np.abs(F[0] + F[1]).max() < 1e-12 * scale
    assert np.abs(F[:, :2]).max() < 1e-12 * scale
    assert np.abs(T).max() < 1e-10 * scale
    assert F[0, 2] > 0  # the wetting bridge pulls plate 1 (below the gap) towards +z


def test_mass_conservation_moving_bodies():
    # P8: with the negative-sum mass correction, the refill and zero-population uncover rule,
    # the total fluid mass is conserved to round-off while bodies move and cells are covered
    # and uncovered.
    o = oracle.Oracle(24, 20, 20, mpf_kinetics=1)
    o.add_body("sphere", (8.0, 10.0, 10.0), radius=4.5, wetting_rho=1.5, mass_density=0.5)
    o.add_body("sphere", (17.0, 10.5, 9.5), radius=3.5, wetting_rho=0.8, mass_density=0.5)
    z, y, x = np.mgrid[0:20, 0:20, 0:24]
    o.init_fluid(RHO_L, RHO_V, (x > 9) & (x < 16))
    o.set_body_velocity(0, V=(0.05, 0.01, 0.0), W=(0.0, 0.0, 0.01))
    o.set_body_velocity(1, V=(-0.04, 0.0, 0.02))
    m0 = o.total_mass()
    s0, _ = o.flags()
    o.step(60)
    s1, _ = o.flags()
    assert (s0 != s1).sum() > 20  # cells were covered and uncovered
    assert abs(o.total_mass() - m0) < 1e-12 * m0
    assert o.lost_refills == 0


def test_momentum_conservation_fluid_plus_bodies():
    # P9: momentum exchange and SC adhesion act as equal and opposite pairs, so fluid plus body
    # momentum is conserved in a periodic box (no solid-solid contact).
    o = oracle.Oracle(20, 18, 16)
    o.add_body("sphere", (9.0, 9.0, 8.0), radius=4.0, wetting_rho=1.4, mass_density=0.3)
    z, y, x = np.mgrid[0:16, 0:18, 0:20]
    o.init_fluid(RHO_L, RHO_V, (x > 11) & (x < 17))
    o.set_body_velocity(0, V=(0.02, -0.01, 0.0), W=(0.0, 0.005, 0.0))
    pf0, pb0 = o.total_momentum()
    p0 = pf0 + pb0
    for _ in range(4):
        o.step(10)
        pf, pb = o.total_momentum()
        assert np.abs(pf + pb - p0).max() < 1e-11, (pf + pb - p0)
    assert np.abs(pb - pb0).max() > 1e-4  # the body did exchange momentum


def test_couette_moving_wall_closed_form():
    # Moving-wall bounce-back (Sec. 3.2.2 Eqs. lb_bounce_back, lb_bounce_back_us): planar Couette
    # flow between a held plate and a plate sliding tangentially at U (very heavy, so its velocity
    # stays U). For BGK with half-way bounce-back the steady profile is exactly linear between the
    # half-way wall positions, u_x = U (z - z_wall)/H, for any tau (the linear profile satisfies the
    # lattice equations with the Chapman-Enskog non-equilibrium part, and the moving-wall term gives
    # the wall velocity at the link midpoint). A wrong factor or sign in g, or a wall term applied
    # to the wrong population, changes the slope or the wall value. Two channels: the gap between
    # the plates, and the gap that closes through the periodic boundary.
    U, nz = 0.02, 24
    o = oracle.Oracle(4, 4, nz, G=0.0, tau=0.8, e0=0.0)
    o.add_body("box", (1.5, 1.5, 3.0), half=(50.0, 50.0, 3.3), wetting_rho=1.0, fixed=True)
    o.add_body("box", (1.5, 1.5, 15.0), half=(50.0, 50.0, 3.3), wetting_rho=1.0, mass_density=1e16)
    o.init_fluid(1.0, 1.0)
    o.set_body_velocity(1, V=(U, 0.0, 0.0))
    solid, owner = o.flags()
    col = solid[:, 0, 0]
    held = np.nonzero(owner[:, 0, 0] == 0)[0]
    moving = np.nonzero(owner[:, 0, 0] == 1)[0]
    assert list(held) == [2, 3, 4] and list(moving) == [14, 15, 16]
    o.step(3000)  # slowest mode decays as exp(-nu (pi/H)^2 t): 1e-16 by then
    r, v, _ = o.fields()
    ux = v[:, :, :, 0]
    exp = np.zeros(nz)
    H = 9.0
    for z in range(5, 14):  # held wall at 4.5, moving wall at 13.5
        exp[z] = U * (z - 4.5) / H
    for z in list(range(17, 24)) + [0, 1]:  # moving wall at 16.5, held wall at 1.5 + nz
        exp[z] = U * ((1.5 + nz - z) % nz) / H
    fluid = col == 0
    for y in range(4):
        for x in range(4):
            assert np.abs(ux[fluid, y, x] - exp[fluid]).max() < 1e-12 * U, (y, x)
    assert np.abs(v[fluid][..., 1:]).max() < 1e-14
    assert np.abs(r[fluid] - 1.0).max() < 1e-12


def test_one_step_brute_force_moving_body():
    # One step with a translating and rotating body, computed by hand: half-way bounce-back with the
    # moving-wall term g_i = 2 rho w_i c_i.u_B / c_s^2, u_B = V + omega x (x_mid - X_B) at the link
    # midpoint x_mid = x - c_i/2 (Eq. lb_bounce_back_us, Eq. solid_velocity), rho the density of the
    # pulled populations, the mass correction delta rho = -sum g_i on the rest population
    # (Eq. lb_bounce_back_mass), BGK; the momentum exchange -c_i (2 f*_opp + g_i) and its torque
    # about X_B with the arm at the link midpoint (Eq. solid_liquid_force).
    tau = 0.9
    o = oracle.Oracle(4, 4, 4, G=0.0, tau=tau)
    o.add_body("sphere", (1.0, 2.0, 1.0), radius=2.0, wetting_rho=1.0)
    o.init_fluid(1.0, 1.0)
    V = np.array([0.011, -0.023, 0.017])
    W = np.array([0.021, -0.013, 0.031])
    o.set_body_velocity(0, V=V, W=W)
    solid, _ = o.flags()
    assert solid.sum() == 1 and solid[1, 2, 1] == 1
    X = o.bodies()["X"][0].copy()
    c, w = o.velocity_set()
    Q = len(w)
    rest = int(np.where((c == 0).all(1))[0][0])
    opp = [int(np.where((c == -c[i]).all(1))[0][0]) for i in range(Q)]
    rng = np.random.default_rng(1)
    f = 0.02 + 0.05 * rng.random((Q, 4, 4, 4))
    f[:, 1, 2, 1] = 0.0
    o.set_populations(f)

    def mi(d):
        return (d + 2.0) % 4.0 - 2.0

    exp = np.zeros_like(f)
    F = np.zeros(3)
    T = np.zeros(3)
    for z in range(4):
        for y in range(4):
            for x in range(4):
                if solid[z, y, x]:
                    continue
                fi = np.zeros(Q)
                links = []
                for i in range(Q):
                    sx, sy, sz = (x - c[i, 0]) % 4, (y - c[i, 1]) % 4, (z - c[i, 2]) % 4
                    if i != rest and solid[sz, sy, sx]:
                        fi[i] = f[opp[i], z, y, x]
                        links.append(i)
                    else:
                        fi[i] = f[i, sz, sy, sx]
                rho = fi.sum()
                drho = 0.0
                for i in links:
                    mid = np.array([x, y, z], float) - 0.5 * c[i]
                    arm = mi(mid - X)
                    uB = V + np.cross(W, arm)
                    g = 2.0 * rho * w[i] * (c[i] @ uB) * 3.0
                    dP = -c[i] * (2.0 * f[opp[i], z, y, x] + g)
                    F += dP
                    T += np.cross(arm, dP)
                    fi[i] += g
                    drho -= g
                fi[rest] += drho
                u = (c.T @ fi) / rho
                cu = c @ u
                feq = rho * w * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * u @ u)
                exp[:, z, y, x] = fi - (fi - feq) / tau
    o.step(1)
    s1, _ = o.flags()
    assert np.array_equal(s1, solid)  # no cover event: the populations are the collision's
    got = o.populations()
    assert np.abs(got - exp).max() < 1e-15
    _, _, parts = o.body_forces()
    assert np.allclose(parts[0, 0, :3], F, rtol=1e-12, atol=1e-16)
    assert np.allclose(parts[0, 0, 3:], T, rtol=1e-11, atol=1e-16)


def test_storage_model_rounding():
    # the storage model's binary16 rounding (analysis option store_prec = 2) against numpy's IEEE
    # binary16 conversion, over normal and subnormal magnitudes and both signs
    rng = np.random.default_rng(4)
    vals = np.concatenate([rng.uniform(-2, 2, 2000), rng.uniform(-1e-4, 1e-4, 2000), rng.uniform(-1e-7, 1e-7, 500),
                           [0.0, 1.0, -1.0, 0.5, 2.0 ** -14, 2.0 ** -24, 3 * 2.0 ** -25, 1 + 2.0 ** -11]])
    vals = vals.astype(np.float32).astype(np.float64)  # the model rounds the float value
    got = np.array([oracle.round_binary16(v) for v in vals])
    assert np.array_equal(got, vals.astype(np.float16).astype(np.float64))
    # a run with FP32 storage stays within FP32 rounding of the FP64 run over a few steps
    rho = 0.12 + 1.77 * (np.random.default_rng(5).random((6, 5, 4)) > 0.5)
    a, b = oracle.Oracle(4, 5, 6), oracle.Oracle(4, 5, 6, store_prec=1)
    for o in (a, b):
        o.init_fluid_fields(rho)
        o.step(3)
    fa, fb = a.populations(), b.populations()
    assert np.array_equal(fb, fb.astype(np.float32).astype(np.float64))
    assert 0 < np.abs(fa - fb).max() < 1e-6
