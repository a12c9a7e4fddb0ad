"""Closed forms and measurement helpers used to pin the oracle (test infrastructure only).

Each function states the passage of arXiv:1902.10432 it restates. None of them is used by
the CUDA library.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate, optimize

CS2 = 1.0 / 3.0


# --- Sec. 3.2.3: pseudo-potential, equation of state, interface tension --------------------
def psi(rho, rho0=1.0):
    """Eq. mean_field_potential: psi = 1 - exp(-rho / rho0)."""
    return 1.0 - np.exp(-np.asarray(rho) / rho0)


def eos_pressure(rho, G=-5.0, rho0=1.0):
    """Eq. pressure: p = c_s^2 rho + (1/2) c_s^2 G psi^2."""
    return CS2 * np.asarray(rho) + 0.5 * CS2 * G * psi(rho, rho0) ** 2


def coexistence(G=-5.0, rho0=1.0, eps=0.0, guess=(1.9, 0.12)):
    """Flat-interface coexistence densities of the pseudo-potential fluid.

    Mechanical stability across a flat interface gives p(rho_l) = p(rho_v) = p0 and
    int_{rho_v}^{rho_l} (p0 - p(rho)) psi'(rho) / psi(rho)^(1 + eps) d rho = 0. eps = 0 is the
    rule whose liquid branch reproduces the paper's rho_L = 1.888 (parameter table, Sec. 3.3).
    """

    def dpsi(r):
        return np.exp(-r / rho0) / rho0

    def eqs(v):
        rl, rv = v
        p0 = float(eos_pressure(rl, G, rho0))
        f = lambda r: (p0 - float(eos_pressure(r, G, rho0))) * dpsi(r) / float(psi(r, rho0)) ** (1.0 + eps)
        return [float(eos_pressure(rl, G, rho0) - eos_pressure(rv, G, rho0)),
                integrate.quad(f, rv, rl, limit=200)[0]]

    rl, rv = optimize.fsolve(eqs, guess, xtol=1e-13)
    return float(rl), float(rv)


def planar_tension(psi_profile, G=-5.0):
    """Eq. interface_tension (with c_x read as c_s): sigma = -1/2 c_s^4 G int |d psi/dn|^2 dn.

    psi_profile is psi on unit-spaced nodes across ONE interface; the derivative is the central
    difference and the integral the node sum.
    """
    p = np.asarray(psi_profile, np.float64)
    d = 0.5 * (p[2:] - p[:-2])
    return -0.5 * CS2 * CS2 * G * float(np.sum(d * d))


# --- Sec. 2.1: plates -------------------------------------------------------------------------
def plate_force_planar(sigma, L):
    """Eq. plate_force_planar: F_p = 2 sigma L."""
    return 2.0 * sigma * L


def plate_force_cylinder(sigma, R):
    """Eq. plate_force: F_c = pi sigma R (90 degree wetting)."""
    return math.pi * sigma * R


def plate_force_volume(sigma, R0, h0, h):
    """App. A: F = pi sigma R0 sqrt(h0 / h) at constant liquid volume."""
    return math.pi * sigma * R0 * math.sqrt(h0 / h)


def plate_gap_planar(h0, sigma, L, m, t):
    """Eq. theory_plates_motion_2d: h_p = h0 - (2 sigma L / m) t^2 (both plates free)."""
    return h0 - 2.0 * sigma * L / m * np.asarray(t, float) ** 2


def plate_gap_cylinder(h0, sigma, R0, m, t):
    """Eq. theory_plate_motion_approx: h_c = h0 - (pi sigma R0 / m) t^2."""
    return h0 - math.pi * sigma * R0 / m * np.asarray(t, float) ** 2


# --- Sec. 2.2 and App. B: two spheres ------------------------------------------------------
def theta_spherical(c):
    """Eq. theory_2_spheres_spherical: wetting angle of a spherical bridge vs liquid fraction."""
    c = float(c)
    chi = 2.0 / 3.0 ** 0.25 * math.sqrt((1.0 - c) * math.sqrt(c * (1.0 - c))) / (1.0 - c)
    return math.acos((chi * chi - 2.0) / 2.0) - math.acos(chi / 2.0)


def theta_cylindrical(c):
    """Eq. theory_2_spheres_cylindrical: wetting angle of a cylindrical bridge."""
    c = float(c)
    chi = -math.cos(math.acos((1.0 - 9.0 * c) / (1.0 - c)) / 3.0 + math.pi / 3.0) + 0.5
    return math.pi / 2.0 - math.acos(1.0 - chi)


def liquid_fraction(VL, VS):
    """Sec. 2.2: c = V_L / (V_L + V_S)."""
    return VL / (VL + VS)


# --- Sec. 4.1: Laplace fit ----------------------------------------------------------------
def laplace_slope(inv_R, dp):
    """Eq. young_laplace: dp = sigma kappa; least-squares slope through the origin."""
    x = np.asarray(inv_R, float)
    y = np.asarray(dp, float)
    return float(np.dot(x, y) / np.dot(x, x))


# --- Young's law (Sec. 2.1.1): contact angle of a cap on a flat wall --------------------------
def cap_angle(base_halfwidth, height):
    """Contact angle of a circular cap (2D cut) from its base half-width a and height h:
    tan(theta/2) = h / a."""
    return 2.0 * math.atan2(height, base_halfwidth)


# --- Sec. 2.1: a bridge between parallel plates away from 90 degrees ---------------------------
def toroidal_bridge(sigma, theta, h, V):
    """Toroidal (circular-meridian) approximation of an axisymmetric liquid bridge between two
    parallel plates with the same contact angle theta (radians, 0 < theta <= pi/2), gap h and liquid
    volume V. The paper's force on a plate (Sec. 2.1, Eq. plate_force) is the surface-tension pull
    along the contact line plus the Laplace pressure on the wetted area; evaluated at the neck
    (radius a) it is F = 2 pi sigma a - pi a^2 dp, with dp = sigma (1/a - 1/r1) from Eq.
    young_laplace with the two principal curvatures, the meridian being a circle of radius
    r1 = h / (2 cos theta) that meets both plates at theta. Hence F = pi sigma a (1 + a / r1); at
    90 degrees r1 is infinite and F = pi sigma a with V = pi a^2 h (the cylinder of Eq.
    plate_force). a follows from V = pi int_{-h/2}^{h/2} (a + r1 - sqrt(r1^2 - z^2))^2 dz.
    Returns (a, r1, F)."""
    if abs(theta - math.pi / 2) < 1e-12:
        a = math.sqrt(V / (math.pi * h))
        return a, math.inf, math.pi * sigma * a
    r1 = h / (2.0 * math.cos(theta))

    def vol(a):
        f = lambda z: (a + r1 - math.sqrt(r1 * r1 - z * z)) ** 2
        return math.pi * integrate.quad(f, -0.5 * h, 0.5 * h)[0]

    a = optimize.brentq(lambda x: vol(x) - V, 1e-9, math.sqrt(V / (math.pi * h)) + r1)
    return a, r1, math.pi * sigma * a * (1.0 + a / r1)
