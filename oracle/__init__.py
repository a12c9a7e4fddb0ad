"""FP64 CPU oracle for the multi-phase-field / lattice-Boltzmann step (arXiv:1902.10432).

TEST INFRASTRUCTURE ONLY: this package is the slow, plain reference the CUDA library is
checked against. Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it; the product path never does. It shares no code with the CUDA
library (``paper_1902_10432_gb300``) and imports nothing from it.

The C++ source ``cbl_oracle.cpp`` implements the time step in the paper's order (Sec. 3.2.1
LB collision/streaming, Sec. 3.2.2 bounce-back / momentum exchange / refill, Sec. 3.2.3
Shan-Chen force with wetting, Sec. 3.1 rigid bodies and phase-field advection, Sec. 3.3
phase-field kinetics). ``Oracle`` below is argument marshalling only.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cbl_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (plain g++, OpenMP, no FMA contraction so x86 and Arm agree)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
               _SRC, "-o", tmp]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


class orc_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("q", ctypes.c_int),
        ("tau", ctypes.c_double), ("G", ctypes.c_double), ("rho0", ctypes.c_double),
        ("ext_force", ctypes.c_double * 3),
        ("mpf_kinetics", ctypes.c_int),
        ("mobility", ctypes.c_double), ("eta", ctypes.c_double),
        ("sigma_sf", ctypes.c_double), ("sigma_ss", ctypes.c_double),
        ("e0", ctypes.c_double), ("rc", ctypes.c_double),
        ("nrep", ctypes.c_int),
        ("solid_threshold", ctypes.c_double),
        ("member_threshold", ctypes.c_double),
        ("nthreads", ctypes.c_int),
        ("store_prec", ctypes.c_int),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            D = ctypes.POINTER(ctypes.c_double)
            lib.orc_create.restype = P
            lib.orc_create.argtypes = [ctypes.POINTER(orc_params)]
            lib.orc_destroy.argtypes = [P]
            lib.orc_add_body.restype = ctypes.c_int
            lib.orc_add_body.argtypes = [P, ctypes.c_int, D, ctypes.c_double, D, D,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_int]
            lib.orc_init_fluid.argtypes = [P, ctypes.c_double, ctypes.c_double, ctypes.c_void_p]
            lib.orc_init_fluid_fields.argtypes = [P, D, ctypes.c_void_p]
            lib.orc_step.argtypes = [P, ctypes.c_int]
            for name in ("orc_num_cells", "orc_time", "orc_lost_refills"):
                getattr(lib, name).restype = ctypes.c_long
                getattr(lib, name).argtypes = [P]
            lib.orc_num_bodies.restype = ctypes.c_int
            lib.orc_num_bodies.argtypes = [P]
            lib.orc_read_fields.argtypes = [P, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            lib.orc_read_flags.argtypes = [P, ctypes.c_void_p, ctypes.c_void_p]
            lib.orc_read_phi.argtypes = [P, ctypes.c_int, D]
            lib.orc_read_populations.argtypes = [P, D]
            lib.orc_write_populations.argtypes = [P, D]
            lib.orc_velocity_set.argtypes = [P, ctypes.POINTER(ctypes.c_int), D]
            lib.orc_read_body_forces.argtypes = [P, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            lib.orc_get_bodies.argtypes = [P] + [ctypes.c_void_p] * 6
            lib.orc_set_body_velocity.argtypes = [P, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
            lib.orc_set_body_fixed.argtypes = [P, ctypes.c_int, ctypes.c_int]
            lib.orc_integrate_body.argtypes = [P, ctypes.c_int, D, D]
            lib.orc_total_mass.restype = ctypes.c_double
            lib.orc_total_mass.argtypes = [P]
            lib.orc_total_momentum.argtypes = [P, D, D]
            lib.orc_phase_only.argtypes = [P, ctypes.c_int]
            lib.orc_round_binary16.restype = ctypes.c_double
            lib.orc_round_binary16.argtypes = [ctypes.c_double]
            _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _vp(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


DEFAULTS = dict(q=19, tau=1.0, G=-5.0, rho0=1.0, ext_force=(0.0, 0.0, 0.0), mpf_kinetics=0,
                mobility=1e-5, eta=5.0, sigma_sf=3.583e-2, sigma_ss=0.5 * 3.583e-2, e0=1e-3, rc=3.0, nrep=4,
                solid_threshold=0.05, member_threshold=0.5, nthreads=0, store_prec=0)


class Oracle:
    """One FP64 simulation. Arrays are numpy, cell index = x + nx*(y + ny*z)."""

    def __init__(self, nx, ny, nz, **kw):
        lib = _load()
        cfg = dict(DEFAULTS)
        unknown = set(kw) - set(cfg)
        if unknown:
            raise TypeError("unknown oracle parameters: %s" % sorted(unknown))
        cfg.update(kw)
        p = orc_params()
        p.nx, p.ny, p.nz = nx, ny, nz
        for k, v in cfg.items():
            if k == "ext_force":
                p.ext_force[:] = list(v)
            else:
                setattr(p, k, v)
        self.params = cfg
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz
        self._lib = lib
        self._h = lib.orc_create(ctypes.byref(p))
        if not self._h:
            raise ValueError("oracle rejected the parameters")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_destroy(h)
            self._h = None

    # -- set-up -------------------------------------------------------------------------------
    def add_body(self, shape, center, radius=0.0, half=(0.0, 0.0, 0.0), quat=(1.0, 0.0, 0.0, 0.0),
                 mass_density=4.0, wetting_rho=2.0, fixed=False):
        c = np.asarray(center, np.float64)
        h = np.asarray(half, np.float64)
        q = np.asarray(quat, np.float64)
        sid = {"sphere": 0, "box": 1}[shape] if isinstance(shape, str) else int(shape)
        bid = self._lib.orc_add_body(self._h, sid, _dp(c), float(radius), _dp(h), _dp(q),
                                     float(mass_density), float(wetting_rho), int(bool(fixed)))
        if bid < 0:
            raise RuntimeError("add_body after init_fluid")
        return bid

    def init_fluid(self, rho_l, rho_v, mask=None):
        m = None if mask is None else np.ascontiguousarray(mask, np.uint8).reshape(-1)
        self._lib.orc_init_fluid(self._h, float(rho_l), float(rho_v), _vp(m))

    def init_fluid_fields(self, rho, u=None):
        r = np.ascontiguousarray(rho, np.float64).reshape(-1)
        uu = None if u is None else np.ascontiguousarray(u, np.float64).reshape(-1)
        self._lib.orc_init_fluid_fields(self._h, _dp(r), _vp(uu))

    # -- stepping -----------------------------------------------------------------------------
    def step(self, n=1):
        if self._lib.orc_step(self._h, int(n)) != 0:
            raise RuntimeError("step before init_fluid")

    def phase_only(self, kinetics=False):
        self._lib.orc_phase_only(self._h, int(bool(kinetics)))

    # -- read-out -----------------------------------------------------------------------------
    @property
    def t(self):
        return self._lib.orc_time(self._h)

    @property
    def nbodies(self):
        return self._lib.orc_num_bodies(self._h)

    @property
    def lost_refills(self):
        return self._lib.orc_lost_refills(self._h)

    def fields(self):
        rho = np.empty(self.N)
        vel = np.empty(3 * self.N)
        phf = np.empty(self.N)
        self._lib.orc_read_fields(self._h, _vp(rho), _vp(vel), _vp(phf))
        return rho.reshape(self.shape), vel.reshape(self.shape + (3,)), phf.reshape(self.shape)

    def flags(self):
        s = np.empty(self.N, np.uint8)
        o = np.empty(self.N, np.int32)
        self._lib.orc_read_flags(self._h, _vp(s), _vp(o))
        return s.reshape(self.shape), o.reshape(self.shape)

    def phi(self, body):
        out = np.empty(self.N)
        self._lib.orc_read_phi(self._h, int(body), _dp(out))
        return out.reshape(self.shape)

    def velocity_set(self):
        q = self.params["q"]
        c = np.empty(3 * q, np.int32)
        w = np.empty(q)
        self._lib.orc_velocity_set(self._h, c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(w))
        return c.reshape(q, 3), w

    def populations(self):
        out = np.empty(self.params["q"] * self.N)
        self._lib.orc_read_populations(self._h, _dp(out))
        return out.reshape((self.params["q"],) + self.shape)

    def set_populations(self, f):
        a = np.ascontiguousarray(f, np.float64).reshape(-1)
        assert a.size == self.params["q"] * self.N
        self._lib.orc_write_populations(self._h, _dp(a))

    def body_forces(self):
        nb = self.nbodies
        F = np.empty(3 * nb)
        T = np.empty(3 * nb)
        parts = np.empty(18 * nb)
        self._lib.orc_read_body_forces(self._h, _vp(F), _vp(T), _vp(parts))
        return F.reshape(nb, 3), T.reshape(nb, 3), parts.reshape(nb, 3, 6)

    def bodies(self):
        nb = self.nbodies
        X, V, W = (np.empty(3 * nb) for _ in range(3))
        Q = np.empty(4 * nb)
        M = np.empty(nb)
        I = np.empty(9 * nb)
        self._lib.orc_get_bodies(self._h, _vp(X), _vp(V), _vp(W), _vp(Q), _vp(M), _vp(I))
        return dict(X=X.reshape(nb, 3), V=V.reshape(nb, 3), W=W.reshape(nb, 3), Q=Q.reshape(nb, 4),
                    M=M, I=I.reshape(nb, 3, 3))

    def set_body_velocity(self, body, V=None, W=None):
        v = None if V is None else np.asarray(V, np.float64)
        w = None if W is None else np.asarray(W, np.float64)
        self._lib.orc_set_body_velocity(self._h, int(body), _vp(v), _vp(w))

    def set_fixed(self, fixed):
        if len(fixed) != self.nbodies:
            raise ValueError("one flag per body")
        for b, f in enumerate(fixed):
            self._lib.orc_set_body_fixed(self._h, b, 1 if f else 0)

    def integrate_body(self, body, F, T=(0.0, 0.0, 0.0)):
        self._lib.orc_integrate_body(self._h, int(body), _dp(np.asarray(F, np.float64)),
                                     _dp(np.asarray(T, np.float64)))

    def total_mass(self):
        return self._lib.orc_total_mass(self._h)

    def total_momentum(self):
        a = np.empty(3)
        b = np.empty(3)
        self._lib.orc_total_momentum(self._h, _dp(a), _dp(b))
        return a, b


def round_binary16(h):
    """The binary16 rounding of the oracle's storage model (store_prec = 2)."""
    return _load().orc_round_binary16(float(h))
