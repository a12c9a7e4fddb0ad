"""Thin ctypes binding of the C ABI in include/cbl.h (argument marshalling only).

Every step of the method runs in the CUDA library ``_lib/libcbl.so``; this module only converts
arguments. Device memory comes from PyTorch's caching allocator through the ``cbl_allocator``
callbacks, and work runs on a PyTorch stream. If the library has not been built the import of
the library fails loudly: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libcbl.so")

CBL_FP64, CBL_FP32, CBL_FP16DEV = 0, 1, 2
PRECISIONS = {"fp64": CBL_FP64, "fp32": CBL_FP32, "fp16dev": CBL_FP16DEV}
STATUS = {0: "CBL_OK", 1: "CBL_ERR_ARG", 2: "CBL_ERR_STATE", 3: "CBL_ERR_OOM", 4: "CBL_ERR_CUDA",
          5: "CBL_ERR_TIMEOUT", 6: "CBL_ERR_UNSTABLE", 7: "CBL_ERR_UNSUPPORTED"}


class cbl_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("q", ctypes.c_int),
        ("tau", ctypes.c_double), ("G", ctypes.c_double), ("rho0", ctypes.c_double),
        ("ext_force", ctypes.c_double * 3),
        ("prec", ctypes.c_int),
        ("mpf_kinetics", ctypes.c_int),
        ("mobility", ctypes.c_double), ("eta", ctypes.c_double),
        ("sigma_sf", ctypes.c_double), ("sigma_ss", ctypes.c_double),
        ("e0", ctypes.c_double), ("rc", ctypes.c_double),
        ("nrep", ctypes.c_int),
        ("solid_threshold", ctypes.c_double), ("member_threshold", ctypes.c_double),
        ("stream", ctypes.c_void_p),
    ]


class cbl_body(ctypes.Structure):
    _fields_ = [
        ("shape", ctypes.c_int),
        ("center", ctypes.c_double * 3),
        ("radius", ctypes.c_double),
        ("half", ctypes.c_double * 3),
        ("quat", ctypes.c_double * 4),
        ("mass_density", ctypes.c_double),
        ("wetting_rho", ctypes.c_double),
        ("fixed", ctypes.c_int),
    ]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class cbl_allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", ctypes.c_void_p)]


# name -> (restype, argtypes); the names are those of include/cbl.h
_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
SIGNATURES = {
    "cbl_create": (ctypes.c_int, [ctypes.POINTER(cbl_params), ctypes.POINTER(cbl_allocator), ctypes.POINTER(_P)]),
    "cbl_add_body": (ctypes.c_int, [_P, ctypes.POINTER(cbl_body), ctypes.POINTER(ctypes.c_int)]),
    "cbl_init_fluid": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_double, _P]),
    "cbl_init_fluid_fields": (ctypes.c_int, [_P, _P, _P]),
    "cbl_step": (ctypes.c_int, [_P, ctypes.c_int]),
    "cbl_read_fields": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int]),
    "cbl_read_populations": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "cbl_velocity_set": (ctypes.c_int, [_P, _P, _P, _P]),
    "cbl_read_flags": (ctypes.c_int, [_P, _P, _P]),
    "cbl_read_phi": (ctypes.c_int, [_P, ctypes.c_int, _P]),
    "cbl_read_body_forces": (ctypes.c_int, [_P, _P, _P, _P]),
    "cbl_get_bodies": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P]),
    "cbl_read_force_mean": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(ctypes.c_longlong), ctypes.c_int]),
    "cbl_set_body_velocities": (ctypes.c_int, [_P, _P, _P]),
    "cbl_set_bodies_fixed": (ctypes.c_int, [_P, _P]),
    "cbl_save": (ctypes.c_int, [_P, ctypes.c_char_p]),
    "cbl_load": (ctypes.c_int, [_P, ctypes.c_char_p]),
    "cbl_move_bodies": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "cbl_total_mass": (ctypes.c_int, [_P, _D]),
    "cbl_info": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int64),
                                ctypes.POINTER(ctypes.c_int)]),
    "cbl_time_phases": (ctypes.c_int, [_P, ctypes.c_int, _D]),
    "cbl_kernel_times": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_int)]),
    "cbl_set_option": (ctypes.c_int, [_P, ctypes.c_char_p, ctypes.c_double]),
    "cbl_get_option": (ctypes.c_int, [_P, ctypes.c_char_p, ctypes.POINTER(ctypes.c_double)]),
    "cbl_lbm_step_noalloc": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                            ctypes.c_double, ctypes.c_double, _P, _P, _P]),
    "cbl_batch_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, _P, ctypes.POINTER(_P)]),
    "cbl_batch_step": (ctypes.c_int, [_P, ctypes.c_int]),
    "cbl_batch_sync": (ctypes.c_int, [_P]),
    "cbl_batch_destroy": (ctypes.c_int, [_P]),
    "cbl_batch_set_option": (ctypes.c_int, [_P, ctypes.c_char_p, ctypes.c_double]),
    "cbl_batch_info": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_int)]),
    "cbl_mlp_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P,
                                      ctypes.POINTER(_P)]),
    "cbl_mlp_num_params": (ctypes.c_int64, [_P]),
    "cbl_mlp_set_params": (ctypes.c_int, [_P, _P]),
    "cbl_mlp_get_params": (ctypes.c_int, [_P, _P]),
    "cbl_mlp_forward": (ctypes.c_int, [_P, _P, _P, ctypes.c_int]),
    "cbl_mlp_grad": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.POINTER(ctypes.c_float)]),
    "cbl_mlp_read_grad": (ctypes.c_int, [_P, _P]),
    "cbl_mlp_zero_grad": (ctypes.c_int, [_P]),
    "cbl_mlp_adam_step": (ctypes.c_int, [_P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float]),
    "cbl_mlp_sync": (ctypes.c_int, [_P]),
    "cbl_mlp_advance": (ctypes.c_int, [_P] + [_P] * 10 + [ctypes.c_int, ctypes.c_int, ctypes.c_int, _P,
                                                          ctypes.c_double, _P, ctypes.c_double]),
    "cbl_mlp_destroy": (ctypes.c_int, [_P]),
    "cbl_destroy": (ctypes.c_int, [_P]),
    "cbl_last_error": (ctypes.c_char_p, [_P]),
}

_lib = None


def load():
    """Load the CUDA library; raises if it has not been built (no CPU fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("CUDA library %s is missing: run __graft_entry__.build()" % LIB_PATH)
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class CblError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


def _vp(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def torch_allocator(device=None, stream=None):
    """cbl_allocator backed by PyTorch's caching allocator. Keep the returned object alive."""
    import torch

    dev = torch.cuda.current_device() if device is None else device

    def _alloc(nbytes, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), device=dev, stream=stream)
        except Exception:  # OOM -> NULL, reported by the library as CBL_ERR_OOM
            return None

    def _free(ptr, user):
        torch.cuda.caching_allocator_delete(ptr)

    a = cbl_allocator(ALLOC_FN(_alloc), FREE_FN(_free), None)
    a._keep = (_alloc, _free)
    return a


class Sim:
    """One simulation on the GPU through the C ABI. Arrays are numpy; cell index x + nx*(y + ny*z)."""

    DEFAULTS = dict(q=19, tau=1.0, G=-5.0, rho0=1.0, ext_force=(0.0, 0.0, 0.0), prec="fp32",
                    mpf_kinetics=0, mobility=1e-5, eta=5.0, sigma_sf=3.583e-2, sigma_ss=0.5 * 3.583e-2,
                    e0=1e-3, rc=3.0, nrep=4, solid_threshold=0.05, member_threshold=0.5)

    def __init__(self, nx, ny, nz, use_torch=True, **kw):
        self._lib = load()
        cfg = dict(self.DEFAULTS)
        unknown = set(kw) - set(cfg)
        if unknown:
            raise TypeError("unknown parameters: %s" % sorted(unknown))
        cfg.update(kw)
        p = cbl_params()
        p.nx, p.ny, p.nz = nx, ny, nz
        for k, v in cfg.items():
            if k == "ext_force":
                p.ext_force[:] = list(v)
            elif k == "prec":
                p.prec = PRECISIONS[v] if isinstance(v, str) else int(v)
            else:
                setattr(p, k, v)
        self._alloc = None
        self._stream = None
        if use_torch:
            import torch

            # a stream of its own: the legacy default stream cannot be captured into a graph
            self._stream = torch.cuda.Stream()
            p.stream = ctypes.c_void_p(self._stream.cuda_stream)
            self._alloc = torch_allocator(stream=self._stream)
        self.params = cfg
        self.q = int(cfg["q"])
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz
        h = ctypes.c_void_p()
        st = self._lib.cbl_create(ctypes.byref(p), ctypes.byref(self._alloc) if self._alloc else None,
                                  ctypes.byref(h))
        if st != 0:
            raise CblError(st, self._lib.cbl_last_error(None).decode())
        self._h = h
        self.nb = 0

    def _ck(self, st):
        if st != 0:
            raise CblError(st, self._lib.cbl_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.cbl_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_body(self, shape, center, radius=0.0, half=(0.0, 0.0, 0.0), quat=(1.0, 0.0, 0.0, 0.0),
                 mass_density=4.0, wetting_rho=2.0, fixed=False):
        b = cbl_body()
        b.shape = {"sphere": 0, "box": 1}[shape] if isinstance(shape, str) else int(shape)
        b.center[:] = [float(v) for v in center]
        b.radius = float(radius)
        b.half[:] = [float(v) for v in half]
        b.quat[:] = [float(v) for v in quat]
        b.mass_density = float(mass_density)
        b.wetting_rho = float(wetting_rho)
        b.fixed = int(bool(fixed))
        bid = ctypes.c_int()
        self._ck(self._lib.cbl_add_body(self._h, ctypes.byref(b), ctypes.byref(bid)))
        self.nb += 1
        return bid.value

    def init_fluid(self, rho_l, rho_v, mask=None):
        m = None if mask is None else np.ascontiguousarray(mask, np.uint8).reshape(-1)
        self._ck(self._lib.cbl_init_fluid(self._h, float(rho_l), float(rho_v), _vp(m)))

    def init_fluid_fields(self, rho, u=None):
        r = np.ascontiguousarray(rho, np.float64).reshape(-1)
        uu = None if u is None else np.ascontiguousarray(u, np.float64).reshape(-1)
        self._ck(self._lib.cbl_init_fluid_fields(self._h, _vp(r), _vp(uu)))

    def step(self, n=1):
        self._ck(self._lib.cbl_step(self._h, int(n)))

    def fields(self, out=None):
        """Density, velocity and fluid phase field of the last step, float64 numpy arrays. out: three
        float64 C-contiguous host arrays of N, 3N and N values to read into (e.g. views of pinned
        memory, which the copies use directly); new arrays otherwise."""
        if out is None:
            rho, vel, phf = np.empty(self.N), np.empty(3 * self.N), np.empty(self.N)
        else:
            rho, vel, phf = out
            for a, n in ((rho, self.N), (vel, 3 * self.N), (phf, self.N)):
                if a.dtype != np.float64 or a.size != n or not a.flags["C_CONTIGUOUS"]:
                    raise ValueError("out: float64 C-contiguous arrays of N, 3N and N values")
        self._ck(self._lib.cbl_read_fields(self._h, _vp(rho), _vp(vel), _vp(phf), 0))
        return rho.reshape(self.shape), vel.reshape(self.shape + (3,)), phf.reshape(self.shape)

    def fields_device(self, rho, vel=None, phi_fluid=None):
        """Read into device tensors (torch, float64, contiguous)."""
        ptr = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())
        self._ck(self._lib.cbl_read_fields(self._h, ptr(rho), ptr(vel), ptr(phi_fluid), 1))

    def velocity_set(self):
        """Directions c (q x 3 ints) and weights w (q) in the order of populations()."""
        q = ctypes.c_int()
        c = np.empty(3 * self.q, np.int32)
        w = np.empty(self.q)
        self._ck(self._lib.cbl_velocity_set(self._h, ctypes.byref(q), _vp(c), _vp(w)))
        return c.reshape(self.q, 3), w

    def populations(self):
        """Current post-collision populations, float64 [q][nz][ny][nx] in the library's order
        (velocity_set() gives the directions and weights)."""
        out = np.empty(self.q * self.N)
        self._ck(self._lib.cbl_read_populations(self._h, _vp(out), 0))
        return out.reshape((self.q,) + self.shape)

    def flags(self):
        s = np.empty(self.N, np.uint8)
        o = np.empty(self.N, np.int32)
        self._ck(self._lib.cbl_read_flags(self._h, _vp(s), _vp(o)))
        return s.reshape(self.shape), o.reshape(self.shape)

    def phi(self, body):
        out = np.empty(self.N)
        self._ck(self._lib.cbl_read_phi(self._h, int(body), _vp(out)))
        return out.reshape(self.shape)

    def body_forces(self):
        nb = self.nb
        F = np.empty(3 * nb)
        T = np.empty(3 * nb)
        parts = np.empty(18 * nb)
        self._ck(self._lib.cbl_read_body_forces(self._h, _vp(F), _vp(T), _vp(parts)))
        return F.reshape(nb, 3), T.reshape(nb, 3), parts.reshape(nb, 3, 6)

    def force_mean(self, reset=True):
        """Mean total force and torque per body over the steps since the last reset (device-side sums),
        and that number of steps; reset starts the sums anew."""
        nb = self.nb
        F = np.empty(3 * nb)
        T = np.empty(3 * nb)
        n = ctypes.c_longlong()
        self._ck(self._lib.cbl_read_force_mean(self._h, _vp(F), _vp(T), ctypes.byref(n), int(bool(reset))))
        return F.reshape(nb, 3), T.reshape(nb, 3), n.value

    def bodies(self):
        nb = self.nb
        X, V, W = (np.empty(3 * nb) for _ in range(3))
        Q = np.empty(4 * nb)
        M = np.empty(nb)
        I = np.empty(9 * nb)
        self._ck(self._lib.cbl_get_bodies(self._h, _vp(X), _vp(V), _vp(W), _vp(Q), _vp(M), _vp(I)))
        return dict(X=X.reshape(nb, 3), V=V.reshape(nb, 3), W=W.reshape(nb, 3), Q=Q.reshape(nb, 4), M=M,
                    I=I.reshape(nb, 3, 3))

    def set_body_velocities(self, V=None, W=None):
        v = None if V is None else np.ascontiguousarray(V, np.float64).reshape(-1)
        w = None if W is None else np.ascontiguousarray(W, np.float64).reshape(-1)
        self._ck(self._lib.cbl_set_body_velocities(self._h, _vp(v), _vp(w)))

    def save(self, path):
        self._ck(self._lib.cbl_save(self._h, os.fsencode(path)))

    def load(self, path):
        """Restore a checkpoint instead of init_fluid (same parameters and bodies as the saved run)."""
        self._ck(self._lib.cbl_load(self._h, os.fsencode(path)))

    def set_fixed(self, fixed):
        f = np.ascontiguousarray([1 if v else 0 for v in fixed], np.int32)
        if f.size != self.nb:
            raise ValueError("one flag per body")
        self._ck(self._lib.cbl_set_bodies_fixed(self._h, _vp(f)))

    def move_bodies(self, X, Q=None, V=None, W=None):
        f = lambda a: None if a is None else np.ascontiguousarray(a, np.float64).reshape(-1)
        X, Q, V, W = f(X), f(Q), f(V), f(W)
        self._ck(self._lib.cbl_move_bodies(self._h, _vp(X), _vp(Q), _vp(V), _vp(W)))

    def total_mass(self):
        m = ctypes.c_double()
        self._ck(self._lib.cbl_total_mass(self._h, ctypes.byref(m)))
        return m.value

    PHASES = ("density", "collide", "boundary", "repulsion", "bodies", "advect", "kinetics", "flags", "refill")

    def time_phases(self, n):
        """Mean per-step duration (ms) of each kernel phase over n steps, CUDA events on the stream."""
        ms = (ctypes.c_double * len(self.PHASES))()
        self._ck(self._lib.cbl_time_phases(self._h, int(n), ms))
        return dict(zip(self.PHASES, list(ms)))

    def kernel_times(self, max_n=512):
        """Durations (ms) of the bulk collision in the replays of the last step() call, measured by
        event nodes inside the step graph (needs set_option("kernel_events", 1) before stepping)."""
        buf = (ctypes.c_float * max_n)()
        n = ctypes.c_int()
        self._ck(self._lib.cbl_kernel_times(self._h, int(max_n), buf, ctypes.byref(n)))
        return list(buf[:n.value])

    def set_option(self, key, value):
        self._ck(self._lib.cbl_set_option(self._h, key.encode(), float(value)))

    def get_option(self, key):
        v = ctypes.c_double()
        self._ck(self._lib.cbl_get_option(self._h, key.encode(), ctypes.byref(v)))
        return v.value

    @property
    def stream(self):
        return self._stream

    def info(self):
        nb = ctypes.c_int()
        nc = ctypes.c_int64()
        err = ctypes.c_int()
        self._ck(self._lib.cbl_info(self._h, ctypes.byref(nb), ctypes.byref(nc), ctypes.byref(err)))
        return dict(nbodies=nb.value, ncells=nc.value, device_error=err.value)


class Batch:
    """Independent simulations advanced together: one CUDA graph holds one step of every instance, the
    bulk lattice-Boltzmann pass of all instances in one persistent launch (cbl_batch_* in
    include/cbl.h). The simulations must outlive the batch."""

    def __init__(self, sims, stream=None):
        self._lib = load()
        self.sims = list(sims)
        arr = (_P * len(self.sims))(*[s._h.value for s in self.sims])
        h = _P()
        st = self._lib.cbl_batch_create(arr, len(self.sims),
                                        None if stream is None else _P(stream.cuda_stream), ctypes.byref(h))
        if st != 0:
            raise CblError(st, self._lib.cbl_last_error(None).decode())
        self._h = h

    def step(self, n=1):
        st = self._lib.cbl_batch_step(self._h, int(n))
        if st != 0:
            raise CblError(st, self._lib.cbl_last_error(None).decode())

    def sync(self):
        st = self._lib.cbl_batch_sync(self._h)
        if st != 0:
            raise CblError(st, self._lib.cbl_last_error(None).decode())

    def set_option(self, key, value):
        st = self._lib.cbl_batch_set_option(self._h, key.encode(), float(value))
        if st != 0:
            raise CblError(st, self._lib.cbl_last_error(None).decode())

    def info(self):
        m, t, g = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        it = ctypes.c_longlong()
        st = self._lib.cbl_batch_info(self._h, ctypes.byref(m), ctypes.byref(t), ctypes.byref(it), ctypes.byref(g))
        if st != 0:
            raise CblError(st, self._lib.cbl_last_error(None).decode())
        return dict(mode=m.value, tile=t.value, items=it.value, grid=g.value)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.cbl_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MLP:
    """Force surrogate network on the GPU (cbl_mlp_* in include/cbl.h): 4 -> 64 -> 64 -> 64 -> 6, tanh,
    bfloat16 weights with FP32 accumulation, FP32 master weights updated by Adam. Tensors are torch
    CUDA float32, [sample][feature]."""

    def __init__(self, stream=None):
        import torch

        self._lib = load()
        self._stream = stream if stream is not None else torch.cuda.Stream()
        h = _P()
        st = self._lib.cbl_mlp_create(4, 64, 3, 6, _P(self._stream.cuda_stream), ctypes.byref(h))
        if st != 0:
            raise CblError(st, "cbl_mlp_create")
        self._h = h
        self.n_params = int(self._lib.cbl_mlp_num_params(h))

    def _ck(self, st, what):
        if st != 0:
            raise CblError(st, what)

    def set_params(self, p):
        a = np.ascontiguousarray(p, np.float32)
        assert a.size == self.n_params
        self._ck(self._lib.cbl_mlp_set_params(self._h, _vp(a)), "set_params")

    def params(self):
        a = np.empty(self.n_params, np.float32)
        self._ck(self._lib.cbl_mlp_get_params(self._h, _vp(a)), "get_params")
        return a

    def forward(self, x, y=None):
        import torch

        n = x.shape[0]
        if y is None:
            y = torch.empty((n, 6), dtype=torch.float32, device=x.device)
        # inputs written on the caller's stream must be complete; the result is complete on return
        torch.cuda.current_stream().synchronize()
        self._ck(self._lib.cbl_mlp_forward(self._h, _P(x.data_ptr()), _P(y.data_ptr()), n), "forward")
        self._lib.cbl_mlp_sync(self._h)
        return y

    def grad(self, x, t, want_loss=True):
        import torch

        torch.cuda.current_stream().synchronize()
        loss = ctypes.c_float()
        self._ck(self._lib.cbl_mlp_grad(self._h, _P(x.data_ptr()), _P(t.data_ptr()), x.shape[0],
                                        ctypes.byref(loss) if want_loss else None), "grad")
        return loss.value if want_loss else None

    def read_grad(self):
        a = np.empty(self.n_params, np.float32)
        self._ck(self._lib.cbl_mlp_read_grad(self._h, _vp(a)), "read_grad")
        return a

    def zero_grad(self):
        self._ck(self._lib.cbl_mlp_zero_grad(self._h), "zero_grad")

    def adam_step(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self._ck(self._lib.cbl_mlp_adam_step(self._h, lr, beta1, beta2, eps), "adam_step")

    def sync(self):
        self._lib.cbl_mlp_sync(self._h)

    def advance(self, X, V, W, M, Iinv, R, fixed, bias, pairs, VL, steps, dims, cos_theta, norm, sigma):
        """Bodies advanced `steps` steps under the network's pair forces on the device (cbl_mlp_advance):
        X, V, W (nb x 3 float64), M, Iinv, R (nb float64), fixed (nb int32), bias (nb x 3 float64), pairs
        (npairs x 2 int32), VL (npairs float64) are CUDA tensors on the network's device; X, V, W are
        updated in place. dims (3 ints) and norm (28 floats) are host sequences."""
        import torch

        torch.cuda.current_stream().synchronize()
        ptr = lambda t: _P(t.data_ptr()) if t is not None and t.numel() else None
        d = (ctypes.c_int * 3)(*[int(v) for v in dims])
        nm = (ctypes.c_float * 28)(*[float(v) for v in norm])
        self._ck(self._lib.cbl_mlp_advance(self._h, ptr(X), ptr(V), ptr(W), ptr(M), ptr(Iinv), ptr(R), ptr(fixed),
                                           ptr(bias), ptr(pairs), ptr(VL), int(X.shape[0]), int(pairs.shape[0]),
                                           int(steps), d, float(cos_theta), nm, float(sigma)), "advance")
        self._lib.cbl_mlp_sync(self._h)

    @property
    def stream(self):
        return self._stream

    def close(self):
        if getattr(self, "_h", None):
            self._lib.cbl_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


NOALLOC_MAX_CELLS = 1 << 20


def _check_noalloc_args(f_in, f_out, nx, ny, nz, mass_out):
    """The C entry point cannot see buffer sizes or devices, so a wrong buffer would be a memory fault
    on the GPU: every property it relies on is checked here, before the call (ValueError)."""
    import torch

    n = 19 * int(nx) * int(ny) * int(nz)
    for name, t in (("f_in", f_in), ("f_out", f_out)):
        if not isinstance(t, torch.Tensor):
            raise ValueError("%s must be a torch tensor" % name)
        if t.dtype != torch.float32:
            raise ValueError("%s must be float32, got %s" % (name, t.dtype))
        if not t.is_contiguous():
            raise ValueError("%s must be contiguous" % name)
        if t.numel() < n:
            raise ValueError("%s holds %d floats, the lattice needs 19*nx*ny*nz = %d" % (name, t.numel(), n))
    a0, a1 = f_in.data_ptr(), f_in.data_ptr() + 4 * n
    b0, b1 = f_out.data_ptr(), f_out.data_ptr() + 4 * n
    if a0 < b1 and b0 < a1:
        raise ValueError("f_in and f_out overlap")
    if mass_out is not None:
        if not isinstance(mass_out, torch.Tensor) or mass_out.dtype != torch.float64 or mass_out.numel() < 1:
            raise ValueError("mass_out must be a float64 tensor with at least one element")
    dev = None
    for name, t in (("f_in", f_in), ("f_out", f_out), ("mass_out", mass_out)):
        if t is None:
            continue
        if not t.is_cuda:
            raise ValueError("%s must be a CUDA tensor" % name)
        if dev is None:
            dev = torch.cuda.current_device()
        if t.device.index != dev:
            raise ValueError("%s is on cuda:%d, the current device is cuda:%d" % (name, t.device.index, dev))


def lbm_step_noalloc(f_in, f_out, nx, ny, nz, tau=1.0, G=-5.0, rho0=1.0, ext_force=None, mass_out=None,
                     stream=None):
    """One fluid-only LBM step on caller-owned device tensors (float32, 19*nx*ny*nz each, on the current
    device, not overlapping) with no device allocation inside the library (cbl_lbm_step_noalloc in
    include/cbl.h). mass_out: optional float64 CUDA tensor. The work is enqueued on `stream`
    (a torch.cuda.Stream), by default on torch's current stream, so it is ordered with the caller's
    other work on that stream. Arguments the library cannot check are checked here (ValueError)."""
    import torch

    _check_noalloc_args(f_in, f_out, nx, ny, nz, mass_out)
    lib = load()
    ext = None
    if ext_force is not None:
        ext = (ctypes.c_double * 3)(*ext_force)
    s = (stream if stream is not None else torch.cuda.current_stream()).cuda_stream
    st = lib.cbl_lbm_step_noalloc(ctypes.c_void_p(f_in.data_ptr()), ctypes.c_void_p(f_out.data_ptr()), nx, ny, nz,
                                  float(tau), float(G), float(rho0), ext,
                                  None if mass_out is None else ctypes.c_void_p(mass_out.data_ptr()),
                                  ctypes.c_void_p(s))
    if st != 0:
        raise CblError(st, "cbl_lbm_step_noalloc")
