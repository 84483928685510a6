"""FP64 CPU oracle of the porous lattice Boltzmann model (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA library
and never imports it.  The arithmetic lives in ``vans_oracle.c`` (plain loops in
double precision, one function per step of the method); this module compiles it
with gcc and exposes it through ctypes on numpy arrays.

Conventions (same as the C file): populations ``f`` are ``float64[Q, nz, ny, nx]``
(``nz == 1`` for D2Q9), ``eps`` is ``[nz, ny, nx]``, velocities are
``[D, nz, ny, nx]``.  Directions follow the D2Q9 / D3Q19 ordering of the C file.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

# OpenMP threads sleep instead of spinning when idle, so the oracle degrades
# gracefully when the host cores are shared (set before the runtime loads)
os.environ.setdefault("OMP_WAIT_POLICY", "PASSIVE")

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vans_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libvans_oracle.so")
_lock = threading.Lock()
_lib = None
# The test of the pins (tests/test_oracle_mutants.py) points this module at a
# build of the oracle with one mistake planted in it, in a child process of its
# own; nothing else sets this variable.
_MUTANT = os.environ.get("VANS_ORACLE_MUTANT_LIB")


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/libvans_oracle.so``.

    ``-ffp-contract=off`` keeps gcc from fusing multiply-adds, so the FP64 results
    are the same on x86-64 and aarch64 hosts.
    """
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC",
           "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Params(ctypes.Structure):
    _fields_ = [
        ("q", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("nz", ctypes.c_int), ("wall_mask", ctypes.c_int),
        ("tau", ctypes.c_double), ("g", ctypes.c_double * 3),
        ("drag_mode", ctypes.c_int), ("k_mode", ctypes.c_int),
        ("d_p", ctypes.c_double), ("K", ctypes.c_double), ("F_eps", ctypes.c_double),
        ("u_wall", ctypes.c_double * 3), ("wall_kind", ctypes.c_int),
    ]


@dataclass
class Params:
    """Model and domain parameters (mirrors ``or_params`` in the C file)."""
    q: int = 9
    nx: int = 1
    ny: int = 1
    nz: int = 1
    wall_mask: int = 0
    tau: float = 0.8
    g: tuple = (0.0, 0.0, 0.0)
    drag_mode: int = 0
    k_mode: int = 0
    d_p: float = 1.0
    K: float = 1.0
    F_eps: float = 0.0
    u_wall: tuple = (0.0, 0.0, 0.0)
    wall_kind: int = 0

    def _c(self) -> _Params:
        g = tuple(float(v) for v in self.g) + (0.0,) * (3 - len(self.g))
        uw = tuple(float(v) for v in self.u_wall) + (0.0,) * (3 - len(self.u_wall))
        return _Params(int(self.q), int(self.nx), int(self.ny), int(self.nz),
                       int(self.wall_mask), float(self.tau), (ctypes.c_double * 3)(*g),
                       int(self.drag_mode), int(self.k_mode), float(self.d_p),
                       float(self.K), float(self.F_eps), (ctypes.c_double * 3)(*uw),
                       int(self.wall_kind))

    @property
    def dim(self) -> int:
        return 2 if self.q == 9 else 3

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(_MUTANT if _MUTANT else build())
        P = ctypes.POINTER(_Params)
        d = ctypes.POINTER(ctypes.c_double)
        i = ctypes.POINTER(ctypes.c_int)
        sig = {
            "or_lattice": (ctypes.c_int, [ctypes.c_int, i, d, i]),
            "or_feq": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_double, d, d]),
            "or_source": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, d, d, d]),
            "or_velocity": (None, [ctypes.c_double, d, ctypes.c_double, ctypes.c_double, d]),
            "or_drag_coeffs": (ctypes.c_int, [P, ctypes.c_double, d, d]),
            "or_grad_eps": (ctypes.c_int, [P, d, d]),
            "or_init": (ctypes.c_int, [P, d, d]),
            "or_moments": (ctypes.c_int, [P, d, d, d, d]),
            "or_collide": (ctypes.c_int, [P, d, d]),
            "or_stream": (ctypes.c_int, [P, d, d, d]),
            "or_run": (ctypes.c_int, [P, d, d, ctypes.c_int]),
            "or_flux": (ctypes.c_int, [P, d, d, ctypes.c_int, d]),
            "or_adjoint": (ctypes.c_int, [P, d, ctypes.c_int, ctypes.c_int, d, d]),
            "or_num_threads": (ctypes.c_int, []),
            "or_set_num_threads": (None, [ctypes.c_int]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"oracle {what} failed (status {rc})")


def lattice(q: int):
    """Velocity set ``e[q,3]`` (int), weights ``w[q]`` and opposite table ``opp[q]``."""
    lib = _load()
    e = np.zeros((q, 3), dtype=np.int32)
    w = np.zeros(q)
    opp = np.zeros(q, dtype=np.int32)
    ip = ctypes.POINTER(ctypes.c_int)
    _check(lib.or_lattice(q, e.ctypes.data_as(ip), _dp(w), opp.ctypes.data_as(ip)), "lattice")
    return e, w, opp


def feq(q: int, eps: float, rho: float, u) -> np.ndarray:
    """Eq. d2q9eq for one cell."""
    lib = _load()
    uu = _f64(list(u) + [0.0] * (3 - len(u)))
    out = np.zeros(q)
    _check(lib.or_feq(q, eps, rho, _dp(uu), _dp(out)), "feq")
    return out


def source(q: int, tau: float, u, V) -> np.ndarray:
    """Eq. pi / Eq. Fi: the source term for the vector V (p grad eps or F)."""
    lib = _load()
    uu = _f64(list(u) + [0.0] * (3 - len(u)))
    vv = _f64(list(V) + [0.0] * (3 - len(V)))
    out = np.zeros(q)
    _check(lib.or_source(q, tau, _dp(uu), _dp(vv), _dp(out)), "source")
    return out


def velocity(R: float, m, alpha: float, beta: float) -> np.ndarray:
    """Closed-form solution u of (R + alpha/2 + beta/2 |u|) u = m."""
    lib = _load()
    mm = _f64(list(m) + [0.0] * (3 - len(m)))
    out = np.zeros(3)
    lib.or_velocity(R, _dp(mm), alpha, beta, _dp(out))
    return out


def drag_coeffs(p: Params, eps: float):
    """(alpha, beta): F_drag = -alpha u - beta |u| u for porosity eps."""
    lib = _load()
    a = ctypes.c_double()
    b = ctypes.c_double()
    pc = p._c()
    _check(lib.or_drag_coeffs(ctypes.byref(pc), eps, ctypes.byref(a), ctypes.byref(b)), "drag")
    return a.value, b.value


def _eps(p: Params, eps) -> np.ndarray:
    e = _f64(eps).reshape(p.shape)
    return np.ascontiguousarray(e)


def grad_eps(p: Params, eps) -> np.ndarray:
    lib = _load()
    e = _eps(p, eps)
    out = np.zeros((3,) + p.shape)
    _check(lib.or_grad_eps(ctypes.byref(p._c()), _dp(e), _dp(out)), "grad_eps")
    return out[: p.dim]


def init(p: Params, eps) -> np.ndarray:
    """f(x, 0) = w_i eps(x) (rho = 1, u = 0)."""
    lib = _load()
    e = _eps(p, eps)
    f = np.zeros((p.q,) + p.shape)
    _check(lib.or_init(ctypes.byref(p._c()), _dp(e), _dp(f)), "init")
    return f


def moments(p: Params, eps, f):
    """(rho[nz,ny,nx], u[D,nz,ny,nx]) of the state f."""
    lib = _load()
    e = _eps(p, eps)
    ff = _f64(f).reshape((p.q,) + p.shape)
    rho = np.zeros(p.shape)
    u = np.zeros((p.dim,) + p.shape)
    _check(lib.or_moments(ctypes.byref(p._c()), _dp(e), _dp(ff), _dp(rho), _dp(u)), "moments")
    return rho, u


def collide(p: Params, eps, f) -> np.ndarray:
    lib = _load()
    e = _eps(p, eps)
    ff = _f64(f).reshape((p.q,) + p.shape).copy()
    _check(lib.or_collide(ctypes.byref(p._c()), _dp(e), _dp(ff)), "collide")
    return ff


def stream(p: Params, eps, fstar) -> np.ndarray:
    lib = _load()
    e = _eps(p, eps)
    fs = _f64(fstar).reshape((p.q,) + p.shape)
    out = np.zeros_like(fs)
    _check(lib.or_stream(ctypes.byref(p._c()), _dp(e), _dp(fs), _dp(out)), "stream")
    return out


def run(p: Params, eps, f, nsteps: int) -> np.ndarray:
    """Advance f(x,t) by nsteps of the final LBE; returns a new array."""
    lib = _load()
    e = _eps(p, eps)
    ff = _f64(f).reshape((p.q,) + p.shape).copy()
    _check(lib.or_run(ctypes.byref(p._c()), _dp(e), _dp(ff), int(nsteps)), "run")
    return ff


def flux(p: Params, eps, f, x_out: int) -> float:
    """J = sum over the plane x = x_out of eps*rho*u_x."""
    lib = _load()
    e = _eps(p, eps)
    ff = _f64(f).reshape((p.q,) + p.shape)
    J = ctypes.c_double()
    _check(lib.or_flux(ctypes.byref(p._c()), _dp(e), _dp(ff), int(x_out), ctypes.byref(J)), "flux")
    return J.value


def adjoint(p: Params, eps, nsteps: int, x_out: int):
    """(J, dJ/deps) for J = flux(f(nsteps)) from f(0) = w eps (discrete adjoint)."""
    lib = _load()
    e = _eps(p, eps)
    out = np.zeros(p.shape)
    J = ctypes.c_double()
    _check(lib.or_adjoint(ctypes.byref(p._c()), _dp(e), int(nsteps), int(x_out), _dp(out),
                          ctypes.byref(J)), "adjoint")
    return J.value, out


def num_threads() -> int:
    return int(_load().or_num_threads())


def set_num_threads(n: int) -> None:
    _load().or_set_num_threads(int(n))
