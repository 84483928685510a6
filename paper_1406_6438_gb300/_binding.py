"""Thin ctypes binding of libvans.so (include/vans.h).

Argument marshalling only: every step of the method runs in the library's CUDA
kernels.  PyTorch supplies device memory (the caller-owned workspace and
buffers) and the stream.  There is no CPU fallback: if the library cannot be
loaded, or no CUDA device is present, the classes below raise.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import asdict, dataclass

from . import build as _build

VANS_OK = 0
STATUS = {
    0: "VANS_OK", -1: "VANS_ERR_ARG", -2: "VANS_ERR_CUDA", -3: "VANS_ERR_DIVERGED",
    -4: "VANS_ERR_TIMEOUT", -5: "VANS_ERR_UNSUPPORTED", -6: "VANS_ERR_STATE",
}


class VansError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {STATUS.get(status, status)}")


class _CParams(ctypes.Structure):
    _fields_ = [
        ("q", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("wall_mask", ctypes.c_int), ("tau", ctypes.c_float), ("g", ctypes.c_float * 3),
        ("drag_mode", ctypes.c_int), ("k_mode", ctypes.c_int), ("d_p", ctypes.c_float),
        ("K", ctypes.c_float), ("F_eps", ctypes.c_float), ("u_wall", ctypes.c_float * 3),
        ("wall_kind", ctypes.c_int),
    ]


class _CLaunch(ctypes.Structure):
    _fields_ = [("cpt", ctypes.c_int), ("warps", ctypes.c_int), ("rows", ctypes.c_int),
                ("kind", ctypes.c_int), ("ctas", ctypes.c_int)]


@dataclass
class Params:
    """Fields of ``vans_params`` (see include/vans.h)."""
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

    @classmethod
    def of(cls, p) -> "Params":
        return p if isinstance(p, Params) else cls(**p)

    def c(self) -> _CParams:
        g = tuple(float(v) for v in self.g) + (0.0,) * (3 - len(self.g))
        uw = tuple(float(v) for v in self.u_wall) + (0.0,) * (3 - len(self.u_wall))
        return _CParams(int(self.q), int(self.nx), int(self.ny), int(self.nz), int(self.wall_mask),
                        float(self.tau), (ctypes.c_float * 3)(*g), int(self.drag_mode),
                        int(self.k_mode), float(self.d_p), float(self.K), float(self.F_eps),
                        (ctypes.c_float * 3)(*uw), int(self.wall_kind))

    @property
    def dim(self) -> int:
        return 2 if self.q == 9 else 3

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    def as_dict(self) -> dict:
        return asdict(self)


@dataclass
class Launch:
    """``vans_launch`` (see include/vans.h).  kind 0: register-load kernel (cpt
    cells per lane, warps x rows per block); kind 2: bulk-copy pipeline over
    row strips with a porosity ring (32*warps threads, cpt cells per thread per
    tile, rows = pipeline stages); kinds 4, 5: kind 2 with a producer warp and
    per-warp stage release (5: consecutive cells per thread); kinds 6, 7:
    persistent CTAs over interleaved row tiles; kind 8: every step of a call
    in one launch of one thread-block cluster holding the state in shared
    memory (rows = the largest cluster, warps 8 or 16, cpt 1).  Kinds 1 and 3
    are not built.  ctas: at most that many CTAs per SM for the pipelined
    kinds (0: as many as fit)."""
    cpt: int
    warps: int
    rows: int
    kind: int = 0
    ctas: int = 0


_lib = None
_lock = threading.Lock()

_P = ctypes.POINTER(_CParams)
_LP = ctypes.POINTER(_CLaunch)
_H = ctypes.c_void_p
_F = ctypes.c_void_p   # device pointers travel as integers


def load_library(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libvans.so, building it first if needed (nvcc required)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"libvans.so not built ({_build.LIB}); run __graft_entry__.build()")
        lib = ctypes.CDLL(_build.LIB)
        sig = {
            "vans_state_floats": (ctypes.c_longlong, [_P]),
            "vans_workspace_bytes": (ctypes.c_size_t, [_P]),
            "vans_create": (ctypes.c_int, [_P, _F, ctypes.c_size_t, ctypes.c_void_p,
                                           ctypes.POINTER(_H)]),
            "vans_destroy": (None, [_H]),
            "vans_set_eps": (ctypes.c_int, [_H, _F]),
            "vans_set_eps_async": (ctypes.c_int, [_H, _F]),
            "vans_update_eps": (ctypes.c_int, [_H, _F]),
            "vans_step": (ctypes.c_int, [_H, ctypes.c_int]),
            "vans_step_raw": (ctypes.c_int, [_H, _F, _F]),
            "vans_step_monitored": (ctypes.c_int, [_H, ctypes.c_int, ctypes.c_int, _F, _F, _F]),
            "vans_moments": (ctypes.c_int, [_H, _F, _F]),
            "vans_get_populations": (ctypes.c_int, [_H, _F]),
            "vans_set_populations": (ctypes.c_int, [_H, _F]),
            "vans_get_state": (ctypes.c_int, [_H, _F]),
            "vans_set_state": (ctypes.c_int, [_H, _F]),
            "vans_autotune": (ctypes.c_int, [_H, _LP]),
            "vans_get_launch": (ctypes.c_int, [_H, _LP]),
            "vans_set_launch": (ctypes.c_int, [_H, _LP]),
            "vans_flux": (ctypes.c_int, [_H, _F, ctypes.c_int, _F]),
            "vans_flux_seed": (ctypes.c_int, [_H, _F, ctypes.c_int, _F, _F]),
            "vans_step_adjoint": (ctypes.c_int, [_H, _F, _F, _F, _F]),
            "vans_grad_finalize": (ctypes.c_int, [_H, _F, _F, _F]),
            "vans_adjoint_segment": (ctypes.c_int, [_H, _F, _F, ctypes.c_int, _F, _F, _F]),
            "vans_set_adjoint_precision": (ctypes.c_int, [_H, ctypes.c_int]),
            "vans_set_adjoint_launch": (ctypes.c_int, [_H, _LP]),
            "vans_batch_workspace_bytes": (ctypes.c_size_t, [_P, ctypes.c_int]),
            "vans_batch_create": (ctypes.c_int, [_P, ctypes.c_int, _F, ctypes.c_size_t,
                                                 ctypes.c_void_p, ctypes.POINTER(_H)]),
            "vans_batch_set_eps": (ctypes.c_int, [_H, ctypes.c_int, _F]),
            "vans_batch_step": (ctypes.c_int, [_H, ctypes.c_int]),
            "vans_batch_moments": (ctypes.c_int, [_H, ctypes.c_int, _F, _F]),
            "vans_batch_get_populations": (ctypes.c_int, [_H, ctypes.c_int, _F]),
            "vans_batch_autotune": (ctypes.c_int, [_H, _LP]),
            "vans_batch_profile_step": (ctypes.c_int, [_H, _F, ctypes.c_longlong,
                                                       ctypes.POINTER(ctypes.c_longlong)]),
            "vans_batch_cells": (ctypes.c_longlong, [_H]),
            "vans_cells": (ctypes.c_longlong, [_H]),
            "vans_halo_floats": (ctypes.c_longlong, [_H]),
            "vans_set_eps_slab": (ctypes.c_int, [_H, _F, _F, _F]),
            "vans_halo_pack": (ctypes.c_int, [_H, _F, _F]),
            "vans_halo_unpack": (ctypes.c_int, [_H, _F, _F]),
            "vans_launch_count": (ctypes.c_longlong, [_H]),
            "vans_check": (ctypes.c_int, [_H]),
            "vans_status_string": (ctypes.c_char_p, [ctypes.c_int]),
            "vans_version": (ctypes.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(rc: int, what: str):
    if rc != VANS_OK:
        raise VansError(rc, what)


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("no CUDA device: the porous LBM library runs on the GPU only")
    return torch


def _ptr(t) -> int:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _f32(t, n: int, what: str):
    torch = _torch()
    if t.dtype != torch.float32 or t.numel() != n:
        raise ValueError(f"{what}: expected {n} float32 values, got {t.numel()} {t.dtype}")
    return _ptr(t)


class Solver:
    """One domain: ``vans_create`` on a torch-allocated workspace.

    All calls enqueue on the CUDA stream current at construction."""

    def __init__(self, params, device=None):
        torch = _torch()
        self.lib = load_library()
        self.params = Params.of(params)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        cp = self.params.c()
        nbytes = self.lib.vans_workspace_bytes(ctypes.byref(cp))
        if nbytes == 0:
            raise VansError(-1, "vans_workspace_bytes (invalid parameters)")
        self.state_floats = int(self.lib.vans_state_floats(ctypes.byref(cp)))
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        self._ws = base + ((-base) % 256)
        self.stream = torch.cuda.current_stream(self.device)
        h = _H()
        _check(self.lib.vans_create(ctypes.byref(cp), self._ws, nbytes, self.stream.cuda_stream,
                                    ctypes.byref(h)), "vans_create")
        self._h = h

    # -- lifecycle --------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            self.lib.vans_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    # -- forward ----------------------------------------------------------
    def set_eps(self, eps):
        _check(self.lib.vans_set_eps(self._h, _f32(eps, self.params.cells, "eps")), "vans_set_eps")

    def set_eps_async(self, eps):
        """``vans_set_eps`` without the stream synchronisation: an out-of-range
        field leaves the state undefined and makes the next ``check()`` fail."""
        _check(self.lib.vans_set_eps_async(self._h, _f32(eps, self.params.cells, "eps")),
               "vans_set_eps_async")

    def run_jobs(self, eps_host, nsteps: int, rho_host, u_host):
        """Jobs back to back, each one porosity field: its upload from pinned
        host memory, ``vans_set_eps_async`` (rest state), ``nsteps`` steps,
        ``vans_moments``, and rho and u back into pinned host memory.  The
        copies run on a second stream and overlap the steps of the neighbouring
        jobs (two device buffers of each kind take turns).  eps_host: pinned
        float32 CPU tensors of N values; rho_host, u_host: pinned float32 CPU
        tensors of N and D*N values that receive each job's results.  Returns
        when the last results are on the host."""
        torch = _torch()
        p = self.params
        n = len(eps_host)
        if len(rho_host) != n or len(u_host) != n:
            raise ValueError("one rho and one u buffer per job")
        for t in list(eps_host) + list(rho_host) + list(u_host):
            if t.is_cuda or not t.is_pinned() or t.dtype != torch.float32:
                raise ValueError("host buffers must be pinned float32 CPU tensors")
        dev = self.device
        copy = torch.cuda.Stream(device=dev)
        eps_d = [torch.empty(p.cells, dtype=torch.float32, device=dev) for _ in range(2)]
        rho_d = [torch.empty(p.cells, dtype=torch.float32, device=dev) for _ in range(2)]
        u_d = [torch.empty(p.dim * p.cells, dtype=torch.float32, device=dev) for _ in range(2)]
        ev = lambda: torch.cuda.Event()  # noqa: E731
        up, used, done, down = ([ev() for _ in range(n)] for _ in range(4))
        with torch.cuda.stream(copy):
            copy.wait_stream(self.stream)          # buffers allocated on the solver's stream
            for k in range(min(2, n)):
                eps_d[k].copy_(eps_host[k], non_blocking=True)
                up[k].record(copy)
        for k in range(n):
            b = k % 2
            self.stream.wait_event(up[k])
            self.set_eps_async(eps_d[b])
            used[k].record(self.stream)            # eps_d[b] has been read
            self.step(nsteps)
            if k >= 2:
                self.stream.wait_event(down[k - 2])   # rho_d[b], u_d[b] are free again
            self.moments(rho_d[b], u_d[b])
            done[k].record(self.stream)
            with torch.cuda.stream(copy):
                copy.wait_event(done[k])
                rho_host[k].copy_(rho_d[b], non_blocking=True)
                u_host[k].copy_(u_d[b], non_blocking=True)
                down[k].record(copy)
                if k + 2 < n:
                    copy.wait_event(used[k])
                    eps_d[b].copy_(eps_host[k + 2], non_blocking=True)
                    up[k + 2].record(copy)
        copy.synchronize()
        self.stream.synchronize()

    # -- slabs along x -----------------------------------------------------
    @property
    def halo_floats(self) -> int:
        return int(self.lib.vans_halo_floats(self._h))

    def set_eps_slab(self, eps, eps_left, eps_right):
        """The slab's own porosity field and the columns just left and right of
        it (ny * nz values each)."""
        rows = self.params.ny * self.params.nz
        _check(self.lib.vans_set_eps_slab(self._h, _f32(eps, self.params.cells, "eps"),
                                          _f32(eps_left, rows, "eps_left"),
                                          _f32(eps_right, rows, "eps_right")), "vans_set_eps_slab")

    def halo_pack(self, to_left, to_right):
        n = self.halo_floats
        _check(self.lib.vans_halo_pack(self._h, _f32(to_left, n, "to_left"),
                                       _f32(to_right, n, "to_right")), "vans_halo_pack")

    def halo_unpack(self, from_left, from_right):
        n = self.halo_floats
        _check(self.lib.vans_halo_unpack(self._h, _f32(from_left, n, "from_left"),
                                         _f32(from_right, n, "from_right")), "vans_halo_unpack")

    def update_eps(self, eps):
        """New porosity field, same physical populations (eps varying in time)."""
        _check(self.lib.vans_update_eps(self._h, _f32(eps, self.params.cells, "eps")),
               "vans_update_eps")

    def step(self, nsteps: int = 1):
        _check(self.lib.vans_step(self._h, int(nsteps)), "vans_step")

    def step_monitored(self, nsteps: int, every: int, rho=None, u=None, stats=None):
        """nsteps steps; every `every` steps the step kernel also writes rho and u
        and reduces (max|du|, max|u|, diverged, count) into stats."""
        torch = _torch()
        p = self.params
        if rho is None:
            rho = torch.empty(p.shape, dtype=torch.float32, device=self.device)
        if u is None:
            u = torch.zeros((p.dim,) + p.shape, dtype=torch.float32, device=self.device)
        if stats is None:
            stats = torch.empty(4, dtype=torch.float32, device=self.device)
        _check(self.lib.vans_step_monitored(self._h, int(nsteps), int(every),
                                            _f32(rho, p.cells, "rho"), _f32(u, p.dim * p.cells, "u"),
                                            _f32(stats, 4, "stats")), "vans_step_monitored")
        return rho, u, stats

    def step_raw(self, state_in, state_out):
        _check(self.lib.vans_step_raw(self._h, _f32(state_in, self.state_floats, "state_in"),
                                      _f32(state_out, self.state_floats, "state_out")),
               "vans_step_raw")

    def moments(self, rho=None, u=None):
        torch = _torch()
        p = self.params
        if rho is None:
            rho = torch.empty(p.shape, dtype=torch.float32, device=self.device)
        if u is None:
            u = torch.empty((p.dim,) + p.shape, dtype=torch.float32, device=self.device)
        _check(self.lib.vans_moments(self._h, _f32(rho, p.cells, "rho"),
                                     _f32(u, p.dim * p.cells, "u")), "vans_moments")
        return rho, u

    def populations(self, out=None):
        torch = _torch()
        p = self.params
        if out is None:
            out = torch.empty((p.q,) + p.shape, dtype=torch.float32, device=self.device)
        _check(self.lib.vans_get_populations(self._h, _f32(out, p.q * p.cells, "f")),
               "vans_get_populations")
        return out

    def set_populations(self, f):
        p = self.params
        _check(self.lib.vans_set_populations(self._h, _f32(f, p.q * p.cells, "f")),
               "vans_set_populations")

    def new_state(self):
        torch = _torch()
        return torch.zeros(self.state_floats, dtype=torch.float32, device=self.device)

    def get_state(self, out=None):
        if out is None:
            out = self.new_state()
        _check(self.lib.vans_get_state(self._h, _f32(out, self.state_floats, "state")),
               "vans_get_state")
        return out

    def set_state(self, state):
        _check(self.lib.vans_set_state(self._h, _f32(state, self.state_floats, "state")),
               "vans_set_state")

    def check(self) -> bool:
        rc = self.lib.vans_check(self._h)
        if rc == -3:
            return False
        _check(rc, "vans_check")
        return True

    # -- launch configuration -------------------------------------------------
    def autotune(self) -> Launch:
        c = _CLaunch()
        _check(self.lib.vans_autotune(self._h, ctypes.byref(c)), "vans_autotune")
        return Launch(c.cpt, c.warps, c.rows, c.kind, c.ctas)

    @property
    def launch(self) -> Launch:
        c = _CLaunch()
        _check(self.lib.vans_get_launch(self._h, ctypes.byref(c)), "vans_get_launch")
        return Launch(c.cpt, c.warps, c.rows, c.kind, c.ctas)

    @launch.setter
    def launch(self, L: Launch):
        c = _CLaunch(int(L.cpt), int(L.warps), int(L.rows), int(L.kind), int(L.ctas))
        _check(self.lib.vans_set_launch(self._h, ctypes.byref(c)), "vans_set_launch")

    @property
    def launch_count(self) -> int:
        return int(self.lib.vans_launch_count(self._h))

    # -- reverse mode ---------------------------------------------------------
    def grad_floats(self) -> int:
        """Floats of grad_acc: sums and compensation words of dJ/deps and dJ/d(grad eps)."""
        return 2 * (1 + self.params.dim) * self.params.cells

    def flux(self, x_out: int, state=None, out=None):
        torch = _torch()
        if out is None:
            out = torch.empty(1, dtype=torch.float32, device=self.device)
        st = None if state is None else _f32(state, self.state_floats, "state")
        _check(self.lib.vans_flux(self._h, st, int(x_out), _f32(out, 1, "J")), "vans_flux")
        return out

    def flux_seed(self, x_out: int, lam, grad, state=None):
        st = None if state is None else _f32(state, self.state_floats, "state")
        _check(self.lib.vans_flux_seed(self._h, st, int(x_out),
                                       _f32(lam, self.state_floats, "lam"),
                                       _f32(grad, self.grad_floats(), "grad_acc")),
               "vans_flux_seed")

    def step_adjoint(self, state_t, lam_in, lam_out, grad):
        _check(self.lib.vans_step_adjoint(self._h, _f32(state_t, self.state_floats, "state_t"),
                                          _f32(lam_in, self.state_floats, "lam_in"),
                                          _f32(lam_out, self.state_floats, "lam_out"),
                                          _f32(grad, self.grad_floats(), "grad_acc")),
               "vans_step_adjoint")

    def set_adjoint_launch(self, L: Launch):
        c = _CLaunch(int(L.cpt), int(L.warps), int(L.rows), int(L.kind), int(L.ctas))
        _check(self.lib.vans_set_adjoint_launch(self._h, ctypes.byref(c)), "vans_set_adjoint_launch")

    def set_adjoint_precision(self, bits: int):
        _check(self.lib.vans_set_adjoint_precision(self._h, int(bits)), "vans_set_adjoint_precision")

    def adjoint_segment(self, ckpt, seg, length: int, lam, tmp, grad):
        """Recompute a segment from its checkpoint and walk lam back through it."""
        if seg.numel() < (length + 1) * self.state_floats or seg.dtype != _torch().float32:
            raise ValueError("seg: expected (length+1) float32 state buffers")
        _check(self.lib.vans_adjoint_segment(self._h, _f32(ckpt, self.state_floats, "ckpt"),
                                             _ptr(seg), int(length),
                                             _f32(lam, self.state_floats, "lam"),
                                             _f32(tmp, self.state_floats, "tmp"),
                                             _f32(grad, self.grad_floats(), "grad_acc")),
               "vans_adjoint_segment")

    def grad_finalize(self, lam0, grad, out=None):
        torch = _torch()
        p = self.params
        if out is None:
            out = torch.empty(p.shape, dtype=torch.float32, device=self.device)
        _check(self.lib.vans_grad_finalize(self._h, _f32(lam0, self.state_floats, "lam0"),
                                           _f32(grad, self.grad_floats(), "grad_acc"),
                                           _f32(out, p.cells, "dJdeps")),
               "vans_grad_finalize")
        return out


class Batch:
    """Many independent D2Q9 domains advanced by one persistent kernel per step."""

    def __init__(self, params_list, device=None):
        torch = _torch()
        self.lib = load_library()
        self.params = [Params.of(p) for p in params_list]
        self.n = len(self.params)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        arr = (_CParams * self.n)(*[p.c() for p in self.params])
        nbytes = self.lib.vans_batch_workspace_bytes(arr, self.n)
        if nbytes == 0:
            raise VansError(-1, "vans_batch_workspace_bytes (invalid parameters)")
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        self._ws = base + ((-base) % 256)
        self.stream = torch.cuda.current_stream(self.device)
        h = _H()
        _check(self.lib.vans_batch_create(arr, self.n, self._ws, nbytes, self.stream.cuda_stream,
                                          ctypes.byref(h)), "vans_batch_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self.lib.vans_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_eps(self, d: int, eps):
        _check(self.lib.vans_batch_set_eps(self._h, int(d), _f32(eps, self.params[d].cells, "eps")),
               "vans_batch_set_eps")

    def step(self, nsteps: int = 1):
        _check(self.lib.vans_batch_step(self._h, int(nsteps)), "vans_batch_step")

    def moments(self, d: int):
        torch = _torch()
        p = self.params[d]
        rho = torch.empty(p.shape, dtype=torch.float32, device=self.device)
        u = torch.empty((2,) + p.shape, dtype=torch.float32, device=self.device)
        _check(self.lib.vans_batch_moments(self._h, int(d), _ptr(rho), _ptr(u)), "vans_batch_moments")
        return rho, u

    def populations(self, d: int):
        torch = _torch()
        p = self.params[d]
        out = torch.empty((9,) + p.shape, dtype=torch.float32, device=self.device)
        _check(self.lib.vans_batch_get_populations(self._h, int(d), _ptr(out)),
               "vans_batch_get_populations")
        return out

    def autotune(self) -> Launch:
        c = _CLaunch()
        _check(self.lib.vans_batch_autotune(self._h, ctypes.byref(c)), "vans_batch_autotune")
        return Launch(c.cpt, c.warps, c.rows, c.kind, c.ctas)

    def profile_step(self) -> dict:
        """One step with per-CTA timing records (vans_batch_profile_step) and
        the load balance they give: the mean over all SMs of each SM's busy span
        (first CTA start to last CTA end on it) over the step's makespan."""
        torch = _torch()
        n = ctypes.c_longlong(0)
        _check(self.lib.vans_batch_profile_step(self._h, None, 0, ctypes.byref(n)),
               "vans_batch_profile_step")
        rec = torch.zeros(3 * n.value, dtype=torch.int64, device=self.device)
        _check(self.lib.vans_batch_profile_step(self._h, _ptr(rec), 3 * n.value, ctypes.byref(n)),
               "vans_batch_profile_step")
        r = rec.view(-1, 3).cpu().numpy()
        r = r[r[:, 1] != 0]
        t0, t1 = int(r[:, 1].min()), int(r[:, 2].max())
        spans = {}
        for sm, a, b in r:
            lo, hi = spans.get(int(sm), (a, b))
            spans[int(sm)] = (min(lo, a), max(hi, b))
        sms = torch.cuda.get_device_properties(self.device).multi_processor_count
        busy = sum(int(b) - int(a) for a, b in spans.values())
        per_sm = {}
        for sm in r[:, 0]:
            per_sm[int(sm)] = per_sm.get(int(sm), 0) + 1
        return {"ctas": int(len(r)), "sms_used": len(spans), "makespan_us": (t1 - t0) / 1e3,
                "efficiency": busy / (sms * (t1 - t0)),
                "max_ctas_per_sm": max(per_sm.values())}

    @property
    def launch(self) -> Launch:
        c = _CLaunch()
        _check(self.lib.vans_get_launch(self._h, ctypes.byref(c)), "vans_get_launch")
        return Launch(c.cpt, c.warps, c.rows, c.kind, c.ctas)

    @launch.setter
    def launch(self, L: Launch):
        c = _CLaunch(int(L.cpt), int(L.warps), int(L.rows), int(L.kind), int(L.ctas))
        _check(self.lib.vans_set_launch(self._h, ctypes.byref(c)), "vans_set_launch")

    @property
    def cells(self) -> int:
        return int(self.lib.vans_batch_cells(self._h))

    @property
    def launch_count(self) -> int:
        return int(self.lib.vans_launch_count(self._h))

    def check(self) -> bool:
        rc = self.lib.vans_check(self._h)
        if rc == -3:
            return False
        _check(rc, "vans_check")
        return True
