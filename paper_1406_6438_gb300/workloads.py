"""Seeded synthetic inputs and workload definitions.

This module holds no arithmetic of the method.  It only draws the inputs that
both the CUDA path and the FP64 oracle consume: porosity fields, domain sizes,
relaxation times, random populations, and the parameter sets of the workloads.
Every float parameter is rounded to float32 here, once, so that the GPU (FP32)
and the oracle (FP64) read identical numbers.

Porosity fields: i.i.d. N(0,1) noise from ``numpy.random.default_rng(seed)`` in
float64, a periodic FFT Gaussian filter of standard deviation ``sigma`` cells
(the "correlation length"), a min-max map onto ``[lo, hi]``, one cast to float32.
"""
from __future__ import annotations

import numpy as np

# Ergun particle diameter used wherever a workload gives no Darcy number.  It
# makes K(eps = 0.6) equal the K = Da * H^2 = 1e-3 * 64^2 of the 128x64 channel.
D_P = 21.33


def f32(x: float) -> float:
    """Round a parameter to the nearest float32 (and return it as a Python float)."""
    return float(np.float32(x))


def smoothed_noise(shape, sigma: float, lo: float, hi: float, seed: int) -> np.ndarray:
    """Gaussian-smoothed white noise on a periodic grid, mapped onto [lo, hi], float32."""
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal(shape)
    spec = np.fft.fftn(noise)
    for ax, n in enumerate(shape):
        k = 2.0 * np.pi * np.fft.fftfreq(n)
        filt = np.exp(-0.5 * (sigma * k) ** 2)
        sh = [1] * len(shape)
        sh[ax] = n
        spec = spec * filt.reshape(sh)
    sm = np.real(np.fft.ifftn(spec))
    a, b = sm.min(), sm.max()
    if b > a:
        sm = (sm - a) / (b - a)
    else:
        sm = np.zeros_like(sm)
    return (lo + (hi - lo) * sm).astype(np.float32)


def uniform_eps(shape, value: float) -> np.ndarray:
    return np.full(shape, np.float32(value), dtype=np.float32)


def params(q=9, nx=1, ny=1, nz=1, wall_mask=0, tau=0.8, g=(0.0, 0.0, 0.0), drag_mode=0,
           k_mode=0, d_p=1.0, K=1.0, F_eps=0.0, u_wall=(0.0, 0.0, 0.0), wall_kind=0) -> dict:
    """A parameter set (the fields of ``vans_params``), floats rounded to float32."""
    g = tuple(f32(v) for v in g) + (0.0,) * (3 - len(g))
    uw = tuple(f32(v) for v in u_wall) + (0.0,) * (3 - len(u_wall))
    return dict(q=int(q), nx=int(nx), ny=int(ny), nz=int(nz), wall_mask=int(wall_mask),
                tau=f32(tau), g=g, drag_mode=int(drag_mode), k_mode=int(k_mode),
                d_p=f32(d_p), K=f32(K), F_eps=f32(F_eps), u_wall=uw, wall_kind=int(wall_kind))


# --------------------------------------------------------------------------
# Workloads.  Each returns (params dict, eps float32 [nz, ny, nx], nsteps).
# --------------------------------------------------------------------------

def channel_128x64():
    """D2Q9 porous Poiseuille channel 128x64, uniform eps = 0.6, Da = 1e-3
    (K = Da * H^2 = 4.096 with H = 64), F_eps from the paper's formula of eps,
    tau = 0.8, body force g_x = 2.3e-5 (Re = U H / nu ~ 1), periodic x,
    bounce-back y, 5000 steps."""
    p = params(q=9, nx=128, ny=64, wall_mask=2, tau=0.8, g=(2.3e-5, 0, 0), drag_mode=2,
               k_mode=2, K=1e-3 * 64 * 64)
    return p, uniform_eps((1, 64, 128), 0.6), 5000


def periodic_2d(n: int = 4096, seed: int = 2, nsteps: int = 1000):
    """D2Q9 periodic n x n domain, eps from seeded smoothed noise (sigma = 16) in
    [0.4, 1.0], tau = 0.6, Ergun drag with d_p = 21.33, body force along x."""
    p = params(q=9, nx=n, ny=n, wall_mask=0, tau=0.6, g=(5e-5, 0, 0), drag_mode=2, k_mode=0,
               d_p=D_P)
    return p, smoothed_noise((1, n, n), 16.0, 0.4, 1.0, seed), nsteps


def periodic_2d_shape(nx: int, ny: int, seed: int = 2, nsteps: int = 200):
    """The periodic D2Q9 workload on an nx x ny grid (downsized parity cases)."""
    p = params(q=9, nx=nx, ny=ny, wall_mask=0, tau=0.6, g=(5e-5, 0, 0), drag_mode=2, k_mode=0,
               d_p=D_P)
    return p, smoothed_noise((1, ny, nx), 16.0, 0.4, 1.0, seed), nsteps


def duct_3d(nx: int = 256, ny: int = 256, nz: int = 256, seed: int = 3, nsteps: int = 500):
    """D3Q19 porous duct, eps from smoothed noise in [0.35, 0.95], Forchheimer on,
    tau = 0.6, bounce-back on y and z, periodic x, body force along x (Re ~ 50)."""
    p = params(q=19, nx=nx, ny=ny, nz=nz, wall_mask=6, tau=0.6, g=(2e-5, 0, 0), drag_mode=2,
               k_mode=0, d_p=D_P)
    return p, smoothed_noise((nz, ny, nx), 16.0, 0.35, 0.95, seed), nsteps


def batched_channels(n: int = 256, seed: int = 4, nx_range=(64, 1024), ny_range=(32, 512),
                     tau_range=(0.55, 1.0)):
    """Independent D2Q9 porous channels (periodic x, bounce-back y): sizes drawn
    uniformly from nx_range x ny_range, tau from tau_range, eps of domain k from
    smoothed noise (seed 1000*seed + k) in [0.4, 1.0]."""
    rng = np.random.default_rng(seed)
    nxs = rng.integers(nx_range[0], nx_range[1] + 1, size=n)
    nys = rng.integers(ny_range[0], ny_range[1] + 1, size=n)
    taus = rng.uniform(tau_range[0], tau_range[1], size=n)
    doms = []
    for k in range(n):
        p = params(q=9, nx=nxs[k], ny=nys[k], wall_mask=2, tau=taus[k], g=(1e-5, 0, 0),
                   drag_mode=2, k_mode=0, d_p=D_P)
        eps = smoothed_noise((1, int(nys[k]), int(nxs[k])), 16.0, 0.4, 1.0, 1000 * seed + k)
        doms.append((p, eps))
    return doms


def adjoint_channel(nx: int = 512, ny: int = 512, seed: int = 5, nsteps: int = 2000,
                    every: int = 100):
    """D2Q9 channel for the outlet-flux gradient: eps from smoothed noise in
    [0.4, 1.0], tau = 0.8, Ergun drag, body force along x, bounce-back y,
    nsteps forward steps with checkpoints every ``every`` steps."""
    p = params(q=9, nx=nx, ny=ny, wall_mask=2, tau=0.8, g=(2e-5, 0, 0), drag_mode=2, k_mode=0,
               d_p=D_P)
    return p, smoothed_noise((1, ny, nx), 16.0, 0.4, 1.0, seed), nsteps, every


def couette_80(Re: float = 1.0, Da: float = 1e-2, eps: float = 0.1, n: int = 80, nx: int = 80,
               wall_kind: int = 0):
    """The paper's validation case: Couette flow through a porous medium of
    uniform porosity eps = 0.1 between plates H = L = 80 apart, the upper plate
    moving at u0 (the characteristic velocity), periodic in x; tau = 0.6574 at
    Re = 50, 0.8 otherwise; rho = 1, u = 0 at start; Re = L u0 / nu, Da = K / L^2;
    drag law with K = Da L^2 and F_eps = 1.75/sqrt(150 eps^3); no body force.
    wall_kind 0: half-way bounce-back plates, n rows of nodes; wall_kind 1: the
    non-equilibrium extrapolation scheme with the plates on nodes, n + 1 rows."""
    tau = 0.6574 if Re == 50 else 0.8
    nu = (f32(tau) - 0.5) / 3.0
    u0 = Re * nu / n
    ny = n + 1 if wall_kind == 1 else n
    p = params(q=9, nx=nx, ny=ny, wall_mask=2, tau=tau, drag_mode=2, k_mode=2, K=Da * n * n,
               u_wall=(u0, 0.0, 0.0), wall_kind=wall_kind)
    return p, uniform_eps((1, ny, nx), eps)


def fd_cells(shape, count: int = 32, seed: int = 5):
    """``count`` distinct random cells (z, y, x) of a grid, for finite differences."""
    rng = np.random.default_rng(seed)
    n = int(np.prod(shape))
    flat = rng.choice(n, size=count, replace=False)
    return [tuple(int(v) for v in np.unravel_index(i, shape)) for i in sorted(flat)]


def lattice_weights(q: int) -> np.ndarray:
    """Rest-state weights only used to build random test states near rest.  (They
    are data of the velocity sets, listed in the same order as the library's.)"""
    if q == 9:
        return np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    return np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


def random_state(q: int, eps: np.ndarray, seed: int, amp: float = 0.02) -> np.ndarray:
    """Populations near rest, f_i = w_i eps (1 + amp * N(0,1)), float32 [q, nz, ny, nx]."""
    rng = np.random.default_rng(seed)
    w = lattice_weights(q).reshape((q, 1, 1, 1))
    noise = rng.standard_normal((q,) + eps.shape)
    return (w * eps.astype(np.float64)[None] * (1.0 + amp * noise)).astype(np.float32)
