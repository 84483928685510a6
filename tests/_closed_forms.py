"""Closed forms and a boundary-value solver that the oracle is pinned to.

Nothing here reuses the oracle's code: these are textbook solutions of the
continuum equations the model must reproduce, written from the mathematics.
"""
import numpy as np
from scipy.linalg import solve_banded


def poiseuille_series(y, t, g, nu, H, nterms=400):
    """Start-up plane Poiseuille flow between walls at 0 and H driven by g:
    u = g/(2nu) y (H-y) - sum_{n odd} 4 g H^2/(nu n^3 pi^3) sin(n pi y/H) exp(-nu n^2 pi^2 t/H^2)."""
    u = g / (2 * nu) * y * (H - y)
    for n in range(1, 2 * nterms, 2):
        u = u - 4 * g * H * H / (nu * n ** 3 * np.pi ** 3) * np.sin(n * np.pi * y / H) \
            * np.exp(-nu * n * n * np.pi ** 2 * t / H ** 2)
    return u


def duct_series(y, z, g, nu, A, B, nterms=200):
    """Steady laminar flow along x in the rectangular duct 0 < y < A, 0 < z < B
    (no slip on all four walls) driven by g: nu (u_yy + u_zz) = -g.  Sine series
    in y of the plane-channel parabola, each mode corrected by the cosh term
    that brings it to zero on the z walls:
    u = sum_{n odd} 4 g A^2/(nu n^3 pi^3) sin(n pi y/A)
        [1 - cosh(n pi (z - B/2)/A) / cosh(n pi B/(2A))]."""
    u = np.zeros(np.broadcast(y, z).shape)
    for n in range(1, 2 * nterms, 2):
        k = n * np.pi / A
        u = u + 4 * g * A * A / (nu * n ** 3 * np.pi ** 3) * np.sin(k * y) \
            * (1 - np.cosh(k * (z - B / 2)) / np.cosh(k * B / 2))
    return u


def brinkman(y, g, nu, eps, K, H):
    """Steady solution of nu u'' - (eps nu/K) u + g = 0, u(0) = u(H) = 0."""
    r = np.sqrt(eps / K)
    return g * K / (eps * nu) * (1 - np.cosh(r * (y - H / 2)) / np.cosh(r * H / 2))


def porous_bvp(nu, eps, K, Feps, g, H, n=4001, u_top=0.0):
    """Fine-grid solution of the fully developed porous channel equation
    nu u'' - (eps nu / K) u - (eps^2 F_eps / sqrt K) |u| u + g = 0,
    u(0) = 0, u(H) = u_top, by Newton iteration on a second-order FD grid."""
    y = np.linspace(0.0, H, n)
    h = y[1] - y[0]
    u = np.zeros(n)
    u[-1] = u_top
    a = eps * nu / K
    b = eps ** 2 * Feps / np.sqrt(K)
    for _ in range(100):
        ui = u[1:-1]
        r = nu * (u[2:] - 2 * ui + u[:-2]) / h ** 2 - a * ui - b * ui * np.abs(ui) + g
        d = -2 * nu / h ** 2 - a - 2 * b * np.abs(ui)
        ab = np.zeros((3, n - 2))
        ab[0, 1:] = nu / h ** 2
        ab[1] = d
        ab[2, :-1] = nu / h ** 2
        du = solve_banded((1, 1), ab, -r)
        u[1:-1] += du
        if np.abs(du).max() <= 1e-15 * max(1e-300, np.abs(u).max()):
            break
    return y, u
