"""Pins of the oracle's per-cell arithmetic (CPU only).

Each test checks the FP64 oracle against something fixed by the paper or by the
mathematics rather than against itself: lattice isotropy, the moment identities
the paper states for f^eq and P_i, the same identities for the Guo term F_i,
brute-force root finding for the implicit velocity, and the paper's own K and
F_eps formulas for the drag coefficients.
"""
import itertools

import numpy as np
import pytest

import oracle as O

CS2 = 1.0 / 3.0


@pytest.mark.parametrize("q,dim", [(9, 2), (19, 3)])
def test_lattice_isotropy(q, dim):
    """Velocity-set pins: weights sum to 1, odd moments vanish, the second moment
    is cs^2 delta and the fourth is cs^4 (dd + dd + dd) (Qian et al. 1992, the
    lattices the paper's equilibrium is written for)."""
    e, w, opp = O.lattice(q)
    e = e[:, :dim].astype(float)
    assert len({tuple(v) for v in e}) == q
    assert abs(w.sum() - 1) < 1e-15
    assert np.abs((w[:, None] * e).sum(0)).max() < 1e-15
    d = np.eye(dim)
    m2 = np.einsum("i,ia,ib->ab", w, e, e)
    assert np.abs(m2 - CS2 * d).max() < 1e-15
    m3 = np.einsum("i,ia,ib,ic->abc", w, e, e, e)
    assert np.abs(m3).max() < 1e-15
    m4 = np.einsum("i,ia,ib,ic,id->abcd", w, e, e, e, e)
    iso = CS2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                      + np.einsum("ad,bc->abcd", d, d))
    assert np.abs(m4 - iso).max() < 1e-15
    for i in range(q):
        assert np.all(e[opp[i]] == -e[i])


def _rand_cell(rng, dim):
    eps = rng.uniform(0.3, 1.0)
    rho = rng.uniform(0.9, 1.1)
    u = np.zeros(3)
    u[:dim] = rng.normal(size=dim) * 0.05
    return eps, rho, u


@pytest.mark.parametrize("q,dim", [(9, 2), (19, 3)])
def test_feq_moments(q, dim):
    """Moments of Eq. d2q9eq (the identities listed after it): sum f^eq = eps rho,
    sum e f^eq = eps rho u, sum e e f^eq = cs^2 eps rho delta + eps rho u u, and the
    third moment cs^2 eps rho (d_ab u_c + d_ac u_b + d_bc u_a) (the printed indices
    are garbled; this is the symmetric reading)."""
    e, _, _ = O.lattice(q)
    e = e[:, :dim].astype(float)
    rng = np.random.default_rng(11)
    d = np.eye(dim)
    for _ in range(50):
        eps, rho, u3 = _rand_cell(rng, dim)
        u = u3[:dim]
        f = O.feq(q, eps, rho, u3)
        R = eps * rho
        assert abs(f.sum() - R) < 1e-14
        assert np.abs(e.T @ f - R * u).max() < 1e-15
        m2 = np.einsum("i,ia,ib->ab", f, e, e)
        assert np.abs(m2 - (CS2 * R * d + R * np.outer(u, u))).max() < 1e-14
        m3 = np.einsum("i,ia,ib,ic->abc", f, e, e, e)
        ref = CS2 * R * (np.einsum("ab,c->abc", d, u) + np.einsum("ac,b->abc", d, u)
                         + np.einsum("bc,a->abc", d, u))
        assert np.abs(m3 - ref).max() < 1e-15


@pytest.mark.parametrize("q,dim", [(9, 2), (19, 3)])
def test_source_moments(q, dim):
    """Moments of Eq. pi (listed after it) and of Eq. Fi, which has the same form:
    sum S = 0, sum e S = (1 - 1/(2 tau)) V, sum e e S = (1 - 1/(2 tau)) (u V + V u).
    With V = p grad eps the first moment is (1 - 1/(2 tau)) cs^2 rho grad eps."""
    e, _, _ = O.lattice(q)
    e = e[:, :dim].astype(float)
    rng = np.random.default_rng(12)
    for _ in range(50):
        tau = rng.uniform(0.51, 2.0)
        u = np.zeros(3)
        u[:dim] = rng.normal(size=dim) * 0.05
        V = np.zeros(3)
        V[:dim] = rng.normal(size=dim) * 1e-3
        S = O.source(q, tau, u, V)
        c = 1 - 1 / (2 * tau)
        assert abs(S.sum()) < 1e-18
        assert np.abs(e.T @ S - c * V[:dim]).max() < 1e-18
        m2 = np.einsum("i,ia,ib->ab", S, e, e)
        ref = c * (np.outer(u[:dim], V[:dim]) + np.outer(V[:dim], u[:dim]))
        assert np.abs(m2 - ref).max() < 1e-18
    # pressure-correction form
    rho, gradeps = 1.03, np.array([0.02, -0.01, 0.005])
    tau = 0.7
    V = CS2 * rho * gradeps
    S = O.source(q, tau, np.zeros(3), V)
    assert np.abs(e.T @ S - (1 - 1 / (2 * tau)) * CS2 * rho * gradeps[:dim]).max() < 1e-18


def _bisect_speed(a, b, mm):
    """|u| with |u| (a + b |u|) = |m|, by bisection."""
    lo, hi = 0.0, mm / a
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if mid * (a + b * mid) < mm:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def test_velocity_solve_bruteforce():
    """The closed form for the implicit Eq. 1moment against bisection: the speed
    solves |u| (R + alpha/2 + beta/2 |u|) = |m| and u is parallel to m."""
    rng = np.random.default_rng(13)
    for _ in range(200):
        R = rng.uniform(0.3, 1.2)
        alpha = rng.uniform(0, 0.1)
        beta = rng.choice([0.0, rng.uniform(0, 2.0)])
        m = rng.normal(size=3) * rng.choice([1e-4, 1e-2, 0.1])
        u = O.velocity(R, m, alpha, beta)
        mm = np.linalg.norm(m)
        s = _bisect_speed(R + alpha / 2, beta / 2, mm)
        assert abs(np.linalg.norm(u) - s) <= 1e-13 * s + 1e-300
        assert np.abs(np.cross(u, m)).max() <= 1e-14 * np.linalg.norm(u) * mm + 1e-300
        # residual of (R + alpha/2 + beta/2 |u|) u = m
        res = (R + alpha / 2 + beta / 2 * np.linalg.norm(u)) * u - m
        assert np.abs(res).max() <= 1e-14 * mm
    assert np.all(O.velocity(1.0, [0, 0, 0], 0.1, 0.3) == 0)


def test_drag_coefficients_match_paper_formulas():
    """alpha = eps^2 nu / K and beta = eps^3 F_eps / sqrt K with the Ergun K and
    F_eps printed in the paper, against the oracle's finite-at-eps=1 closed form."""
    tau, d_p = 0.6, 21.33
    nu = CS2 * (tau - 0.5)
    for eps in np.linspace(0.1, 0.95, 12):
        K = eps ** 3 * d_p ** 2 / (150 * (1 - eps) ** 2)
        Feps = 1.75 / np.sqrt(150 * eps ** 3)
        p = O.Params(tau=tau, drag_mode=2, k_mode=0, d_p=d_p)
        a, b = O.drag_coeffs(p, eps)
        assert abs(a - eps ** 2 * nu / K) <= 1e-14 * a
        assert abs(b - eps ** 3 * Feps / np.sqrt(K)) <= 1e-14 * b
        p2 = O.Params(tau=tau, drag_mode=2, k_mode=2, K=K)
        a2, b2 = O.drag_coeffs(p2, eps)
        assert abs(a2 - a) <= 1e-13 * a and abs(b2 - b) <= 1e-13 * b
        p1 = O.Params(tau=tau, drag_mode=2, k_mode=1, K=K, F_eps=Feps)
        a1, b1 = O.drag_coeffs(p1, eps)
        assert abs(a1 - a) <= 1e-13 * a and abs(b1 - b) <= 1e-13 * b
    p = O.Params(tau=tau, drag_mode=2, k_mode=0, d_p=d_p)
    assert O.drag_coeffs(p, 1.0) == (0.0, 0.0)
    assert O.drag_coeffs(O.Params(tau=tau, drag_mode=1, k_mode=0, d_p=d_p), 0.5)[1] == 0.0
    assert O.drag_coeffs(O.Params(tau=tau, drag_mode=0, k_mode=0, d_p=d_p), 0.5) == (0.0, 0.0)


@pytest.mark.parametrize("q", [9, 19])
def test_grad_eps_stencil_exact_on_linear_fields(q):
    """The lattice gradient (1/cs^2) sum w_i e_i eps(x+e_i) is exact for a linear
    field away from walls and wrap seams, and zero for a uniform field."""
    e, w, _ = O.lattice(q)
    nz = 1 if q == 9 else 6
    p = O.Params(q=q, nx=7, ny=6, nz=nz, wall_mask=0)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(6), np.arange(7), indexing="ij")
    c = np.array([0.013, -0.021, 0.007])
    lin = 0.5 + c[0] * x + c[1] * y + (c[2] * z if q == 19 else 0)
    G = O.grad_eps(p, lin)
    inner = (slice(1, -1) if nz > 2 else slice(None), slice(1, -1), slice(1, -1))
    for k in range(p.dim):
        assert np.abs(G[k][inner] - c[k]).max() < 1e-14
    G0 = O.grad_eps(p, np.full(p.shape, 0.7))
    assert np.abs(G0).max() < 1e-15


def test_streaming_single_population():
    """Brute force: a single population moves one cell along e_i per step,
    wraps on periodic axes and comes back reversed at a bounce-back wall."""
    for q, shape, wm in [(9, (1, 5, 4), 2), (19, (4, 3, 5), 6), (9, (1, 3, 3), 0)]:
        nz, ny, nx = shape
        p = O.Params(q=q, nx=nx, ny=ny, nz=nz, wall_mask=wm)
        e, _, opp = O.lattice(q)
        walls = [(wm >> a) & 1 for a in range(3)]
        for i, (z, y, x) in itertools.product(range(q), itertools.product(range(nz), range(ny), range(nx))):
            fs = np.zeros((q,) + shape)
            fs[i, z, y, x] = 1.0
            fn = O.stream(p, np.ones(shape), fs)
            dest = [x + e[i, 0], y + e[i, 1], z + e[i, 2]]
            out = False
            for a, n in enumerate((nx, ny, nz)):
                if dest[a] < 0 or dest[a] >= n:
                    if walls[a]:
                        out = True
                    dest[a] %= n
            exp = np.zeros_like(fs)
            if out:
                exp[opp[i], z, y, x] = 1.0
            else:
                exp[i, dest[2], dest[1], dest[0]] = 1.0
            assert np.array_equal(fn, exp), (q, i, z, y, x)
