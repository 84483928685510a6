"""Pins of the oracle's outlet flux J (CPU only).

J is the sum over the plane x = x_out of eps*rho*u_x, with eps*rho*u the
momentum of Eq. 1moment (its half-force and half-pressure terms included): the
objective whose gradient the reverse pass computes.  Three independent facts
fix it:

* it is the plane sum of the moments the oracle reports (pinned themselves by
  the flow tests), column by column, so the plane and the component are right;
* for a state that does not vary along x on a lattice without walls the plane
  momentum changes by exactly the plane sum of p grad eps + F in one step, and
  Eq. 1moment puts eps*rho*u half-way between the momentum before and after the
  step, so J is the mean of the plane momentum at t and t + 1 -- this fixes
  the halves in front of the force and pressure terms;
* in a steady Darcy channel it equals eps times the flux of the Brinkman closed
  form, to second order in 1/H.
"""
import numpy as np
import pytest

import oracle as O
from paper_1406_6438_gb300 import workloads as W
from tests._closed_forms import brinkman

CS2 = 1.0 / 3.0


def _plane_momentum(q, f, x):
    """sum over the plane x of sum_i e_ix f_i: the x-momentum stored in the
    populations of that plane (no force terms)."""
    e, _, _ = O.lattice(q)
    return float(np.einsum("i,izy->", e[:, 0].astype(np.float64), f[:, :, :, x]))


@pytest.mark.parametrize("q,shape,wm", [(9, (1, 11, 7), 2), (9, (1, 6, 9), 0),
                                        (19, (5, 4, 6), 6), (19, (3, 5, 4), 2)])
def test_flux_is_the_plane_sum_of_the_moments(q, shape, wm):
    """J(x_out) = sum over y, z of eps * rho * u_x at column x_out, for every
    x_out, on a random state with a non-uniform eps, drag and a body force."""
    nz, ny, nx = shape
    p = O.Params(q=q, nx=nx, ny=ny, nz=nz, wall_mask=wm, tau=0.7, g=(4e-4, -1e-4, 2e-4),
                 drag_mode=2, k_mode=0, d_p=5.0)
    eps = W.smoothed_noise(shape, 1.5, 0.4, 1.0, seed=sum(shape) + wm).astype(np.float64)
    f = W.random_state(q, eps.astype(np.float32), seed=5 + wm, amp=0.05).astype(np.float64)
    rho, u = O.moments(p, eps, f)
    for x in range(nx):
        want = float((eps * rho * u[0])[:, :, x].sum())
        scale = float(np.abs(eps * rho * u[0])[:, :, x].sum())
        assert abs(O.flux(p, eps, f, x) - want) <= 1e-14 * scale
    # the columns differ, so a wrong plane could not pass
    Js = [O.flux(p, eps, f, x) for x in range(nx)]
    assert np.ptp(Js) > 1e-3 * np.abs(Js).max()


@pytest.mark.parametrize("q,shape,dm", [(9, (1, 13, 3), 2), (9, (1, 8, 2), 1),
                                        (19, (5, 6, 2), 2), (19, (4, 3, 3), 1)])
def test_flux_is_the_mean_of_the_plane_momentum_before_and_after_a_step(q, shape, dm):
    """A state that does not vary along x, periodic in every direction: one
    step moves each plane's populations into the next plane, which holds the
    same ones, so the plane momentum changes by the plane sum of the force
    alone; Eq. 1moment with its half-force terms puts J half-way:
    J(t) = (P(t) + P(t+1)) / 2 with P the plane sum of sum_i e_ix f_i.  eps
    varies across the planes (pressure term on), drag and body force on."""
    nz, ny, nx = shape
    p = O.Params(q=q, nx=nx, ny=ny, nz=nz, wall_mask=0, tau=0.77, g=(3e-3, 1e-3, -1e-3),
                 drag_mode=dm, k_mode=0, d_p=2.0)
    col = W.smoothed_noise((nz, ny, 1), 1.0, 0.4, 1.0, seed=ny + nz).astype(np.float64)
    eps = np.repeat(col, nx, axis=2)
    f1 = W.random_state(q, col.astype(np.float32), seed=11 * ny + dm, amp=0.1).astype(np.float64)
    f = np.repeat(f1, nx, axis=3)
    g = O.run(p, eps, f, 1)
    for x in range(nx):
        P0, P1 = _plane_momentum(q, f, x), _plane_momentum(q, g, x)
        J = O.flux(p, eps, f, x)
        assert abs(P1 - P0) > 1e-3 * abs(J)         # the force did change the momentum
        assert abs(J - 0.5 * (P0 + P1)) <= 1e-13 * (abs(P0) + abs(P1))


def test_flux_of_a_steady_darcy_channel_against_the_brinkman_closed_form():
    """Uniform eps, Darcy drag only, walls in y: at steady state rho = 1 and
    J = eps * sum_y u(y) with u the Brinkman profile of nu u'' - (eps nu / K) u
    + g = 0, sampled at the cell centres y = j + 1/2.  The relative error falls
    at second order in 1/H."""
    tau, e, Da, g = 0.8, 0.6, 1e-2, 1e-6
    nu = CS2 * (tau - 0.5)
    errs = []
    for H in (16, 32, 64):
        K = Da * H * H
        p = O.Params(q=9, nx=2, ny=H, wall_mask=2, tau=tau, g=(g, 0, 0), drag_mode=1,
                     k_mode=1, K=K)
        eps = np.full(p.shape, e)
        f = O.run(p, eps, O.init(p, eps), int(20 * H * H / (100 * nu)) + 3000)
        y = np.arange(H) + 0.5
        want = e * brinkman(y, g, nu, e, K, H).sum()
        errs.append(abs(O.flux(p, eps, f, 1) - want) / want)
    # measured 9.8e-4, 2.4e-4, 6.1e-5: the plane momentum without the half
    # force (the populations' own sum_i e_ix f_i) is 5 times further off
    assert errs[-1] < 1e-4, errs
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all(ratios > 3.5), (errs, ratios)
