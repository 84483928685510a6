"""Pin of the oracle's discrete adjoint: dJ/deps against FP64 central finite
differences of the oracle's forward run, on every cell of tiny grids (CPU only).

J is the outlet flux, the sum of eps*rho*u_x (Eq. 1moment) over the plane
x = nx - 1 after T steps from the rest state f = w eps."""
import numpy as np
import pytest

import oracle as O

CASES = [
    # (q, shape (nz, ny, nx), wall_mask, drag_mode, k_mode, u_wall)
    (9, (1, 5, 6), 2, 2, 0, (0, 0, 0)),
    (9, (1, 4, 5), 0, 2, 0, (0, 0, 0)),
    (9, (1, 5, 4), 2, 1, 1, (0, 0, 0)),
    (9, (1, 5, 4), 2, 2, 2, (0, 0, 0)),
    (9, (1, 5, 4), 2, 2, 0, (0.01, 0, 0)),
    (19, (3, 4, 5), 6, 2, 0, (0, 0, 0)),
]


@pytest.mark.parametrize("q,shape,wm,dm,km,uw", CASES)
def test_adjoint_matches_central_differences(q, shape, wm, dm, km, uw):
    nz, ny, nx = shape
    p = O.Params(q=q, nx=nx, ny=ny, nz=nz, wall_mask=wm, tau=0.7, g=(2e-3, 5e-4, 1e-4),
                 drag_mode=dm, k_mode=km, d_p=3.0, K=2.0, F_eps=0.3, u_wall=uw)
    rng = np.random.default_rng(17 + q + wm + dm + km)
    eps = rng.uniform(0.4, 0.95, size=shape)
    T, xo = 10, nx - 1
    J, grad = O.adjoint(p, eps, T, xo)

    def Jof(e):
        f = O.run(p, e, O.init(p, e), T)
        return O.flux(p, e, f, xo)

    assert abs(J - Jof(eps)) <= 1e-15 * abs(J)
    h = 1e-6
    fd = np.zeros_like(eps)
    for idx in np.ndindex(shape):
        ep = eps.copy()
        ep[idx] += h
        em = eps.copy()
        em[idx] -= h
        fd[idx] = (Jof(ep) - Jof(em)) / (2 * h)
    scale = np.abs(fd).max()
    assert scale > 0
    assert np.abs(grad - fd).max() <= 1e-6 * scale
