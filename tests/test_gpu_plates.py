"""Plates on nodes with the non-equilibrium extrapolation scheme (wall_kind 1,
the boundary scheme of the paper's validation runs) on the GPU against the
oracle: random states through every kernel kind that has plate rows, the
paper's porous Couette case, and the combinations the library refuses."""
import numpy as np
import pytest

from paper_1406_6438_gb300 import workloads as W
from paper_1406_6438_gb300._binding import Launch
from tests._gpu import gpu_run, oracle_run, rel_u, solver, torch_cuda

pytestmark = pytest.mark.gpu


def _case(q, shape, uw, seed):
    nz, ny, nx = shape
    p = W.params(q=q, nx=nx, ny=ny, nz=nz, wall_mask=2, tau=0.7, g=(3e-4, -1e-4, 5e-5),
                 drag_mode=2, k_mode=0, d_p=6.0, u_wall=uw, wall_kind=1)
    eps = W.smoothed_noise(shape, 2.0, 0.4, 1.0, seed)
    f0 = W.random_state(q, eps, seed + 100, amp=0.02)
    return p, eps, f0


PLATE_CASES = [
    # q, (nz, ny, nx), u_wall, launches (the shapes with a plates-on-nodes instance)
    (9, (1, 13, 37), (0.01, 0.0, 0.0),
     [Launch(1, 1, 2), Launch(2, 2, 1), Launch(4, 4, 1), Launch(4, 1, 2), Launch(2, 4, 3, 2),
      Launch(4, 4, 3, 2), Launch(4, 4, 3, 5), Launch(4, 2, 2, 5), Launch(4, 4, 2, 7),
      Launch(4, 2, 3, 7)]),
    (9, (1, 3, 20), (0.02, 0.0, 0.0),       # one fluid row between the plates
     [Launch(2, 2, 1), Launch(4, 4, 3, 2), Launch(4, 4, 3, 5), Launch(4, 4, 2, 7)]),
    (9, (1, 40, 700), (0.0, 0.0, 0.0),
     [Launch(4, 4, 1), Launch(2, 4, 3, 2), Launch(4, 4, 4, 5), Launch(4, 4, 4, 7)]),
    (19, (7, 9, 21), (0.01, 0.0, 0.004),
     [Launch(1, 2, 1), Launch(2, 2, 2), Launch(1, 4, 3, 2), Launch(2, 4, 3, 5),
      Launch(2, 4, 2, 7)]),
    (19, (6, 30, 300), (0.0, 0.0, 0.0), [Launch(1, 4, 3, 2), Launch(2, 4, 3, 7)]),
    (19, (5, 8, 64), (0.01, 0.0, 0.0), [Launch(2, 4, 2, 7), Launch(2, 4, 3, 7)]),
]


@pytest.mark.parametrize("q,shape,uw,launches", PLATE_CASES)
def test_plates_on_nodes_random_states(q, shape, uw, launches):
    """Every population (the plate rows hold f^eq of the plate plus the
    neighbour's non-equilibrium part) and the velocity after 1 and 5 steps from
    a random state, for each kernel kind with plate rows."""
    p, eps, f0 = _case(q, shape, uw, seed=61 + sum(shape))
    for nsteps in (1, 5):
        _, u_o, f_o = oracle_run(p, eps, nsteps, f0)
        for L in launches:
            _, u, f = gpu_run(p, eps, nsteps, f0, launch=L)
            assert np.abs(f - f_o).max() <= 2e-7, (L, nsteps, np.abs(f - f_o).max())
            assert rel_u(u, u_o) <= 1e-5, (L, nsteps)


@pytest.mark.parametrize("Re,Da", [(1, 1e-3), (50, 1e-2)])
def test_porous_couette_with_plates_on_nodes(Re, Da):
    """The paper's validation case with its boundary scheme (81 x 80 nodes,
    plates H = 80 apart, eps = 0.1) from rest, 3000 steps in the autotuned
    launch: velocity within 1e-5 of the oracle."""
    p, eps = W.couette_80(Re=Re, Da=Da, wall_kind=1)
    s = solver(p, eps)
    L = s.autotune()
    assert L.kind in (0, 2, 5, 7, 8)        # the shapes with a plates-on-nodes instance
    s.step(3000)
    _, u = s.moments()
    _, u_o, _ = oracle_run(p, eps, 3000)
    assert rel_u(u.cpu().numpy().astype(np.float64), u_o) <= 1e-5
    assert s.check()


def test_plates_on_nodes_refusals():
    torch = torch_cuda()
    import paper_1406_6438_gb300 as V
    from paper_1406_6438_gb300._binding import VansError
    p, eps, _ = _case(9, (1, 12, 40), (0.01, 0.0, 0.0), seed=3)
    s = solver(p, eps)
    for L in (Launch(2, 8, 2, 6), Launch(2, 4, 2, 4)):
        with pytest.raises(VansError):      # shapes without a plates-on-nodes instance
            s.launch = L
    with pytest.raises(VansError):
        s.step_monitored(10, 5)
    lam = s.new_state()
    grad = torch.empty(s.grad_floats(), device="cuda")
    with pytest.raises(VansError):
        s.flux_seed(39, lam, grad)
    with pytest.raises(VansError):
        V.Batch([p])
    # the flux (a diagnostic) is defined: sum of eps rho u_x over the column
    J = s.flux(20)
    assert np.isfinite(float(J.item()))
    # the 192-, 320- and 384-cell D3Q19 tiles have no plates-on-nodes instance
    p3, eps3, _ = _case(19, (3, 10, 192), (0.01, 0.0, 0.0), seed=4)
    s3 = solver(p3, eps3)
    for L in (Launch(2, 3, 2, 7), Launch(2, 5, 2, 7), Launch(2, 6, 2, 7)):
        with pytest.raises(VansError):
            s3.launch = L
    s3.launch = Launch(2, 4, 2, 7)
