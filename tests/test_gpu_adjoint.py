"""GPU reverse mode (adjoint step kernel + checkpointed recomputation behind a
torch.autograd.Function) against the oracle's FP64 discrete adjoint."""
import numpy as np
import pytest

import oracle as O
from paper_1406_6438_gb300 import workloads as W
from tests._gpu import solver, torch_cuda

pytestmark = pytest.mark.gpu


def _gpu_grad(p, eps, nsteps, every, x_out):
    torch = torch_cuda()
    from paper_1406_6438_gb300.adjoint import outlet_flux
    s = solver(p, eps)
    e = torch.from_numpy(np.ascontiguousarray(eps)).cuda().requires_grad_(True)
    J = outlet_flux(e, s, nsteps, every, x_out)
    J.backward()
    torch.cuda.synchronize()
    return float(J.item()), e.grad.cpu().numpy().astype(np.float64)


ADJ_CASES = [
    # params, nsteps, every
    (W.adjoint_channel(nx=64, ny=48)[0], 200, 20),
    (W.params(q=9, nx=40, ny=32, wall_mask=0, tau=0.6, g=(5e-5, 2e-5, 0), drag_mode=2, k_mode=0,
              d_p=W.D_P), 120, 50),
    (W.params(q=9, nx=37, ny=20, wall_mask=2, tau=0.9, g=(1e-4, 0, 0), drag_mode=2, k_mode=2,
              K=4.0), 90, 30),
    (W.params(q=19, nx=12, ny=8, nz=6, wall_mask=6, tau=0.7, g=(1e-4, 0, 0), drag_mode=2,
              k_mode=0, d_p=5.0), 30, 10),
]


@pytest.mark.parametrize("p,nsteps,every", ADJ_CASES)
def test_adjoint_matches_oracle_discrete_adjoint(p, nsteps, every):
    """dJ/deps of every cell from the GPU adjoint (FP32, FP32 accumulation)
    within 1e-4 of the oracle's FP64 adjoint, relative to max |dJ/deps|."""
    shape = (p["nz"], p["ny"], p["nx"])
    eps = W.smoothed_noise(shape, 4.0, 0.4, 1.0, seed=shape[1] + nsteps)
    x_out = p["nx"] - 1
    J_o, g_o = O.adjoint(O.Params(**p), eps.astype(np.float64), nsteps, x_out)
    J, g = _gpu_grad(p, eps, nsteps, every, x_out)
    assert abs(J - J_o) <= 1e-5 * abs(J_o)
    err = np.abs(g - g_o).max() / np.abs(g_o).max()
    assert err <= 1e-4, err


def test_checkpoint_interval_does_not_change_the_gradient():
    torch = torch_cuda()
    p = W.adjoint_channel(nx=48, ny=32)[0]
    eps = W.smoothed_noise((1, 32, 48), 4.0, 0.4, 1.0, seed=3)
    _, g1 = _gpu_grad(p, eps, 60, 60, 47)
    _, g2 = _gpu_grad(p, eps, 60, 7, 47)
    assert np.array_equal(g1, g2)
