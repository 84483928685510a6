"""The adjoint workload at full size: a 512x512 porous channel, 2000 steps from
rest, checkpoints every 100 steps.  The GPU gradient of the outlet flux with
respect to eps (FP32 adjoint kernel, FP32 accumulation) is compared with FP64
central finite differences of the oracle at 32 random cells, stored in
tests/golden/adjoint_channel_512_fd.json by tests/golden/make_adjoint_fd.py
(which calls the oracle only)."""
import json
import os

import numpy as np
import pytest

from paper_1406_6438_gb300 import workloads as W
from tests._gpu import solver, torch_cuda

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "adjoint_channel_512_fd.json")


@pytest.mark.parametrize("bits,tol", [(64, 1e-4), (32, 1e-4)])
def test_adjoint_gradient_matches_fp64_finite_differences_at_32_cells(bits, tol):
    """Within 1e-4 of the FD values, relative to their maximum.  bits = 64:
    per-cell reverse arithmetic in FP64 (FP32 states and lambda; each term
    enters the compensated FP32 accumulation as its leading part and
    remainder; measured 6.1e-5, the level the FP32 storage sets).  bits = 32:
    all-FP32 reverse step, its square roots and reciprocals formed like the
    forward step's (measured 7.2e-5; the eps gradient is a ~700x smaller
    residual of the grad-eps sensitivities, so the per-cell FP32 rounding
    adds to the storage's share)."""
    torch = torch_cuda()
    from paper_1406_6438_gb300.adjoint import outlet_flux
    gold = json.load(open(GOLDEN))
    p, eps, nsteps, every = W.adjoint_channel()
    assert nsteps == gold["nsteps"]
    cells = [tuple(c) for c in gold["cells_zyx"]]
    assert cells == W.fd_cells(eps.shape, 32, seed=5)
    s = solver(p, eps)
    s.set_adjoint_precision(bits)
    e = torch.from_numpy(eps).cuda().requires_grad_(True)
    J = outlet_flux(e, s, nsteps, every, gold["x_out"])
    J.backward()
    torch.cuda.synchronize()
    g = e.grad.cpu().numpy().astype(np.float64)
    fd = np.array(gold["dJdeps_fd"])
    got = np.array([g[c] for c in cells])
    assert abs(J.item() - gold["J"]) <= 1e-5 * abs(gold["J"])
    err = np.abs(got - fd).max() / np.abs(fd).max()
    assert err <= tol, err
    assert np.isfinite(g).all()
