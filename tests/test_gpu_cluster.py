"""Launch kind 8: every step of a call in one launch of one thread-block
cluster that keeps the whole state in its distributed shared memory (domains
of up to a few hundred KB: the 128x64 channel, the 80x80 Couette case).
Against the FP64 oracle and against the step-by-step register-load kernel."""
import numpy as np
import pytest

from paper_1406_6438_gb300 import workloads as W
from paper_1406_6438_gb300._binding import Launch, VansError
from tests._gpu import gpu_run, oracle_run, rel_u, solver, torch_cuda

pytestmark = pytest.mark.gpu

K8 = [Launch(1, 8, 16, 8), Launch(1, 16, 16, 8), Launch(1, 8, 8, 8), Launch(1, 16, 4, 8)]


def _case(q, shape, wm, **kw):
    nz, ny, nx = shape
    base = dict(q=q, nx=nx, ny=ny, nz=nz, wall_mask=wm, tau=0.7, g=(3e-4, -1e-4, 5e-5),
                drag_mode=2, k_mode=0, d_p=6.0)
    base.update(kw)
    p = W.params(**base)
    eps = W.smoothed_noise(shape, 2.0, 0.4, 1.0, sum(shape) + wm)
    f0 = W.random_state(q, eps, sum(shape) + 100, amp=0.02)
    return p, eps, f0


CASES = [
    (9, (1, 13, 37), 2, {}),
    (9, (1, 20, 64), 0, {}),
    (9, (1, 17, 45), 2, dict(u_wall=(0.02, 0.005, 0.0))),
    (19, (7, 9, 21), 6, {}),
    (19, (5, 6, 12), 2, dict(u_wall=(0.01, 0.0, 0.004))),
    # plates on nodes (the paper's boundary scheme): rows 0 and ny-1 are not
    # stepped, the rows next to them write the plates' inward populations,
    # across the bands of two CTAs where a band ends next to a plate
    (9, (1, 19, 40), 2, dict(wall_kind=1, u_wall=(0.015, 0.0, 0.0))),
    (9, (1, 3, 24), 2, dict(wall_kind=1, u_wall=(0.01, 0.0, 0.0))),
    (19, (4, 9, 16), 2, dict(wall_kind=1, u_wall=(0.01, 0.0, 0.005))),
]


@pytest.mark.parametrize("q,shape,wm,kw", CASES)
@pytest.mark.parametrize("nsteps", [1, 8, 29])
def test_cluster_steps_match_the_oracle(q, shape, wm, kw, nsteps):
    p, eps, f0 = _case(q, shape, wm, **kw)
    rho_o, u_o, f_o = oracle_run(p, eps, nsteps, f0)
    _, _, f_ref = gpu_run(p, eps, nsteps, f0, launch=Launch(1, 4, 1))
    for L in K8:
        rho, u, f = gpu_run(p, eps, nsteps, f0, launch=L)
        assert np.abs(f - f_o).max() <= 2e-7, (L, np.abs(f - f_o).max())
        assert rel_u(u, u_o) <= 1e-5, L
        assert np.abs(rho - rho_o).max() <= 1e-6, L
        # the register-load kernel, one launch per step: within an ulp or two
        assert np.abs(f - f_ref).max() <= 6e-8, (L, np.abs(f - f_ref).max())


def test_channel_128x64_5000_steps_in_one_launch():
    """The 128x64 porous Poiseuille channel after its 5000 steps, all of them in
    one cluster launch: the same 1e-5 velocity bound against the oracle."""
    p, eps, n = W.channel_128x64()
    rho_o, u_o, _ = oracle_run(p, eps, n)
    rho, u, _ = gpu_run(p, eps, n, launch=Launch(1, 16, 16, 8))
    assert rel_u(u, u_o) <= 1e-5, rel_u(u, u_o)
    assert np.abs(rho - rho_o).max() <= 1e-5


def test_cluster_calls_compose_and_refusals():
    """Calls of several lengths continue each other (the state and its parity
    are where single steps leave them); domains too large for one cluster are
    refused."""
    torch = torch_cuda()
    p, eps, _ = W.periodic_2d_shape(90, 40, nsteps=0)
    a = solver(p, eps, launch=Launch(1, 16, 16, 8))
    b = solver(p, eps, launch=Launch(1, 4, 1))
    for n in (3, 1, 10, 64, 7):
        a.step(n)
        b.step(n)
    fa, fb = a.populations(), b.populations()
    torch.cuda.synchronize()
    assert (fa - fb).abs().max().item() <= 6e-8
    big, eps_big, _ = W.periodic_2d_shape(1024, 1024, nsteps=0)
    s = solver(big, eps_big)
    with pytest.raises(VansError) as ex:
        s.launch = Launch(1, 16, 16, 8)
    assert ex.value.status == -5


@pytest.mark.parametrize("Re,Da", [(1.0, 1e-3), (50.0, 1e-2)])
def test_porous_couette_of_the_paper_in_one_cluster_launch(Re, Da):
    """The paper's porous Couette case with its own boundary scheme (plates on
    nodes, 81 rows), all steps in one cluster launch, against the oracle and
    against the register-load kernel's single steps."""
    p, eps = W.couette_80(Re=Re, Da=Da, wall_kind=1)
    n = 400
    rho_o, u_o, f_o = oracle_run(p, eps, n)
    _, _, f_ref = gpu_run(p, eps, n, launch=Launch(1, 4, 1))
    rho, u, f = gpu_run(p, eps, n, launch=Launch(1, 16, 16, 8))
    assert rel_u(u, u_o) <= 1e-5, rel_u(u, u_o)
    assert np.abs(f - f_o).max() <= 2e-7
    assert np.abs(f - f_ref).max() <= 6e-8
