"""Slabs along x on one GPU: the pack / exchange / unpack cycle of the
multi-GPU decomposition, run here between slabs that share a GPU (the exchange
a device copy), against the FP64 oracle of the whole domain cell by cell and
against the single-domain solver bit for bit (the same step kernel instance,
so the same per-cell arithmetic)."""
import numpy as np
import pytest

from paper_1406_6438_gb300 import workloads as W
from paper_1406_6438_gb300._binding import Launch, VansError
from tests._gpu import gpu_run, oracle_run, rel_u, solver, torch_cuda

pytestmark = pytest.mark.gpu


def _params(q, shape, wm, **kw):
    nz, ny, nx = shape
    base = dict(q=q, nx=nx, ny=ny, nz=nz, wall_mask=wm, tau=0.66, g=(2e-4, -5e-5, 3e-5),
                drag_mode=2, k_mode=0, d_p=6.0)
    base.update(kw)
    return W.params(**base)


CASES = [
    # q, shape (nz, ny, nx), wall_mask, cuts, extra parameters
    (9, (1, 40, 96), 2, [(0, 50), (50, 96)], {}),
    (9, (1, 33, 70), 0, [(0, 13), (13, 47), (47, 70)], {}),
    (9, (1, 24, 64), 2, [(0, 32), (32, 64)], dict(u_wall=(0.02, 0.0, 0.0))),
    # plates on nodes: cut at a multiple of 4 columns, so that every cell keeps
    # its place among the 4 cells of a lane of the register-load kernel (its
    # unrolled copies may round the plate arithmetic differently by an ulp)
    (9, (1, 21, 60), 2, [(0, 28), (28, 60)], dict(wall_kind=1, u_wall=(0.01, 0.0, 0.0))),
    (19, (10, 12, 40), 6, [(0, 16), (16, 40)], {}),
    (19, (6, 7, 30), 2, [(0, 9), (9, 20), (20, 30)], dict(u_wall=(0.01, 0.0, 0.004))),
]


@pytest.mark.parametrize("q,shape,wm,cuts,kw", CASES)
def test_slabs_match_the_oracle_and_the_whole_domain(q, shape, wm, cuts, kw):
    torch = torch_cuda()
    from paper_1406_6438_gb300.slabs import Slabs
    p = _params(q, shape, wm, **kw)
    eps = W.smoothed_noise(shape, 3.0, 0.4, 1.0, seed=sum(shape) + len(cuts))
    n = 20
    sl = Slabs(p, eps, cuts=cuts)
    sl.step(n)
    f = sl.populations()
    rho, u = sl.moments()
    torch.cuda.synchronize()
    rho_o, u_o, f_o = oracle_run(p, eps, n)
    err_f = float(np.abs(f.cpu().numpy() - f_o).max())
    assert err_f <= 2e-7, err_f
    assert rel_u(u.cpu().numpy().astype(np.float64), u_o) <= 1e-5
    assert np.abs(rho.cpu().numpy() - rho_o).max() <= 1e-6
    # the whole domain on one handle, the same (default) launch: identical bits
    _, _, f_w = gpu_run(p, eps, n)
    assert np.array_equal(f.cpu().numpy().astype(np.float64), f_w)
    sl.close()


@pytest.mark.parametrize("case", ["d2q9", "d3q19 rows of one tile", "d2q9 cluster-resident",
                                  "d3q19 cluster-resident"])
def test_slabs_in_a_pipelined_launch(case):
    """The interleaved bulk-copy step (kind 7) and the cluster-resident step
    (kind 8) on slabs, against the oracle.  D3Q19 slabs of 64 columns are rows
    of one tile, which a periodic domain stages cells only, taking the x wrap
    from the row's other end; a slab's halo columns are its neighbours', so it
    must stage them."""
    torch = torch_cuda()
    from paper_1406_6438_gb300.slabs import Slabs
    if case == "d2q9":
        p, eps, _ = W.periodic_2d_shape(600, 64, nsteps=0)
        L = Launch(4, 4, 3, 7, 2)
    elif case == "d3q19 rows of one tile":
        p, eps, _ = W.duct_3d(nx=128, ny=12, nz=10, nsteps=0)
        L = Launch(2, 4, 2, 7)
    elif case == "d2q9 cluster-resident":
        # kind 8, one step per call: the halo columns the exchange wrote are
        # loaded with the band
        p, eps, _ = W.periodic_2d_shape(96, 40, nsteps=0)
        L = Launch(1, 16, 16, 8)
    else:
        p, eps, _ = W.duct_3d(nx=24, ny=9, nz=7, nsteps=0)
        L = Launch(1, 16, 16, 8)
    sl = Slabs(p, eps, nslabs=2, launch=L)
    sl.step(15)
    f = sl.populations()
    torch.cuda.synchronize()
    _, _, f_o = oracle_run(p, eps, 15)
    assert np.abs(f.cpu().numpy() - f_o).max() <= 2e-7
    sl.close()


def test_one_slab_exchanging_with_itself_is_the_periodic_step():
    """A single slab whose messages come back to it (from_left = its own
    to_right) reproduces vans_step's own periodic wrap bit for bit."""
    torch = torch_cuda()
    p, eps, _ = W.periodic_2d_shape(77, 30, nsteps=0)
    a = solver(p, eps)
    b = solver(p, eps)
    n = b.halo_floats
    assert n == 3 * 30
    tl, tr = (torch.empty(n, device="cuda") for _ in range(2))
    for _ in range(9):
        a.step(1)
        b.step(1)
        b.halo_pack(tl, tr)
        b.halo_unpack(tr, tl)
    torch.cuda.synchronize()
    assert torch.equal(a.get_state(), b.get_state())


def test_slab_refusals():
    torch = torch_cuda()
    p, eps, _ = W.periodic_2d_shape(40, 16, nsteps=0)
    s = solver(p, eps)
    col = torch.full((16,), 0.5, device="cuda")
    bad = col.clone()
    bad[3] = 0.0
    e = torch.from_numpy(eps).cuda().view(-1)
    with pytest.raises(VansError) as ex:
        s.set_eps_slab(e, bad, col)
    assert ex.value.status == -1
    s.set_eps_slab(e, col, col)
    for call in (lambda: s.step(2), lambda: s.step_monitored(3, 1), lambda: s.update_eps(e)):
        with pytest.raises(VansError) as ex:
            call()
        assert ex.value.status == -5
    s.step(1)                       # one step at a time is the slab's cycle
    s.set_eps(e)                    # a plain field makes it a periodic domain again
    s.step(3)
