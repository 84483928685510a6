"""GPU parity of the fused step, the moments and the state I/O against the FP64
oracle, on seeded inputs, through the C ABI (libvans.so)."""
import numpy as np
import pytest

import oracle as O
from paper_1406_6438_gb300 import workloads as W
from paper_1406_6438_gb300._binding import Launch, VansError
from tests._gpu import gpu_run, oracle_run, rel_u, solver, torch_cuda

pytestmark = pytest.mark.gpu


def _case(q, shape, wall_mask, seed, tau=0.7, k_mode=0):
    nz, ny, nx = shape
    p = W.params(q=q, nx=nx, ny=ny, nz=nz, wall_mask=wall_mask, tau=tau,
                 g=(3e-4, -1e-4, 5e-5), drag_mode=2, k_mode=k_mode, d_p=6.0, K=2.5, F_eps=0.3)
    eps = W.smoothed_noise(shape, 2.0, 0.4, 1.0, seed)
    f0 = W.random_state(q, eps, seed + 100, amp=0.02)
    return p, eps, f0


STEP_CASES = [
    # q, (nz, ny, nx), wall_mask, launches (kinds 0, 2, 4-7)
    (9, (1, 13, 37), 2, [Launch(1, 1, 2), Launch(2, 2, 1), Launch(4, 1, 2), Launch(4, 4, 1),
                         Launch(2, 4, 3, 2), Launch(2, 4, 3, 4), Launch(4, 4, 3, 5),
                         Launch(4, 2, 2, 5), Launch(2, 4, 2, 6), Launch(2, 8, 3, 6),
                         Launch(4, 4, 2, 7), Launch(4, 2, 3, 7), Launch(4, 4, 2, 7, 2),
                         Launch(4, 4, 3, 5, 1), Launch(2, 4, 3, 2, 3)]),
    (9, (1, 6, 5), 0, [Launch(4, 2, 1), Launch(1, 2, 1), Launch(1, 8, 2, 2), Launch(4, 2, 3, 5)]),
    (9, (1, 1, 1), 0, [Launch(4, 2, 1), Launch(2, 4, 3, 2), Launch(2, 4, 3, 4), Launch(4, 4, 3, 5),
                       Launch(2, 4, 2, 6), Launch(4, 4, 2, 7)]),
    (9, (1, 1, 3), 2, [Launch(1, 2, 1), Launch(2, 8, 2, 2), Launch(4, 2, 2, 7)]),
    (9, (1, 9, 300), 2, [Launch(2, 2, 2), Launch(4, 2, 1), Launch(4, 4, 3, 2), Launch(1, 8, 4, 2),
                         Launch(4, 4, 3, 4), Launch(1, 8, 4, 4), Launch(4, 2, 4, 5),
                         Launch(2, 4, 3, 6), Launch(4, 4, 2, 7)]),
    (9, (1, 7, 1100), 0, [Launch(2, 4, 4, 2), Launch(4, 4, 3, 5, 2), Launch(4, 4, 3, 7, 2)]),
    (9, (1, 40, 700), 2, [Launch(2, 8, 3, 2), Launch(1, 8, 5, 2), Launch(2, 8, 3, 4),
                          Launch(4, 4, 6, 5), Launch(2, 8, 4, 6), Launch(4, 2, 5, 7)]),
    (19, (7, 9, 21), 6, [Launch(1, 2, 1), Launch(2, 2, 2), Launch(4, 1, 2), Launch(1, 4, 3, 2),
                         Launch(2, 4, 2, 2), Launch(1, 4, 3, 4), Launch(2, 4, 2, 4),
                         Launch(2, 4, 2, 5), Launch(2, 2, 4, 5), Launch(1, 4, 2, 6),
                         Launch(1, 8, 3, 6), Launch(2, 4, 2, 7), Launch(2, 2, 3, 7),
                         Launch(2, 4, 2, 7, 1)]),
    (19, (5, 4, 33), 2, [Launch(2, 2, 1), Launch(1, 8, 2, 2), Launch(2, 4, 4, 5)]),
    (19, (3, 3, 4), 0, [Launch(1, 2, 1), Launch(1, 4, 4, 2), Launch(2, 4, 2, 7)]),
    (19, (1, 1, 2), 6, [Launch(1, 2, 1), Launch(1, 4, 3, 2), Launch(2, 4, 2, 5),
                        Launch(1, 4, 2, 6), Launch(2, 4, 2, 7)]),
    (19, (6, 30, 300), 4, [Launch(2, 4, 3, 2), Launch(1, 8, 3, 2), Launch(1, 8, 3, 4),
                           Launch(2, 4, 3, 5), Launch(1, 8, 2, 6),
                           Launch(2, 4, 3, 7), Launch(2, 4, 2, 7, 2)]),
    # D3Q19 rows of a multiple of 8 cells, each row one tile (or two): the
    # halo columns sit in sectors of their own
    (19, (4, 6, 64), 0, [Launch(2, 4, 2, 7), Launch(2, 2, 2, 7), Launch(2, 4, 3, 7, 2),
                         Launch(1, 4, 2, 6), Launch(1, 8, 3, 6)]),
    (19, (3, 5, 128), 6, [Launch(2, 2, 2, 7), Launch(1, 4, 2, 6), Launch(2, 4, 2, 7),
                          Launch(1, 8, 2, 6)]),
    (19, (2, 4, 256), 2, [Launch(2, 4, 2, 7), Launch(2, 2, 3, 7), Launch(1, 8, 2, 6),
                          Launch(1, 4, 3, 6)]),
    (19, (2, 3, 8), 6, [Launch(2, 4, 2, 7), Launch(1, 4, 2, 6)]),
    # rows shorter than the tile staged cells-only: lanes past nx idle, the x
    # wrap read from the other end of the staged cells
    (19, (3, 7, 96), 6, [Launch(2, 4, 2, 7), Launch(2, 4, 3, 7, 2), Launch(2, 2, 2, 7)]),
    (19, (5, 3, 40), 2, [Launch(2, 2, 3, 7), Launch(2, 4, 2, 7)]),
    # 384-cell tiles (6 compute warps): rows of 384 and 264 cells staged
    # cells-only, 300 (not a multiple of 8) and 600 cells with their halos
    (19, (2, 3, 384), 6, [Launch(2, 6, 2, 7), Launch(2, 6, 3, 7, 1)]),
    (19, (3, 2, 264), 2, [Launch(2, 6, 2, 7)]),
    (19, (2, 2, 300), 6, [Launch(2, 6, 2, 7)]),
    (19, (2, 3, 600), 0, [Launch(2, 6, 2, 7)]),
    # 192-cell tiles (3 compute warps)
    (19, (3, 3, 192), 6, [Launch(2, 3, 2, 7), Launch(2, 3, 3, 7, 2)]),
    (19, (2, 5, 136), 2, [Launch(2, 3, 2, 7)]),
    (19, (2, 2, 250), 6, [Launch(2, 3, 2, 7)]),
    # 320-cell tiles (5 compute warps): rows of one tile and of two
    (19, (2, 3, 320), 6, [Launch(2, 5, 2, 7), Launch(2, 5, 3, 7, 1)]),
    (19, (3, 2, 512), 2, [Launch(2, 5, 2, 7)]),
    (19, (2, 2, 296), 0, [Launch(2, 5, 2, 7)]),
]


@pytest.mark.parametrize("q,shape,wm,launches", STEP_CASES)
@pytest.mark.parametrize("nsteps", [1, 7])
def test_step_matches_oracle_on_random_states(q, shape, wm, launches, nsteps):
    """Every population after 1 and 7 steps from a random near-rest state, for
    several launch shapes (cells per thread, warps, rows), ragged nx, tiny
    grids, periodic and bounce-back axes.  Tolerance: a few FP32 ulps of f."""
    p, eps, f0 = _case(q, shape, wm, seed=sum(shape) + wm)
    rho_o, u_o, f_o = oracle_run(p, eps, nsteps, f0)
    for L in launches:
        rho, u, f = gpu_run(p, eps, nsteps, f0, launch=L)
        assert np.abs(f - f_o).max() <= 2e-7, (L, np.abs(f - f_o).max())
        assert np.abs(rho - rho_o).max() <= 1e-6, L
        assert rel_u(u, u_o) <= 1e-5, (L, rel_u(u, u_o))


@pytest.mark.parametrize("k_mode", [0, 1, 2])
def test_drag_modes(k_mode):
    p, eps, f0 = _case(9, (1, 12, 20), 2, seed=5 + k_mode, k_mode=k_mode)
    for dm in (0, 1, 2):
        p["drag_mode"] = dm
        rho_o, u_o, f_o = oracle_run(p, eps, 20, f0)
        rho, u, f = gpu_run(p, eps, 20, f0)
        assert np.abs(f - f_o).max() <= 2e-7
        assert rel_u(u, u_o) <= 1e-5


def test_channel_128x64_5000_steps():
    """The 128x64 porous Poiseuille channel (uniform eps = 0.6, Da = 1e-3,
    Forchheimer on, tau = 0.8) after 5000 steps from rest: FP32 GPU velocity
    within 1e-5 of the FP64 oracle, relative to max|u|."""
    p, eps, n = W.channel_128x64()
    rho_o, u_o, _ = oracle_run(p, eps, n)
    rho, u, _ = gpu_run(p, eps, n)
    assert rel_u(u, u_o) <= 1e-5, rel_u(u, u_o)
    assert np.abs(rho - rho_o).max() <= 1e-5


def test_periodic_noise_field_downsized():
    """The periodic smoothed-noise workload (eps in [0.4, 1], tau = 0.6, Ergun
    drag, body force) on a 96x80 grid for 200 steps."""
    p, eps, n = W.periodic_2d_shape(96, 80, nsteps=200)
    rho_o, u_o, _ = oracle_run(p, eps, n)
    rho, u, _ = gpu_run(p, eps, n)
    assert rel_u(u, u_o) <= 1e-5, rel_u(u, u_o)
    assert np.abs(rho - rho_o).max() <= 1e-5


def test_d3q19_duct_downsized():
    """The D3Q19 porous duct (walls on y and z, eps in [0.35, 0.95]) on a
    40x24x20 grid for 100 steps."""
    p, eps, n = W.duct_3d(nx=40, ny=24, nz=20, nsteps=100)
    rho_o, u_o, _ = oracle_run(p, eps, n)
    rho, u, _ = gpu_run(p, eps, n)
    assert rel_u(u, u_o) <= 1e-5, rel_u(u, u_o)
    assert np.abs(rho - rho_o).max() <= 1e-5


@pytest.mark.parametrize("L", [Launch(4, 4, 1), Launch(2, 8, 3, 2), Launch(4, 4, 3, 4),
                               Launch(4, 4, 3, 5),
                               Launch(2, 4, 2, 6), Launch(4, 4, 2, 7)])
def test_graph_replay_equals_single_launches(L):
    """vans_step(n) replays a captured CUDA graph for long runs; the result is
    bit-identical to n single steps."""
    torch = torch_cuda()
    p, eps, n = W.periodic_2d_shape(70, 50, nsteps=0)
    a = solver(p, eps, launch=L)
    b = solver(p, eps, launch=L)
    a.step(64 * 2 + 3)
    for _ in range(64 * 2 + 3):
        b.step(1)
    fa, fb = a.get_state(), b.get_state()
    torch.cuda.synchronize()
    assert torch.equal(fa, fb)
    # and an odd start parity before the graph
    a.step(1)
    a.step(65)
    for _ in range(66):
        b.step(1)
    assert torch.equal(a.get_state(), b.get_state())


def test_checkpoint_resume_is_bitwise():
    """Stop, save the state, continue; restore, continue again: identical."""
    torch = torch_cuda()
    p, eps, _ = W.periodic_2d_shape(64, 40, nsteps=0)
    s = solver(p, eps)
    s.step(30)
    ck = s.get_state()
    s.step(77)
    ref = s.get_state().clone()
    s.set_state(ck)
    s.step(77)
    torch.cuda.synchronize()
    assert torch.equal(s.get_state(), ref)


def test_autotune_leaves_state_unchanged():
    torch = torch_cuda()
    p, eps, _ = W.periodic_2d_shape(200, 64, nsteps=0)
    a = solver(p, eps)
    b = solver(p, eps)
    a.step(10)
    b.step(10)
    L = a.autotune()
    assert L.cpt in (1, 2, 4) and L.kind in (0, 2, 4, 5, 6, 7, 8)
    b.launch = L
    a.step(10)
    b.step(10)
    torch.cuda.synchronize()
    assert torch.equal(a.get_state(), b.get_state())


def test_populations_roundtrip():
    torch = torch_cuda()
    p, eps, f0 = _case(9, (1, 10, 23), 2, seed=3)
    s = solver(p, eps)
    ft = torch.from_numpy(f0).cuda()
    s.set_populations(ft)
    back = s.populations()
    torch.cuda.synchronize()
    assert (back - ft).abs().max().item() <= 6e-8


def test_launch_shapes_agree_on_a_long_run():
    p, eps, n = W.periodic_2d_shape(150, 40, nsteps=300)
    ref = None
    for L in (Launch(1, 2, 1), Launch(2, 4, 2), Launch(4, 4, 1), Launch(4, 2, 4),
              Launch(2, 8, 3, 2), Launch(2, 8, 3, 4), Launch(4, 4, 2, 5), Launch(2, 8, 2, 6),
              Launch(4, 4, 2, 7)):
        rho, u, f = gpu_run(p, eps, n, launch=L)
        if ref is None:
            ref = u
        else:
            assert rel_u(u, ref) <= 1e-6


@pytest.mark.parametrize("wm", [0, 2])
def test_mass_conserved_on_gpu(wm):
    """Total mass over 2000 steps drifts by FP32 rounding only."""
    torch = torch_cuda()
    p, eps, _ = W.periodic_2d_shape(128, 96, nsteps=0)
    p["wall_mask"] = wm
    s = solver(p, eps)
    m0 = s.populations().double().sum().item()
    s.step(2000)
    m1 = s.populations().double().sum().item()
    assert abs(m1 - m0) <= 1e-6 * m0


def test_errors_reported():
    torch = torch_cuda()
    import paper_1406_6438_gb300 as V
    p, eps, _ = W.periodic_2d_shape(16, 8, nsteps=0)
    s = V.Solver(p)
    with pytest.raises(VansError) as e:
        s.step(1)
    assert e.value.status == -6
    bad = torch.from_numpy(eps.copy()).cuda().view(-1)
    bad[5] = 0.0
    with pytest.raises(VansError) as e:
        s.set_eps(bad)
    assert e.value.status == -1
    bad[5] = float("nan")
    with pytest.raises(VansError):
        s.set_eps(bad)
    bad[5] = 1.5
    with pytest.raises(VansError):
        s.set_eps(bad)
    s.set_eps(torch.from_numpy(eps).cuda().view(-1))
    with pytest.raises(VansError):
        s.step(-1)
    assert s.check()
    f = s.populations()
    f[3, 0, 2, 2] = float("nan")          # a fault injected on the host side
    s.set_populations(f)
    assert not s.check()


def test_set_eps_async_and_pipelined_jobs():
    """vans_set_eps_async gives the same state as vans_set_eps; an out-of-range
    field surfaces at the next check and a valid one clears it.  run_jobs
    (uploads, steps, moments and downloads of consecutive jobs overlapped on
    two streams) returns what one job at a time through the synchronous calls
    returns, bit for bit."""
    torch = torch_cuda()
    p, eps, _ = W.periodic_2d_shape(200, 72, nsteps=0)
    fields = [W.smoothed_noise((1, 72, 200), 8.0, 0.4, 1.0, seed=20 + k) for k in range(5)]
    a, b = solver(p, eps), solver(p, eps)
    e_dev = torch.from_numpy(fields[1]).cuda().view(-1)
    a.set_eps(e_dev)
    b.set_eps_async(e_dev)
    a.step(9)
    b.step(9)
    assert torch.equal(a.get_state(), b.get_state())
    assert b.check()
    bad = e_dev.clone()
    bad[17] = 1.5
    b.set_eps_async(bad)
    with pytest.raises(VansError) as e:
        b.check()
    assert e.value.status == -1
    b.set_eps_async(e_dev)
    assert b.check()
    # pipelined jobs against one job at a time
    n = len(fields)
    eps_h = [torch.from_numpy(f).view(-1).pin_memory() for f in fields]
    rho_h = [torch.empty(p["nx"] * p["ny"]).pin_memory() for _ in range(n)]
    u_h = [torch.empty(2 * p["nx"] * p["ny"]).pin_memory() for _ in range(n)]
    b.run_jobs(eps_h, 23, rho_h, u_h)
    for k in range(n):
        a.set_eps(torch.from_numpy(fields[k]).cuda().view(-1))
        a.step(23)
        rho, u = a.moments()
        torch.cuda.synchronize()
        assert torch.equal(rho.cpu().view(-1), rho_h[k]), k
        assert torch.equal(u.cpu().view(-1), u_h[k]), k


@pytest.mark.parametrize("Re,Da", [(1, 1e-3), (50, 1e-2)])
def test_porous_couette_of_the_paper_80x80(Re, Da):
    """The paper's validation case on the GPU: Couette flow through a porous
    medium (eps = 0.1, 80 x 80, upper plate moving at u0, tau = 0.8, or 0.6574
    at Re = 50), 3000 steps from rest, velocity within 1e-5 of the oracle."""
    p, eps = W.couette_80(Re=Re, Da=Da)
    rho_o, u_o, _ = oracle_run(p, eps, 3000)
    rho, u, _ = gpu_run(p, eps, 3000)
    assert rel_u(u, u_o) <= 1e-5, rel_u(u, u_o)
    assert np.abs(rho - rho_o).max() <= 1e-5


MOVING = [
    (9, (1, 13, 37), 2, (0.01, 0.002, 0.0),
     [Launch(4, 4, 1), Launch(1, 2, 1), Launch(2, 4, 3, 2), Launch(2, 4, 3, 4),
      Launch(4, 4, 3, 5)]),
    (9, (1, 1, 5), 2, (0.02, 0.0, 0.0), [Launch(2, 2, 1), Launch(2, 4, 2, 2), Launch(2, 4, 2, 6),
                                         Launch(4, 4, 3, 7)]),
    (19, (7, 9, 21), 6, (0.01, 0.003, -0.002),
     [Launch(1, 2, 1), Launch(2, 2, 2), Launch(2, 4, 2, 2), Launch(2, 4, 3, 5),
      Launch(1, 4, 2, 6), Launch(2, 4, 2, 7)]),
    (19, (4, 5, 9), 2, (0.0, 0.0, 0.01), [Launch(2, 2, 1), Launch(1, 8, 2, 2), Launch(1, 8, 2, 4),
                                          Launch(2, 4, 2, 5)]),
    (19, (5, 7, 64), 6, (0.01, 0.0, 0.004), [Launch(2, 4, 2, 7), Launch(1, 4, 2, 6),
                                             Launch(2, 2, 2, 7)]),
    # the 192-, 320- and 384-cell D3Q19 tiles (3, 5 and 6 warps)
    (19, (3, 5, 192), 6, (0.01, 0.0, 0.004), [Launch(2, 3, 2, 7), Launch(2, 5, 2, 7),
                                              Launch(2, 6, 2, 7)]),
]


@pytest.mark.parametrize("q,shape,wm,uw,launches", MOVING)
def test_moving_wall_random_states(q, shape, wm, uw, launches):
    """Populations through a moving upper wall (including the D3Q19 edge rows
    where a z wall is crossed too), every kernel kind, 1 and 5 steps."""
    p, eps, f0 = _case(q, shape, wm, seed=31 + sum(shape))
    p["u_wall"] = tuple(W.f32(v) for v in uw)
    for nsteps in (1, 5):
        rho_o, u_o, f_o = oracle_run(p, eps, nsteps, f0)
        for L in launches:
            rho, u, f = gpu_run(p, eps, nsteps, f0, launch=L)
            assert np.abs(f - f_o).max() <= 2e-7, (L, nsteps, np.abs(f - f_o).max())
            assert rel_u(u, u_o) <= 1e-5, (L, nsteps)


def test_rest_state_next_to_a_moving_wall():
    """After vans_set_eps the populations are f = w eps everywhere, also in the
    row under the moving plate (the initial state of the validation case)."""
    torch = torch_cuda()
    p, eps = W.couette_80(Re=50, Da=1e-2, nx=16)
    s = solver(p, eps)
    f = s.populations().cpu().numpy()
    w = W.lattice_weights(9).reshape(9, 1, 1, 1)
    assert np.abs(f - w * eps[None].astype(np.float64)).max() <= 1e-8


@pytest.mark.parametrize("q,shape,wm,uw,L", [(9, (1, 30, 41), 2, (0.0, 0.0, 0.0), None),
                                           (9, (1, 24, 33), 2, (0.01, 0.0, 0.0), None),
                                           (19, (8, 10, 17), 6, (0.0, 0.0, 0.0), None),
                                           # rows of one tile staged without their halos
                                           (19, (6, 8, 32), 6, (0.01, 0.0, 0.0),
                                            Launch(2, 4, 2, 7))])
def test_porosity_varying_in_time(q, shape, wm, uw, L):
    """eps(x, t): the field changes every few steps (a translating smoothed
    field) while the populations carry on; the oracle runs the same schedule
    on its own state.  Velocity within 1e-5 after 60 steps."""
    torch = torch_cuda()
    import oracle as O
    nz, ny, nx = shape
    p = W.params(q=q, nx=nx, ny=ny, nz=nz, wall_mask=wm, tau=0.7, g=(4e-5, 0, 0),
                 drag_mode=2, k_mode=0, d_p=6.0, u_wall=uw)
    base = W.smoothed_noise(shape, 3.0, 0.4, 1.0, seed=51)
    fields = [np.ascontiguousarray(np.roll(base, k, axis=2)) for k in range(6)]
    s = solver(p, fields[0], launch=L)
    po = O.Params(**p)
    f = O.init(po, fields[0].astype(np.float64))
    for k, e in enumerate(fields):
        if k:
            s.update_eps(torch.from_numpy(e).cuda().view(-1))
        s.step(10)
        f = O.run(po, e.astype(np.float64), f, 10)
    rho, u = s.moments()
    torch.cuda.synchronize()
    rho_o, u_o = O.moments(po, fields[-1].astype(np.float64), f)
    assert rel_u(u.cpu().numpy().astype(np.float64), u_o) <= 1e-5
    assert np.abs(rho.cpu().numpy() - rho_o).max() <= 1e-5
    # the populations survive the update itself
    fa = s.populations()
    s.update_eps(torch.from_numpy(fields[0]).cuda().view(-1))
    fb = s.populations()
    torch.cuda.synchronize()
    assert (fa - fb).abs().max().item() <= 1e-7


def test_monitored_steps_emit_the_moments_and_reductions():
    """vans_step_monitored: the moments written by the step kernel equal those of
    vans_moments on the same state, the run itself matches plain steps, and the
    in-kernel reductions report max |u|, the change since the last emission,
    the number of emissions and a divergence."""
    torch = torch_cuda()
    p, eps, _ = W.periodic_2d_shape(150, 70, nsteps=0)
    a = solver(p, eps)
    b = solver(p, eps)
    a.step(40)
    rho_ref, u_ref = a.moments()                 # state after 40 steps
    rho, u, st = b.step_monitored(41, 41)        # one emission, reading the state after 40
    torch.cuda.synchronize()
    assert (rho - rho_ref).abs().max().item() <= 1e-6
    assert (u - u_ref).abs().max().item() <= 1e-6 * u_ref.abs().max().item() + 1e-12
    s = st.cpu().numpy()
    assert s[3] == 1.0 and s[2] == 0.0
    assert abs(s[1] - float(torch.linalg.vector_norm(u_ref, dim=0).max())) <= 1e-6 * s[1]
    assert abs(s[0] - s[1]) <= 1e-6 * s[1]       # previous u was zero
    a.step(1)
    assert (a.populations() - b.populations()).abs().max().item() <= 1e-7
    # several emissions; converging flow reports a small change between them
    rho, u, st = b.step_monitored(300, 100, rho, u)
    s = st.cpu().numpy()
    assert s[3] == 3.0 and 0.0 < s[0] < s[1]
    # a non-finite state is flagged
    f = b.populations()
    f[2, 0, 5, 5] = float("nan")
    b.set_populations(f)
    _, _, st = b.step_monitored(1, 1, rho, u)
    assert st[2].item() == 1.0


@pytest.mark.parametrize("q,shape,wm", [(9, (1, 70, 150), 0), (9, (1, 37, 53), 2),
                                        (19, (12, 10, 30), 6)])
def test_monitored_emission_matches_the_oracle(q, shape, wm):
    """F1 against the FP64 oracle: 60 monitored steps from rest with an emission
    every 20 steps.  The emissions read the states after 19, 39 and 59 steps;
    the last one's rho and u are the oracle's moments of the state after 59
    steps, and the reductions are the oracle's: max over cells and emissions of
    |u| and of |u - u_prev| (u_prev = zero before the first emission)."""
    torch = torch_cuda()
    nz, ny, nx = shape
    p = W.params(q=q, nx=nx, ny=ny, nz=nz, wall_mask=wm, tau=0.62, g=(4e-5, 1e-5, -1e-5),
                 drag_mode=2, k_mode=0, d_p=W.D_P)
    eps = W.smoothed_noise(shape, 6.0, 0.4, 1.0, seed=sum(shape))
    s = solver(p, eps)
    rho, u, st = s.step_monitored(60, 20)
    torch.cuda.synchronize()
    po = O.Params(**p)
    e64 = eps.astype(np.float64)
    f = O.init(po, e64)
    us, prev, dmax, umax = [], 0.0, 0.0, 0.0
    for n in (19, 20, 20):
        f = O.run(po, e64, f, n)
        rho_o, u_o = O.moments(po, e64, f)
        dmax = max(dmax, float(np.sqrt(((u_o - prev) ** 2).sum(axis=0)).max()))
        umax = max(umax, float(np.sqrt((u_o ** 2).sum(axis=0)).max()))
        prev = u_o
        us.append(u_o)
    assert rel_u(u.cpu().numpy().astype(np.float64), us[-1]) <= 1e-5
    assert np.abs(rho.cpu().numpy() - rho_o).max() <= 1e-6
    got = st.cpu().numpy().astype(np.float64)
    assert got[3] == 3.0 and got[2] == 0.0
    assert abs(got[1] - umax) <= 1e-5 * umax
    assert abs(got[0] - dmax) <= 1e-5 * umax


def test_cta_cap_refusals_and_roundtrip():
    """ctas (CTAs per SM) is taken by the pipelined kinds only, within 1..4;
    the reverse step takes none; a capped shape reads back unchanged."""
    torch_cuda()
    p, eps, _ = W.periodic_2d_shape(64, 16, nsteps=0)
    s = solver(p, eps)
    for L in (Launch(4, 4, 1, 0, 1), Launch(4, 4, 2, 7, 5), Launch(4, 4, 2, 7, -1),
              Launch(2, 4, 3, 1), Launch(4, 4, 3, 3),       # kinds 1 and 3 are not built
              Launch(4, 6, 2, 7)):                          # 6 warps: D3Q19 only
        with pytest.raises(VansError):
            s.launch = L
    with pytest.raises(VansError):
        s.set_adjoint_launch(Launch(1, 4, 4, 1, 2))
    s.launch = Launch(4, 4, 2, 7, 2)
    assert s.launch == Launch(4, 4, 2, 7, 2)
