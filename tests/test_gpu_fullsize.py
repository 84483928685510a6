"""Parity at the full sizes of the benchmark workloads, in the launch
configuration bench.py uses (the autotuner's pick): every cell against the
FP64 oracle for a few steps (the oracle finishes them in seconds on the host
cores), and properties that hold at any length for the long runs."""
import numpy as np
import pytest

from paper_1406_6438_gb300 import workloads as W
from tests._gpu import oracle_run, rel_u, torch_cuda

pytestmark = pytest.mark.gpu


def _autotuned(p, eps):
    torch = torch_cuda()
    import paper_1406_6438_gb300 as V
    s = V.Solver(p)
    s.set_eps(torch.from_numpy(eps).cuda().view(-1))
    s.autotune()
    return s


def test_periodic_4096_every_cell_after_200_steps():
    """The 4096^2 workload, 200 of its 1000 steps (the oracle takes about a
    minute of host time for them), every population, rho and u against the
    FP64 oracle."""
    torch = torch_cuda()
    p, eps, _ = W.periodic_2d(4096)
    s = _autotuned(p, eps)
    s.step(200)
    rho, u = s.moments()
    f = s.populations()
    torch.cuda.synchronize()
    rho_o, u_o, f_o = oracle_run(p, eps, 200)
    err_f = float(np.abs(f.cpu().numpy() - f_o).max())
    err_u = rel_u(u.cpu().numpy().astype(np.float64), u_o)
    err_r = float(np.abs(rho.cpu().numpy() - rho_o).max())
    print(f"4096^2 x 200: f {err_f:.2e}, u {err_u:.2e}, rho {err_r:.2e}, launch {s.launch}")
    assert err_f <= 1e-6 and err_u <= 1e-5 and err_r <= 2e-6, (err_f, err_u, err_r)


def test_periodic_4096_long_run_properties():
    """1000 steps (the workload's length): finite, subsonic, mass conserved to
    FP32 rounding, and the monitoring step's reductions agree."""
    torch = torch_cuda()
    p, eps, n = W.periodic_2d(4096)
    s = _autotuned(p, eps)
    m0 = s.populations().double().sum().item()
    rho, u, st = s.step_monitored(n, n)
    m1 = s.populations().double().sum().item()
    assert s.check()
    stats = st.cpu().numpy()
    assert stats[2] == 0.0 and stats[3] == 1.0 and 0.0 < stats[1] < 0.3
    assert abs(m1 - m0) <= 1e-6 * m0


def test_duct_256cubed_every_cell_after_50_steps():
    """The 256^3 duct, 50 of its 500 steps, every population, rho and u against
    the FP64 oracle."""
    torch = torch_cuda()
    p, eps, _ = W.duct_3d()
    s = _autotuned(p, eps)
    s.step(50)
    rho, u = s.moments()
    f = s.populations()
    torch.cuda.synchronize()
    rho_o, u_o, f_o = oracle_run(p, eps, 50)
    err_f = float(np.abs(f.cpu().numpy() - f_o).max())
    err_u = rel_u(u.cpu().numpy().astype(np.float64), u_o)
    err_r = float(np.abs(rho.cpu().numpy() - rho_o).max())
    print(f"256^3 x 50: f {err_f:.2e}, u {err_u:.2e}, rho {err_r:.2e}, launch {s.launch}")
    assert err_f <= 1e-6 and err_u <= 1e-5 and err_r <= 2e-6, (err_f, err_u, err_r)


def test_duct_256cubed_long_run_properties():
    """The duct's 500 steps (the workload's length) in the autotuned launch:
    finite, subsonic, mass conserved to FP32 rounding (bounce-back walls and a
    body force conserve it), and the monitoring step's reductions agree."""
    torch = torch_cuda()
    p, eps, n = W.duct_3d()
    s = _autotuned(p, eps)
    m0 = s.populations().double().sum().item()
    rho, u, st = s.step_monitored(n, n)
    m1 = s.populations().double().sum().item()
    assert s.check()
    stats = st.cpu().numpy()
    assert stats[2] == 0.0 and stats[3] == 1.0 and 0.0 < stats[1] < 0.3
    assert abs(m1 - m0) <= 1e-6 * m0
    speed = float(u.double().pow(2).sum(0).sqrt().max().item())
    assert abs(speed - float(stats[1])) <= 1e-5 * float(stats[1])


def test_batched_256_domains_sampled():
    """The 256-domain batch in its autotuned configuration: eight domains
    (the largest, the smallest and six drawn with a seed) against the oracle
    after 300 steps; every domain finite after the workload's 2000 steps."""
    torch = torch_cuda()
    import paper_1406_6438_gb300 as V
    doms = W.batched_channels()
    b = V.Batch([p for p, _ in doms])
    for d, (_, e) in enumerate(doms):
        b.set_eps(d, torch.from_numpy(e).cuda().view(-1))
    b.autotune()
    b.step(300)
    torch.cuda.synchronize()
    sizes = [p["nx"] * p["ny"] for p, _ in doms]
    pick = {int(np.argmax(sizes)), int(np.argmin(sizes))}
    pick |= set(int(k) for k in np.random.default_rng(7).choice(len(doms), 6, replace=False))
    for d in sorted(pick):
        p, e = doms[d]
        _, u_o, f_o = oracle_run(p, e, 300)
        f = b.populations(d).cpu().numpy()
        _, u = b.moments(d)
        assert np.abs(f - f_o).max() <= 1e-6, (d, np.abs(f - f_o).max())
        assert rel_u(u.cpu().numpy().astype(np.float64), u_o) <= 1e-5, d
    b.step(2000 - 300)
    assert b.check()
