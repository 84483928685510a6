"""GPU batched step (one persistent launch per step over a tile list drawn from
many domains of uneven size, each with its own eps and tau) against the oracle
run domain by domain."""
import numpy as np
import pytest

from paper_1406_6438_gb300 import workloads as W
from paper_1406_6438_gb300._binding import Launch
from tests._gpu import oracle_run, rel_u, torch_cuda

pytestmark = pytest.mark.gpu


def _batch(doms):
    torch = torch_cuda()
    import paper_1406_6438_gb300 as V
    b = V.Batch([p for p, _ in doms])
    for d, (_, eps) in enumerate(doms):
        b.set_eps(d, torch.from_numpy(eps).cuda().view(-1))
    return b


def test_batched_matches_oracle_per_domain():
    torch = torch_cuda()
    doms = W.batched_channels(n=7, seed=41, nx_range=(5, 150), ny_range=(3, 60))
    b = _batch(doms)
    L = b.autotune()
    assert L.cpt in (1, 2, 4)
    nsteps = 150
    b.step(nsteps)
    torch.cuda.synchronize()
    for d, (p, eps) in enumerate(doms):
        rho_o, u_o, f_o = oracle_run(p, eps, nsteps)
        rho, u = b.moments(d)
        f = b.populations(d).cpu().numpy()
        assert np.abs(f - f_o).max() <= 5e-7, d
        assert rel_u(u.cpu().numpy(), u_o) <= 1e-5, d
        assert np.abs(rho.cpu().numpy() - rho_o).max() <= 1e-5, d


@pytest.mark.parametrize("L", [Launch(1, 2, 1), Launch(2, 1, 2), Launch(4, 4, 1), Launch(4, 2, 2),
                               Launch(4, 4, 3, 2), Launch(2, 8, 2, 2), Launch(1, 8, 3, 2),
                               Launch(2, 8, 2, 4), Launch(1, 8, 3, 4), Launch(4, 4, 4, 5),
                               Launch(4, 2, 2, 5), Launch(2, 4, 2, 6), Launch(2, 8, 3, 6),
                               Launch(4, 4, 4, 7), Launch(4, 2, 3, 7), Launch(4, 4, 2, 7, 2),
                               Launch(4, 4, 2, 5, 2)])
def test_batched_launch_shapes(L):
    torch = torch_cuda()
    doms = W.batched_channels(n=4, seed=43, nx_range=(20, 300), ny_range=(4, 40))
    b = _batch(doms)
    b.launch = L
    b.step(70)
    torch.cuda.synchronize()
    for d, (p, eps) in enumerate(doms):
        _, u_o, f_o = oracle_run(p, eps, 70)
        f = b.populations(d).cpu().numpy()
        assert np.abs(f - f_o).max() <= 5e-7, (L, d)


@pytest.mark.parametrize("L", [Launch(4, 4, 1), Launch(4, 4, 3, 2), Launch(4, 4, 4, 5),
                               Launch(4, 4, 4, 7)])
def test_batched_equals_single_domain_solver(L):
    """The batched kernels and the single-domain kernels run the same per-cell
    arithmetic (the compiler may contract a multiply-add differently in the two
    instantiations): populations within one FP32 ulp after a graph-replayed run."""
    torch = torch_cuda()
    import paper_1406_6438_gb300 as V
    doms = W.batched_channels(n=3, seed=44, nx_range=(60, 700), ny_range=(20, 90))
    b = _batch(doms)
    b.launch = L
    b.step(130)
    for d, (p, eps) in enumerate(doms):
        s = V.Solver(p)
        s.set_eps(torch.from_numpy(eps).cuda().view(-1))
        s.launch = L
        s.step(130)
        assert (s.populations() - b.populations(d)).abs().max().item() <= 6e-8


@pytest.mark.parametrize("L", [Launch(4, 4, 1), Launch(2, 4, 2, 4), Launch(4, 4, 2, 7),
                               Launch(2, 8, 2, 6)])
def test_batched_domains_with_moving_walls(L):
    """Domains whose upper wall moves (each at its own speed) next to resting
    ones in one batch: populations of every domain against the oracle."""
    torch = torch_cuda()
    doms = W.batched_channels(n=4, seed=45, nx_range=(30, 600), ny_range=(5, 50))
    speeds = [0.02, 0.0, 0.008, 0.015]
    doms = [(dict(p, u_wall=(W.f32(v), 0.0, 0.0)), e) for (p, e), v in zip(doms, speeds)]
    b = _batch(doms)
    b.launch = L
    b.step(60)
    torch.cuda.synchronize()
    for d, (p, eps) in enumerate(doms):
        _, u_o, f_o = oracle_run(p, eps, 60)
        f = b.populations(d).cpu().numpy()
        assert np.abs(f - f_o).max() <= 5e-7, (L, d)


@pytest.mark.parametrize("L", [Launch(2, 4, 3, 2), Launch(2, 4, 3, 4), Launch(4, 4, 2, 7),
                               Launch(4, 4, 2, 5, 2)])
def test_profiled_step_equals_a_step(L):
    """vans_batch_profile_step advances the batch exactly like one step (every
    population bitwise) and returns one timing record per CTA, from which the
    load balance lies in (0, 1]; the register-load kind has no records."""
    torch = torch_cuda()
    from paper_1406_6438_gb300._binding import VansError
    doms = W.batched_channels(n=9, seed=43, nx_range=(40, 700), ny_range=(8, 90))
    a, b = _batch(doms), _batch(doms)
    a.launch = L
    b.launch = L
    a.step(3)
    b.step(2)
    lb = b.profile_step()
    torch.cuda.synchronize()
    for d in range(len(doms)):
        assert torch.equal(a.populations(d), b.populations(d)), d
    assert lb["ctas"] > 0 and lb["sms_used"] > 0
    assert 0.0 < lb["efficiency"] <= 1.0 and lb["makespan_us"] > 0.0
    b.launch = Launch(4, 4, 1)
    with pytest.raises(VansError):
        b.profile_step()


def test_cta_cap_holds():
    """A persistent batched launch capped at 2 CTAs per SM puts at most 2 on any
    SM (from the profiled step's records); uncapped, the same shape fits more."""
    torch_cuda()
    doms = W.batched_channels(n=24, seed=44, nx_range=(200, 900), ny_range=(40, 200))
    b = _batch(doms)
    b.launch = Launch(4, 4, 2, 7, 2)
    capped = b.profile_step()
    b.launch = Launch(4, 4, 2, 7)
    free = b.profile_step()
    assert capped["max_ctas_per_sm"] <= 2 < free["max_ctas_per_sm"]
