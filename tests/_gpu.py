"""Helpers shared by the GPU parity tests: run the CUDA path and the oracle on
the same seeded inputs and measure their differences."""
import numpy as np
import pytest

import oracle as O


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    return torch


def solver(params, eps, launch=None):
    torch = torch_cuda()
    import paper_1406_6438_gb300 as V
    s = V.Solver(params)
    s.set_eps(torch.from_numpy(np.ascontiguousarray(eps, dtype=np.float32)).cuda().view(-1))
    if launch is not None:
        s.launch = launch
    return s


def gpu_run(params, eps, nsteps, f0=None, launch=None):
    """Moments and populations after nsteps on the GPU (numpy, float64)."""
    torch = torch_cuda()
    s = solver(params, eps, launch)
    if f0 is not None:
        s.set_populations(torch.from_numpy(np.ascontiguousarray(f0, dtype=np.float32)).cuda())
    s.step(nsteps)
    rho, u = s.moments()
    f = s.populations()
    torch.cuda.synchronize()
    out = (rho.cpu().numpy().astype(np.float64), u.cpu().numpy().astype(np.float64),
           f.cpu().numpy().astype(np.float64))
    s.close()
    return out


def oracle_run(params, eps, nsteps, f0=None):
    p = O.Params(**params)
    e = np.asarray(eps, dtype=np.float64)
    f = O.init(p, e) if f0 is None else np.asarray(f0, dtype=np.float64)
    f = O.run(p, e, f, nsteps)
    rho, u = O.moments(p, e, f)
    return rho, u, f


def rel_u(u_gpu, u_ora):
    """max over cells and components of |u_gpu - u_ora| / max |u_ora|."""
    return float(np.abs(u_gpu - u_ora).max() / np.abs(u_ora).max())
