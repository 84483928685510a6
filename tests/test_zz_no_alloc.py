"""vans_step_static: the one step that needs no workspace and allocates nothing.

Some callers cannot give the library device memory: code running inside
another framework's memory pool, code that may not call cudaMalloc while a CUDA
graph is being captured, or hosts with a fixed device-memory budget.  For them
the library keeps the step's only scratch (the padded porosity rows) in a fixed
16 MiB device array of its own.  These tests call that entry point through the
C ABI and check that two calls in a row give the same states as the ordinary
workspace-based step (vans_step_raw on a handle) for every kind of boundary the
entry point accepts, and that domains beyond the array's limit and overlapping
buffers are refused.  This file is collected last on purpose (test_zz_*)."""
import ctypes

import numpy as np
import pytest

from paper_1406_6438_gb300 import workloads as W
from paper_1406_6438_gb300._binding import Launch, Params, load_library
from tests._gpu import solver, torch_cuda

ATOL = 2e-7   # the population tolerance of the other GPU parity tests


def _lib():
    lib = load_library()
    fn = lib.vans_step_static
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                   ctypes.c_void_p]
    return lib


def _case(case):
    """(params, eps, launch of the workspace step) of each boundary kind."""
    if case == "d2q9 channel":
        p, eps, _ = W.periodic_2d_shape(150, 90, nsteps=0)
        p["wall_mask"] = 2
        return p, eps, Launch(4, 4, 1)
    if case == "d2q9 fixed K, F_eps(eps)":
        p, eps, _ = W.periodic_2d_shape(77, 41, nsteps=0)
        p.update(wall_mask=2, k_mode=2, K=W.f32(3.5))
        return p, eps, Launch(4, 4, 1)
    if case == "d2q9 moving wall":
        p, eps, _ = W.periodic_2d_shape(96, 40, nsteps=0)
        p.update(wall_mask=2, u_wall=(W.f32(0.02), 0.0, 0.0))
        return p, eps, Launch(4, 4, 1)
    if case == "d2q9 plates on nodes":
        p, eps, _ = W.periodic_2d_shape(64, 33, nsteps=0)
        p.update(wall_mask=2, wall_kind=1, u_wall=(W.f32(0.01), 0.0, 0.0))
        return p, eps, Launch(4, 4, 1)
    if case == "d3q19 duct":
        p, eps, _ = W.duct_3d(nx=30, ny=20, nz=14, nsteps=0)
        return p, eps, Launch(2, 4, 1)
    if case == "d3q19 duct, moving wall":
        p, eps, _ = W.duct_3d(nx=24, ny=18, nz=12, nsteps=0)
        p.update(u_wall=(W.f32(0.015), 0.0, W.f32(0.005)))
        return p, eps, Launch(2, 4, 1)
    if case == "d3q19 128^3, the largest cube":
        p, eps, _ = W.duct_3d(nx=128, ny=128, nz=128, nsteps=0)
        return p, eps, Launch(2, 4, 1)
    raise ValueError(case)


CASES = ["d2q9 channel", "d2q9 fixed K, F_eps(eps)", "d2q9 moving wall", "d2q9 plates on nodes",
         "d3q19 duct", "d3q19 duct, moving wall", "d3q19 128^3, the largest cube"]


@pytest.mark.gpu
@pytest.mark.parametrize("case", CASES)
def test_static_step_matches_workspace_step_twice(case):
    torch = torch_cuda()
    lib = _lib()
    p, eps, default = _case(case)
    s = solver(p, eps, launch=default)
    s.step(25)                                   # a state away from rest
    st = s.get_state()
    ref1, ref2 = s.new_state(), s.new_state()
    s.step_raw(st, ref1)
    s.step_raw(ref1, ref2)
    out1, out2 = s.new_state(), s.new_state()
    eps_dev = torch.from_numpy(np.ascontiguousarray(eps)).cuda().view(-1)
    cp = Params.of(p).c()
    stream = torch.cuda.current_stream().cuda_stream
    assert lib.vans_step_static(ctypes.byref(cp), eps_dev.data_ptr(), st.data_ptr(),
                                out1.data_ptr(), stream) == 0
    assert lib.vans_step_static(ctypes.byref(cp), eps_dev.data_ptr(), out1.data_ptr(),
                                out2.data_ptr(), stream) == 0
    torch.cuda.synchronize()
    assert (out1 - ref1).abs().max().item() <= ATOL
    assert (out2 - ref2).abs().max().item() <= ATOL
    assert (ref2 - st).abs().max().item() > 0    # the steps did move the state


def test_static_step_refuses_domains_beyond_its_scratch_and_overlapping_buffers():
    """Refusals happen before any CUDA call, so this runs without a GPU: the
    pointers are never dereferenced."""
    lib = _lib()
    a, b, e = 1 << 32, 1 << 40, 1 << 36          # far apart, never touched
    big = Params(q=9, nx=2048, ny=2048, wall_mask=2, tau=0.7)   # 2048 rows x 2080 floats > 4 Mi
    assert lib.vans_step_static(ctypes.byref(big.c()), e, a, b, None) == -1
    cube = Params(q=19, nx=129, ny=129, nz=129, wall_mask=6, tau=0.7)   # pitch 320: 5.3 Mi floats
    assert lib.vans_step_static(ctypes.byref(cube.c()), e, a, b, None) == -1
    small = Params(q=9, nx=100, ny=50, wall_mask=2, tau=0.7)
    n = lib.vans_state_floats(ctypes.byref(small.c()))
    assert n > 0
    for out in (a, a + 4 * (n - 1), a - 4 * (n - 1)):   # equal or partly overlapping ranges
        assert lib.vans_step_static(ctypes.byref(small.c()), e, a, out, None) == -1
