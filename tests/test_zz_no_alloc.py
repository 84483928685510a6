"""vans_step_static: the one step that needs no workspace and allocates nothing.

Some callers cannot give the library device memory: code running inside
another framework's memory pool, code that may not call cudaMalloc while a CUDA
graph is being captured, or hosts with a fixed device-memory budget.  For them
the library keeps the step's only scratch (the padded porosity rows) in a fixed
16 MiB device array of its own.  These tests call that entry point through the
C ABI and check that two calls in a row give the same states as the ordinary
workspace-based step, and that a domain beyond the array's limit is refused.
This file is collected last on purpose (test_zz_*)."""
import ctypes

import numpy as np
import pytest

from paper_1406_6438_gb300 import workloads as W
from paper_1406_6438_gb300._binding import Launch, Params, load_library
from tests._gpu import solver, torch_cuda

pytestmark = pytest.mark.gpu

ATOL = 2e-7   # the population tolerance of the other GPU parity tests


def _lib():
    lib = load_library()
    fn = lib.vans_step_static
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                   ctypes.c_void_p]
    return lib


@pytest.mark.parametrize("case", ["d2q9", "d3q19"])
def test_static_step_matches_workspace_step_twice(case):
    torch = torch_cuda()
    lib = _lib()
    if case == "d2q9":
        p, eps, _ = W.periodic_2d_shape(150, 90, nsteps=0)
        p["wall_mask"] = 2
        default = Launch(4, 4, 1)
    else:
        p, eps, _ = W.duct_3d(nx=30, ny=20, nz=14, nsteps=0)
        default = Launch(2, 4, 1)
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


def test_static_step_refuses_domains_beyond_its_scratch():
    torch = torch_cuda()
    lib = _lib()
    p = Params(q=9, nx=2048, ny=2048, tau=0.7)   # 2048 rows x 2080 floats > 4 Mi floats
    dummy = torch.zeros(16, device="cuda")
    rc = lib.vans_step_static(ctypes.byref(p.c()), dummy.data_ptr(), dummy.data_ptr(),
                              dummy[8:].data_ptr(), None)
    assert rc == -1
