"""GB300 (sm_103a) lattice Boltzmann solver for the volume-averaged
Navier-Stokes equations (Zhang, Wang & Ouyang).

The compute path is libvans.so (hand-written CUDA kernels behind the C ABI of
include/vans.h).  This package only marshals arguments to it:

    Solver   one domain (D2Q9 or D3Q19): set_eps, step, moments, populations,
             checkpoints, adjoint step, outlet flux
    Batch    many independent D2Q9 domains, one persistent kernel per step
    adjoint  torch.autograd.Function for d(outlet flux)/d(eps)
    workloads  seeded synthetic inputs (porosity fields, domain sizes)
"""
from ._binding import Batch, Launch, Params, Solver, VansError, load_library  # noqa: F401
from . import workloads  # noqa: F401

__all__ = ["Batch", "Launch", "Params", "Solver", "VansError", "load_library", "workloads"]
