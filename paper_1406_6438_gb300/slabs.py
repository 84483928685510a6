"""Domains cut along x into slabs: one solver handle per slab, on one GPU or one
slab per rank.

x is the periodic axis of every domain here, so a cut never meets a wall.  The
update of a cell needs only its neighbours' post-collision populations (the
final LBE), so across a cut only the populations that stream over it move,
once per step.  One step of a slab: ``vans_step(h, 1)``; ``vans_halo_pack``
(its last column's e_x = +1 populations go right, its first column's e_x = -1
populations go left); the exchange of the messages; ``vans_halo_unpack``.
The exchange is the caller's part of the cycle: a device copy between slabs on
one GPU (``Slabs``), point-to-point sends and receives between ranks through
``torch.distributed`` (``DistributedSlab``, NCCL between GPUs).
"""
from __future__ import annotations

import numpy as np

from ._binding import Params, Solver, _torch


def cut_points(nx: int, nslabs: int):
    """Column ranges [x0, x1) of nslabs slabs of nearly equal width (>= 1)."""
    if not 1 <= nslabs <= nx:
        raise ValueError(f"cannot cut {nx} columns into {nslabs} slabs")
    edges = [nx * k // nslabs for k in range(nslabs + 1)]
    return [(edges[k], edges[k + 1]) for k in range(nslabs)]


def halo_exchange(to_left, to_right, from_left, from_right, rank: int, world: int, group=None):
    """One step's exchange between the ranks of a ring of slabs (rank r's
    neighbours are r - 1 and r + 1, modulo world): to_right goes to the right
    neighbour, where it is from_left, and to_left to the left neighbour, where
    it is from_right.  The four operations are issued as one batch in the same
    order on every rank, rightward messages with tag 0 and leftward ones with
    tag 1, so they pair up whether the backend matches by tag (gloo) or by call
    order per peer (NCCL, also when both neighbours are the same rank).  A
    single rank is its own neighbour on both sides."""
    if world == 1:
        from_left.copy_(to_right)
        from_right.copy_(to_left)
        return
    import torch.distributed as dist
    right, left = (rank + 1) % world, (rank - 1) % world
    ops = [dist.P2POp(dist.isend, to_right, right, group, 0),
           dist.P2POp(dist.isend, to_left, left, group, 1),
           dist.P2POp(dist.irecv, from_left, left, group, 0),
           dist.P2POp(dist.irecv, from_right, right, group, 1)]
    for req in dist.batch_isend_irecv(ops):
        req.wait()


def _columns(eps: np.ndarray, x: int) -> np.ndarray:
    """Column x (periodic) of a [nz, ny, nx] field as ny * nz values, row = z * ny + y."""
    return np.ascontiguousarray(eps[:, :, x % eps.shape[2]]).reshape(-1)


class Slabs:
    """A domain cut into slabs along x on one GPU.  Every slab is a Solver of
    its own width; all of them enqueue on the stream current at construction,
    as do the device copies that stand for the exchange, so the cycle of a step
    is ordered by the stream alone."""

    def __init__(self, params, eps: np.ndarray, nslabs: int = 2, cuts=None, launch=None):
        torch = _torch()
        self.params = Params.of(params)
        p = self.params
        eps = np.asarray(eps, dtype=np.float32).reshape(p.shape)
        self.cuts = cuts if cuts is not None else cut_points(p.nx, nslabs)
        self.stream = torch.cuda.current_stream()
        self.slabs = []
        for x0, x1 in self.cuts:
            q = Params(**dict(p.as_dict(), nx=x1 - x0))
            s = Solver(q)
            dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda().view(-1)  # noqa: E731
            s.set_eps_slab(dev(eps[:, :, x0:x1]), dev(_columns(eps, x0 - 1)), dev(_columns(eps, x1)))
            if launch is not None:
                s.launch = launch
            self.slabs.append(s)
        n = self.slabs[0].halo_floats
        buf = lambda: [torch.empty(n, dtype=torch.float32, device="cuda") for _ in self.slabs]  # noqa: E731
        self.to_left, self.to_right, self.from_left, self.from_right = buf(), buf(), buf(), buf()

    def step(self, nsteps: int = 1):
        torch = _torch()
        S = len(self.slabs)
        with torch.cuda.stream(self.stream):
            for _ in range(nsteps):
                for k, s in enumerate(self.slabs):
                    s.step(1)
                    s.halo_pack(self.to_left[k], self.to_right[k])
                for k in range(S):          # the exchange: device copies between the slabs
                    self.from_left[k].copy_(self.to_right[(k - 1) % S])
                    self.from_right[k].copy_(self.to_left[(k + 1) % S])
                for k, s in enumerate(self.slabs):
                    s.halo_unpack(self.from_left[k], self.from_right[k])

    def populations(self):
        """Physical populations of the whole domain, [q, nz, ny, nx]."""
        torch = _torch()
        return torch.cat([s.populations() for s in self.slabs], dim=3)

    def moments(self):
        torch = _torch()
        parts = [s.moments() for s in self.slabs]
        return (torch.cat([r for r, _ in parts], dim=2), torch.cat([u for _, u in parts], dim=3))

    def close(self):
        for s in self.slabs:
            s.close()


class DistributedSlab:
    """Slab ``rank`` of a domain cut into ``world`` slabs, one per rank and
    GPU; the exchange runs through torch.distributed (NCCL) point-to-point
    operations, which follow the solver's stream."""

    def __init__(self, params, eps: np.ndarray, rank: int, world: int, group=None, launch=None):
        torch = _torch()
        self.params = Params.of(params)
        p = self.params
        eps = np.asarray(eps, dtype=np.float32).reshape(p.shape)
        self.rank, self.world, self.group = rank, world, group
        self.x0, self.x1 = cut_points(p.nx, world)[rank]
        q = Params(**dict(p.as_dict(), nx=self.x1 - self.x0))
        self.solver = Solver(q)
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda().view(-1)  # noqa: E731
        self.solver.set_eps_slab(dev(eps[:, :, self.x0:self.x1]), dev(_columns(eps, self.x0 - 1)),
                                 dev(_columns(eps, self.x1)))
        if launch is not None:
            self.solver.launch = launch
        n = self.solver.halo_floats
        self.bufs = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(4)]

    def step(self, nsteps: int = 1):
        to_left, to_right, from_left, from_right = self.bufs
        for _ in range(nsteps):
            self.solver.step(1)
            self.solver.halo_pack(to_left, to_right)
            halo_exchange(to_left, to_right, from_left, from_right, self.rank, self.world, self.group)
            self.solver.halo_unpack(from_left, from_right)
