"""The halo exchange schedule of slabs along x, on CPU with gloo ranks.

Each rank stands for one slab of a ring: after one exchange, a rank's
from_left must hold its left neighbour's to_right and its from_right its right
neighbour's to_left, for rings of 1, 2 (both neighbours the same rank) and 3
ranks, over several exchanges in a row.  The CUDA pack and unpack of the
messages are tested on the GPU (tests/test_gpu_slabs.py); the cut points and
the porosity columns the slabs are given are checked here too."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_1406_6438_gb300.slabs import _columns, cut_points, halo_exchange


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _message(rank, side, step, n=7):
    # a message that names its sender, its direction and the step
    return torch.arange(n, dtype=torch.float32) + 1000.0 * rank + 100.0 * side + 10.0 * step


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ok = True
    for step in range(3):
        to_left, to_right = _message(rank, 0, step), _message(rank, 1, step)
        from_left, from_right = torch.full((7,), -1.0), torch.full((7,), -1.0)
        halo_exchange(to_left, to_right, from_left, from_right, rank, world)
        left, right = (rank - 1) % world, (rank + 1) % world
        ok = ok and torch.equal(from_left, _message(left, 1, step))
        ok = ok and torch.equal(from_right, _message(right, 0, step))
    q.put((rank, ok))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_ring_exchange_delivers_each_message_to_its_neighbour(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(world))
    assert out == [(r, True) for r in range(world)]


def test_single_slab_is_its_own_neighbour():
    to_left, to_right = _message(0, 0, 0), _message(0, 1, 0)
    from_left, from_right = torch.zeros(7), torch.zeros(7)
    halo_exchange(to_left, to_right, from_left, from_right, 0, 1)
    assert torch.equal(from_left, to_right) and torch.equal(from_right, to_left)


def test_cut_points_and_edge_columns():
    assert cut_points(10, 3) == [(0, 3), (3, 6), (6, 10)]
    assert cut_points(5, 5) == [(k, k + 1) for k in range(5)]
    with pytest.raises(ValueError):
        cut_points(4, 5)
    eps = np.arange(2 * 3 * 5, dtype=np.float32).reshape(2, 3, 5)   # [nz, ny, nx]
    # the column left of slab [0, x1) is the domain's last (periodic x), row = z * ny + y
    assert np.array_equal(_columns(eps, -1), eps[:, :, 4].reshape(-1))
    assert np.array_equal(_columns(eps, 5), eps[:, :, 0].reshape(-1))
    assert _columns(eps, 2)[4] == eps[1, 1, 2]
