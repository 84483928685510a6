"""The multi-rank path of bench.py on CPU: two gloo ranks (world_size 2) take
the slowest rank's time and sum the cells of both replicas, and the reference
arm does no work on ranks other than 0."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.max_over_ranks(0.5 + rank, dist, "cpu")      # rank r timed 0.5 + r s
    q.put((rank, t, bench.job_mlups(world, 1000, 10, t)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t, v in out:
        assert t == 1.5                                     # the slower rank's time
        assert v == pytest.approx(2 * 1000 * 10 / 1.5 / 1e6)


def test_single_process_needs_no_group():
    assert bench.max_over_ranks(0.25, None, "cpu") == 0.25
    assert bench.job_mlups(1, 16777216, 1000, 0.2) == pytest.approx(83886.08)


def test_reference_arm_idles_on_nonzero_ranks(monkeypatch):
    monkeypatch.setenv("RANK", "1")

    class A:
        steps, warmup, gpus = 5, 3, 2

    assert bench.reference_arm(A()) == 0


def test_reference_arm_prints_one_json_line_on_cpu():
    """`bench.py --impl reference` (the FP64 oracle on host cores) needs no GPU
    and prints one JSON line with the keys the contract names."""
    import json
    import subprocess
    import sys
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "MLUPS" and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["higher_is_better"] is True and d["steps"] == 1
