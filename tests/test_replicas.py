"""The multi-process (replica) path of bench.py on CPU with the gloo backend,
world size 2: each rank runs its own replica, the job reports the slowest
rank's times and the pairs summed over ranks; the reference arm runs on rank 0
only and the other ranks leave without work."""
import argparse
import os
import socket
import sys

import pytest

from conftest import ROOT


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    out = bench.combine_ranks(ms=10.0 + rank, e2e=20.0 + 3 * rank, pairs=1000 * (rank + 1), device="cpu")
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, out))


def test_combine_ranks_gloo_world_size_2():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        assert res[r] == (11.0, 23.0, 3000.0)


def test_combine_ranks_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_ranks(5.0, 7.0, 42, "cpu") == (5.0, 7.0, 42.0)


def test_reference_arm_runs_on_rank_0_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    args = argparse.Namespace(steps=2, warmup=3, ref_points=8, gpus=2, impl="reference", cpu_seconds=1.0)
    assert bench.run_reference(args) is None
    assert capsys.readouterr().out == ""
