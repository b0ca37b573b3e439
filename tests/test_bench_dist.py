"""The multi-rank (replicas) path of bench.py on CPU with the gloo backend, world size 2: every
rank learns the slowest rank's time, the whole-job rate counts every rank's maps over that time,
ranks draw disjoint maps, and in the reference arm only rank 0 works and prints."""
import argparse
import contextlib
import io
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t_ms = 100.0 + 50.0 * rank           # rank 1 is the slow one
        t_max = bench.max_over_ranks(t_ms, world, "cpu")
        rate = bench.whole_job_rate(world, 32, 2, t_max)
        seeds = bench.rank_map_seeds(rank, 4)
        out = io.StringIO()
        args = argparse.Namespace(L=64, lam=2.0, J0=2, B=4, steps=1, warmup=0, gpus=world, unrotated=False,
                                  mode="mixed")
        with contextlib.redirect_stdout(out):
            if rank != 0:
                bench.run_reference(args, rank, world)
        dist.barrier()
        q.put((rank, t_max, rate, seeds, out.getvalue()))
    finally:
        dist.destroy_process_group()


def test_replicas_max_time_rate_and_rank_work():
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, v0, s0, o0), (r1, t1, v1, s1, o1) = res
    assert t0 == t1 == 150.0                  # both ranks see the slowest rank's time
    assert v0 == v1 == pytest.approx(2 * 32 * 2 / 0.150)
    assert not set(s0) & set(s1)              # disjoint maps per rank
    assert o1 == ""                           # the reference arm: rank 1 does nothing


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, 1, "cpu") == 12.5
    assert bench.whole_job_rate(1, 32, 2, 1000.0) == 64.0
