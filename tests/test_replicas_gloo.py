"""Host logic of the multi-GPU bench (independent replicas, weak scaling) on
CPU with two gloo ranks: distinct seeds per rank, and the job throughput =
cell updates summed over ranks / slowest rank's time."""
import datetime
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=60))
    updates = [3_000_000, 5_000_000][rank]
    ms = [100.0, 250.0][rank]
    value, ms_max = bench.job_throughput(updates, ms, dist, "cpu")
    q.put((rank, bench.replica_seed(4, rank), value, ms_max))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_throughput_and_distinct_seeds():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        res = sorted(q.get(timeout=120) for _ in procs)
        for p in procs:
            p.join(timeout=60)
            assert p.exitcode == 0
    finally:
        for p in procs:
            if p.is_alive():
                p.kill()
    (r0, s0, v0, m0), (r1, s1, v1, m1) = res
    assert s0 != s1
    assert m0 == m1 == 250.0
    assert v0 == v1 == pytest.approx(8_000_000 / 0.25 / 1e9)


def test_single_process_throughput():
    v, ms = bench.job_throughput(1_000_000, 10.0)
    assert ms == 10.0 and v == pytest.approx(0.1)
