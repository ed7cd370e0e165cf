"""Host logic of the multi-rank benchmark (replicas only: every rank runs
the whole workload, the job's step time is the slowest rank's, the job's
throughput is the work of all ranks over that time), checked with two gloo
ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [3.5, 7.25][rank]
        got = bench.max_over_ranks(ms, dist, "cpu")
        out.put((rank, got, bench.replicas_throughput(2e9, world, got)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [7.25, 7.25]
    # 2 replicas x 2 GFLOP in 7.25 ms
    assert res[0][2] == pytest.approx(2 * 2e9 / 7.25e-3 / 1e9)


def test_single_rank_is_local_time():
    assert bench.max_over_ranks(4.0, None, "cpu") == 4.0
    assert bench.replicas_throughput(1e9, 1, 2.0) == pytest.approx(500.0)
