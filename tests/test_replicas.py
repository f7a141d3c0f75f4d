"""The multi-GPU form of the benchmark is independent replicas (one per rank,
no data exchange).  Its host logic -- barrier bracket, max over ranks, whole-job
throughput -- checked with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    bench._barrier_sync(torch)
    seconds = 0.5 + 0.25 * rank                    # rank 1 is the slower replica
    v = bench.replica_value(torch, 1000.0, seconds)
    m = bench._max_over_ranks(torch, seconds)
    bench._barrier_sync(torch)
    out[rank] = (v, m)
    dist.destroy_process_group()


def test_two_replicas_whole_job_value():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    # both ranks agree: 2 x 1000 points over the slowest rank's 0.75 s
    for r in range(2):
        v, m = out[r]
        assert m == 0.75 and abs(v - 2000.0 / 0.75) < 1e-9


def test_single_process_is_identity():
    import bench
    assert bench.replica_value(torch, 10.0, 2.0) == 5.0
    assert bench._max_over_ranks(torch, 3.0) == 3.0
