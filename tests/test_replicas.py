"""Multi-GPU is replicas only: the factorization does not shard, N ranks run N
independent copies and the job throughput uses the slowest rank's time.
The host-side logic of bench.py is exercised here with two gloo ranks on CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    ms = 100.0 + 50.0 * rank  # rank 1 is the slow one
    bench.barrier(ws)
    m = bench.max_over_ranks(ws, ms)
    v = bench.job_value(2.0e12, 4, ws, m)
    out[rank] = (m, v)
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_job_value():
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
    for r in range(2):
        m, v = out[r]
        assert m == 150.0
        assert v == pytest.approx(2.0e12 * 4 * 2 / 0.150)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(1, 3.5) == 3.5
    assert bench.job_value(1e12, 2, 1, 1000.0) == pytest.approx(2e12)
