"""The benchmark's multi-rank logic on CPU: two gloo ranks (replicas), the job
time is the slowest rank's, and the job value counts every rank's work."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, ws, port, ms_by_rank, out):
    import torch.distributed as dist
    import bench
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(ws), "LOCAL_RANK": str(rank)})
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    ms = bench.reduce_max_ms(ms_by_rank[rank], ws, device="cpu")
    dist.barrier()
    out.put((rank, ms, bench.job_value(1000, ws, ms)))
    dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ms_by_rank = [12.5, 20.0]
    procs = [ctx.Process(target=_rank, args=(r, 2, port, ms_by_rank, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, val in res:
        assert ms == 20.0
        assert val == pytest.approx(1000 * 2 / 0.020)


def test_single_rank_identity():
    import bench
    assert bench.reduce_max_ms(7.0, 1) == 7.0
    assert bench.job_value(500, 1, 10.0) == pytest.approx(50000.0)
