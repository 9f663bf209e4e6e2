"""The multi-GPU path of bench.py is replicas only (one independent problem per
rank, no collective on the data path): its only cross-rank step is the timing
aggregation, checked here with two CPU ranks over gloo."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, times, out):
    import torch
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    t_ms, value = bench.aggregate_ranks(torch, dist, times[rank], ws, 3, torch.device("cpu"))
    out.put((rank, t_ms, value))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_timing_is_max_over_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    times = [1200.0, 1500.0]
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t_ms, value in res:
        assert t_ms == 1500.0  # the slowest rank
        assert value == pytest.approx(2 * 3 / 1.5)  # all ranks' solves / that time
