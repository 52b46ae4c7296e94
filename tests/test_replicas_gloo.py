"""Multi-GPU runs of bench.py are independent replicas (the transform has no
exchange step here): each rank times the full workload on its own GPU, the
ranks agree on the slowest rank's time with one MAX all-reduce, and the
whole-job throughput is the points of all ranks over that time.  This checks
that aggregation with two CPU ranks on the gloo backend (no GPU)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                       "RANK": str(rank), "WORLD_SIZE": str(ws), "LOCAL_RANK": str(rank)})
    import torch
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        got_ws, got_rank, got_local = bench._dist()
        ms = [0.30, 0.45][rank]  # rank 1 is the slowest replica
        slowest = bench.ranks_max(ms, got_ws, torch.device("cpu"))
        value = bench.replica_throughput(2 << 20, slowest, got_ws)
        out.put((rank, got_ws, got_rank, got_local, slowest, value))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_time():
    import torch.multiprocessing as mp
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
    for rank, ws, got_rank, local, slowest, value in res:
        assert (ws, got_rank, local) == (2, rank, rank)
        assert slowest == pytest.approx(0.45)
        assert value == pytest.approx(2 * (2 << 20) / 0.45e-3)


def test_single_replica_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.ranks_max(0.3, 1, None) == 0.3
    assert bench.replica_throughput(100, 1.0, 1) == pytest.approx(1e5)
