"""The multi-GPU path of bench.py is replicas only (independent MGVI systems,
no exchange step): every rank times the same work and the job reports all
ranks' units over the slowest rank's time.  These CPU tests run that host
logic on two gloo ranks (no GPU)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        t_local = [0.5, 0.8][rank]  # the second rank is slower
        t_max = bench.max_over_ranks(t_local, world, torch.device("cpu"))
        value = bench.replica_throughput(1000, world, t_max)
        out.put((rank, t_max, value))
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas_report_slowest_rank():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t_max, value in res:
        assert t_max == 0.8
        assert value == pytest.approx(2 * 1000 / 0.8)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(0.3, 1, None) == 0.3
    assert bench.replica_throughput(10, 1, 0.5) == 20.0
