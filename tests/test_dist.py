"""The multi-rank host logic of bench.py on CPU: two gloo ranks set up the
process group from the torchrun environment, take the max over ranks of
their timings, pass the barrier, and aggregate weak-scaling throughput."""
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


def _rank(rank, world, port, q):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist

    class A:
        impl = "ours"

    w, r, loc = bench.dist_setup(A())
    assert (w, r, loc) == (world, rank, rank)
    assert dist.get_backend() == "gloo"
    got = bench.max_over_ranks(10.0 + rank, w)
    bench.barrier(w)
    rate = bench.aggregate_rate(1000, 2.0, w)
    q.put((rank, got, rate))
    dist.destroy_process_group()


def test_two_rank_gloo_timing_and_aggregation():
    import torch.multiprocessing as mp
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    res = sorted(q.get(timeout=5) for _ in range(world))
    assert [r[1] for r in res] == [11.0, 11.0]          # max over ranks on every rank
    assert [r[2] for r in res] == [1000.0, 1000.0]      # 2 ranks x 1000 units / 2 s
