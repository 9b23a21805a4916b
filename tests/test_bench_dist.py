"""The multi-rank host logic of bench.py on CPU (gloo, world size 2): ranks
reach the barriers, the timed region takes the maximum over ranks and the
work sums over ranks (replicas; no data-path collective)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      CTD_BENCH_BACKEND="gloo")
    import bench
    r, w = bench.dist_init(world)
    bench.barrier(w)
    t = bench.max_over_ranks(1.0 + r, w)
    n = bench.sum_over_ranks(10.0 * (r + 1), w)
    out.put((r, w, t, n))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_rank_replicas_reduce_time_and_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, 2, 2.0, 30.0), (1, 2, 2.0, 30.0)]
