"""The sharded run's host logic (paper_1109_3266_gb300.shard.run_sharded_with)
on CPU: two gloo ranks, each transporting its share of every batch with the
binary64 oracle in place of the device, summing the batch tallies with a gloo
all-reduce and folding the sum.  The result must be the single-process run of
the same problem: the same counts, and the same dose and standard error up to
the order of binary64 additions (Sec. 4: histories distributed among
processors that run without interfering; batch statistics of Sec. 2.2.1)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def problem():
    from paper_1109_3266_gb300 import inputs as I
    return I.head(n_hist=40_003, n_batches=7, seed=17, shape=(24, 24, 16), d=1.0)


class OracleShard:
    """One rank's transport and fold with the oracle (binary64), for the CPU test."""

    def __init__(self, p):
        from oracle import oracle as O
        self.O, self.p = O, p
        self.s = O.Setup(p, 64)
        self.mass = O.voxel_mass_kg(p.phantom)

    def begin(self, n_hist, seed, n_batches):
        from paper_1109_3266_gb300 import shard
        self.sizes = shard.batch_sizes(n_hist, n_batches)
        self.starts = np.concatenate([[0], np.cumsum(self.sizes)[:-1]]).astype(np.int64)
        self.sum_d = np.zeros(self.mass.size)
        self.sum_d2 = np.zeros(self.mass.size)
        self.counts_ = {k: 0 for k in self.O.COUNT_KEYS}
        self.e = np.zeros(2)

    def transport(self, b, lo, hi):
        import torch
        h0 = int(self.starts[b])
        edep, c = self.s.transport(h0 + lo, h0 + hi)
        for k in self.O.COUNT_KEYS:
            self.counts_[k] += c[k]
        self.e += [c["e_emitted"], c["e_escaped"]]
        return torch.from_numpy(edep)

    def fold(self, b, buf):
        d = self.O.dose_per_history(buf.numpy(), self.mass, self.sizes[b])
        self.sum_d += d
        self.sum_d2 += d * d

    def counts(self):
        return np.array([self.counts_[k] for k in self.O.COUNT_KEYS], dtype=np.uint64), self.e.copy()

    def finish(self, c, e):
        nb = len(self.sizes)
        D = self.sum_d / nb
        var = np.maximum(self.sum_d2 / nb - D * D, 0.0) * nb / (nb - 1)
        return {"dose": D, "std": np.sqrt(var / nb), "counts": dict(zip(self.O.COUNT_KEYS, c.tolist())),
                "energies": e}


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch
    import torch.distributed as dist

    from paper_1109_3266_gb300 import shard
    dist.init_process_group("gloo")
    p = problem()

    def tally(buf):
        dist.all_reduce(buf, op=dist.ReduceOp.SUM)

    def counts(c, e):
        tc = torch.from_numpy(c.astype(np.int64))
        te = torch.from_numpy(e)
        dist.all_reduce(tc, op=dist.ReduceOp.SUM)
        dist.all_reduce(te, op=dist.ReduceOp.SUM)
        return tc.numpy().astype(np.uint64), te.numpy()

    res = shard.run_sharded_with(OracleShard(p), p.n_hist, p.seed, p.n_batches, rank, world, tally, counts)
    out.put((rank, res["dose"], res["std"], res["counts"], res["energies"]))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_run_equals_single_process_run(oracle, world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for pr in ps:
        pr.start()
    res = sorted((q.get(timeout=300) for _ in ps), key=lambda x: x[0])
    for pr in ps:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    p = problem()
    ref = oracle.run(p, precision=64, threads=1)
    for _, dose, std, counts, energies in res:
        for k in oracle.COUNT_KEYS:
            assert counts[k] == ref.counts[k], k
        np.testing.assert_allclose(dose, ref.dose, rtol=1e-12, atol=0)
        m = ref.dose > 0.1 * ref.dose.max()
        np.testing.assert_allclose(std[m], ref.std[m], rtol=1e-6)
        assert energies[0] == pytest.approx(ref.counts["e_emitted"], rel=1e-12)


def test_shards_cover_every_history_once():
    from paper_1109_3266_gb300 import shard
    for n in (0, 1, 7, 1000, 10 ** 9 + 7):
        for world in (1, 2, 3, 8):
            parts = [shard.shard_of(n, r, world) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            assert all(parts[r][1] == parts[r + 1][0] for r in range(world - 1))
            assert all(0 <= hi - lo <= n // world + 1 for lo, hi in parts)
    assert sum(shard.batch_sizes(1003, 7)) == 1003
