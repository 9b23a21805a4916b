"""The sharded run (ctd_shard_*, paper_1109_3266_gb300.shard) on one GPU: W
ranks emulated as host threads, each with its own context and copy of the
phantom, summing their batch tallies through host barriers (the collective a
multi-GPU run takes from NCCL).  Every rank must end with the single-GPU
ctd_run result: the same counts, the dose up to the order of binary64
additions (Sec. 4; Sec. 2.2.1)."""
import threading

import numpy as np
import pytest

from paper_1109_3266_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctd():
    from paper_1109_3266_gb300 import build, ctd as binding
    build.build()
    return binding


KEYS = ("pe", "compton", "rayleigh", "fictitious", "escaped", "missed", "cutoff", "terminated", "aborted", "steps",
        "histories", "n_batches")


class ThreadCollective:
    """Sums over W threads of one process: every thread hands in its tensor, the last
    to arrive adds them, and each copies the sum back."""

    def __init__(self, world):
        self.world = world
        self.bar = threading.Barrier(world)
        self.slots = [None] * world
        self.total = None

    def tally(self, rank):
        import torch

        def f(buf):
            torch.cuda.synchronize()
            self.slots[rank] = buf
            if self.bar.wait() == 0:
                self.total = sum(self.slots[1:], self.slots[0].clone())
                torch.cuda.synchronize()
            self.bar.wait()
            buf.copy_(self.total)
            torch.cuda.synchronize()
            self.bar.wait()
        return f

    def counts(self, rank):
        def f(c, e):
            self.slots[rank] = (c.copy(), e.copy())
            if self.bar.wait() == 0:
                self.total = (sum(s[0] for s in self.slots), sum(s[1] for s in self.slots))
            self.bar.wait()
            out = (self.total[0].copy(), self.total[1].copy())
            self.bar.wait()
            return out
        return f


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_run_equals_single_gpu_run(ctd, world):
    import torch

    from paper_1109_3266_gb300 import shard
    p = I.head(n_hist=3_000_001, n_batches=10, seed=41, shape=(64, 64, 40), d=0.4)
    c0 = ctd.ctd_create(device=0)
    h0 = ctd.load_problem(c0, p)
    ctd.ctd_run(c0, h0, p.n_hist, p.seed, p.n_batches)
    ref_dose, ref_sd, ref = ctd.ctd_get_dose_and_stddev(c0, h0, p.phantom.nvox)
    ctd.ctd_destroy(c0)

    coll = ThreadCollective(world)
    results, errors = [None] * world, []

    def rank_main(r):
        try:
            ctx = ctd.ctd_create(device=0, stream=torch.cuda.current_stream().cuda_stream)
            h = ctd.load_problem(ctx, p)
            sh = shard.LibraryShard(ctx, h, p.phantom.nvox, torch.device("cuda", 0))
            st = shard.run_sharded_with(sh, p.n_hist, p.seed, p.n_batches, r, world, coll.tally(r), coll.counts(r))
            dose, sd, _ = ctd.ctd_get_dose_and_stddev(ctx, h, p.phantom.nvox)
            results[r] = (st, dose, sd)
            ctd.ctd_destroy(ctx)
        except Exception as e:      # surfaced below
            errors.append(e)
            coll.bar.abort()

    ts = [threading.Thread(target=rank_main, args=(r,)) for r in range(world)]
    for t in ts:
        t.start()
    for t in ts:
        t.join(timeout=300)
    assert not errors, errors
    for st, dose, sd in results:
        diff = {k: (st[k], ref[k]) for k in KEYS if st[k] != ref[k]}
        assert not diff, diff
        np.testing.assert_allclose(dose, ref_dose, rtol=1e-9, atol=0)
        np.testing.assert_allclose(sd, ref_sd, rtol=1e-6, atol=1e-30)
        assert st["avg_rsd"] == pytest.approx(ref["avg_rsd"], rel=1e-6)
        assert st["e_emitted_kev"] == pytest.approx(ref["e_emitted_kev"], rel=1e-12)


def test_shard_calls_refuse_bad_arguments(ctd):
    import torch
    p = I.tiny_water(1000)
    ctx = ctd.ctd_create(device=0)
    h = ctd.load_problem(ctx, p)
    buf = torch.zeros(p.phantom.nvox, dtype=torch.float64, device="cuda")
    with pytest.raises(ctd.CtdError):
        ctd.ctd_shard_batch(ctx, h, 0, 0, 10, buf.data_ptr())        # no run begun
    ctd.ctd_shard_begin(ctx, h, 1000, 1, 10)
    with pytest.raises(ctd.CtdError):
        ctd.ctd_shard_batch(ctx, h, 10, 0, 10, buf.data_ptr())       # batch out of range
    with pytest.raises(ctd.CtdError):
        ctd.ctd_shard_batch(ctx, h, 0, 0, 101, buf.data_ptr())       # past the batch's 100 histories
    with pytest.raises(ctd.CtdError):
        ctd.ctd_shard_begin(ctx, h, 10, 1, 11)
    ctd.ctd_destroy(ctx)
