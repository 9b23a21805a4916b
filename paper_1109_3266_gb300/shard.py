"""One dose calculation sharded over several GPUs (Sec. 4: the histories are
distributed among GPUs that run without interfering).

Every rank holds the phantom and runs its share of each batch: rank r of W
transports the local histories [floor(n_b r / W), floor(n_b (r + 1) / W)) of a
batch of n_b.  Histories draw their random numbers from (seed, history) alone,
so the union of the shards is the single-GPU run.  The ranks then sum their
partial batch tallies with one binary64 all-reduce and each folds the sum, so
every rank ends with the batch statistics of Sec. 2.2.1; the counts are summed
once at the end.  The transport, the folds and the statistics run in the
library (LibraryShard); the collective is the caller's (NCCL across GPUs).
"""
from __future__ import annotations

import numpy as np

from . import ctd


def batch_sizes(n_hist: int, n_batches: int):
    lo, rem = divmod(n_hist, n_batches)
    return [lo + 1 if b < rem else lo for b in range(n_batches)]


def shard_of(n: int, rank: int, world: int):
    """Local history range [lo, hi) of rank `rank` in a batch of n histories."""
    return (n * rank) // world, (n * (rank + 1)) // world


class LibraryShard:
    """One rank's side of a sharded run in the CUDA library: a phantom loaded in a
    context, and a device buffer for the batch tally the ranks sum."""

    def __init__(self, ctx, handle, nvox, device):
        import torch
        self.ctx, self.h = ctx, handle
        self.buf = torch.zeros(nvox, dtype=torch.float64, device=device)

    def begin(self, n_hist, seed, n_batches):
        ctd.ctd_shard_begin(self.ctx, self.h, n_hist, seed, n_batches)

    def transport(self, batch, lo, hi):
        ctd.ctd_shard_batch(self.ctx, self.h, batch, lo, hi, self.buf.data_ptr())
        return self.buf

    def fold(self, batch, buf):
        ctd.ctd_shard_fold(self.ctx, self.h, batch, buf.data_ptr())

    def counts(self):
        return ctd.ctd_shard_counts(self.ctx, self.h)

    def finish(self, counts, energies):
        ctd.ctd_shard_finish(self.ctx, self.h, counts, energies)
        return ctd.ctd_get_dose_and_stddev(self.ctx, self.h, 0, want_arrays=False)[2]


def run_sharded_with(shard, n_hist, seed, n_batches, rank, world, allreduce, allreduce_counts):
    """The sharded run of one rank.  allreduce(tensor) sums a batch tally over the
    ranks in place; allreduce_counts(counts uint64[10], energies float64[2]) returns
    their sums over the ranks.  Returns the shard's finish() value."""
    shard.begin(n_hist, seed, n_batches)
    for b, nb in enumerate(batch_sizes(n_hist, n_batches)):
        lo, hi = shard_of(nb, rank, world)
        buf = shard.transport(b, lo, hi)
        allreduce(buf)
        shard.fold(b, buf)
    c, e = shard.counts()
    c, e = allreduce_counts(c, e)
    return shard.finish(c, e)


def nccl_allreduce(device):
    """The collectives of torch.distributed (NCCL on GPUs): a tally summed in place,
    counts and energies summed through one device tensor each."""
    import torch
    import torch.distributed as dist

    def tally(buf):
        dist.all_reduce(buf, op=dist.ReduceOp.SUM)

    def counts(c, e):
        tc = torch.from_numpy(c.astype(np.int64)).to(device)
        te = torch.from_numpy(e).to(device)
        dist.all_reduce(tc, op=dist.ReduceOp.SUM)
        dist.all_reduce(te, op=dist.ReduceOp.SUM)
        return tc.cpu().numpy().astype(np.uint64), te.cpu().numpy()

    return tally, counts


_SHARDS = {}


def run_sharded(ctd_mod, ctx, handle, n_hist, seed, n_batches, rank, world, reduce, device, nvox=None):
    """run_sharded_with on the library's shard of this rank (kept per phantom, so that
    its tally buffer is allocated once); reduce = nccl_allreduce(device)."""
    key = (ctx.value, handle)
    if key not in _SHARDS:
        if nvox is None:
            raise ValueError("nvox is needed the first time a phantom is sharded")
        _SHARDS[key] = LibraryShard(ctx, handle, nvox, device)
    tally, counts = reduce
    return run_sharded_with(_SHARDS[key], n_hist, seed, n_batches, rank, world, tally, counts)
