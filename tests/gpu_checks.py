"""Checks of a device run against the binary64 oracle shared by the GPU tests.

histories_match_binary64 runs histories of a loaded problem through the C
ABI's per-history records (ctd_trace_range) and compares them with the
binary64 oracle's records and decision margins (track_compare): in primary-only
mode no history whose margins are all >= 1 may differ; in full transport,
where the margins no longer bound the error after a scatter, at most
`full_frac` of the histories may take another path."""
from track_compare import assert_consistent, compare

FULL_FRAC = 5e-3


def histories_match_binary64(ctd, ctx, h, p, oracle, ranges=None, full_frac=FULL_FRAC, max_flagged=0.05):
    ranges = ranges or [(0, p.n_hist)]
    s64 = oracle.Setup(p, 64)
    primary = p.physics.mode == "max_real" and p.physics.max_real == 1
    out = []
    for a, b in ranges:
        dev = ctd.ctd_trace_range(ctx, h, p.n_hist, p.seed, p.n_batches, a, b)
        ref = s64.track(a, b, threads=16)
        if primary:
            s = assert_consistent(dev, ref, max_flagged)
        else:
            s = compare(dev, ref)
            assert s["never_ended"] == 0 and s["mismatches"] <= full_frac * s["histories"], s
        out.append(s)
    return out
