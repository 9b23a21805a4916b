"""History-by-history comparison of a binary32 run (the device, or the oracle's
binary32 mode) with the binary64 oracle's records and decision margins.

A history whose smallest decision margin is at least 1 must end the same way,
after the same number of Woodcock steps, with the same type of last real
interaction; if its margin over deposit-moving voxel boundaries is also at
least 1, its last real interaction must sit in the same voxel.  The energy its
ending event deposited must agree within E_TOL.  Histories below a margin of 1
may differ: their decision came within binary32 resolution of the other branch
(the oracle states the bound of each decision)."""
import numpy as np

# keV: 64 units of 2^-24 of the largest photon energy of the node grids (150 keV)
E_TOL = 64 * 2.0 ** -24 * 150.0


def compare(run32, ref64):
    """Summary of the comparison; `unflagged_mismatches` and `unflagged_idx` must be 0."""
    assert run32.shape == ref64.shape
    robust = ref64["margin"] >= 1.0
    robust_loc = ref64["margin_loc"] >= 1.0
    differ = ((run32["end"] != ref64["end"]) | (run32["last_type"] != ref64["last_type"]) |
              (run32["steps"] != ref64["steps"]))
    has_real = ref64["last_type"] >= 0
    idx_differ = has_real & (run32["idx"] != ref64["idx"])
    de = np.abs(run32["e_end"] - ref64["e_end"])
    return {
        "histories": int(run32.size),
        "flagged": int(np.count_nonzero(~robust)),
        "mismatches": int(np.count_nonzero(differ)),
        "unflagged_mismatches": int(np.count_nonzero(differ & robust)),
        "idx_mismatches": int(np.count_nonzero(idx_differ)),
        "unflagged_idx": int(np.count_nonzero(idx_differ & robust_loc & robust)),
        "max_de_unflagged": float(de[robust & ~differ].max()) if np.any(robust & ~differ) else 0.0,
        "never_ended": int(np.count_nonzero(run32["end"] < 0)),
    }


def assert_consistent(run32, ref64, max_flagged_frac=0.05):
    s = compare(run32, ref64)
    assert s["never_ended"] == 0, s
    assert s["unflagged_mismatches"] == 0, s
    assert s["unflagged_idx"] == 0, s
    assert s["max_de_unflagged"] <= E_TOL, s
    assert s["flagged"] <= max_flagged_frac * s["histories"], s
    return s


def counts_of(tracks):
    """End-state counts of a set of records (names as in the run stats)."""
    names = ("pe", "cutoff", "escaped", "missed", "terminated", "aborted")
    b = np.bincount(tracks["end"][tracks["end"] >= 0], minlength=6)
    return {n: int(b[i]) for i, n in enumerate(names)}
