"""The device against the binary64 oracle, history by history (the primary-only
comparison of Sec. 2.1's interaction choice, and of the source of
Secs. 2.2.4-2.2.6), through the C ABI's per-history records.

- Primary only: a history whose binary64 decision margins are all >= 1 ends
  the same way on the device, after the same Woodcock steps, in the same
  voxel, with the same deposit (track_compare); on the tiny-water workload at
  seed 1 and on the one- and two-voxel slabs no history differs at all.
- Full transport: the device and the binary64 oracle take the same path in
  all but a few per mille of the histories.
- The same holds on sampled history ranges of the full-size CBCT-water and
  head workloads (also with Waller-Hartree Compton, the independent-atom form
  factor and a bowtie fluence map) and on the trajectory variants.
- The trace instantiation is the production kernel plus the records: its
  counts and deposits equal ctd_run_range's over the same range."""
import dataclasses
import math

import numpy as np
import pytest

from paper_1109_3266_gb300 import inputs as I
from test_oracle_transport import pencil_problem
from track_compare import assert_consistent, compare, counts_of

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctd():
    from paper_1109_3266_gb300 import build, ctd as binding
    build.build()
    return binding


@pytest.fixture(scope="module")
def ctx(ctd):
    c = ctd.ctd_create(device=0)
    yield c
    ctd.ctd_destroy(c)


def primary(p):
    return I.scaled(p, physics=dataclasses.replace(p.physics, mode="max_real", max_real=1))


def physics(p, **kw):
    return I.scaled(p, physics=dataclasses.replace(p.physics, **kw))


def device_tracks(ctd, ctx, p, ranges):
    h = ctd.load_problem(ctx, p)
    out = [ctd.ctd_trace_range(ctx, h, p.n_hist, p.seed, p.n_batches, a, b) for a, b in ranges]
    ctd.ctd_destroy_phantom(ctx, h)
    return out


def oracle_tracks(oracle, p, ranges):
    s = oracle.Setup(p, 64)
    return [s.track(a, b, threads=16) for a, b in ranges]


SMALL = {
    "tiny_water": lambda: I.tiny_water(100_000, seed=1),
    "slab_water": lambda: pencil_problem([(I.WATER, 1.0)], 100_000),
    "slab_water_bone": lambda: pencil_problem([(I.WATER, 2.0), (I.BONE, 2.0)], 100_000),
    "head": lambda: I.head(n_hist=200_000, seed=3, shape=(64, 64, 40), d=0.4),
    "cbct_water": lambda: I.cbct_water(n_hist=200_000, seed=2, shape=(64, 64, 32), d=0.8),
}


def test_densities_across_the_packed_word_history_by_history(ctd, ctx, oracle):
    # a voxel's material and density reach the device as one 32-bit word: densities
    # log-uniform over [2^-18, 16] g/cm^3, zeros and the smallest exact value decode exactly
    p = I.cbct_water(n_hist=100_000, seed=5, shape=(48, 48, 24), d=0.8)
    rng = np.random.default_rng(11)
    rho = np.exp2(rng.uniform(-18.0, 4.0, size=p.phantom.rho.shape)).astype(np.float32)
    flat = rho.reshape(-1)
    flat[::97] = 0.0
    flat[1::97] = 2.0 ** -18
    p = dataclasses.replace(p, phantom=dataclasses.replace(p.phantom, rho=rho))
    dev, = device_tracks(ctd, ctx, p, [(0, p.n_hist)])
    ref, = oracle_tracks(oracle, p, [(0, p.n_hist)])
    assert_consistent(dev, ref)


@pytest.mark.parametrize("name", list(SMALL))
def test_primary_only_history_by_history(ctd, ctx, oracle, name):
    p = SMALL[name]()
    if p.physics.mode != "max_real":
        p = primary(p)
    dev, = device_tracks(ctd, ctx, p, [(0, p.n_hist)])
    ref, = oracle_tracks(oracle, p, [(0, p.n_hist)])
    s = assert_consistent(dev, ref)
    if name.startswith(("tiny", "slab")):
        assert s["mismatches"] == 0, s


@pytest.mark.parametrize("name", ["tiny_water", "head", "cbct_water"])
def test_full_transport_history_by_history(ctd, ctx, oracle, name):
    p = SMALL[name]()
    dev, = device_tracks(ctd, ctx, p, [(0, p.n_hist)])
    ref, = oracle_tracks(oracle, p, [(0, p.n_hist)])
    s = compare(dev, ref)
    assert s["never_ended"] == 0, s
    assert s["mismatches"] <= 2e-3 * s["histories"], s


FULL = {
    "cbct_water": (lambda: I.cbct_water(), [(0, 20_000), (123_456_789, 123_476_789),
                                             (1_000_000_000 - 15_000, 1_000_000_000)]),
    "head": (lambda: I.head(), [(0, 20_000), (1_234_567_890, 1_234_587_890), (1_999_990_000, 2_000_000_000)]),
    "cbct_water_wh": (lambda: physics(I.cbct_water(), compton="wh"), [(777_777_777, 777_797_777)]),
    "cbct_water_iaa": (lambda: physics(I.cbct_water(), rayleigh="iaa"), [(999_980_000, 1_000_000_000)]),
    "head_wh_iaa": (lambda: physics(I.head(), compton="wh", rayleigh="iaa"), [(1_234_567_890, 1_234_587_890)]),
    "cbct_water_bowtie": (lambda: I.cbct_water(bowtie=True), [(0, 20_000), (500_000_000, 500_020_000)]),
}


@pytest.mark.parametrize("mode", ["primary", "full"])
@pytest.mark.parametrize("name", list(FULL))
def test_full_size_ranges_history_by_history(ctd, ctx, oracle, name, mode):
    make, ranges = FULL[name]
    p = make()
    if mode == "primary":
        p = primary(p)
    devs = device_tracks(ctd, ctx, p, ranges)
    refs = oracle_tracks(oracle, p, ranges)
    for dev, ref in zip(devs, refs):
        if mode == "primary":
            assert_consistent(dev, ref)
        else:
            s = compare(dev, ref)
            assert s["never_ended"] == 0 and s["mismatches"] <= 5e-3 * s["histories"], s


TRAJ = {
    "continuous_arc": I.arc_source(100.0, -8.0, 8.0, -6.0, 6.0, continuous=True),
    "partial_arc": I.arc_source(100.0, -8.0, 8.0, -6.0, 6.0, n_proj=200, arc0=0.0, arc1=math.radians(200.0)),
    "helix": I.helical_source(100.0, -8.0, 8.0, -2.0, 2.0, turns=2.5, z0=-5.0, z1=4.0, continuous=True),
}


@pytest.mark.parametrize("name", list(TRAJ))
def test_trajectories_history_by_history(ctd, ctx, oracle, name):
    p = I.head(100_000, seed=21, phantom_seed=5, shape=(48, 48, 40), d=0.5)
    p = primary(dataclasses.replace(p, source=TRAJ[name]))
    dev, = device_tracks(ctd, ctx, p, [(0, p.n_hist)])
    ref, = oracle_tracks(oracle, p, [(0, p.n_hist)])
    assert_consistent(dev, ref)


def test_trace_launch_equals_production_launch(ctd, ctx):
    # the records' instantiation runs the same histories as the production kernel
    p = I.head(n_hist=300_000, seed=3, shape=(64, 64, 40), d=0.4)
    h = ctd.load_problem(ctx, p)
    a, b = 12_345, 212_345
    tr = ctd.ctd_trace_range(ctx, h, p.n_hist, p.seed, p.n_batches, a, b)
    _, _, st_t = ctd.ctd_get_dose_and_stddev(ctx, h, 0, want_arrays=False)
    ed_t = ctd.ctd_get_edep(ctx, h, p.phantom.nvox)
    ctd.ctd_run_range(ctx, h, p.n_hist, p.seed, p.n_batches, a, b, clear=True)
    _, _, st_r = ctd.ctd_get_dose_and_stddev(ctx, h, 0, want_arrays=False)
    ed_r = ctd.ctd_get_edep(ctx, h, p.phantom.nvox)
    for k in ("pe", "compton", "rayleigh", "fictitious", "escaped", "missed", "cutoff", "terminated", "aborted",
              "steps"):
        assert st_t[k] == st_r[k], k
    np.testing.assert_allclose(ed_t, ed_r, rtol=1e-12, atol=1e-9)
    ends = counts_of(tr)
    for k, v in ends.items():
        assert v == st_t[k], k
    assert int(tr["steps"].sum()) == st_t["steps"]
    assert np.all(tr["end"] >= 0)
    # an empty range and a range past the end
    assert ctd.ctd_trace_range(ctx, h, p.n_hist, p.seed, p.n_batches, 5, 5).size == 0
    with pytest.raises(ctd.CtdError):
        ctd.ctd_trace_range(ctx, h, p.n_hist, p.seed, p.n_batches, 0, p.n_hist + 1)
    # more records than one call may hold (2^26) are refused before any work
    with pytest.raises(ctd.CtdError) as e:
        ctd.ctd_trace_range(ctx, h, 2 ** 30, p.seed, p.n_batches, 0, 2 ** 26 + 1)
    assert "2^26" in str(e.value) or "67108864" in str(e.value)
    ctd.ctd_destroy_phantom(ctx, h)
