"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

- The device's logarithm and sincos stay within stated bounds of binary64 on
  every uniform the transport draws; the uniform mapping is exact.
- The binary32 tables and surfaces equal the host-built binary64 ones rounded
  (the library's host physics is pinned on its own in the CPU suite).
- The device's surface samplers follow Eqs. 1-2.
- Transport: history by history against the binary64 oracle's records and
  decision margins (gpu_checks); the dose within 3 combined standard errors
  of the binary64 oracle for >= 99 % of the voxels above 10 % of the maximum,
  with the total deposit within 0.5 %.
- Properties that hold at any size are checked on the full 1e9-history
  CBCT-water run."""
import math

import numpy as np
import pytest

from paper_1109_3266_gb300 import inputs as I
from gpu_checks import histories_match_binary64

pytestmark = pytest.mark.gpu

COUNT_KEYS = ("pe", "compton", "rayleigh", "fictitious", "escaped", "missed", "cutoff", "terminated", "aborted",
              "steps")


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


def small_cbct(n_hist=200_000, seed=2):
    return I.cbct_water(n_hist=n_hist, seed=seed, shape=(64, 64, 32), d=0.8)


def small_head(n_hist=200_000, seed=3):
    return I.head(n_hist=n_hist, seed=seed, shape=(64, 64, 40), d=0.4)


def dose_parity(dose, sd, ref, ref_sd, frac=0.99):
    dmax = ref.max()
    m = ref > 0.1 * dmax
    z = np.abs(dose[m] - ref[m]) / np.sqrt(sd[m] ** 2 + ref_sd[m] ** 2 + 1e-300)
    return float(np.mean(z < 3.0)), int(m.sum())


# ----------------------------------------------------------------- elementary functions
def test_device_log_and_sincos_within_bounds_on_every_uniform(ctd, ctx):
    # the decision margins of the oracle allow 2^-18 of absolute error in ln u
    u = ((2 * np.arange(2 ** 23, dtype=np.float64) + 1) * 2.0 ** -24).astype(np.float32)
    u64 = u.astype(np.float64)
    dev = ctd.ctd_eval_math(ctx, 0, u).astype(np.float64)
    assert np.max(np.abs(dev - np.log(u64))) <= 2.0 ** -18
    dev = ctd.ctd_eval_math(ctx, 1, u).reshape(-1, 2).astype(np.float64)
    assert np.max(np.abs(dev[:, 0] - np.cos(2 * np.pi * u64))) <= 2.0 ** -20
    assert np.max(np.abs(dev[:, 1] - np.sin(2 * np.pi * u64))) <= 2.0 ** -20


def test_device_uniform_mapping_equals_oracle_on_every_significand(ctd, ctx, oracle):
    # every 23-bit significand k = x >> 9, with random low bits below it
    k = np.arange(2 ** 23, dtype=np.uint32)
    low = np.random.default_rng(11).integers(0, 512, k.size, dtype=np.uint32)
    words = (k << np.uint32(9)) | low
    dev = ctd.ctd_eval_math(ctx, 2, words.view(np.float32))
    assert np.array_equal(dev.view(np.uint32), oracle.uniform_f32(words).view(np.uint32))


# ----------------------------------------------------------------- tables
@pytest.mark.parametrize("make", [lambda: I.tiny_water(1000), lambda: small_head(1000)])
def test_tables_and_surfaces_equal_oracle_bitwise(ctd, ctx, oracle, make):
    p = make()
    h = ctd.load_problem(ctx, p)
    cum, mm, cs, rs = ctd.ctd_get_tables(ctx, h)
    s = oracle.Setup(p, 32)
    ocum, omm = s.tables()
    ocs, ors = s.surfaces()
    assert np.array_equal(cum, ocum)
    assert np.array_equal(mm, omm)
    assert np.array_equal(cs, ocs)
    assert np.array_equal(rs, ors)
    ctd.ctd_destroy_phantom(ctx, h)


# ----------------------------------------------------------------- samplers (Figs. 3-4)
@pytest.mark.parametrize("kind,e", [("compton", 10.0), ("compton", 60.0), ("rayleigh", 10.0), ("rayleigh", 60.0),
                                    ("compton", 60.5)])
def test_device_sampler_matches_oracle_and_eq1_eq2(ctd, ctx, oracle, kind, e):
    from scipy import stats
    from test_oracle_sampling import _chi2_equal_prob, cdf_factory
    p = small_head(1000)
    h = ctd.load_problem(ctx, p)
    mat = 3 if kind == "rayleigh" else 0          # brain, q0 = 1
    n = 2_000_000
    dev = ctd.ctd_sample_mu(ctx, h, kind, mat, e, 77, n)
    ref = oracle.Setup(p, 32).sample_mu(kind, mat, e, 200_000, seed=77)
    assert np.array_equal(dev[:200_000], ref)
    assert _chi2_equal_prob(dev, cdf_factory(kind, e, 1.0)) > 1e-4
    ctd.ctd_destroy_phantom(ctx, h)


# ----------------------------------------------------------------- primary-only counts
@pytest.mark.parametrize("make", [lambda: I.tiny_water(100_000), lambda: small_head(100_000),
                                  lambda: small_cbct(100_000)])
def test_primary_only_matches_binary64(ctd, ctx, oracle, make):
    p = make()
    p = I.scaled(p, physics=I.Physics(p.physics.e_min, p.physics.e_max, mode="max_real", max_real=1))
    dose, sd, st, h = ctd.run_problem(ctx, p)
    assert st["histories"] == p.n_hist
    r = oracle.run(p, precision=64)
    # every history is either the same on both sides or within its margins; the totals follow
    s, = histories_match_binary64(ctd, ctx, h, p, oracle)
    for k in ("pe", "compton", "rayleigh", "escaped", "missed", "cutoff", "terminated", "aborted"):
        assert abs(st[k] - r.counts[k]) <= s["flagged"], (k, st[k], r.counts[k], s)
    assert st["e_deposited_kev"] == pytest.approx(r.counts["e_deposited"], rel=1e-5)
    ctd.ctd_destroy_phantom(ctx, h)


# ----------------------------------------------------------------- full transport
@pytest.mark.parametrize("make", [lambda: I.tiny_water(100_000), lambda: small_head(300_000),
                                  lambda: small_cbct(300_000)])
def test_full_transport_matches_oracles(ctd, ctx, oracle, make):
    p = make()
    dose, sd, st, h = ctd.run_problem(ctx, p)
    r64 = oracle.run(p, precision=64)
    frac, nmask = dose_parity(dose, sd, r64.dose, r64.std)
    assert nmask > 50 and frac >= 0.99, (frac, nmask)
    e64 = r64.counts["e_deposited"]
    assert abs(st["e_deposited_kev"] - e64) <= 0.005 * e64
    # energy bookkeeping on the device
    assert abs(st["e_deposited_kev"] + st["e_escaped_kev"] - st["e_emitted_kev"]) <= 1e-9 * st["e_emitted_kev"]
    # avg RSD as the oracle defines it, from the device's own dose and stddev
    assert st["avg_rsd"] == pytest.approx(oracle.avg_rsd(dose, sd, p.phantom.rho), rel=1e-9)
    assert st["paper_sigma_bar"] == pytest.approx(oracle.paper_sigma_bar(dose, sd, p.phantom.rho), rel=1e-9)
    histories_match_binary64(ctd, ctx, h, p, oracle)
    ctd.ctd_destroy_phantom(ctx, h)


def test_independent_seeds_agree_statistically(ctd, ctx, oracle):
    p = small_head(400_000)
    dose, sd, st, h = ctd.run_problem(ctx, p)
    r64 = oracle.run(I.scaled(p, seed=99), precision=64)
    frac, nmask = dose_parity(dose, sd, r64.dose, r64.std)
    assert frac >= 0.99, (frac, nmask)
    e64 = r64.counts["e_deposited"] / r64.counts["e_emitted"]
    eg = st["e_deposited_kev"] / st["e_emitted_kev"]
    assert abs(eg - e64) < 0.005 * e64
    ctd.ctd_destroy_phantom(ctx, h)


@pytest.mark.parametrize("mode", ["full", "max_real"])
@pytest.mark.parametrize("scale", [2.0, 10.0])
def test_majorant_scale_matches_binary64(ctd, ctx, oracle, scale, mode):
    p = small_head(50_000)
    p = I.scaled(p, physics=I.Physics(1, 150, majorant_scale=scale, mode=mode, max_real=1))
    h = ctd.load_problem(ctx, p)
    histories_match_binary64(ctd, ctx, h, p, oracle)
    ctd.ctd_destroy_phantom(ctx, h)


# ----------------------------------------------------------------- full-size workloads, sampled
def _physics(p, **kw):
    import dataclasses
    return I.scaled(p, physics=dataclasses.replace(p.physics, **kw))


def test_full_size_cbct_run_properties(ctd, ctx):
    # the whole 1e9-history workload in its 10 batches: bookkeeping and end states add up
    p = I.cbct_water()
    dose, sd, st, h = ctd.run_problem(ctx, p)
    ends = st["pe"] + st["cutoff"] + st["escaped"] + st["missed"] + st["terminated"] + st["aborted"]
    assert ends == p.n_hist and st["aborted"] == 0
    assert abs(st["e_deposited_kev"] + st["e_escaped_kev"] - st["e_emitted_kev"]) <= 1e-9 * st["e_emitted_kev"]
    assert np.all(dose >= 0) and np.all(sd >= 0)
    assert 0 < st["avg_rsd"] < 0.5
    # the spectrum's mean energy is what was emitted
    sp = p.spectrum
    mean_e = float(np.sum(sp.w * 0.5 * (sp.e_lo + sp.e_hi)) / sp.w.sum())
    assert st["e_emitted_kev"] / p.n_hist == pytest.approx(mean_e, rel=1e-3)
    ctd.ctd_destroy_phantom(ctx, h)


# ----------------------------------------------------------------- edge cases
def test_edge_cases(ctd, ctx, oracle):
    # ragged batches and a history count equal to the batch count
    for n, nb in ((1003, 7), (10, 10), (2, 2)):
        p = I.tiny_water(n_hist=n, n_batches=nb)
        dose, sd, st, h = ctd.run_problem(ctx, p)
        histories_match_binary64(ctd, ctx, h, p, oracle)
        ctd.ctd_destroy_phantom(ctx, h)
    # a single voxel, a field that misses the phantom, a vacuum phantom
    one = I.Problem("one", I.uniform_box(1, 1, 1, 2.0, I.WATER), I.static_source(10.0, 0.5, 0.5),
                    I.spectrum_line(40.0), I.Physics(10, 150), 5000, 5, 4)
    miss = I.Problem("miss", I.uniform_box(4, 4, 4, 1.0, I.WATER), I.Source("static", 50.0, 20.0, 30.0, 20.0, 30.0),
                     I.spectrum_line(40.0), I.Physics(10, 150), 5000, 5, 4)
    vac = I.Problem("vac", I.uniform_box(4, 4, 4, 1.0, I.WATER, density=0.0), I.static_source(50.0, 1.0, 1.0),
                    I.spectrum_line(40.0), I.Physics(10, 150), 5000, 5, 4)
    for p in (one, miss, vac):
        dose, sd, st, h = ctd.run_problem(ctx, p)
        assert np.all(np.isfinite(dose)) and np.all(np.isfinite(sd))
        histories_match_binary64(ctd, ctx, h, p, oracle)
        ctd.ctd_destroy_phantom(ctx, h)
    assert st["escaped"] == 5000 and st["steps"] == 5000
    # an empty range does nothing; bad arguments are refused
    p = I.tiny_water(1000)
    h = ctd.load_problem(ctx, p)
    ctd.ctd_run_range(ctx, h, 1000, 1, 10, 500, 500)
    assert np.all(ctd.ctd_get_edep(ctx, h, p.phantom.nvox) == 0)
    with pytest.raises(ctd.CtdError):
        ctd.ctd_run(ctx, h, 1000, 1, 1)
    with pytest.raises(ctd.CtdError):
        ctd.ctd_run_range(ctx, h, 1000, 1, 10, 10, 2000)
    with pytest.raises(ctd.CtdError):
        ctd.ctd_set_spectrum(ctx, h, [200.0], [201.0], [1.0]) or ctd.ctd_run(ctx, h, 1000, 1, 10)
    ctd.ctd_destroy_phantom(ctx, h)
    with pytest.raises(ctd.CtdError):
        ctd.ctd_destroy_phantom(ctx, h)


@pytest.mark.gpu
def test_memory_probes_report_rates(ctd):
    """The memory-ceiling probes run on L2- and HBM-sized buffers and give
    positive, finite rates; arguments out of range are refused."""
    c = ctd.ctd_create(device=0)
    try:
        for kind in (ctd.PROBE_L2_RED, ctd.PROBE_GATHER4, ctd.PROBE_VOXEL):
            for n_slots in (1, 1 << 20, 1 << 28):
                r = ctd.ctd_probe_memory(c, kind, n_slots, 1 << 24)
                assert np.isfinite(r) and r > 0
        for bad in ((3, 1 << 20, 1 << 20), (0, 0, 1 << 20), (0, 1 << 32, 1 << 20), (1, 1 << 20, 0),
                    (2, 1 << 20, 1 << 33)):
            with pytest.raises(ctd.CtdError):
                ctd.ctd_probe_memory(c, *bad)
    finally:
        ctd.ctd_destroy(c)


def test_phantom_checks_on_the_device(ctd, ctx):
    # the voxel scan at creation names the first voxel that breaks a rule
    nx, ny, nz = 64, 48, 40
    mat = np.zeros(nx * ny * nz, dtype=np.uint8)
    rho = np.ones(nx * ny * nz, dtype=np.float32)
    mats = [I.WATER, I.BONE]

    def make(m, r):
        return ctd.ctd_create_phantom(ctx, nx, ny, nz, 0.5, 0.5, 0.5, m, r, mats)

    def msg(m, r):
        with pytest.raises(ctd.CtdError) as e:
            make(m, r)
        return str(e.value)

    m1 = mat.copy()
    m1[[100_000, 20_000]] = [2, 7]
    assert "voxel 20000 has material 7" in msg(m1, rho)
    # densities travel packed with the material in one word: 0 or [2^-18, 2^13) g/cm^3
    below, top = np.float32(2.0 ** -18), np.float32(2.0 ** 13)
    for bad in (np.nan, np.inf, -1.0, -1e-30, np.nextafter(below, np.float32(0)), 1e-6, top, 1e30):
        r1 = rho.copy()
        r1[[99_999, 5_001]] = bad
        assert "voxel 5001 has density" in msg(mat, r1)
    for good in (below, np.nextafter(top, np.float32(0)), 0.0, 1e-5, 5000.0):
        r1 = rho.copy()
        r1[[99_999, 5_001]] = good
        ctd.ctd_destroy_phantom(ctx, make(mat, r1))
    r1 = rho.copy()
    r1[4_000] = np.nan
    assert "voxel 3000 has material" in msg(np.where(np.arange(mat.size) == 3000, 5, mat).astype(np.uint8), r1)
    assert "voxel 4000 has density" in msg(np.where(np.arange(mat.size) == 5000, 5, mat).astype(np.uint8), r1)
    # -0 is a valid density
    m2 = mat.copy()
    m2[:10] = 1
    r2 = rho.copy()
    r2[:10] = -0.0
    h = make(m2, r2)
    ctd.ctd_destroy_phantom(ctx, h)


def test_odd_voxel_count_dose_equals_oracle(ctd, ctx, oracle):
    # dose, stddev and energy per voxel on a grid of odd size; the binary64 oracle
    # follows the same histories, so dose and stddev agree far inside 3 sigma
    p = I.head(60_000, seed=12, phantom_seed=4, shape=(33, 31, 21), d=0.8)
    assert p.phantom.nvox % 2 == 1
    dose, sd, st, h = ctd.run_problem(ctx, p)
    r64 = oracle.run(p, precision=64)
    frac, nmask = dose_parity(dose, sd, r64.dose, r64.std)
    assert frac >= 0.99, (frac, nmask)
    m = r64.dose > 0.1 * r64.dose.max()
    assert np.median(np.abs(sd[m] / r64.std[m] - 1)) < 0.01
    ed = ctd.ctd_get_edep(ctx, h, p.phantom.nvox)
    assert ed.sum() == pytest.approx(r64.edep.sum(), rel=1e-4)
    histories_match_binary64(ctd, ctx, h, p, oracle)
    ctd.ctd_destroy_phantom(ctx, h)
