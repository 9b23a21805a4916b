"""Parity of the independent-atom Rayleigh form factor (Sec. 2.2.2, Eq. 1) on
the GPU: tables and per-material R surfaces equal to the oracle's bit for bit,
device sampling equal to the oracle's binary32 sampler and to Eq. 1, bit-exact
counts against the binary32 oracle, dose within 3 sigma of the binary64
oracle, argument checks of ctd_set_material_elements, and the batched form
equal to separate runs."""
import dataclasses

import numpy as np
import pytest

from paper_1109_3266_gb300 import inputs as I
from gpu_checks import histories_match_binary64
from test_gpu_parity import COUNT_KEYS, dose_parity, small_cbct, small_head

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


def iaa(p):
    return I.scaled(p, physics=dataclasses.replace(p.physics, rayleigh="iaa"))


def test_iaa_tables_and_surfaces_equal_oracle_bitwise(ctd, ctx, oracle):
    p = iaa(small_head(1000))
    h = ctd.load_problem(ctx, p)
    cum, mm, cs, rs = ctd.ctd_get_tables(ctx, h)
    s = oracle.Setup(p, 32)
    ocum, omm = s.tables()
    ocs, ors = s.surfaces()
    # the library integrates the Compton / Rayleigh totals by Gauss-Legendre, the oracle by
    # Simpson (5e-9 apart): the binary32 tables agree to one unit in the last place
    np.testing.assert_allclose(cum, ocum, rtol=2.0 ** -23, atol=0)
    np.testing.assert_allclose(mm, omm, rtol=2.0 ** -23, atol=0)
    assert np.array_equal(cs, ocs) and np.array_equal(rs, ors)
    # the Rayleigh column and the R surfaces differ from the analytic form factor's
    hg = ctd.load_problem(ctx, small_head(1000))
    g_cum, _, _, g_rs = ctd.ctd_get_tables(ctx, hg)
    assert np.all((cum[:, :, 2] - cum[:, :, 1]) != (g_cum[:, :, 2] - g_cum[:, :, 1]))
    assert not np.array_equal(rs, g_rs)
    # clearing the elements restores the analytic tables bit for bit
    for m in range(len(p.phantom.materials)):
        ctd.ctd_set_material_elements(ctx, h, m, ())
    cum2, _, _, rs2 = ctd.ctd_get_tables(ctx, h)
    assert np.array_equal(cum2, g_cum) and np.array_equal(rs2, g_rs)
    ctd.ctd_destroy_phantom(ctx, hg)
    ctd.ctd_destroy_phantom(ctx, h)


@pytest.mark.parametrize("mat,e", [(0, 10.0), (1, 60.0), (2, 150.0), (3, 60.0), (3, 30.5)])
def test_iaa_device_sampler_matches_oracle_and_eq1(ctd, ctx, oracle, mat, e):
    from test_oracle_iaa import _chi2_equal_prob, iaa_cdf
    p = iaa(small_head(1000))
    h = ctd.load_problem(ctx, p)
    dev = ctd.ctd_sample_mu(ctx, h, "rayleigh", mat, e, 71, 2_000_000)
    ref = oracle.Setup(p, 32).sample_mu("rayleigh", mat, e, 200_000, seed=71)
    assert np.array_equal(dev[:200_000], ref)
    if e == int(e):
        assert _chi2_equal_prob(dev, iaa_cdf(p.phantom.materials[mat], e)) > 1e-4
    ctd.ctd_destroy_phantom(ctx, h)


@pytest.mark.parametrize("make", [lambda: I.tiny_water(100_000), lambda: small_head(300_000),
                                  lambda: small_cbct(300_000)])
def test_iaa_full_transport_matches_oracles(ctd, ctx, oracle, make):
    p = iaa(make())
    dose, sd, st, h = ctd.run_problem(ctx, p)
    r64 = oracle.run(p, precision=64)
    frac, nmask = dose_parity(dose, sd, r64.dose, r64.std)
    assert nmask > 50 and frac >= 0.99, (frac, nmask)
    e64 = r64.counts["e_deposited"]
    assert abs(st["e_deposited_kev"] - e64) <= 0.005 * e64
    assert abs(st["e_deposited_kev"] + st["e_escaped_kev"] - st["e_emitted_kev"]) <= 1e-9 * st["e_emitted_kev"]
    histories_match_binary64(ctd, ctx, h, p, oracle)
    ctd.ctd_destroy_phantom(ctx, h)


def test_iaa_primary_only_matches_binary64(ctd, ctx, oracle):
    p = small_head(100_000)
    p = I.scaled(p, physics=I.Physics(1, 150, mode="max_real", max_real=1, rayleigh="iaa"))
    h = ctd.load_problem(ctx, p)
    histories_match_binary64(ctd, ctx, h, p, oracle)
    ctd.ctd_destroy_phantom(ctx, h)


def test_material_elements_are_checked(ctd, ctx):
    p = small_head(1000)
    h = ctd.load_problem(ctx, p)
    n_mat = len(p.phantom.materials)
    bad = [(0, ((0, 1.0),)), (0, ((101, 1.0),)), (0, ((8, 0.0),)), (0, ((8, float("nan")),)), (0, ((8, -1.0),)),
           (0, tuple((1, 1.0) for _ in range(17))), (n_mat, ((8, 1.0),)), (-1, ((8, 1.0),))]
    for m, els in bad:
        with pytest.raises(ctd.CtdError):
            ctd.ctd_set_material_elements(ctx, h, m, els)
    ctd.ctd_set_material_elements(ctx, h, 0, ((8, 1.0),))
    ctd.ctd_set_material_elements(ctx, h, n_mat - 1, tuple((1, 0.5) for _ in range(16)))
    ctd.ctd_destroy_phantom(ctx, h)
    with pytest.raises(ctd.CtdError):
        ctd.ctd_set_material_elements(ctx, h, 0, ((8, 1.0),))


def test_iaa_and_analytic_requests_batched_together(ctd, ctx):
    ps = [iaa(small_head(80_000)), small_head(60_000, seed=5), iaa(small_cbct(50_000))]
    ref = []
    for p in ps:
        dose, sd, st, h = ctd.run_problem(ctx, p)
        ref.append((dose, st))
        ctd.ctd_destroy_phantom(ctx, h)
    for shared in (0, 1):
        c = ctd.ctd_create(device=0, shared_launch=shared)
        hs = [ctd.load_problem(c, p) for p in ps]
        ctd.ctd_run_batch(c, hs, [p.n_hist for p in ps], [p.seed for p in ps], 10)
        for p, h, (dose, st) in zip(ps, hs, ref):
            d2, _, st2 = ctd.ctd_get_dose_and_stddev(c, h, p.phantom.nvox)
            assert all(st[k] == st2[k] for k in COUNT_KEYS)
            assert np.allclose(d2, dose, rtol=1e-9, atol=0)
        ctd.ctd_destroy(c)
