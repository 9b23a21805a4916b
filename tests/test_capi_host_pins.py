"""The library's own host physics and host logic, pinned without the oracle
and without a GPU (through the host-only C calls ctd_material_columns,
ctd_angular_surface, ctd_allocate_histories and ctd_alias_table).

The pins are the ones the oracle meets, applied to the library directly:
  - the cross sections: the photoelectric and Rayleigh power laws and their
    unit values (Sec. 2.1), the Klein-Nishina total against numeric
    integration of Eq. 2, the Waller-Hartree total against its free-electron,
    Thomson and high-energy limits (Sec. 2.2.3), the independent-atom Rayleigh
    total against the exact antiderivative (Sec. 2.2.2);
  - the R and C surfaces (Secs. 2.2.2-2.2.3): each row inverts the CDF of
    Eq. 1 or Eq. 2 obtained here by quadrature;
  - the allocation of histories to spectrum bins (Sec. 2.2.5): exact rational
    largest remainder, and refusal of unusable weights;
  - the alias table of a fluence map (Sec. 2.2.4): the probability each beamlet
    gets from the table equals its share of the intensity."""
import math
from fractions import Fraction

import numpy as np
import pytest
from scipy import integrate

from paper_1109_3266_gb300 import inputs as I
from test_oracle_iaa import closed_sigma, iaa_cdf, tf_radius
from test_oracle_physics import kn_dsigma_domega
from test_oracle_sampling import cdf_factory
from test_oracle_wh import SQ0, a_of, g_closed, wh_cdf

NA = 6.02214076e23
R0 = 2.8179403262e-13
MEC2 = 510.99895


@pytest.fixture(scope="module")
def ctd():
    from paper_1109_3266_gb300 import build, ctd as binding
    build.build()
    return binding


def parts(ctd, m, e_min=1, e_max=150, compton="kn", elements=()):
    """Photoelectric, Compton and Rayleigh mass attenuation at the nodes, from the
    cumulative columns."""
    c = ctd.ctd_material_columns(m, e_min, e_max, compton, elements)
    return c[:, 0], c[:, 1] - c[:, 0], c[:, 2] - c[:, 1]


def at(e, e_min=1):
    return int(e) - e_min


# ----------------------------------------------------------------- cross sections
def test_photoelectric_power_law_and_unit_value(ctd):
    w = I.WATER
    pe, _, _ = parts(ctd, w)
    for e in (10, 33, 60):
        assert pe[at(2 * e)] / pe[at(e)] == pytest.approx(1 / 8, rel=1e-13)
    heavy = I.Material("h", w.z_over_a, w.a_mol, 2 * w.z_eff, 1.0, 1.0)
    light = I.Material("l", w.z_over_a, 2 * w.a_mol, w.z_eff, 1.0, 1.0)
    assert parts(ctd, heavy)[0][at(50)] / pe[at(50)] == pytest.approx(16, rel=1e-13)
    assert parts(ctd, light)[0][at(50)] / pe[at(50)] == pytest.approx(0.5, rel=1e-13)
    # Z = 1, E = 1 MeV, one formula unit per N_A grams: 1e-2 microbarn times N_A
    unit = I.Material("u", 0.5, 1.0, 1.0, 1.0, 1.0)
    pe_u, _, _ = parts(ctd, unit, 1000, 1001)
    assert pe_u[0] == pytest.approx(1e-2 * 1e-30 * NA, rel=1e-13)


def test_rayleigh_power_law_and_calibration(ctd):
    w = I.WATER
    _, _, r = parts(ctd, w)
    assert r[at(120)] / r[at(60)] == pytest.approx(0.25, rel=1e-9)
    z2 = I.Material("z", w.z_over_a, w.a_mol, 2 * w.z_eff, 1.0, 1.0)
    assert parts(ctd, z2)[2][at(60)] / r[at(60)] == pytest.approx(4, rel=1e-9)
    assert r[at(60)] == pytest.approx(0.008, rel=2e-3)


@pytest.mark.parametrize("e", [1, 10, 60, 150])
def test_compton_is_electrons_per_gram_times_integral_of_eq2(ctd, e):
    _, c, _ = parts(ctd, I.WATER)
    num, _ = integrate.quad(lambda mu: 2 * math.pi * kn_dsigma_domega(mu, e), -1, 1, epsabs=0, epsrel=1e-13)
    assert c[at(e)] == pytest.approx(NA * I.WATER.z_over_a * num, rel=1e-9)


def test_waller_hartree_limits(ctd):
    # free electrons (sq0 <= 0): the Klein-Nishina total
    free = I.Material("f", I.WATER.z_over_a, I.WATER.a_mol, I.WATER.z_eff, 1.0, 1.0, sq0=0.0)
    _, c_kn, _ = parts(ctd, I.WATER, compton="kn")
    _, c_free, _ = parts(ctd, free, compton="wh")
    np.testing.assert_allclose(c_free, c_kn, rtol=1e-9)   # Simpson on 20000 intervals
    m = I.Material("m", I.WATER.z_over_a, I.WATER.a_mol, I.WATER.z_eff, 1.0, 1.0, sq0=SQ0)
    _, c_wh, _ = parts(ctd, m, compton="wh")
    ne = NA * m.z_over_a
    # Thomson limit at 1 keV (k = 0.002): (r0^2/2)(1 + mu^2) S/Z integrated, O(k) off
    assert c_wh[at(1)] / ne == pytest.approx(math.pi * R0 * R0 * g_closed(a_of(1.0)), rel=1e-2)
    # high energy: S/Z removes a forward cone, (2/a)(1 - (1 + 2k)/a) of the KN integral
    for e in (120, 150):
        k, a = e / MEC2, a_of(float(e))
        i_kn = c_kn[at(e)] / ne / (math.pi * R0 * R0)
        expect = (2.0 / a) * (1.0 - (1.0 + 2.0 * k) / a) / i_kn
        assert 1.0 - c_wh[at(e)] / c_kn[at(e)] == pytest.approx(expect, rel=1e-4)
    # binding lowers the incoherent total, most at low energy
    r = c_wh / c_kn
    assert np.all((r > 0) & (r < 1)) and np.all(np.diff(r) > 0)


@pytest.mark.parametrize("m", [I.WATER, I.BONE, I.AIR])
def test_iaa_rayleigh_total_equals_the_closed_form(ctd, m):
    _, _, r = parts(ctd, m, elements=m.elements)
    for e in (5, 20, 60, 100, 150):
        assert r[at(e)] == pytest.approx(closed_sigma(m, float(e)) * NA / m.a_mol, rel=1e-12)


# ----------------------------------------------------------------- surfaces
def _max_cdf_error(row, cdf, npts=64):
    n_zeta = row.size
    assert row[0] == -1.0 and row[-1] == 1.0 and np.all(np.diff(row) >= 0)
    zeta = np.arange(n_zeta) / (n_zeta - 1)
    idx = np.unique(np.linspace(0, n_zeta - 1, npts).astype(int))
    return max(abs(cdf(row[i]) - zeta[i]) for i in idx)


@pytest.mark.parametrize("e", [10, 60, 150])
def test_kn_and_rayleigh_surface_rows(ctd, e):
    kn = ctd.ctd_angular_surface("kn", I.WATER, e, e + 1)[0]
    assert _max_cdf_error(kn, cdf_factory("compton", e)) < 1e-8
    ray = ctd.ctd_angular_surface("rayleigh", I.WATER, e, e + 1)[0]
    # trapezoid CDF on 20000 intervals: about (h a)^2 / 12 where the density is steepest
    assert _max_cdf_error(ray, cdf_factory("rayleigh", e, 1.0)) < 2e-4
    thomson = ctd.ctd_angular_surface("rayleigh", I.thomson(I.WATER), e, e + 1)[0]
    assert _max_cdf_error(thomson, cdf_factory("rayleigh", e, 0.0)) < 1e-8


@pytest.mark.parametrize("e", [10, 60, 150])
def test_waller_hartree_surface_rows(ctd, e):
    m = I.Material("m", I.WATER.z_over_a, I.WATER.a_mol, I.WATER.z_eff, 1.0, 1.0, sq0=SQ0)
    row = ctd.ctd_angular_surface("wh", m, e, e + 1)[0]
    assert _max_cdf_error(row, wh_cdf(float(e))) < 1e-6


@pytest.mark.parametrize("m", [I.WATER, I.BONE])
@pytest.mark.parametrize("e", [10, 60, 150])
def test_iaa_surface_rows(ctd, m, e):
    row = ctd.ctd_angular_surface("rayleigh", m, e, e + 1, elements=m.elements)[0]
    k = e / 12.398419843320026
    beta = max((2 * math.pi * tf_radius(z)) ** 2 for z, _ in m.elements) * k * k / 2
    assert _max_cdf_error(row, iaa_cdf(m, e), 48) < max(2e-7, (1e-4 * beta) ** 2 / 12 * 4)


# ----------------------------------------------------------------- allocation (Sec. 2.2.5)
def largest_remainder(n, w):
    """Exact rational largest remainder: floors of n w_j / W, then one more to the
    largest fractions (lower bin first among equals), none to empty bins."""
    W = sum(Fraction(x) for x in w)
    q = [Fraction(n) * Fraction(x) / W for x in w]
    out = [int(math.floor(x)) for x in q]
    order = sorted((j for j in range(len(w)) if w[j] > 0), key=lambda j: (-(q[j] - out[j]), j))
    for j in order[:n - sum(out)]:
        out[j] += 1
    return np.array(out, dtype=np.uint64)


@pytest.mark.parametrize("case", ["kramers120", "kramers80", "random", "zeros", "one_bin", "ties"])
def test_allocation_is_exact_largest_remainder(ctd, case):
    rng = np.random.default_rng(7)
    w = {"kramers120": I.spectrum_kramers(120, 2.5, 1).w,
         "kramers80": I.spectrum_kramers(80, 0.0, 10).w,
         "random": rng.random(60),
         "zeros": np.where(rng.random(40) < 0.3, 0.0, rng.random(40)),
         "one_bin": np.array([3.0]),
         "ties": np.ones(7)}[case]
    for n in (0, 1, 9, 1_000_003, 10**9 + 7):
        got = ctd.ctd_allocate_histories(n, w)
        assert int(got.sum()) == n
        assert np.all(got[w == 0] == 0)
        quota = n * w / w.sum()
        assert np.all(np.abs(got - quota) < 1.0 + 1e-9 * n)
        # the binary64 quotas and the exact ones order the fractions alike here
        assert np.array_equal(got, largest_remainder(n, w)), case


@pytest.mark.parametrize("bad", [[1.0, np.inf], [np.nan, 1.0], [-1.0, 2.0], [0.0, 0.0], [1e308, 1e308]])
def test_allocation_refuses_unusable_weights(ctd, bad):
    with pytest.raises(ctd.CtdError):
        ctd.ctd_allocate_histories(1_000_000_000, np.array(bad))


def test_oracle_allocation_refuses_unusable_weights(oracle):
    for bad in ([1.0, np.inf], [1e308, 1e308], [np.nan, 1.0]):
        with pytest.raises(ValueError):
            oracle.allocate(1000, np.array(bad))


# ----------------------------------------------------------------- alias table (Sec. 2.2.4)
def implied_probabilities(thr, al):
    """P(beamlet I) of the draw k = floor(x n / 2^32), I = k if y < thr[k] else alias[k],
    x and y uniform 32-bit words: (1/n) sum_k [thr_k/2^32 (k = I) + (1 - thr_k/2^32) (alias_k = I)]."""
    n = thr.size
    keep = thr.astype(np.float64) / 2.0 ** 32
    p = keep.copy()
    np.add.at(p, al, 1.0 - keep)
    return p / n


@pytest.mark.parametrize("case", ["bowtie", "random", "uniform", "one_hot", "zeros", "spiky"])
def test_alias_table_gives_each_beamlet_its_share(ctd, case):
    rng = np.random.default_rng(9)
    f = {"bowtie": I.bowtie_fluence(128, 32, seed=1).ravel(),
         "random": rng.exponential(size=1000),
         "uniform": np.ones(777),
         "one_hot": np.eye(1, 50, 17).ravel(),
         "zeros": np.where(rng.random(300) < 0.3, 0.0, rng.random(300)),
         "spiky": np.concatenate([np.full(500, 1e-6), [1e3, 5e2]])}[case]
    thr, al = ctd.ctd_alias_table(f)
    n = f.size
    assert np.all((al >= 0) & (al < n))
    p = implied_probabilities(thr, al)
    # each column's threshold is floor(p 2^32): at most 2^-32 / n lost per column a beamlet appears in
    touches = 1 + np.bincount(al, minlength=n)
    assert np.all(np.abs(p - f / f.sum()) <= touches * 2.0 ** -32 / n + 1e-14)
    assert np.all(p[f == 0] <= touches[f == 0] * 2.0 ** -32 / n)


@pytest.mark.parametrize("bad", [[0.0, 0.0], [1.0, -1.0], [1.0, np.nan], [1.0, np.inf], [1e308, 1e308]])
def test_alias_table_refuses_unusable_intensities(ctd, bad):
    with pytest.raises(ctd.CtdError):
        ctd.ctd_alias_table(np.array(bad))
