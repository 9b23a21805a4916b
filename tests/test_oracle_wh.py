"""Pins of the Waller-Hartree Compton model (Sec. 2.2.3, Eq. 2 with S(q)).

The oracle's reading: S(q)/Z = 1 - exp(-q^2/sq0^2) with q^2 = 2 k^2 (1 - mu),
k = E/hc, the momentum transfer of the analytic form factor.  The oracle's
total cross section is a composite Simpson integral of Eq. 2.  It is pinned by
  (i)   the Klein-Nishina closed form when S/Z = 1;
  (ii)  the Thomson limit (E -> 0), where the integral of (1 + mu^2) S/Z over
        mu has a closed form (and a power series, checked against each other);
  (iii) the Laplace expansion at high energy, where S/Z suppresses only a
        forward cone of width ~ 1/a in 1 - mu.
The exact sampler (a Klein-Nishina draw kept with probability S/Z) and the
C-surface rows are checked against the density itself, and the transport in
Waller-Hartree mode by narrow-beam attenuation and energy conservation."""
import math

import numpy as np
import pytest
from scipy import integrate, optimize, stats

from paper_1109_3266_gb300 import inputs as I

MEC2 = 510.99895
HC = 12.398419843320026
R0 = 2.8179403262e-13
SQ0 = 0.55


def a_of(e, sq0=SQ0):
    return 2.0 * (e / HC) ** 2 / sq0 ** 2


def g_closed(a):
    """int_{-1}^{1} (1 + mu^2) (1 - exp(-a (1 - mu))) dmu, t = 1 - mu in [0, 2]."""
    x = math.exp(-2.0 * a)
    i0 = (1.0 - x) / a
    i1 = (1.0 - x * (1.0 + 2.0 * a)) / a ** 2
    i2 = (2.0 - x * (4.0 * a * a + 4.0 * a + 2.0)) / a ** 3
    return 8.0 / 3.0 - (2.0 * i0 - 2.0 * i1 + i2)


def g_series(a, terms=40):
    """The same integral from 1 - e^{-at} = sum_n (-1)^{n+1} (at)^n / n!."""
    s = 0.0
    for n in range(1, terms):
        m_n = 2.0 ** (n + 2) / (n + 1) - 2.0 ** (n + 3) / (n + 2) + 2.0 ** (n + 3) / (n + 3)
        s += (-1) ** (n + 1) * a ** n / math.factorial(n) * m_n
    return s


def wh_density(e, sq0=SQ0):
    k = e / MEC2
    a = a_of(e, sq0)

    def p(mu):
        r = 1.0 / (1.0 + k * (1.0 - mu))
        return r * r * (r + 1.0 / r - (1.0 - mu * mu)) * (-math.expm1(-a * (1.0 - mu)))
    return p


def wh_cdf(e, sq0=SQ0):
    p = wh_density(e, sq0)
    pts = [-1.0, 0.0, 0.9, 0.99, 0.999, 1.0]
    pieces = [integrate.quad(p, pts[i], pts[i + 1], epsabs=0, epsrel=1e-12, limit=200)[0] for i in range(5)]
    total = sum(pieces)

    def cdf(mu):
        acc = 0.0
        for i in range(5):
            lo, hi = pts[i], pts[i + 1]
            if mu >= hi:
                acc += pieces[i]
            else:
                if mu > lo:
                    acc += integrate.quad(p, lo, mu, epsabs=0, epsrel=1e-12, limit=200)[0]
                break
        return acc / total
    return cdf


def test_thomson_integral_closed_form_and_series_agree():
    # the closed form cancels catastrophically for small a, so the two meet where both hold
    for a in (0.1, 0.3, 0.5, 1.0, 2.0):
        assert g_closed(a) == pytest.approx(g_series(a, terms=80), rel=1e-9)
    # small a: S/Z ~ a (1 - mu), so the integral ~ a * int (1 + mu^2)(1 - mu) = a * 8/3
    assert g_series(1e-6) == pytest.approx(8.0 / 3.0 * 1e-6, rel=1e-5)


@pytest.mark.parametrize("e", [1.0, 10.0, 60.0, 150.0])
def test_free_electron_limit_is_klein_nishina(oracle, e):
    assert oracle.sigma_wh(e, 0.0) == pytest.approx(oracle.sigma_kn(e), rel=1e-12)


@pytest.mark.parametrize("e,tol", [(0.01, 2e-4), (1.0, 1e-2)])
def test_thomson_limit(oracle, e, tol):
    # at k = E/mc^2 -> 0 Eq. 2 becomes (r0^2/2)(1 + mu^2) S/Z; the KN correction is O(k)
    ref = math.pi * R0 * R0 * g_closed(a_of(e)) if a_of(e) > 0.5 else math.pi * R0 * R0 * g_series(a_of(e))
    assert oracle.sigma_wh(e, SQ0) == pytest.approx(ref, rel=tol)


@pytest.mark.parametrize("e", [120.0, 150.0])
def test_high_energy_laplace_expansion(oracle, e):
    # 1 - sigma_WH/sigma_KN = int p_KN exp(-a t) dt / int p_KN, t = 1 - mu; with
    # p_KN = 2 - (2 + 4k) t + O(t^2) near t = 0 the numerator is (2/a)(1 - (1 + 2k)/a) + O(a^-3)
    k = e / MEC2
    a = a_of(e)
    i_kn = oracle.sigma_kn(e) / (math.pi * R0 * R0)
    expect = (2.0 / a) * (1.0 - (1.0 + 2.0 * k) / a) / i_kn
    got = 1.0 - oracle.sigma_wh(e, SQ0) / oracle.sigma_kn(e)
    assert got == pytest.approx(expect, rel=1e-4)


def test_mass_attenuation_uses_electrons_per_gram(oracle):
    m = I.WATER
    for e in (5.0, 60.0):
        assert oracle.mu_compton_wh(m, e) == pytest.approx(6.02214076e23 * m.z_over_a * oracle.sigma_wh(e, m.sq0),
                                                           rel=1e-14)
    # binding lowers the incoherent total, most at low energy
    r = [oracle.mu_compton_wh(m, e) / oracle.mu_compton(m, e) for e in (5.0, 20.0, 60.0, 150.0)]
    assert all(0.0 < x < 1.0 for x in r) and r == sorted(r)


@pytest.mark.parametrize("e", [10, 60, 150])
def test_wh_surface_rows_invert_the_cdf(oracle, e):
    n_zeta = 1024
    row = oracle.wh_surface(SQ0, e, 1, n_zeta)[0]
    assert row[0] == -1.0 and row[-1] == 1.0
    assert np.all(np.diff(row) >= 0)
    cdf = wh_cdf(e)
    zeta = np.arange(n_zeta) / (n_zeta - 1)
    idx = np.unique(np.linspace(0, n_zeta - 1, 64).astype(int))
    err = max(abs(cdf(row[i]) - zeta[i]) for i in idx)
    assert err < 1e-6, err


def _chi2_equal_prob(samples, cdf, nbins=100):
    edges = [-1.0]
    for q in range(1, nbins):
        edges.append(optimize.brentq(lambda m: cdf(m) - q / nbins, -1.0, 1.0, xtol=1e-14))
    edges.append(1.0)
    h, _ = np.histogram(samples, bins=np.array(edges))
    ex = len(samples) / nbins
    return stats.chi2.sf(((h - ex) ** 2 / ex).sum(), nbins - 1)


def _problem():
    ph = I.uniform_box(1, 1, 1, 1.0, I.WATER)
    return I.Problem("wh", ph, I.pencil_source(), I.spectrum_line(60.0),
                     I.Physics(e_min=10, e_max=150, compton="wh"), 1, 1, 1)


@pytest.mark.parametrize("e,precision,exact", [(10, 64, True), (60, 64, True), (10, 64, False), (60, 64, False),
                                               (60, 32, False), (150, 64, False)])
def test_wh_sampled_cosines_follow_eq2(oracle, e, precision, exact):
    s = oracle.Setup(_problem(), precision)
    mu = s.sample_mu("compton", 0, float(e), 1_000_000, seed=21 + e, exact=exact)
    assert mu.min() >= -1 and mu.max() <= 1
    assert _chi2_equal_prob(mu, wh_cdf(e)) > 1e-4


def test_wh_exact_sampler_at_low_energy(oracle):
    # at 1 keV S/Z keeps only about 4 % of Klein-Nishina draws, mostly backward
    ph = I.uniform_box(1, 1, 1, 1.0, I.WATER)
    p = I.Problem("wh", ph, I.pencil_source(), I.spectrum_line(2.0), I.Physics(e_min=1, e_max=150, compton="wh"),
                  1, 1, 1)
    s = oracle.Setup(p, 64)
    mu = s.sample_mu("compton", 0, 1.0, 200_000, seed=4, exact=True)
    assert _chi2_equal_prob(mu, wh_cdf(1.0), nbins=50) > 1e-4
    assert mu.mean() < -0.1


def _pencil(layers, n, compton):
    ph = I.slab_phantom(layers)
    return I.Problem("pencil", ph, I.pencil_source(), I.spectrum_line(60.0),
                     I.Physics(e_min=10, e_max=150, mode="max_real", max_real=1, compton=compton), n, 10, 7)


@pytest.mark.parametrize("precision", [64, 32])
def test_wh_narrow_beam_primary_attenuation(oracle, precision):
    n = 400_000
    _, c = oracle.Setup(_pencil([(I.WATER, 1.0)] * 6, n, "wh"), precision).transport(0, n)
    mu = oracle.mu_pe(I.WATER, 60.0) + oracle.mu_compton_wh(I.WATER, 60.0) + oracle.mu_rayleigh(I.WATER, 60.0)
    pe = math.exp(-mu * 6.0)
    z = (c["escaped"] - n * pe) / math.sqrt(n * pe * (1 - pe))
    assert abs(z) < 4, z


@pytest.mark.parametrize("precision", [64, 32])
def test_wh_energy_conservation_and_less_compton(oracle, precision):
    base = I.head(20_000, shape=(32, 32, 20), d=0.8)
    wh = I.Problem(base.name, base.phantom, base.source, base.spectrum,
                   I.Physics(compton="wh"), base.n_hist, base.n_batches, base.seed)
    r = oracle.run(wh, precision=precision, threads=2)
    c = r.counts
    assert abs(c["e_deposited"] + c["e_escaped"] - c["e_emitted"]) <= 1e-9 * c["e_emitted"]
    assert c["pe"] + c["cutoff"] + c["escaped"] + c["missed"] + c["terminated"] + c["aborted"] == wh.n_hist
    assert c["aborted"] == 0
    kn = oracle.run(base, precision=precision, threads=2).counts
    assert c["compton"] < kn["compton"]
