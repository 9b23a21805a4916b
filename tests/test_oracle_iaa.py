"""Pins of the independent-atom (IAA) Rayleigh form factor (Sec. 2.2.2, Eq. 1).

The oracle's reading: each element is a screened hydrogenic atom, electron
density Z exp(-2r/a) / (pi a^3) with the Thomas-Fermi radius
a = 0.88534138 a0 Z^(-1/3); a formula unit's F^2 is the sum of its atoms' F^2.
Pins, each independent of the oracle's own expressions:
  (i)   the atomic F is the Fourier transform of that density (numeric
        quadrature of the transform);
  (ii)  at x = 0 the molecule's F^2 is sum n_i Z_i^2, and it is the sum of the
        atoms' F^2 at every x;
  (iii) the Simpson Rayleigh total equals the exact antiderivative of
        (1 + mu^2) / (1 + beta (1 - mu))^4 per element, and tends to the
        Thomson total (8 pi / 3) r0^2 sum n_i Z_i^2 as E -> 0;
  (iv)  the R-surface rows invert the CDF of Eq. 1 (quadrature), and the exact,
        binary64 and binary32 surface samplers pass chi-square against it;
  (v)   transport with the IAA total: narrow-beam attenuation and energy
        conservation."""
import math

import numpy as np
import pytest
from scipy import integrate, optimize, stats

from paper_1109_3266_gb300 import inputs as I

HC = 12.398419843320026
R0 = 2.8179403262e-13
BOHR = 0.529177210903
TF = 0.88534138


def tf_radius(z):
    return TF * BOHR / z ** (1.0 / 3.0)


def f_transform(z, x):
    """F(Q) = int n(r) sin(Qr)/(Qr) 4 pi r^2 dr for n = Z exp(-2r/a) / (pi a^3), Q = 4 pi x."""
    a = tf_radius(z)
    if x == 0.0:
        return integrate.quad(lambda r: z / (math.pi * a ** 3) * math.exp(-2 * r / a) * 4 * math.pi * r * r,
                              0, np.inf, epsabs=0, epsrel=1e-12)[0]
    q = 4 * math.pi * x
    # the density is below 1e-50 of its peak beyond 60 a
    val = integrate.quad(lambda r: z / (math.pi * a ** 3) * math.exp(-2 * r / a) * 4 * math.pi * r / q,
                         0, 60 * a, weight="sin", wvar=q, epsabs=0, epsrel=1e-12, limit=400)[0]
    return val


def iaa(problem):
    ph = problem.physics
    return I.Problem(problem.name, problem.phantom, problem.source, problem.spectrum,
                     I.Physics(ph.e_min, ph.e_max, ph.n_zeta, ph.majorant_scale, ph.mode, ph.max_real, ph.compton,
                               rayleigh="iaa"),
                     problem.n_hist, problem.n_batches, problem.seed)


@pytest.mark.parametrize("z", [1, 6, 8, 20, 82])
def test_atom_form_factor_is_the_transform_of_the_screened_density(oracle, z):
    for x in (0.0, 0.03, 0.1, 0.3, 1.0, 3.0):
        f = f_transform(z, x)
        assert oracle.ff_atom2(z, x * x) == pytest.approx(f * f, rel=1e-8, abs=1e-12 * z * z)
    # normalisation: the density holds Z electrons
    assert oracle.ff_atom2(z, 0.0) == pytest.approx(z * z, rel=1e-15)


@pytest.mark.parametrize("m", [I.WATER, I.BONE, I.AIR, I.BRAIN])
def test_molecular_form_factor_sums_the_atoms(oracle, m):
    assert oracle.ff_mol2(m, 0.0) == pytest.approx(sum(n * z * z for z, n in m.elements), rel=1e-14)
    for x2 in (1e-4, 0.01, 0.3, 2.0):
        assert oracle.ff_mol2(m, x2) == pytest.approx(sum(n * oracle.ff_atom2(z, x2) for z, n in m.elements),
                                                      rel=1e-13)
    # F^2 falls with x
    xs = [oracle.ff_mol2(m, x2) for x2 in (0.0, 0.01, 0.1, 1.0, 10.0)]
    assert xs == sorted(xs, reverse=True)


def closed_integral(beta):
    """int_{-1}^{1} (1 + mu^2) / (1 + beta (1 - mu))^4 dmu, with w = 1 + beta (1 - mu)."""
    if beta < 1e-4:
        return 8.0 / 3.0 - beta * 16.0 / 3.0
    W = 1.0 + 2.0 * beta
    A = 2.0 + 2.0 / beta + 1.0 / beta ** 2
    B = -2.0 / beta - 2.0 / beta ** 2
    C = 1.0 / beta ** 2
    return (A * (1 - W ** -3) / 3 + B * (1 - W ** -2) / 2 + C * (1 - 1 / W)) / beta


def closed_sigma(m, e):
    k = e / HC
    s = 0.0
    for z, n in m.elements:
        c = (2 * math.pi * tf_radius(z)) ** 2
        beta = c * k * k / 2.0      # F^2 = Z^2 / (1 + c x^2)^4, x^2 = k^2 (1 - mu) / 2
        s += n * z * z * closed_integral(beta)
    return math.pi * R0 * R0 * s


@pytest.mark.parametrize("m", [I.WATER, I.BONE, I.AIR])
@pytest.mark.parametrize("e", [5.0, 20.0, 60.0, 100.0, 150.0])
def test_iaa_total_equals_the_closed_form(oracle, m, e):
    assert oracle.sigma_rayleigh_iaa(m, e) == pytest.approx(closed_sigma(m, e), rel=2e-6)
    assert oracle.mu_rayleigh_iaa(m, e) == pytest.approx(oracle.sigma_rayleigh_iaa(m, e) * 6.02214076e23 / m.a_mol,
                                                         rel=1e-14)


def test_closed_form_itself():
    # the antiderivative against direct quadrature (it pins the closed form, not the oracle)
    for beta in (0.05, 1.0, 30.0, 600.0):
        q = integrate.quad(lambda mu: (1 + mu * mu) / (1 + beta * (1 - mu)) ** 4, -1, 1,
                           points=[1 - 1 / beta] if beta > 1 else None, epsabs=0, epsrel=1e-12, limit=200)[0]
        assert closed_integral(beta) == pytest.approx(q, rel=1e-9)


@pytest.mark.parametrize("m", [I.WATER, I.BONE])
def test_iaa_total_thomson_limit(oracle, m):
    thomson = 8.0 * math.pi / 3.0 * R0 * R0 * sum(n * z * z for z, n in m.elements)
    assert oracle.sigma_rayleigh_iaa(m, 0.01) == pytest.approx(thomson, rel=1e-5)
    # the total falls with energy
    s = [oracle.sigma_rayleigh_iaa(m, e) for e in (1.0, 10.0, 60.0, 150.0)]
    assert s == sorted(s, reverse=True)


def iaa_density(m, e):
    k = e / HC
    els = [(n, z, (2 * math.pi * tf_radius(z)) ** 2) for z, n in m.elements]

    def p(mu):
        x2 = k * k * (1 - mu) / 2
        return (1 + mu * mu) * sum(n * z * z / (1 + c * x2) ** 4 for n, z, c in els)
    return p


def iaa_cdf(m, e):
    p = iaa_density(m, e)
    pts = [-1.0, 0.0, 0.9, 0.99, 0.999, 0.9999, 1.0]
    pieces = [integrate.quad(p, pts[i], pts[i + 1], epsabs=0, epsrel=1e-12, limit=200)[0] for i in range(6)]
    total = sum(pieces)

    def cdf(mu):
        acc = 0.0
        for i in range(6):
            lo, hi = pts[i], pts[i + 1]
            if mu >= hi:
                acc += pieces[i]
            else:
                if mu > lo:
                    acc += integrate.quad(p, lo, mu, epsabs=0, epsrel=1e-12, limit=200)[0]
                break
        return acc / total
    return cdf


@pytest.mark.parametrize("m", [I.WATER, I.BONE])
@pytest.mark.parametrize("e", [10, 60, 150])
def test_iaa_surface_rows_invert_the_cdf(oracle, m, e):
    n_zeta = 1024
    row = oracle.rayleigh_iaa_surface(m, e, 1, n_zeta)[0]
    assert row[0] == -1.0 and row[-1] == 1.0
    assert np.all(np.diff(row) >= 0)
    cdf = iaa_cdf(m, e)
    zeta = np.arange(n_zeta) / (n_zeta - 1)
    idx = np.unique(np.linspace(0, n_zeta - 1, 48).astype(int))
    err = max(abs(cdf(row[i]) - zeta[i]) for i in idx)
    # the trapezoid cdf on h = 1e-4 in mu errs by about (h beta)^2 / 12 where the
    # density is steepest, beta = c k^2 / 2 of the lightest element
    k = e / HC
    beta = max((2 * math.pi * tf_radius(z)) ** 2 for z, _ in m.elements) * k * k / 2
    assert err < max(2e-7, (1e-4 * beta) ** 2 / 12 * 4), err


def _chi2_equal_prob(samples, cdf, nbins=100):
    edges = [-1.0]
    for q in range(1, nbins):
        edges.append(optimize.brentq(lambda x: cdf(x) - q / nbins, -1.0, 1.0, xtol=1e-14))
    edges.append(1.0)
    h, _ = np.histogram(samples, bins=np.array(edges))
    ex = len(samples) / nbins
    return stats.chi2.sf(((h - ex) ** 2 / ex).sum(), nbins - 1)


def _problem(m):
    ph = I.uniform_box(1, 1, 1, 1.0, m)
    return I.Problem("iaa", ph, I.pencil_source(), I.spectrum_line(60.0),
                     I.Physics(e_min=1, e_max=150, rayleigh="iaa"), 1, 1, 1)


@pytest.mark.parametrize("m", [I.WATER, I.BONE])
@pytest.mark.parametrize("e,precision,exact", [(10, 64, True), (60, 64, True), (150, 64, True), (10, 64, False),
                                               (60, 64, False), (60, 32, False), (150, 32, False)])
def test_iaa_sampled_cosines_follow_eq1(oracle, m, e, precision, exact):
    s = oracle.Setup(_problem(m), precision)
    mu = s.sample_mu("rayleigh", 0, float(e), 400_000, seed=31 + e, exact=exact)
    assert mu.min() >= -1 and mu.max() <= 1
    assert _chi2_equal_prob(mu, iaa_cdf(m, e)) > 1e-4


def _pencil(layers, n):
    ph = I.slab_phantom(layers)
    return I.Problem("pencil", ph, I.pencil_source(), I.spectrum_line(40.0),
                     I.Physics(e_min=10, e_max=150, mode="max_real", max_real=1, rayleigh="iaa"), n, 10, 7)


@pytest.mark.parametrize("precision", [64, 32])
def test_iaa_narrow_beam_primary_attenuation(oracle, precision):
    n = 400_000
    _, c = oracle.Setup(_pencil([(I.WATER, 1.0)] * 6, n), precision).transport(0, n)
    mu = oracle.mu_pe(I.WATER, 40.0) + oracle.mu_compton(I.WATER, 40.0) + oracle.mu_rayleigh_iaa(I.WATER, 40.0)
    pe = math.exp(-mu * 6.0)
    z = (c["escaped"] - n * pe) / math.sqrt(n * pe * (1 - pe))
    assert abs(z) < 4, z
    # the test tells the totals apart: the closed-form Rayleigh total is many sigma off
    mu_g = oracle.mu_pe(I.WATER, 40.0) + oracle.mu_compton(I.WATER, 40.0) + oracle.mu_rayleigh(I.WATER, 40.0)
    pg = math.exp(-mu_g * 6.0)
    assert abs((c["escaped"] - n * pg) / math.sqrt(n * pg * (1 - pg))) > 10


@pytest.mark.parametrize("precision", [64, 32])
def test_iaa_energy_conservation(oracle, precision):
    p = iaa(I.head(20_000, shape=(32, 32, 20), d=0.8))
    r = oracle.run(p, precision=precision, threads=2)
    c = r.counts
    assert abs(c["e_deposited"] + c["e_escaped"] - c["e_emitted"]) <= 1e-9 * c["e_emitted"]
    assert c["pe"] + c["cutoff"] + c["escaped"] + c["missed"] + c["terminated"] + c["aborted"] == p.n_hist
    assert c["rayleigh"] > 0
