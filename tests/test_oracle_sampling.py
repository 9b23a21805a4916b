"""Pins of the angular sampling (Sec. 2.2.2, Eq. 1; Sec. 2.2.3, Eq. 2).

The R and C surfaces are checked against cumulative distributions obtained
here by numeric integration of the closed-form densities, and the sampled
polar cosines (surface, binary32 surface and exact rejection samplers) by a
chi-square test at the paper's validation energies 10 and 60 keV (Figs. 3-4)
and at 150 keV."""
import math

import numpy as np
import pytest
from scipy import integrate, optimize, stats

from paper_1109_3266_gb300 import inputs as I

MEC2 = 510.99895
HC = 12.398419843320026


def density(kind, e, q0=1.0):
    if kind == "compton":
        k = e / MEC2

        def p(mu):
            r = 1.0 / (1.0 + k * (1.0 - mu))
            return r * r * (r + 1.0 / r - (1.0 - mu * mu))
        return p
    a = 2.0 * (e / HC) ** 2 / q0 ** 2 if q0 > 0 else 0.0
    return lambda mu: (1.0 + mu * mu) * math.exp(-a * (1.0 - mu))


def cdf_factory(kind, e, q0=1.0):
    p = density(kind, e, q0)
    # split near mu = 1 where the Rayleigh density is peaked
    pts = [-1.0, 0.0, 0.9, 0.99, 0.999, 1.0]
    pieces = [integrate.quad(p, pts[i], pts[i + 1], epsabs=0, epsrel=1e-12, limit=200)[0] for i in range(5)]
    total = sum(pieces)

    def cdf(mu):
        acc = 0.0
        for i in range(5):
            a, b = pts[i], pts[i + 1]
            if mu >= b:
                acc += pieces[i]
            else:
                if mu > a:
                    acc += integrate.quad(p, a, mu, epsabs=0, epsrel=1e-12, limit=200)[0]
                break
        return acc / total
    return cdf


def _problem(q0):
    w = I.Material("w", I.WATER.z_over_a, I.WATER.a_mol, I.WATER.z_eff, q0, 1.0)
    ph = I.uniform_box(1, 1, 1, 1.0, w)
    return I.Problem("s", ph, I.pencil_source(), I.spectrum_line(60.0), I.Physics(e_min=10, e_max=150), 1, 1, 1)


@pytest.mark.parametrize("kind,q0,tol", [("compton", 1.0, 1e-8), ("rayleigh", 1.0, 2e-4), ("rayleigh", 0.0, 1e-8)])
@pytest.mark.parametrize("e", [10, 60, 150])
def test_surface_rows_invert_the_cdf(oracle, kind, q0, tol, e):
    n_zeta = 1024
    if kind == "compton":
        row = oracle.kn_surface(e, 1, n_zeta)[0]
    else:
        row = oracle.rayleigh_surface(q0, e, 1, n_zeta)[0]
    assert row[0] == -1.0 and row[-1] == 1.0
    assert np.all(np.diff(row) >= 0)
    cdf = cdf_factory(kind, e, q0)
    zeta = np.arange(n_zeta) / (n_zeta - 1)
    idx = np.unique(np.linspace(0, n_zeta - 1, 64).astype(int))
    err = max(abs(cdf(row[i]) - zeta[i]) for i in idx)
    # trapezoid cdf on 20000 intervals: error ~ (h a)^2/12 with a the Rayleigh exponent
    assert err < tol, err


def _chi2_equal_prob(samples, cdf, nbins=100):
    edges = [-1.0]
    for q in range(1, nbins):
        target = q / nbins
        edges.append(optimize.brentq(lambda m: cdf(m) - target, -1.0, 1.0, xtol=1e-14))
    edges.append(1.0)
    h, _ = np.histogram(samples, bins=np.array(edges))
    e = len(samples) / nbins
    chi2 = ((h - e) ** 2 / e).sum()
    return stats.chi2.sf(chi2, nbins - 1)


CASES = [
    ("compton", 1.0, 10, 64, False), ("compton", 1.0, 60, 64, False), ("compton", 1.0, 150, 64, False),
    ("compton", 1.0, 60, 32, False), ("compton", 1.0, 10, 64, True), ("compton", 1.0, 60, 64, True),
    ("rayleigh", 1.0, 10, 64, False), ("rayleigh", 1.0, 60, 64, False), ("rayleigh", 1.0, 60, 32, False),
    ("rayleigh", 1.0, 60, 64, True), ("rayleigh", 1.0, 10, 64, True),
    ("rayleigh", 0.0, 60, 64, False), ("rayleigh", 0.0, 60, 64, True),
]


@pytest.mark.parametrize("kind,q0,e,precision,exact", CASES)
def test_sampled_cosines_follow_eq1_eq2(oracle, kind, q0, e, precision, exact):
    s = oracle.Setup(_problem(q0), precision)
    mu = s.sample_mu(kind, 0, float(e), 1_000_000, seed=11 + e, exact=exact)
    assert mu.min() >= -1 and mu.max() <= 1
    p = _chi2_equal_prob(mu, cdf_factory(kind, e, q0))
    assert p > 1e-4, p


def test_surface_sampler_between_nodes(oracle):
    # at 60.5 keV the sampler interpolates two node rows; the distribution stays that of Eq. 2
    s = oracle.Setup(_problem(1.0), 64)
    mu = s.sample_mu("compton", 0, 60.5, 1_000_000, seed=3)
    assert _chi2_equal_prob(mu, cdf_factory("compton", 60.5)) > 1e-4


def test_compton_mean_energy_loss(oracle):
    # mean of E'/E under Eq. 2 (S = 1) from the exact sampler vs numeric integration
    s = oracle.Setup(_problem(1.0), 64)
    for e in (20.0, 80.0):
        mu = s.sample_mu("compton", 0, e, 400_000, seed=5, exact=True)
        k = e / MEC2
        ratio = 1.0 / (1.0 + k * (1.0 - mu))
        p = density("compton", e)
        z = integrate.quad(p, -1, 1, epsrel=1e-12)[0]
        ref = integrate.quad(lambda m: p(m) / (1 + k * (1 - m)), -1, 1, epsrel=1e-12)[0] / z
        assert abs(ratio.mean() - ref) < 5 * ratio.std() / math.sqrt(ratio.size)
