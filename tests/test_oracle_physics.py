"""Pins of the oracle's cross sections and node tables (Sec. 2.1, Eq. 2,
Sec. 2.2.7 item 3).  The Klein-Nishina total is checked against numeric
integration of Eq. 2 with S = 1; the power laws against their exponents;
the tables against the closed forms at the nodes and the majorant invariant."""
import math

import numpy as np
import pytest
from scipy import integrate

from paper_1109_3266_gb300 import inputs as I

R0 = 2.8179403262e-13
MEC2 = 510.99895
NA = 6.02214076e23


def kn_dsigma_domega(mu, e):
    """Eq. 2 with S(q) = 1: r0^2/2 (E'/E)^2 (E'/E + E/E' - sin^2 theta), cm^2/sr."""
    ep = e / (1.0 + (e / MEC2) * (1.0 - mu))
    r = ep / e
    return 0.5 * R0 ** 2 * r * r * (r + 1.0 / r - (1.0 - mu * mu))


@pytest.mark.parametrize("e", [1.0, 10.0, 60.0, 150.0, 511.0, 2000.0])
def test_kn_total_equals_integral_of_eq2(oracle, e):
    num, _ = integrate.quad(lambda mu: 2 * math.pi * kn_dsigma_domega(mu, e), -1, 1, epsabs=0, epsrel=1e-13)
    assert oracle.sigma_kn(e) == pytest.approx(num, rel=1e-9)


def test_kn_thomson_limit(oracle):
    thomson = 8 * math.pi / 3 * R0 ** 2
    assert oracle.sigma_kn(0.01) == pytest.approx(thomson, rel=1e-4)
    assert oracle.sigma_kn(0.01) < thomson


def test_compton_is_electron_density_times_kn(oracle):
    m1 = I.WATER
    m2 = I.Material("x", 2 * m1.z_over_a, m1.a_mol, 3.0, 1.0, 1.0)
    for e in (10.0, 60.0, 140.0):
        assert oracle.mu_compton(m2, e) == pytest.approx(2 * oracle.mu_compton(m1, e), rel=1e-15)
        # electrons per gram N_A Z/A times the per-electron total
        assert oracle.mu_compton(m1, e) / oracle.sigma_kn(e) == pytest.approx(NA * m1.z_over_a, rel=1e-15)
    # water at 60 keV: about 0.18 cm^2/g of incoherent scattering
    assert 0.17 < oracle.mu_compton(I.WATER, 60.0) < 0.19


def test_photoelectric_power_law(oracle):
    w = I.WATER
    for e in (10.0, 33.0, 60.0):
        assert oracle.mu_pe(w, 2 * e) / oracle.mu_pe(w, e) == pytest.approx(1 / 8, rel=1e-14)
    heavy = I.Material("h", w.z_over_a, w.a_mol, 2 * w.z_eff, 1.0, 1.0)
    assert oracle.mu_pe(heavy, 50.0) / oracle.mu_pe(w, 50.0) == pytest.approx(16, rel=1e-14)
    light = I.Material("l", w.z_over_a, 2 * w.a_mol, w.z_eff, 1.0, 1.0)
    assert oracle.mu_pe(light, 50.0) / oracle.mu_pe(w, 50.0) == pytest.approx(0.5, rel=1e-14)
    # unit arguments: Z = 1, E = 1 MeV, one formula unit per N_A * 1 g -> 1e-2 microbarn * N_A
    unit = I.Material("u", 0.5, 1.0, 1.0, 1.0, 1.0)
    assert oracle.mu_pe(unit, 1000.0) == pytest.approx(1e-2 * 1e-30 * NA, rel=1e-14)


def test_rayleigh_power_law_and_calibration(oracle):
    w = I.WATER
    assert oracle.mu_rayleigh(w, 120.0) / oracle.mu_rayleigh(w, 60.0) == pytest.approx(0.25, rel=1e-14)
    z2 = I.Material("z", w.z_over_a, w.a_mol, 2 * w.z_eff, 1.0, 1.0)
    assert oracle.mu_rayleigh(z2, 60.0) / oracle.mu_rayleigh(w, 60.0) == pytest.approx(4, rel=1e-14)
    # the Rayleigh constant is fixed so that water at 60 keV has 0.008 cm^2/g
    assert oracle.mu_rayleigh(w, 60.0) == pytest.approx(0.008, rel=2e-3)


def _two_material_problem(scale=1.0):
    ph = I.slab_phantom([(I.WATER, 2.0), (I.BONE, 2.0)])
    return I.Problem("slab", ph, I.pencil_source(), I.spectrum_line(60.0),
                     I.Physics(e_min=10, e_max=150, majorant_scale=scale), 1000, 10, 1)


@pytest.mark.parametrize("precision", [64, 32])
def test_tables_are_closed_forms_at_nodes(oracle, precision):
    p = _two_material_problem()
    s = oracle.Setup(p, precision)
    cum, mm = s.tables()
    for mi, m in enumerate(p.phantom.materials):
        for j, e in enumerate(range(10, 151)):
            pe, c, r = oracle.mu_pe(m, e), oracle.mu_compton(m, e), oracle.mu_rayleigh(m, e)
            ref = np.array([pe, pe + c, pe + c + r])
            if precision == 32:
                ref = ref.astype(np.float32).astype(np.float64)
                assert np.array_equal(cum[mi, j], ref)
            else:
                assert np.allclose(cum[mi, j], ref, rtol=1e-15, atol=0)
    assert np.all(np.diff(cum, axis=2) > 0)           # PE < PE+C < PE+C+R
    assert np.all(np.diff(cum[..., 2], axis=1) < 0)   # total falls with E on this grid


def test_majorant_bounds_every_material(oracle):
    p = _two_material_problem()
    s = oracle.Setup(p, 64)
    cum, mm = s.tables()
    rho = p.phantom.rho.ravel()
    for mi in range(len(p.phantom.materials)):
        rmax = rho[p.phantom.mat.ravel() == mi].max()
        assert np.all(mm >= rmax * cum[mi, :, 2] * (1 - 1e-15))
    # the majorant is attained by bone here
    assert np.allclose(mm, float(rho.max()) * cum[1, :, 2], rtol=1e-15)
    s2 = oracle.Setup(_two_material_problem(2.5), 64)
    assert np.allclose(s2.tables()[1], 2.5 * mm, rtol=1e-15)
