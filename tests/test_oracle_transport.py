"""Pins of the oracle's transport (Sec. 2.1, Fig. 2): direction rotation,
source geometry, narrow-beam attenuation, interaction-type fractions,
majorant invariance of Woodcock tracking, energy conservation and a
brute-force quadrature of the 1- and 2-interaction dose in slabs."""
import math

import numpy as np
import pytest
from scipy import integrate

from paper_1109_3266_gb300 import inputs as I

MEC2 = 510.99895


# ------------------------------------------------------------------ rotation
@pytest.mark.parametrize("precision,tol", [(64, 1e-12), (32, 3e-7)])
def test_rotation_keeps_polar_angle_and_norm(oracle, precision, tol):
    rng = np.random.default_rng(3)
    for _ in range(2000):
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        if rng.uniform() < 0.05:
            u = np.array([0.0, 0.0, rng.choice([-1.0, 1.0])])
        mu = rng.uniform(-1, 1)
        t = rng.uniform()
        un = oracle.rotate(u, mu, t, precision).astype(np.float64)
        uin = np.asarray(u, dtype=np.float32 if precision == 32 else np.float64).astype(np.float64)
        assert abs(np.linalg.norm(un) - 1) < tol
        assert abs(np.dot(uin, un) - mu) < 4 * tol


def test_rotation_azimuth_about_z(oracle):
    for t in (0.0, 0.1, 0.25, 0.6):
        un = oracle.rotate([0.0, 0.0, 1.0], 0.3, t, 64)
        st = math.sqrt(1 - 0.09)
        assert np.allclose(un, [st * math.cos(2 * math.pi * t), st * math.sin(2 * math.pi * t), 0.3], atol=1e-14)


def test_rotation_azimuth_is_uniform_about_axis(oracle):
    # for a fixed axis, the scattered directions' azimuth about it must be uniform
    u = np.array([0.3, -0.5, 0.8])
    u /= np.linalg.norm(u)
    e1 = np.cross(u, [1.0, 0, 0])
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(u, e1)
    phis = []
    for t in np.random.default_rng(4).uniform(size=4000):
        v = oracle.rotate(u, 0.2, t, 64)
        phis.append(math.atan2(np.dot(v, e2), np.dot(v, e1)))
    h, _ = np.histogram(phis, bins=20, range=(-math.pi, math.pi))
    chi2 = ((h - 200) ** 2 / 200).sum()
    assert chi2 < 19 + 6 * math.sqrt(38)


# ------------------------------------------------------------------ source
def rect_solid_angle(a, b, d):
    """Solid angle of a 2a x 2b rectangle centred on the axis at distance d."""
    return 4.0 * math.atan(a * b / (d * math.sqrt(a * a + b * b + d * d)))


def test_rect_solid_angle_formula():
    num, _ = integrate.dblquad(lambda y, x: 3.0 / (x * x + y * y + 9.0) ** 1.5, -2, 2, -1, 1)
    assert rect_solid_angle(2, 1, 3) == pytest.approx(num, rel=1e-10)


@pytest.mark.parametrize("precision", [64, 32])
def test_source_is_uniform_in_solid_angle(oracle, precision):
    # field 20 x 20 cm at 50 cm; an 8 cm water cube is hit through its front face only
    ph = I.uniform_box(16, 16, 16, 0.5, I.WATER)
    n = 400_000
    p = I.Problem("src", ph, I.static_source(50.0, 10.0, 10.0), I.spectrum_line(60.0),
                  I.Physics(e_min=10, e_max=150, mode="max_real", max_real=1), n, 1, 9)
    _, c = oracle.Setup(p, precision).transport(0, n)
    hit = rect_solid_angle(4.0, 4.0, 46.0) / rect_solid_angle(10.0, 10.0, 50.0)
    z = (n - c["missed"] - n * hit) / math.sqrt(n * hit * (1 - hit))
    assert abs(z) < 4, z


@pytest.mark.parametrize("precision", [64, 32])
def test_source_uniform_in_solid_angle_asymmetric_box(oracle, precision):
    # a 6 x 16 x 8 cm box: the hit fraction depends on the field's u and v marginals separately
    ph = I.uniform_box(12, 32, 16, 0.5, I.WATER)
    n = 1_000_000
    p = I.Problem("src", ph, I.static_source(50.0, 10.0, 10.0), I.spectrum_line(60.0),
                  I.Physics(e_min=10, e_max=150, mode="max_real", max_real=1), n, 1, 10)
    _, c = oracle.Setup(p, precision).transport(0, n)
    hit = rect_solid_angle(3.0, 8.0, 46.0) / rect_solid_angle(10.0, 10.0, 50.0)
    z = (n - c["missed"] - n * hit) / math.sqrt(n * hit * (1 - hit))
    assert abs(z) < 4, z


# ------------------------------------------------------------------ narrow beams
def mu_lin(oracle, m, e, rho):
    """Linear attenuation per channel at energy e (keV): linear interpolation of
    the closed forms between integer-keV nodes."""
    j = math.floor(e)
    t = e - j

    def at(x):
        return np.array([oracle.mu_pe(m, x), oracle.mu_compton(m, x), oracle.mu_rayleigh(m, x)])
    v = at(j) if t == 0 else at(j) + t * (at(j + 1) - at(j))
    return rho * v


def pencil_problem(layers, n, e=60.0, scale=1.0, max_real=1, seed=5, batches=10, dz=None):
    ph = I.slab_phantom(layers, dz=dz)
    return I.Problem("pencil", ph, I.pencil_source(), I.spectrum_line(e),
                     I.Physics(e_min=10, e_max=150, majorant_scale=scale, mode="max_real", max_real=max_real),
                     n, batches, seed)


@pytest.mark.parametrize("precision", [64, 32])
def test_narrow_beam_primary_attenuation(oracle, precision):
    n = 400_000
    p = pencil_problem([(I.WATER, 1.0)] * 6, n)
    _, c = oracle.Setup(p, precision).transport(0, n)
    mu = mu_lin(oracle, I.WATER, 60.0, 1.0).sum()
    pe = math.exp(-mu * 6.0)
    z = (c["escaped"] - n * pe) / math.sqrt(n * pe * (1 - pe))
    assert abs(z) < 4, z
    assert c["missed"] == 0 and c["fictitious"] == 0


@pytest.mark.parametrize("scale", [1.0, 2.0, 10.0])
def test_two_material_slab_and_majorant_invariance(oracle, scale):
    n = 300_000
    p = pencil_problem([(I.WATER, 2.0), (I.BONE, 2.0)], n, scale=scale)
    _, c = oracle.Setup(p, 64).transport(0, n)
    mw = mu_lin(oracle, I.WATER, 60.0, 1.0).sum()
    mb = mu_lin(oracle, I.BONE, 60.0, 1.85).sum()
    pesc = math.exp(-2 * mw - 2 * mb)
    z = (c["escaped"] - n * pesc) / math.sqrt(n * pesc * (1 - pesc))
    assert abs(z) < 4, z
    # fictitious events: Poisson with rate (M - mu) along the path until the first real event
    M = scale * mb
    tw = (1 - math.exp(-mw * 2)) / mw
    tb = math.exp(-mw * 2) * (1 - math.exp(-mb * 2)) / mb
    expect = n * ((M - mw) * tw + (M - mb) * tb)
    assert abs(c["fictitious"] - expect) < 5 * math.sqrt(expect * (1 + M * 4)) + 1e-9


def test_majorant_homogeneous_fictitious_rate(oracle):
    n = 300_000
    lam = 3.0
    p = pencil_problem([(I.WATER, 2.0)] * 2, n, scale=lam)
    _, c = oracle.Setup(p, 64).transport(0, n)
    mu = mu_lin(oracle, I.WATER, 60.0, 1.0).sum()
    L = 4.0
    r = (lam - 1) * mu
    et = (1 - math.exp(-mu * L)) / mu
    et2 = 2 * (1 - math.exp(-mu * L) * (1 + mu * L)) / mu ** 2
    mean = r * et
    var = r * et + r * r * (et2 - et * et)
    z = (c["fictitious"] - n * mean) / math.sqrt(n * var)
    assert abs(z) < 4, z


def test_interaction_type_fractions(oracle):
    n = 400_000
    p = pencil_problem([(I.WATER, 5.0)] * 4, n)
    _, c = oracle.Setup(p, 64).transport(0, n)
    mu = mu_lin(oracle, I.WATER, 60.0, 1.0)
    obs = np.array([c["pe"], c["compton"], c["rayleigh"]], dtype=float)
    exp = obs.sum() * mu / mu.sum()
    chi2 = ((obs - exp) ** 2 / exp).sum()
    assert chi2 < 18.4          # 2 dof, p = 1e-4


# ------------------------------------------------------------------ conservation
@pytest.mark.parametrize("precision", [64, 32])
def test_energy_conservation(oracle, precision):
    probs = [I.tiny_water(20_000), I.head(20_000, shape=(32, 32, 20), d=0.8)]
    for p in probs:
        r = oracle.run(p, precision=precision, threads=2)
        c = r.counts
        assert abs(c["e_deposited"] + c["e_escaped"] - c["e_emitted"]) <= 1e-9 * c["e_emitted"]
        assert abs(r.edep.sum() - c["e_deposited"]) <= 1e-9 * c["e_emitted"]
        ends = c["pe"] + c["cutoff"] + c["escaped"] + c["missed"] + c["terminated"] + c["aborted"]
        assert ends == p.n_hist
        assert c["aborted"] == 0
        # every Woodcock step ends in exactly one of: escape, fictitious, PE, Compton, Rayleigh
        assert c["steps"] == c["escaped"] + c["fictitious"] + c["pe"] + c["compton"] + c["rayleigh"]


def test_line_spectrum_emitted_energy_is_exact(oracle):
    sp = I.Spectrum(np.array([30.0, 45.0, 80.0]), np.array([30.0, 45.0, 80.0]), np.array([0.2, 0.5, 0.3]))
    ph = I.uniform_box(8, 8, 8, 1.0, I.WATER)
    p = I.Problem("l", ph, I.static_source(50, 2, 2), sp, I.Physics(e_min=10, e_max=150), 10_007, 7, 3)
    r = oracle.run(p, threads=1)
    expect = 0.0
    for n in oracle.batch_sizes(p.n_hist, p.n_batches):
        a = oracle.allocate(n, sp.w)
        expect += float(np.dot(a, sp.e_lo))
    assert r.counts["e_emitted"] == expect


# ------------------------------------------------------------------ brute force
def _kn_pdf(e):
    k = e / MEC2

    def p(mu):
        r = 1.0 / (1.0 + k * (1.0 - mu))
        return r * r * (r + 1.0 / r - (1.0 - mu * mu))
    z = integrate.quad(p, -1, 1, epsrel=1e-13)[0]
    return lambda mu: p(mu) / z


def _thomson_pdf(mu):
    return 0.375 * (1.0 + mu * mu)


def _gl(a, b, n=96):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (b - a) * x + 0.5 * (b + a), 0.5 * (b - a) * w


def _mean_deposit(oracle, m, rho, e):
    """Mean energy left at one real interaction of a photon of energy e."""
    mu = mu_lin(oracle, m, e, rho)
    pdf = _kn_pdf(e)
    k = e / MEC2
    x, w = _gl(-1, 1)
    loss = sum(wi * pdf(xi) * (e - e / (1 + k * (1 - xi))) for xi, wi in zip(x, w))
    return (mu[0] * e + mu[1] * loss) / mu.sum()


def expected_slab_deposit(oracle, m, rho, L, e, k_max):
    mu = mu_lin(oracle, m, e, rho)
    mt = mu.sum()
    first = (1 - math.exp(-mt * L)) * _mean_deposit(oracle, m, rho, e)
    if k_max == 1:
        return first
    kn = _kn_pdf(e)
    kk = e / MEC2
    ts, tw = _gl(0, L, 64)
    dens = mt * np.exp(-mt * ts)
    d_e = _mean_deposit(oracle, m, rho, e)
    second = 0.0
    for half in ((-1.0, 0.0), (0.0, 1.0)):
        ms, mw = _gl(*half, 96)
        for m1, wm in zip(ms, mw):
            # path to the slab face along the scattered direction, for every depth t
            ell = (L - ts) / m1 if m1 > 0 else ts / (-m1)
            e1 = e / (1 + kk * (1 - m1))
            mu1 = mu_lin(oracle, m, e1, rho).sum()
            pc = kn(m1) * (1 - np.exp(-mu1 * ell)) * _mean_deposit(oracle, m, rho, e1)
            pr = _thomson_pdf(m1) * (1 - np.exp(-mt * ell)) * d_e
            second += wm * np.sum(tw * dens * (mu[1] / mt * pc + mu[2] / mt * pr))
    return first + second


@pytest.mark.parametrize("k_max", [1, 2])
def test_slab_dose_matches_quadrature(oracle, k_max):
    m = I.thomson(I.WATER)
    L = 5.0
    n = 600_000
    p = pencil_problem([(m, L)], n, max_real=k_max, batches=50, seed=21)
    r = oracle.run(p, precision=64, threads=4)
    per_batch = r.d_batches.sum(axis=1)                        # Gy per history per batch
    to_kev = (p.phantom.rho.ravel()[0] * p.phantom.dx * p.phantom.dy * p.phantom.dz / 1000.0) / 1.602176634e-16
    mc = per_batch.mean() * to_kev
    se = per_batch.std(ddof=1) / math.sqrt(len(per_batch)) * to_kev
    ref = expected_slab_deposit(oracle, m, 1.0, L, 60.0, k_max)
    assert abs(mc - ref) < 4.5 * se, (mc, ref, se)


def test_two_voxel_slab_deposit_per_voxel(oracle):
    n = 600_000
    p = pencil_problem([(I.WATER, 2.5), (I.BONE, 2.5)], n, max_real=1, batches=40, seed=8)
    r = oracle.run(p, precision=64, threads=4)
    mass = oracle.voxel_mass_kg(p.phantom)
    kev = r.d_batches * mass / 1.602176634e-16            # keV per history per batch and voxel
    mc = kev.mean(axis=0)
    se = kev.std(axis=0, ddof=1) / math.sqrt(kev.shape[0])
    mw = mu_lin(oracle, I.WATER, 60.0, 1.0).sum()
    mb = mu_lin(oracle, I.BONE, 60.0, 1.85).sum()
    ref = [(1 - math.exp(-mw * 2.5)) * _mean_deposit(oracle, I.WATER, 1.0, 60.0),
           math.exp(-mw * 2.5) * (1 - math.exp(-mb * 2.5)) * _mean_deposit(oracle, I.BONE, 1.85, 60.0)]
    for v in range(2):
        assert abs(mc[v] - ref[v]) < 4.5 * se[v], (v, mc[v], ref[v], se[v])


def test_voxel_addressing_and_material_lookup(oracle):
    # pencil along z through the central column of a 3 x 5 x 4 phantom, materials
    # alternating along z; first-interaction deposits only in that column
    mat = np.zeros((4, 5, 3), np.uint8)
    mat[1::2] = 1
    mats = [I.WATER, I.BONE]
    rho = np.array([m.density for m in mats], np.float32)[mat]
    ph = I.Phantom(3, 5, 4, 1.0, 1.0, 1.0, mat, rho, mats)
    n = 400_000
    p = I.Problem("col", ph, I.pencil_source(), I.spectrum_line(60.0),
                  I.Physics(e_min=10, e_max=150, mode="max_real", max_real=1), n, 20, 12)
    r = oracle.run(p, precision=64, threads=4)
    kev = r.d_batches * oracle.voxel_mass_kg(ph) / 1.602176634e-16
    mc, se = kev.mean(axis=0), kev.std(axis=0, ddof=1) / math.sqrt(kev.shape[0])
    reach = 1.0
    for z in range(4):
        m, dens = mats[z % 2], float(rho[z, 0, 0])
        mu = mu_lin(oracle, m, 60.0, dens).sum()
        ref = reach * (1 - math.exp(-mu)) * _mean_deposit(oracle, m, dens, 60.0)
        reach *= math.exp(-mu)
        v = 1 + 3 * (2 + 5 * z)
        assert abs(mc[v] - ref) < 4.5 * se[v], (z, mc[v], ref, se[v])
    others = np.ones(ph.nvox, bool)
    others[[1 + 3 * (2 + 5 * z) for z in range(4)]] = False
    assert np.all(r.edep[others] == 0)


@pytest.mark.parametrize("precision", [64, 32])
def test_arc_projections_aim_at_the_centre(oracle, precision):
    # four projections 90 degrees apart with a pencil field: source at 100 (sin b, cos b, 0)
    # aimed at the origin; first-interaction deposits lie on the central cross of a 5 x 5 x 1 slab
    ph = I.uniform_box(5, 5, 1, 1.0, I.WATER)
    n = 400_000
    src = I.arc_source(100.0, 0.0, 0.0, 0.0, 0.0, n_proj=4)
    p = I.Problem("arc", ph, src, I.spectrum_line(60.0),
                  I.Physics(e_min=10, e_max=150, mode="max_real", max_real=1), n, 20, 13)
    r = oracle.run(p, precision=precision, threads=4)
    kev = r.d_batches * oracle.voxel_mass_kg(ph) / 1.602176634e-16
    mc, se = kev.mean(axis=0), kev.std(axis=0, ddof=1) / math.sqrt(kev.shape[0])
    mu = mu_lin(oracle, I.WATER, 60.0, 1.0).sum()
    dbar = _mean_deposit(oracle, I.WATER, 1.0, 60.0)
    ref = np.zeros((5, 5))                 # [iy, ix]
    for j in range(5):
        # beam along -y (b = 0) enters at iy = 4; along +y (b = 180) at iy = 0; likewise in x
        ref[j, 2] += 0.25 * dbar * (1 - math.exp(-mu)) * (math.exp(-mu * (4 - j)) + math.exp(-mu * j))
        ref[2, j] += 0.25 * dbar * (1 - math.exp(-mu)) * (math.exp(-mu * (4 - j)) + math.exp(-mu * j))
    ref = ref.ravel()
    on = ref > 0
    assert np.all(r.edep[~on] == 0)
    assert np.all(np.abs(mc[on] - ref[on]) < 4.5 * se[on]), (mc[on], ref[on], se[on])


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("continuous", [False, True])
def test_helical_trajectory_heights(oracle, precision, continuous):
    # pencil beams on a helix from z = -3 to z = +3 cm into a 3 x 3 cm water rod, seen
    # from multiples of 90 degrees only (equal chords): the energy of first interactions
    # per 1 cm slice follows the heights the trajectory visits, and is zero outside [-3, 3)
    ph = I.uniform_box(3, 3, 10, 1.0, I.WATER)
    n = 300_000
    if continuous:
        # 1.5 turns: each slice is a 90-degree stretch of the helix, so all get a sixth
        src = I.helical_source(100.0, 0.0, 0.0, 0.0, 0.0, turns=1.5, z0=-3.0, z1=3.0, n_proj_per_turn=4,
                               continuous=True)
        share = np.full(6, 1.0 / 6.0)
    else:
        # 2 turns of 4 projections: z_k = -3 + 0.75 k, k < 8, falls 2, 1, 1, 2, 1, 1 per slice
        src = I.helical_source(100.0, 0.0, 0.0, 0.0, 0.0, turns=2.0, z0=-3.0, z1=3.0, n_proj_per_turn=4)
        share = np.array([2, 1, 1, 2, 1, 1]) / 8.0
    p = I.Problem("helix", ph, src, I.spectrum_line(60.0),
                  I.Physics(e_min=10, e_max=150, mode="max_real", max_real=1), n, 10, 14)
    r = oracle.run(p, precision=precision, threads=4)
    per_z = r.edep.reshape(10, 9).sum(axis=1)
    assert np.all(per_z[:2] == 0) and np.all(per_z[8:] == 0)
    inside = per_z[2:8]
    ex = inside.sum() * share
    assert np.all(np.abs(inside - ex) < 5 * np.sqrt(ex * _mean_deposit(oracle, I.WATER, 1.0, 60.0))), inside / ex
    if continuous:
        # height and angle move together: slice i is lit from angles [90 i, 90 (i + 1)) degrees,
        # the source at 100 (sin b, cos b, z), so the entry side of the rod takes more energy
        e = r.edep.reshape(10, 3, 3)                  # [z, y, x]
        for i, (sx, sy) in enumerate([(1, 1), (1, -1), (-1, -1), (-1, 1), (1, 1), (1, -1)]):
            sl = e[2 + i]
            near_x, far_x = (sl[:, 2].sum(), sl[:, 0].sum()) if sx > 0 else (sl[:, 0].sum(), sl[:, 2].sum())
            near_y, far_y = (sl[2, :].sum(), sl[0, :].sum()) if sy > 0 else (sl[0, :].sum(), sl[2, :].sum())
            assert near_x > 1.2 * far_x and near_y > 1.2 * far_y, (i, near_x / far_x, near_y / far_y)
