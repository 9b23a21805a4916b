"""The library's host physics and host logic against the oracle's, without a GPU.

The two are written separately.  The closed forms and the surfaces agree bit
for bit (both take the same expressions and the same cumulative-trapezoid
construction in binary64); the Waller-Hartree and IAA totals agree to 1e-8,
the library integrating by Gauss-Legendre and the oracle by Simpson.  Checked here through the host-only C calls
ctd_material_columns and ctd_angular_surface (node-table columns under both
Compton models and both Rayleigh form factors; the C and R surfaces of every
kind), ctd_allocate_histories (the largest-remainder spectrum allocation) and
ctd_alias_table (the fluence map's alias table).  The GPU tests check the same
on a phantom's uploaded tables and through the counts of runs."""
import numpy as np
import pytest

from paper_1109_3266_gb300 import inputs as I


@pytest.fixture(scope="module")
def ctd():
    from paper_1109_3266_gb300 import build, ctd as binding
    build.build()
    return binding


def oracle_columns(oracle, m, e_min, e_max, compton, iaa):
    out = []
    for e in range(e_min, e_max + 1):
        pe = oracle.mu_pe(m, float(e))
        c = oracle.mu_compton_wh(m, float(e)) if compton == "wh" else oracle.mu_compton(m, float(e))
        r = oracle.mu_rayleigh_iaa(m, float(e)) if iaa else oracle.mu_rayleigh(m, float(e))
        out.append((pe, pe + c, (pe + c) + r))
    return np.array(out)


@pytest.mark.parametrize("m", [I.WATER, I.BONE, I.BRAIN, I.AIR])
@pytest.mark.parametrize("compton,iaa", [("kn", False), ("wh", False), ("kn", True), ("wh", True)])
def test_material_columns_equal_oracle(ctd, oracle, m, compton, iaa):
    e_min, e_max = 1, 150
    lib = ctd.ctd_material_columns(m, e_min, e_max, compton, m.elements if iaa else ())
    ref = oracle_columns(oracle, m, e_min, e_max, compton, iaa)
    if compton == "kn" and not iaa:
        # closed forms on both sides
        assert np.array_equal(lib.view(np.uint64), ref.view(np.uint64))
    else:
        # the Waller-Hartree and IAA totals: Gauss-Legendre in the library, Simpson in the
        # oracle (its error is about 5e-9)
        np.testing.assert_allclose(lib, ref, rtol=1e-8, atol=0)


@pytest.mark.parametrize("kind,m,iaa", [("kn", I.WATER, False), ("rayleigh", I.WATER, False),
                                        ("rayleigh", I.thomson(I.WATER), False), ("rayleigh", I.BONE, True),
                                        ("rayleigh", I.AIR, True), ("wh", I.BRAIN, False)])
def test_surfaces_equal_oracle(ctd, oracle, kind, m, iaa):
    e_min, e_max, n_zeta = 5, 60, 256
    n_e = e_max - e_min + 1
    lib = ctd.ctd_angular_surface(kind, m, e_min, e_max, n_zeta, m.elements if iaa else ())
    if kind == "kn":
        ref = oracle.kn_surface(e_min, n_e, n_zeta)
    elif kind == "wh":
        ref = oracle.wh_surface(m.sq0, e_min, n_e, n_zeta)
    elif iaa:
        ref = oracle.rayleigh_iaa_surface(m, e_min, n_e, n_zeta)
    else:
        ref = oracle.rayleigh_surface(m.q0, e_min, n_e, n_zeta)
    assert np.array_equal(lib.view(np.uint64), ref.view(np.uint64))


def test_host_physics_refuses_bad_arguments(ctd):
    m = I.WATER
    with pytest.raises(ctd.CtdError):
        ctd.ctd_material_columns(m, 10, 10)
    with pytest.raises(ctd.CtdError):
        ctd.ctd_material_columns(m, 1, 150, compton=7)
    with pytest.raises(ctd.CtdError):
        ctd.ctd_material_columns(m, 1, 150, elements=((0, 1.0),))
    with pytest.raises(ctd.CtdError):
        ctd.ctd_material_columns(m, 1, 150, elements=((8, float("inf")),))
    with pytest.raises(ctd.CtdError):
        ctd.ctd_angular_surface(3, m, 1, 150)
    with pytest.raises(ctd.CtdError):
        ctd.ctd_angular_surface("kn", m, 1, 150, n_zeta=1)


@pytest.mark.parametrize("case", ["kramers120", "kramers80", "ties", "zeros", "one_bin"])
def test_allocation_equals_oracle(ctd, oracle, case):
    rng = np.random.default_rng(5)
    w = {"kramers120": I.spectrum_kramers(120, 2.5, 1).w,
         "kramers80": I.spectrum_kramers(80, 0.0, 10).w,
         "ties": np.ones(7),
         "zeros": np.where(rng.random(40) < 0.3, 0.0, rng.random(40)),
         "one_bin": np.array([3.0])}[case]
    for n in (0, 1, 9, 1_000_003, 10**9 + 7):
        got = ctd.ctd_allocate_histories(n, w)
        assert np.array_equal(got, oracle.allocate(n, w))
        assert int(got.sum()) == n
    with pytest.raises(ctd.CtdError):
        ctd.ctd_allocate_histories(10, np.zeros(3))


@pytest.mark.parametrize("case", ["bowtie", "random", "uniform", "one_hot", "zeros"])
def test_alias_table_equals_oracle(ctd, oracle, case):
    rng = np.random.default_rng(3)
    f = {"bowtie": I.bowtie_fluence(128, 32, seed=1).ravel(),
         "random": rng.exponential(size=1000),
         "uniform": np.ones(777),
         "one_hot": np.eye(1, 50, 17).ravel(),
         "zeros": np.where(rng.random(300) < 0.3, 0.0, rng.random(300))}[case]
    thr, al = ctd.ctd_alias_table(f)
    othr, oal = oracle.alias_table(f)
    assert np.array_equal(thr, othr) and np.array_equal(al, oal)
    for bad in (np.zeros(4), np.array([1.0, -1.0]), np.array([1.0, np.nan])):
        with pytest.raises(ctd.CtdError):
            ctd.ctd_alias_table(bad)
