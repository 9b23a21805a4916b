"""The library's host physics equals the oracle's, bit for bit, without a GPU.

The two are written separately; they agree because both take the same closed
forms and integrals in the same order of operations (binary64, the C
library's functions).  Checked here through the host-only C calls
ctd_material_columns and ctd_angular_surface: node-table columns under both
Compton models and both Rayleigh form factors, and the C and R surfaces of
every kind.  (The GPU tests check the same on a phantom's uploaded tables.)"""
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
    assert np.array_equal(lib.view(np.uint64), ref.view(np.uint64))


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
