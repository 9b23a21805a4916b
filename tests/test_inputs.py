"""Checks of the synthetic input generators (phantoms, spectra, requests)."""
import numpy as np

from paper_1109_3266_gb300 import inputs as I


def test_head_phantom_structure():
    ph = I.head_phantom(64, 64, 40, 0.4, seed=3)
    assert ph.mat.shape == (40, 64, 64) and ph.rho.dtype == np.float32 and ph.mat.dtype == np.uint8
    names = [m.name for m in ph.materials]
    assert names == ["air", "soft_tissue", "bone", "brain"]
    for i, m in enumerate(ph.materials):
        sel = ph.mat == i
        assert sel.any()
        r = ph.rho[sel] / m.density
        assert r.min() >= 1 - 0.06 - 1e-6 and r.max() <= 1 + 0.06 + 1e-6
    # air outside the head: the box corners
    assert ph.mat[0, 0, 0] == 0 and ph.mat[-1, -1, -1] == 0
    # deterministic in the seed, different across seeds
    again = I.head_phantom(64, 64, 40, 0.4, seed=3)
    assert np.array_equal(again.rho, ph.rho)
    other = I.head_phantom(64, 64, 40, 0.4, seed=4)
    assert not np.array_equal(other.rho, ph.rho)


def test_kramers_spectrum_shape():
    sp = I.spectrum_kramers(120, 2.5)
    assert len(sp.w) == 119 and sp.e_lo[0] == 1 and sp.e_hi[-1] == 120
    assert np.all(sp.w >= 0) and sp.w[:5].sum() < 1e-20 * sp.w.sum()
    peak = sp.e_lo[np.argmax(sp.w)]
    assert 25 <= peak <= 50


def test_batched_requests_are_reproducible():
    a = I.batched_requests(8)
    b = I.batched_requests(8)
    assert [p.name for p in a] == [p.name for p in b]
    assert [p.n_hist for p in a] == [p.n_hist for p in b]
    assert all(1e7 <= p.n_hist <= 1e9 for p in a)
    assert [p.seed for p in a] == list(range(1000, 1008))


def test_material_compositions_reproduce_their_mass_fractions():
    from paper_1109_3266_gb300 import inputs as I
    assert I.WATER.elements == ((1, 2.0), (8, 1.0))
    for m in (I.SOFT_TISSUE, I.BRAIN, I.BONE, I.AIR):
        mass = [n * I.ATOMIC_WEIGHT[z] for z, n in m.elements]
        # the atoms of one formula unit weigh its molar mass
        assert abs(sum(mass) - m.a_mol) < 1e-9 * m.a_mol
        # and electrons per gram agree with the material's Z/A to about 1 %
        zsum = sum(z * n for z, n in m.elements)
        assert abs(zsum / m.a_mol - m.z_over_a) < 0.012 * m.z_over_a, m.name
        assert all(n > 0 for _, n in m.elements) and len(m.elements) <= 16
    ev = dict(I.BONE.elements)
    w_ca = ev[20] * I.ATOMIC_WEIGHT[20] / I.BONE.a_mol
    assert abs(w_ca - 0.225) < 1e-12
