"""Pins of the fluence-map source (Sec. 2.2.4).

A photon's beamlet I is drawn with probability f_I / sum f, then its point is
uniform inside the beamlet at the centre plane.  The oracle draws I from a
Walker alias table (Vose's construction); the paper's Metropolis-Hastings
chain (Algorithm A1) is in the oracle too, for the error-versus-particles
comparison of Fig. 5(c).  Pins:
  - any alias table implies, by exact enumeration of its columns, the
    probabilities f / sum f (to the 2^-32 resolution of its thresholds);
  - beamlet frequencies of the alias draws pass chi-square, and their error
    e = ||p - p*|| follows the multinomial expectation sqrt(sum p(1-p)/N);
  - the A1 chain converges to f (e falls with N, as in Fig. 5(c));
  - end to end, a thin photoelectric absorber at the centre plane records the
    map beamlet by beamlet, and uniformly inside each beamlet."""
import math

import numpy as np
import pytest
from scipy import stats

from paper_1109_3266_gb300 import inputs as I


def implied_probabilities(thr, al):
    n = thr.size
    keep = thr.astype(np.float64) / 2.0 ** 32
    p = np.zeros(n)
    np.add.at(p, np.arange(n), keep)
    np.add.at(p, al.astype(np.int64), 1.0 - keep)
    return p / n


@pytest.mark.parametrize("case", ["bowtie", "random", "uniform", "one_hot", "zeros"])
def test_alias_table_implies_the_map(oracle, case):
    rng = np.random.default_rng(3)
    f = {"bowtie": I.bowtie_fluence(64, 16, seed=1).ravel(),
         "random": rng.exponential(size=1000),
         "uniform": np.ones(777),
         "one_hot": np.eye(1, 50, 17).ravel(),
         "zeros": np.where(rng.random(300) < 0.3, 0.0, rng.random(300))}[case]
    thr, al = oracle.alias_table(f)
    assert np.all((al >= 0) & (al < f.size))
    p = implied_probabilities(thr, al)
    assert np.abs(p - f / f.sum()).max() < 1e-9
    # a beamlet of zero intensity is never kept or aliased to
    z = f == 0
    assert np.all(thr[z] == 0) and not np.any(z[al[thr < 0xffffffff]])


def test_alias_table_rejects_unusable_maps(oracle):
    for f in (np.zeros(5), np.array([1.0, -1.0]), np.array([1.0, np.nan])):
        with pytest.raises(ValueError):
            oracle.alias_table(f)


def test_alias_draws_follow_the_map(oracle):
    f = I.bowtie_fluence(32, 8, seed=2).ravel()
    p = f / f.sum()
    thr, al = oracle.alias_table(f)
    n = 4_000_000
    c = oracle.alias_counts(thr, al, n, seed=9).astype(np.float64)
    chi2 = ((c - n * p) ** 2 / (n * p)).sum()
    assert stats.chi2.sf(chi2, f.size - 1) > 1e-4


def test_fluence_error_versus_particles(oracle):
    # Fig. 5(c): e = ||p_sim - p*|| against the number of particles, alias table
    # and the paper's Metropolis-Hastings chain (Algorithm A1)
    f = I.bowtie_fluence(64, 16, seed=4).ravel()
    p = f / f.sum()
    thr, al = oracle.alias_table(f)
    e_alias, e_mh = [], []
    for n in (10 ** 4, 10 ** 5, 10 ** 6, 10 ** 7):
        e_alias.append(np.linalg.norm(oracle.alias_counts(thr, al, n, seed=5) / n - p))
        e_mh.append(np.linalg.norm(oracle.mh_counts(f, n, seed=5, i0=0) / n - p))
        expect = math.sqrt((p * (1 - p)).sum() / n)
        assert 0.9 * expect < e_alias[-1] < 1.1 * expect
    assert all(a > b for a, b in zip(e_mh, e_mh[1:]))
    # the chain's draws are correlated: its error is larger at every N
    assert all(m > a for m, a in zip(e_mh, e_alias))


def test_thin_absorber_records_the_map(oracle):
    # static source 50 cm from a 1e-4 cm absorber in the centre plane; 4 x 4 voxels per beamlet
    nu, nv, sub = 12, 6, 4
    half_u, half_v = 6.0, 2.4          # beamlets 1.0 x 0.8 cm
    f = I.bowtie_fluence(nu, nv, seed=6)
    absorber = I.Material("absorber", 0.4, 150.0, 60.0, 1.0, 5000.0)
    ph = I.uniform_box(nu * sub, nv * sub, 1, 1.0, absorber, density=5000.0)
    ph = I.Phantom(ph.nx, ph.ny, ph.nz, 2 * half_u / (nu * sub), 2 * half_v / (nv * sub), 1e-4,
                   ph.mat, ph.rho, ph.materials)
    src = I.Source("static", 50.0, -half_u, half_u, -half_v, half_v, fluence=f)
    n = 400_000
    p = I.Problem("absorber", ph, src, I.spectrum_line(20.0),
                  I.Physics(e_min=10, e_max=150, mode="max_real", max_real=1), n, 10, 8)
    for precision in (64, 32):
        edep, c = oracle.Setup(p, precision).transport(0, n)
        assert c["missed"] == 0 and c["escaped"] < n * 1e-3
        hits = (edep / 20.0).reshape(nv * sub, nu * sub)
        per_beamlet = hits.reshape(nv, sub, nu, sub).sum(axis=(1, 3))
        pf = f / f.sum()
        chi2 = ((per_beamlet - n * pf) ** 2 / (n * pf)).sum()
        assert stats.chi2.sf(chi2, f.size - 1) > 1e-4
        # uniform inside each beamlet: the 16 sub-voxels share its count evenly
        sub_counts = hits.reshape(nv, sub, nu, sub).transpose(0, 2, 1, 3).reshape(-1, sub * sub)
        ex = sub_counts.sum(axis=1, keepdims=True) / (sub * sub)
        chi2 = ((sub_counts - ex) ** 2 / ex).sum()
        assert stats.chi2.sf(chi2, f.size * (sub * sub - 1)) > 1e-4


def test_mh_chains_one_chain_is_the_single_chain_and_counts_add_up(oracle):
    f = I.bowtie_fluence(16, 4, seed=2).ravel()
    for n in (1, 1000, 123_457):
        assert np.array_equal(oracle.mh_chains(f, n, seed=9, chains=1, i0=5), oracle.mh_counts(f, n, seed=9, i0=5))
        for chains in (2, 7, 1000):
            c = oracle.mh_chains(f, n, seed=9, chains=chains, i0=5)
            assert int(c.sum()) == n
    # chains of one particle each visit the trial or stay at i0: every trial beamlet whose
    # intensity is at least i0's is accepted
    n = 20_000
    c = oracle.mh_chains(f, n, seed=3, chains=n, i0=5)
    assert c[5] >= n // f.size


def test_mh_chains_converge_like_the_single_chain(oracle):
    # long chains: the visit frequencies approach f / sum f; one chain per particle
    # never moves far from i0 and stays biased
    f = I.bowtie_fluence(32, 8, seed=4).ravel()
    p = f / f.sum()
    n = 2_000_000
    e_long = np.linalg.norm(oracle.mh_chains(f, n, seed=5, chains=16) / n - p) / np.linalg.norm(p)
    e_short = np.linalg.norm(oracle.mh_chains(f, n, seed=5, chains=n // 4) / n - p) / np.linalg.norm(p)
    assert e_long < 0.05 and e_short > 2 * e_long
