"""Pin of the stratified spectrum allocation (Sec. 2.2.5): histories are
distributed to the 1 keV intervals in proportion to the spectrum.  The oracle's
largest-remainder allocation is compared with an exact rational enumeration."""
from fractions import Fraction

import numpy as np
import pytest

from paper_1109_3266_gb300 import inputs as I


def exact_largest_remainder(n, w):
    W = sum(Fraction(x) for x in w)
    q = [Fraction(n) * Fraction(x) / W for x in w]
    base = [int(x) for x in q]                 # floor of non-negative rationals
    rem = n - sum(base)
    order = sorted(range(len(w)), key=lambda j: (-(q[j] - base[j]), j))
    order = [j for j in order if w[j] > 0]
    for j in order[:rem]:
        base[j] += 1
    return base


@pytest.mark.parametrize("seed", range(8))
def test_allocation_matches_exact_enumeration(oracle, seed):
    rng = np.random.default_rng(seed)
    nb = int(rng.integers(1, 150))
    w = rng.uniform(0, 1, nb)
    w[rng.uniform(size=nb) < 0.1] = 0.0
    if w.sum() == 0:
        w[0] = 1.0
    for n in (0, 1, 7, 999, 10 ** 5 + 3, 10 ** 8 + 17):
        got = oracle.allocate(n, w)
        assert got.sum() == n
        assert list(got) == exact_largest_remainder(n, list(w))


def test_allocation_ties_go_to_lower_bin(oracle):
    got = oracle.allocate(5, [1.0, 1.0, 1.0, 1.0])
    assert list(got) == [2, 1, 1, 1]
    got = oracle.allocate(2, [0.0, 1.0, 0.0, 1.0, 1.0])
    assert list(got) == [0, 1, 0, 1, 0]


def test_allocation_of_kramers_spectrum(oracle):
    sp = I.spectrum_kramers(120, 2.5)
    got = oracle.allocate(10 ** 8, sp.w)
    assert got.sum() == 10 ** 8
    assert got[:5].sum() == 0                          # below ~6 keV the filter leaves nothing
    q = 10 ** 8 * sp.w / sp.w.sum()
    assert np.all(np.abs(got - q) < 1)
