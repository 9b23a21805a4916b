"""Pins of the oracle's random numbers: Philox4x32-10 against the published
known-answer vectors, and the uniform mapping's exactness and range."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def test_philox_known_answers(oracle):
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert oracle.philox(v[0:4], v[4:6]) == v[6:10]


def test_philox_counter_and_key_sensitivity(oracle):
    base = oracle.philox([1, 2, 3, 4], [5, 6])
    for i in range(4):
        ctr = [1, 2, 3, 4]
        ctr[i] ^= 1
        assert oracle.philox(ctr, [5, 6]) != base
    assert oracle.philox([1, 2, 3, 4], [5, 7]) != base


def test_uniform_grid_is_exact_and_open(oracle):
    # u = (2 (x >> 9) + 1) 2^-24: odd multiples of 2^-24, never 0 or 1
    assert oracle.uniform(0) == 2.0 ** -24
    assert oracle.uniform(0xFFFFFFFF) == 1.0 - 2.0 ** -24
    xs = np.random.default_rng(0).integers(0, 2 ** 32, 20000, dtype=np.uint64)
    us = np.array([oracle.uniform(int(x)) for x in xs])
    assert np.all(us.astype(np.float32).astype(np.float64) == us)
    k = (us * 2 ** 24 - 1) / 2
    assert np.all(k == np.floor(k))
    assert np.all(k == (xs >> np.uint64(9)).astype(np.float64))


def test_uniform_binary32_forms(oracle):
    # the binary32 mapping equals the binary64 definition; and the one-subtraction
    # construction from bits, (1 + k 2^-23) - (1 - 2^-24) in binary32, is exact for
    # every significand k (2k + 1 < 2^24 fits), so it gives the same grid
    xs = np.random.default_rng(1).integers(0, 2 ** 32, 20000, dtype=np.uint64)
    f = oracle.uniform_f32(xs.astype(np.uint32))
    assert np.array_equal(f.astype(np.float64), np.array([oracle.uniform(int(x)) for x in xs]))
    k = np.arange(2 ** 23, dtype=np.uint32)
    a = (k | np.uint32(0x3F800000)).view(np.float32)
    one_sub = a - np.float32(1.0 - 2.0 ** -24)
    assert one_sub.dtype == np.float32
    assert np.array_equal(one_sub, oracle.uniform_f32(k << np.uint32(9)))


def test_philox_uniforms_are_uniform(oracle):
    # a million uniforms from consecutive counters: mean, variance, 64-bin chi-square
    n = 250000
    u = np.array([oracle.uniform(w) for i in range(n) for w in oracle.philox([i, 0, 7, 0], [42, 0])])
    assert abs(u.mean() - 0.5) < 5 * np.sqrt(1 / 12 / u.size)
    assert abs(u.var() - 1 / 12) < 5 * np.sqrt(1 / 180 / u.size)
    h, _ = np.histogram(u, bins=64, range=(0, 1))
    e = u.size / 64
    chi2 = ((h - e) ** 2 / e).sum()
    assert chi2 < 63 + 6 * np.sqrt(2 * 63)
