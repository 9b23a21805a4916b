"""Pins of the single-precision logarithm and sincos of the binary32 method:
exhaustive over every uniform the generator can return, against binary64."""
import numpy as np

GRID = ((2 * np.arange(2 ** 23, dtype=np.float64) + 1) * 2.0 ** -24)


def test_log_f32_every_uniform(oracle):
    u = GRID.astype(np.float32)
    assert np.all(u.astype(np.float64) == GRID)
    got = oracle.log_f32(u).astype(np.float64)
    ref = np.log(GRID)
    ulp = np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
    err = np.abs(got - ref) / ulp
    assert err.max() <= 2.0, err.max()
    assert np.all(got < 0)


def test_log_f32_general_arguments(oracle):
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.uniform(1e-30, 1.0, 100000), rng.uniform(0.5, 2.0, 100000),
                        rng.uniform(1.0, 1e30, 100000)]).astype(np.float32)
    got = oracle.log_f32(x).astype(np.float64)
    ref = np.log(x.astype(np.float64))
    ok = np.abs(ref) > 1e-3
    rel = np.abs(got - ref)[ok] / np.abs(ref[ok])
    assert rel.max() < 3e-7
    assert np.abs(got - ref)[~ok].max() < 2e-9
    assert oracle.log_f32(np.array([1.0], np.float32))[0] == 0.0


def test_sincos_turns_every_uniform(oracle):
    t = GRID.astype(np.float32)
    c, s = oracle.sincos_turns_f32(t)
    a = 2 * np.pi * GRID
    assert np.abs(c - np.cos(a)).max() < 2.5e-7
    assert np.abs(s - np.sin(a)).max() < 2.5e-7
    n = c.astype(np.float64) ** 2 + s.astype(np.float64) ** 2
    assert np.abs(n - 1).max() < 1e-6


def test_sincos_turns_quadrants_exact(oracle):
    t = np.array([0.0, 0.25, 0.5, 0.75, 1.0, 1.25], np.float32)
    c, s = oracle.sincos_turns_f32(t)
    assert list(c) == [1, 0, -1, 0, 1, 0]
    assert list(s) == [0, 1, 0, -1, 0, 1]
