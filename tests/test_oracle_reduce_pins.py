"""Pins of the oracle's latitude-mean reduction (Sec. 6.1): brute-force
loops on a tiny array, a field linear in b returns its middle value, a
constant returns itself.  CPU only."""
import numpy as np

import oracle


def test_brute_force_loops():
    rng = np.random.default_rng(2)
    a = rng.normal(size=(3, 5, 4))
    out = oracle.latitude_mean(a)
    for i in range(3):
        for c in range(4):
            s = 0.0
            for b in range(5):
                s += a[i, b, c]
            assert abs(out[i, c] - s / 5) <= 1e-15 * max(1.0, abs(s))


def test_linear_in_latitude_gives_the_middle_value():
    A, B, C = 2, 7, 3
    b = np.arange(B, dtype=float)[None, :, None]
    a = 1.5 + 0.25 * b + np.zeros((A, B, C))
    np.testing.assert_allclose(oracle.latitude_mean(a), 1.5 + 0.25 * 3.0, rtol=1e-15)
    np.testing.assert_array_equal(oracle.latitude_mean(np.full((2, 4, 5), 3.0)), 3.0)
