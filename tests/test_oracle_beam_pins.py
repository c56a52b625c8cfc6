"""Pins of the oracle's Gaussian beam convolution (Sec. 4.11): a point
source becomes the sampled beam with unit sum and the requested FWHM, a flat
sky stays flat away from the edges, and the separable passes equal a
brute-force 2-D convolution.  CPU only."""
import math

import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("fwhm", [2.0, 3.0, 7.5])
def test_point_source_becomes_the_beam(fwhm):
    n = 61
    img = np.zeros((1, n, n))
    img[0, 30, 30] = 1.0
    out = oracle.beam_convolve(img, fwhm)[0]
    assert out.sum() == pytest.approx(1.0, rel=1e-12)
    # the row through the peak is the sampled beam: ln(G(0) / G(d)) =
    # d^2 / (2 sigma^2), so the neighbours give sigma and thus the FWHM
    row = out[30]
    for d in (1, 2):
        sigma = math.sqrt(d * d / (2.0 * math.log(row[30] / row[30 + d])))
        assert 2.0 * math.sqrt(2.0 * math.log(2.0)) * sigma == pytest.approx(fwhm, rel=1e-10)
    np.testing.assert_allclose(out[30], out[:, 30], rtol=1e-13)   # round beam


def test_flat_sky_stays_flat_inside():
    img = np.full((2, 40, 50), 3.0)
    out = oracle.beam_convolve(img, 4.0)
    R = (len(oracle.beam_kernel(4.0)) - 1) // 2
    np.testing.assert_allclose(out[:, R:-R, R:-R], 3.0, rtol=1e-13)
    assert out[0, 0, 0] < 3.0   # the sky outside the image is empty


def test_separable_passes_equal_brute_force_2d():
    rng = np.random.default_rng(6)
    img = rng.uniform(size=(1, 9, 11))
    w = oracle.beam_kernel(2.5)
    R = (len(w) - 1) // 2
    brute = np.zeros_like(img)
    for y in range(9):
        for x in range(11):
            s = 0.0
            for dy in range(-R, R + 1):
                for dx in range(-R, R + 1):
                    yy, xx = y + dy, x + dx
                    if 0 <= yy < 9 and 0 <= xx < 11:
                        s += w[dy + R] * w[dx + R] * img[0, yy, xx]
            brute[0, y, x] = s
    np.testing.assert_allclose(oracle.beam_convolve(img, 2.5), brute, rtol=1e-13)
