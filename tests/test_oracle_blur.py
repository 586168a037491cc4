"""Pins of the oracle's Gaussian blur of the primitive bitmaps (Sec. 3.2 "Blurring
Primitives for Enriching Gradients"; Tab. S1 blur_sigma 1.0), CPU only: against
scipy.ndimage.gaussian_filter with the same radius and zero padding, the impulse
response, and conservation of mass for a bitmap with a zero border."""
import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("sigma", [0.5, 1.0, 1.1, 2.5])
def test_matches_scipy_gaussian_filter(sigma):
    nd = pytest.importorskip("scipy.ndimage")
    t = np.random.default_rng(0).uniform(0, 1, (2, 21, 30)).astype(np.float32)
    r = oracle.blur_radius(sigma)
    ref = np.stack([nd.gaussian_filter(t[i].astype(np.float64), sigma, mode="constant", cval=0.0, radius=r)
                    for i in range(2)])
    np.testing.assert_allclose(oracle.gaussian_blur(t, sigma), ref, rtol=0, atol=1e-14)


def test_impulse_response_is_the_normalised_kernel():
    sigma = 1.0
    r = oracle.blur_radius(sigma)
    t = np.zeros((1, 15, 15))
    t[0, 7, 7] = 1.0
    out = oracle.gaussian_blur(t, sigma)[0]
    d = np.arange(-r, r + 1)
    g = np.exp(-d ** 2 / 2.0)
    g /= g.sum()
    np.testing.assert_allclose(out[7 - r:8 + r, 7 - r:8 + r], np.outer(g, g), rtol=1e-14, atol=1e-17)
    assert out.sum() == pytest.approx(1.0, abs=1e-14)
    assert np.all(out[:7 - r] == 0) and np.all(out[:, 8 + r:] == 0)


def test_mass_is_kept_when_the_border_is_wide_enough_and_lost_at_the_edge():
    g = np.random.default_rng(1)
    t = np.zeros((1, 30, 30))
    t[0, 5:25, 5:25] = g.uniform(0, 1, (20, 20))
    assert oracle.gaussian_blur(t, 1.5)[0].sum() == pytest.approx(t.sum(), rel=1e-13)
    edge = np.zeros((1, 10, 10))
    edge[0, 0, 0] = 1.0
    # a corner texel keeps the quarter-plane part of its kernel (r = 3 at sigma = 1)
    g1 = np.exp(-np.arange(-3, 4) ** 2 / 2.0)
    g1 /= g1.sum()
    assert oracle.gaussian_blur(edge, 1.0)[0].sum() == pytest.approx(g1[3:].sum() ** 2, rel=1e-13)
