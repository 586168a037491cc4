"""Pins of the oracle's structure-aware initialisation (Sec. 3.2, "Structure-aware
Initialization"; Tab. S1 window 7, base probability 0.1, colour std 0.02), CPU only:
the local variance against brute-force windows and a closed form, the sampling
against the inverse-CDF of its weights and the law of large numbers, and the
parameter formulas at the drawn pixels."""
import math

import numpy as np
import pytest

import oracle


def brute_local_variance(img):
    _, H, W = img.shape
    lv = np.zeros((H, W))
    for y in range(H):
        for x in range(W):
            win = img[:, max(0, y - 3):min(H, y + 4), max(0, x - 3):min(W, x + 4)].astype(np.float64)
            lv[y, x] = np.mean([np.var(win[c]) for c in range(3)])
    return lv


def test_local_variance_is_the_clipped_7x7_window_variance_averaged_over_rgb():
    img = np.random.default_rng(0).uniform(0, 1, (3, 23, 19)).astype(np.float32)
    np.testing.assert_allclose(oracle.local_variance(img), brute_local_variance(img), rtol=1e-12, atol=1e-15)


def test_local_variance_closed_forms():
    assert np.all(oracle.local_variance(np.full((3, 12, 9), 0.37, np.float32)) == 0.0)
    # checkerboard of 0 / 1: an interior 7 x 7 window holds 25 of one value and 24 of
    # the other, variance 25 * 24 / 49^2 in every channel
    yy, xx = np.mgrid[0:15, 0:15]
    cb = np.broadcast_to(((yy + xx) % 2).astype(np.float32), (3, 15, 15)).copy()
    lv = oracle.local_variance(cb)
    np.testing.assert_allclose(lv[3:12, 3:12], 25 * 24 / 49 ** 2, rtol=1e-14)


def draws(seed, N):
    g = np.random.default_rng(seed)
    return g.uniform(0, 1, N), g.uniform(0, 1, N), g.normal(size=(N, 3))


def test_constant_image_draws_each_pixel_at_the_middle_of_its_cdf_interval():
    H, W = 9, 7
    img = np.full((3, H, W), 0.5, np.float32)
    u = (np.arange(H * W) + 0.5) / (H * W)
    p, nlv, pix, total = oracle.structure_init(img, u, np.zeros(H * W), np.zeros((H * W, 3)), (2.0, 8.0))
    assert np.all(nlv == 0.0) and total == H * W * math.floor(0.1 * 2 ** 20)
    np.testing.assert_array_equal(pix, np.arange(H * W))
    np.testing.assert_array_equal(p[:, 0], np.arange(H * W) % W)    # pixel centres
    np.testing.assert_array_equal(p[:, 1], np.arange(H * W) // W)
    assert np.all(p[:, 2] == 8.0)                                   # flat: s_max


def test_draws_follow_the_weights():
    """Left half flat, right half noisy: NLV ~ 0 on the left, so each left pixel
    weighs 0.1 and each right pixel 0.1 + 0.9 NLV; with 200k draws the share landing
    on the right matches its share of the weight within 5 standard deviations."""
    H, W = 32, 32
    g = np.random.default_rng(3)
    img = np.full((3, H, W), 0.4, np.float32)
    img[:, :, 16:] = g.uniform(0, 1, (3, H, 16))
    N = 200_000
    u, ut, nc = draws(4, N)
    p, nlv, pix, total = oracle.structure_init(img, u, ut, nc, (2.0, 8.0))
    w = 0.1 + 0.9 * nlv
    share = w[:, 16:].sum() / w.sum()
    got = np.mean(pix % W >= 16)
    assert abs(got - share) < 5 * math.sqrt(share * (1 - share) / N), (got, share)
    # and per pixel: counts against N w / sum w (chi-square with 1023 dof, generous bound)
    cnt = np.bincount(pix, minlength=H * W)
    exp = N * w.ravel() / w.sum()
    chi2 = float(((cnt - exp) ** 2 / exp).sum())
    assert chi2 < 1023 + 6 * math.sqrt(2 * 1023), chi2


def test_parameters_at_the_drawn_pixels():
    g = np.random.default_rng(5)
    img = g.uniform(0, 1, (3, 40, 30)).astype(np.float32)
    img[:, :10] = 0.8     # a flat band: NLV low there
    N = 3000
    u, ut, nc = draws(6, N)
    s_min, s_max, nu = 2.0, 10.0, -2.0
    p, nlv, pix, _ = oracle.structure_init(img, u, ut, nc, (s_min, s_max), sigma_c=0.0, nu=nu)
    assert nlv.min() == 0.0 and nlv.max() == 1.0
    lv = oracle.local_variance(img).ravel()
    np.testing.assert_allclose(nlv.ravel(), (lv - lv.min()) / (lv.max() - lv.min()), rtol=0, atol=1e-15)
    np.testing.assert_allclose(p[:, 2], s_max - (s_max - s_min) * nlv.ravel()[pix], rtol=1e-15)
    np.testing.assert_allclose(p[:, 3], 2 * math.pi * ut, rtol=1e-15)
    assert np.all(p[:, 4] == nu)
    chat = np.clip(img.reshape(3, -1)[:, pix].T.astype(np.float64), 1e-4, 1 - 1e-4)
    np.testing.assert_allclose(p[:, 5:8], np.log(chat / (1 - chat)), rtol=1e-13, atol=1e-13)
    # the highest-variance pixel gets the smallest scale
    top = int(np.argmax(nlv.ravel()))
    if np.any(pix == top):
        assert np.all(p[pix == top, 2] == s_min)
    # colour noise: sigma_c shifts the activated colour by sigma_c * n (before the clamp)
    p2, _, pix2, _ = oracle.structure_init(img, u, ut, nc, (s_min, s_max), sigma_c=0.02, nu=nu)
    np.testing.assert_array_equal(pix2, pix)
    c2 = 1 / (1 + np.exp(-p2[:, 5:8]))
    inside = (chat + 0.02 * nc > 2e-4) & (chat + 0.02 * nc < 1 - 2e-4)
    np.testing.assert_allclose(c2[inside], (chat + 0.02 * nc)[inside], rtol=0, atol=1e-12)


def test_masked_draws_stay_inside_the_mask_and_an_all_ones_mask_changes_nothing():
    g = np.random.default_rng(7)
    img = g.uniform(0, 1, (3, 30, 40)).astype(np.float32)
    yy, xx = np.mgrid[0:30, 0:40]
    mask = (((yy - 15) ** 2 + (xx - 20) ** 2) < 100).astype(np.float32)
    u, ut, nc = draws(8, 4000)
    p, _, pix, total = oracle.structure_init(img, u, ut, nc, (2.0, 8.0), mask=mask)
    assert total > 0 and np.all(mask.ravel()[pix] > 0)
    p1, _, pix1, _ = oracle.structure_init(img, u, ut, nc, (2.0, 8.0), mask=np.ones((30, 40), np.float32))
    p0, _, pix0, _ = oracle.structure_init(img, u, ut, nc, (2.0, 8.0))
    np.testing.assert_array_equal(pix1, pix0)
    np.testing.assert_array_equal(p1, p0)
    pe, _, pixe, te = oracle.structure_init(img, u, ut, nc, (2.0, 8.0), mask=np.zeros((30, 40), np.float32))
    assert te == 0 and np.all(pixe == -1) and np.all(pe == 0)


def test_reinit_replaces_exactly_the_transparent_primitives():
    """Sec. S3 "Re-initialization Mechanism": sigmoid(nu) < 0.3 -> redrawn."""
    g = np.random.default_rng(9)
    img = g.uniform(0, 1, (3, 32, 32)).astype(np.float32)
    N = 300
    params = g.normal(size=(N, 8))
    params[:, 4] = g.uniform(-3, 3, N)
    u, ut, nc = draws(10, N)
    new, idx = oracle.structure_reinit(params, img, None, u, ut, nc, (2.0, 8.0), threshold=0.3)
    low = 1 / (1 + np.exp(-params[:, 4])) < 0.3
    np.testing.assert_array_equal(np.sort(idx), np.nonzero(low)[0])
    np.testing.assert_array_equal(new[~low], params[~low])
    drawn = oracle.structure_init(img, u, ut, nc, (2.0, 8.0))[0]
    np.testing.assert_array_equal(new[low], drawn[low])


def test_alpha_loss_reduces_to_mse_and_its_gradients_match_finite_differences():
    g = np.random.default_rng(11)
    I = g.uniform(0, 1, (3, 9, 11))
    It = g.uniform(0, 1, (3, 9, 11))
    T = g.uniform(0, 1, (9, 11))
    a = g.uniform(0, 1, (9, 11))
    L, dI, dA = oracle.alpha_loss(I, T, It, np.ones_like(a), 0.0)
    assert L == pytest.approx(oracle.mse(I, It), rel=1e-14)
    np.testing.assert_allclose(dI, oracle.mse_grad(I, It), rtol=1e-14)
    assert np.all(dA == 0)
    a[a < 0.3] = 0.0                           # some pixels outside the object
    L, dI, dA = oracle.alpha_loss(I, T, It, a, 0.3)
    assert np.all(dI[:, a == 0] == 0)
    h = 1e-6
    for (c, y, x) in [(0, 2, 3), (2, 8, 10), (1, 0, 0)]:
        Ip, Im = I.copy(), I.copy()
        Ip[c, y, x] += h
        Im[c, y, x] -= h
        fd = (oracle.alpha_loss(Ip, T, It, a, 0.3)[0] - oracle.alpha_loss(Im, T, It, a, 0.3)[0]) / (2 * h)
        assert fd == pytest.approx(dI[c, y, x], rel=1e-6, abs=1e-12)
    for (y, x) in [(1, 1), (4, 7), (8, 0)]:
        # I_alpha = 1 - T: dL/dI_alpha = -dL/dT
        Tp, Tm = T.copy(), T.copy()
        Tp[y, x] += h
        Tm[y, x] -= h
        fd = (oracle.alpha_loss(I, Tp, It, a, 0.3)[0] - oracle.alpha_loss(I, Tm, It, a, 0.3)[0]) / (2 * h)
        assert -fd == pytest.approx(dA[y, x], rel=1e-6, abs=1e-12)
