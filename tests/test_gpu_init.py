"""Structure-aware initialisation on the GPU against its FP64 oracle, through the C
ABI: the normalised local variance bit for bit (both sides take the same FP64
operations in the same order), the drawn pixels exactly (exact integer cumulative
weights), scale, angle and opacity as the float32 rounding of the oracle's FP64
values, and colours within float32 rounding of the logit."""
import numpy as np
import pytest

import oracle
from paper_2602_22625_gb300 import dbmp as D
from paper_2602_22625_gb300 import inputs
from _helpers import cuda, to_dev, torch

pytestmark = pytest.mark.gpu


def make_image(seed, H, W):
    """A smooth gradient with a noisy rectangle and a few hard-edged discs."""
    g = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:H, 0:W] / max(H, W)
    img = np.stack([0.2 + 0.5 * xx, 0.3 + 0.4 * yy, 0.5 + 0.2 * xx * yy])
    img[:, H // 4:H // 2, W // 3:2 * W // 3] = g.uniform(0, 1, (3, H // 2 - H // 4, 2 * W // 3 - W // 3))
    for _ in range(6):
        cy, cx, r = g.uniform(0, H), g.uniform(0, W), g.uniform(2, max(3, H / 8))
        img[:, (np.mgrid[0:H, 0:W][0] - cy) ** 2 + (np.mgrid[0:H, 0:W][1] - cx) ** 2 < r * r] = g.uniform(0, 1, (3, 1))
    return np.clip(img, 0, 1).astype(np.float32)


def gpu_init(img, N, seed, s_range=(2.0, 8.0), sigma_c=0.02, nu=-2.0):
    cuda()
    _, H, W = img.shape
    u, ut, nc = inputs.init_draws(seed, N)
    params = torch.full((N, 8), -123.0, device="cuda")
    nlv = torch.empty(H, W, dtype=torch.float64, device="cuda")
    D.dbmp_structure_init(to_dev(img), to_dev(u), to_dev(ut), to_dev(nc), s_range[0], s_range[1], sigma_c, nu,
                          params, nlv)
    torch.cuda.synchronize()
    ref, rnlv, pix, _ = oracle.structure_init(img, u, ut, nc, s_range, sigma_c, nu)
    return params.cpu().numpy(), nlv.cpu().numpy(), ref, rnlv, pix


def check(img, N, seed, **kw):
    got, nlv, ref, rnlv, pix = gpu_init(img, N, seed, **kw)
    np.testing.assert_array_equal(nlv, rnlv)                       # FP64, bit for bit
    np.testing.assert_array_equal(got[:, :2], ref[:, :2])          # the drawn pixels
    np.testing.assert_array_equal(got[:, 2:5], ref[:, 2:5].astype(np.float32))
    np.testing.assert_allclose(got[:, 5:8], ref[:, 5:8].astype(np.float32), rtol=1e-6, atol=1e-6)
    return got, pix


@pytest.mark.parametrize("shape", [(37, 53), (16, 16), (100, 7), (64, 200)])
def test_matches_oracle_ragged_shapes(shape):
    H, W = shape
    check(make_image(1, H, W), 2000, 2)


def test_flat_image_and_single_pixel():
    got, pix = check(np.full((3, 24, 40), 0.25, np.float32), 500, 3)
    assert np.all(got[:, 2] == 8.0)
    got, pix = check(np.full((3, 1, 1), 0.7, np.float32), 50, 4)
    assert np.all(got[:, :2] == 0.0)


def test_rendered_target_256():
    """The learned-initialisation targets: a 256 x 256 render of 512 anchored primitives."""
    from paper_2602_22625_gb300 import proposer
    scenes = proposer.SceneRenderer(max_batch=1)
    try:
        tp = torch.from_numpy(inputs.anchored(77, 1)).cuda()
        tgt = torch.empty(1, 3, 256, 256, device="cuda")
        scenes.render(tp, tgt)
        torch.cuda.synchronize()
        check(tgt[0].cpu().numpy(), 512, 5, s_range=(6.0, 14.0))
    finally:
        scenes.close()


def test_full_size_canvas():
    """1024 x 1024, 20 000 draws (the main workload's canvas and primitive count)."""
    check(make_image(6, 1024, 1024), 20000, 7)


def test_argument_errors():
    cuda()
    img = torch.zeros(3, 8, 8, device="cuda")
    u = torch.zeros(4, dtype=torch.float64, device="cuda")
    nc = torch.zeros(4, 3, dtype=torch.float64, device="cuda")
    p = torch.zeros(4, 8, device="cuda")
    with pytest.raises(D.DbmpError):
        D.dbmp_structure_init(img, u, u, nc, 8.0, 2.0, 0.02, -2.0, p)       # s_min > s_max
    with pytest.raises(D.DbmpError):
        D.dbmp_structure_init(img, u, u, nc, 2.0, 8.0, -1.0, -2.0, p)       # sigma_c < 0
    with pytest.raises(D.DbmpError):
        D.dbmp_structure_init_scratch_bytes(0, 5)


def disc_mask(H, W, cy, cx, r):
    yy, xx = np.mgrid[0:H, 0:W]
    return (((yy - cy) ** 2 + (xx - cx) ** 2) < r * r).astype(np.float32)


def test_masked_draws_match_oracle_and_an_empty_mask_draws_nothing():
    cuda()
    img = make_image(8, 90, 120)
    mask = disc_mask(90, 120, 45, 60, 30)
    N = 3000
    u, ut, nc = inputs.init_draws(9, N)
    params = torch.full((N, 8), -123.0, device="cuda")
    D.dbmp_structure_init(to_dev(img), to_dev(u), to_dev(ut), to_dev(nc), 2.0, 8.0, 0.02, -2.0, params,
                          mask=to_dev(mask))
    torch.cuda.synchronize()
    ref, _, pix, _ = oracle.structure_init(img, u, ut, nc, (2.0, 8.0), 0.02, -2.0, mask)
    got = params.cpu().numpy()
    np.testing.assert_array_equal(got[:, :2], ref[:, :2])
    assert np.all(mask.ravel()[pix] > 0)
    np.testing.assert_array_equal(got[:, 2:5], ref[:, 2:5].astype(np.float32))
    params.fill_(-123.0)
    D.dbmp_structure_init(to_dev(img), to_dev(u), to_dev(ut), to_dev(nc), 2.0, 8.0, 0.02, -2.0, params,
                          mask=torch.zeros(90, 120, device="cuda"))
    torch.cuda.synchronize()
    assert bool((params == -123.0).all())


def test_reinit_matches_oracle_and_resets_adam_moments():
    cuda()
    img = make_image(10, 64, 64)
    mask = disc_mask(64, 64, 32, 32, 20)
    N = 2000
    g = np.random.default_rng(11)
    p0 = g.normal(size=(N, 8)).astype(np.float32)
    p0[:, 4] = g.uniform(-3, 3, N).astype(np.float32)
    u, ut, nc = inputs.init_draws(12, N)
    params = to_dev(p0)
    m = torch.ones(N, 8, device="cuda")
    v = torch.full((N, 8), 2.0, device="cuda")
    count = torch.zeros(1, dtype=torch.int32, device="cuda")
    D.dbmp_structure_reinit(to_dev(img), to_dev(u), to_dev(ut), to_dev(nc), 2.0, 8.0, 0.02, -2.0, 0.3, params,
                            m, v, count, mask=to_dev(mask))
    torch.cuda.synchronize()
    ref, idx = oracle.structure_reinit(p0, img, mask, u, ut, nc, (2.0, 8.0), 0.3)
    got = params.cpu().numpy()
    low = np.zeros(N, bool)
    low[idx] = True
    assert int(count.item()) == low.sum() > 0
    np.testing.assert_array_equal(got[~low], p0[~low])
    np.testing.assert_array_equal(got[low, :5], ref[low, :5].astype(np.float32))
    np.testing.assert_allclose(got[low, 5:], ref[low, 5:].astype(np.float32), rtol=1e-6, atol=1e-6)
    mm, vv = m.cpu().numpy(), v.cpu().numpy()
    assert np.all(mm[low] == 0) and np.all(vv[low] == 0) and np.all(mm[~low] == 1) and np.all(vv[~low] == 2)


def test_alpha_loss_matches_oracle():
    """Eq. 9 with the paper's opacity weight 0.3 (Sec. S3)."""
    cuda()
    g = np.random.default_rng(13)
    H, W = 77, 45
    I = g.uniform(0, 1, (3, H, W)).astype(np.float32)
    It = g.uniform(0, 1, (3, H, W)).astype(np.float32)
    T = g.uniform(0, 1, (H, W)).astype(np.float32)
    a = disc_mask(H, W, 38, 22, 18) * g.uniform(0.5, 1, (H, W)).astype(np.float32)
    dI = torch.empty(3, H, W, device="cuda")
    dA = torch.empty(H, W, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    D.dbmp_alpha_loss_grad(to_dev(I), to_dev(T), to_dev(It), to_dev(a), 0.3, dI, dA, loss)
    torch.cuda.synchronize()
    L, gI, gA = oracle.alpha_loss(I, T, It, a, 0.3)
    # differences and residuals are formed in float32 (one rounding each), sums compensated.
    # The opacity residual (1 - T) - alpha* rounds 1 - T first: its absolute error is up
    # to ~1 ulp of 1 (1.2e-7), large relative to a residual that nearly cancels, so its
    # gradient gets an absolute bound of 2.4e-7 times the scale 2 lambda / n.
    assert loss.item() == pytest.approx(L, rel=2e-7)
    np.testing.assert_allclose(dI.cpu().numpy(), gI, rtol=1e-6, atol=1e-12)
    np.testing.assert_allclose(dA.cpu().numpy(), gA, rtol=1e-6, atol=2.4e-7 * 2 * 0.3 / (H * W))
