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
