"""Gaussian blur of the primitive bitmaps on the GPU against the FP64 oracle, through
the C ABI (Sec. 3.2 "Blurring Primitives for Enriching Gradients"; Tab. S1 sigma 1.0).
The kernel sums in float32 in two separable passes of 2r + 1 taps; the bound 2e-6 is
about 2 (2r + 1) float32 roundings of values in [0, 1] at r = 15."""
import numpy as np
import pytest

import oracle
from paper_2602_22625_gb300 import dbmp as D
from paper_2602_22625_gb300 import inputs
from _helpers import cuda, to_dev, torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape,sigma", [((1, 17, 23), 1.0), ((3, 64, 64), 0.5), ((2, 40, 70), 2.5),
                                         ((1, 5, 200), 5.0), ((4, 33, 31), 1.3)])
def test_blur_matches_oracle(shape, sigma):
    cuda()
    t = np.random.default_rng(hash(shape) % 1000).uniform(0, 1, shape).astype(np.float32)
    got = D.dbmp_blur_bitmaps(to_dev(t), sigma)
    torch.cuda.synchronize()
    np.testing.assert_allclose(got.cpu().numpy(), oracle.gaussian_blur(t, sigma), rtol=0, atol=2e-6)


def test_blur_of_the_stroke_atlas():
    """16 hard-edged 128 x 128 strokes at the paper's sigma = 1."""
    cuda()
    t = inputs.stroke_atlas(11, 16, 128, blur_sigma=0.0)
    got = D.dbmp_blur_bitmaps(to_dev(t), 1.0)
    torch.cuda.synchronize()
    np.testing.assert_allclose(got.cpu().numpy(), oracle.gaussian_blur(t, 1.0), rtol=0, atol=2e-6)


def test_blur_argument_errors():
    cuda()
    t = torch.zeros(2, 16, 16, device="cuda")
    with pytest.raises(D.DbmpError):
        D.dbmp_blur_bitmaps(t, 0.0)
    with pytest.raises(D.DbmpError):
        D.dbmp_blur_bitmaps(t, 5.5)
    with pytest.raises(D.DbmpError):
        D.dbmp_blur_bitmaps(t, 1.0, out=t)          # in place is refused
