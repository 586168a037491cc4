"""Pins of the proposal network's FP64 oracle (CPU only): convolution, its adjoint
and the weight gradient against torch float64 conv2d + autograd; the whole
network's gradient against central finite differences; bf16 rounding against
torch's bfloat16 conversion; decode/target round trip."""
import numpy as np
import pytest

from oracle import cnn
from paper_2602_22625_gb300 import inputs

torch = pytest.importorskip("torch")
F = torch.nn.functional


def test_bf16_rounding_matches_torch():
    x = np.random.default_rng(0).normal(size=10000) * np.logspace(-3, 3, 10000)
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).double().numpy()
    np.testing.assert_array_equal(cnn.bf16(x), ref)


def test_conv_forward_and_adjoints_match_torch():
    rng = np.random.default_rng(1)
    B, H, W, C, Cout = 2, 12, 10, 8, 5
    X = rng.normal(size=(B, H, W, C))
    Wt = rng.normal(size=(Cout, C, 4, 4))
    b = rng.normal(size=Cout)
    Xt = torch.tensor(X.transpose(0, 3, 1, 2), requires_grad=True)
    Wtt = torch.tensor(Wt, requires_grad=True)
    bt = torch.tensor(b, requires_grad=True)
    Y = F.conv2d(Xt, Wtt, bt, stride=2, padding=1)
    col, (_, Ho, Wo) = cnn.im2col(X)
    Wm = Wt.transpose(0, 2, 3, 1).reshape(Cout, -1)   # (Cout, (ky, kx, c))
    Yo = (col @ Wm.T + b).reshape(B, Ho, Wo, Cout)
    np.testing.assert_allclose(Yo, Y.detach().numpy().transpose(0, 2, 3, 1), rtol=0, atol=1e-12)
    G = rng.normal(size=Yo.shape)
    (Y * torch.tensor(G.transpose(0, 3, 1, 2))).sum().backward()
    g2 = G.reshape(-1, Cout)
    dW = (g2.T @ col).reshape(Cout, 4, 4, C).transpose(0, 3, 1, 2)
    np.testing.assert_allclose(dW, Wtt.grad.numpy(), rtol=0, atol=1e-11)
    np.testing.assert_allclose(g2.sum(0), bt.grad.numpy(), atol=1e-12)
    dX = cnn.col2im(g2 @ Wm, X.shape)
    np.testing.assert_allclose(dX, Xt.grad.numpy().transpose(0, 2, 3, 1), rtol=0, atol=1e-11)


def test_network_gradient_matches_finite_differences():
    rng = np.random.default_rng(2)
    theta = inputs.cnn_init(3).astype(np.float64)
    theta += rng.normal(size=theta.shape) * 0.01   # non-zero biases too
    images = rng.uniform(0, 1, (1, 3, 256, 256))
    tp = inputs.anchored(4, 1)
    O, cache = cnn.forward(theta, images, rnd=False)
    L, dO = cnn.loss_and_grad(O, tp)
    g = cnn.backward(dO, cache)
    sizes = [(c * k * k * cp, c) for cp, _, c, k in cnn.LAYERS]
    offs = np.cumsum([0] + [a + b for a, b in sizes])
    picks = []
    for li, (nw, nb) in enumerate(sizes):
        picks += list(offs[li] + rng.choice(nw, 2, replace=False)) + [offs[li] + nw + rng.integers(nb)]
    for i in picks:
        h = 1e-7  # small enough that no ReLU pre-activation crosses zero inside the step
        tp_ = theta.copy(); tp_[i] += h
        tm_ = theta.copy(); tm_[i] -= h
        Lp = cnn.loss_and_grad(cnn.forward(tp_, images, rnd=False)[0], tp)[0]
        Lm = cnn.loss_and_grad(cnn.forward(tm_, images, rnd=False)[0], tp)[0]
        fd = (Lp - Lm) / (2 * h)
        # FP64 roundoff of the difference quotient is ~1e-16 * L / h ~ 1e-9 absolute
        assert fd == pytest.approx(g[i], rel=1e-3, abs=2e-9), (i, fd, g[i])


def test_decode_inverts_targets():
    tp = inputs.anchored(5, 2)
    t = cnn.targets(tp)
    O = t.reshape(2, 64, 64).reshape(128, 64)
    p = cnn.decode(O)
    inside = np.all(np.abs((t[..., :3])) < np.log(0.98 / 0.02) - 1e-9, axis=-1)
    np.testing.assert_allclose(p[..., :3][inside], tp[..., :3][inside], atol=1e-4)
    np.testing.assert_allclose(p[..., 4:], np.clip(tp[..., 4:], -6, 6), atol=1e-6)
