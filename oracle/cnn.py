"""FP64 reference of the learned proposal network -- TEST INFRASTRUCTURE.

Only the tests, the smoke check and the benchmark's CPU-baseline leg use this.
It shares no code with the CUDA library.

The network (a learned initialiser; the paper names learned/AR initialisation as
future work, Sec. S5, and shows that initialisation matters, Sec. 3.2.2):
  input   B x 256 x 256 x 4 (NHWC): channels 0-2 = 2 (I - 0.5), 3 = 0
  conv1-5 4x4, stride 2, padding 1, + bias, ReLU: 4(3 used)->32->64->128->256->256,
          spatial 256 -> 128 -> 64 -> 32 -> 16 -> 8
  head    1x1 conv 256 -> 64 (+ bias): 8 slots x 8 outputs per cell of the 8x8 map
Weights are stored (Cout, K) with K ordered (ky, kx, ci), ci fastest.

Mixed precision, mirrored from the GPU path so that both round at the same
points: inputs, weights, post-ReLU activations and the backward's dZ tensors are
rounded to bfloat16 (round to nearest even); a convolution's input gradient is
summed over all its (tap, channel) terms before the one rounding of the dZ it
feeds; everything else is FP64 here.  With round=False
the network is plain FP64 (used by the finite-difference pins).

Output decoding (anchored parameterisation): cell (cy, cx), slot k, outputs o_j:
  x = cx*32 + (k%4)*8 + 8 sigmoid(o0),  y = cy*32 + (k//4)*16 + 16 sigmoid(o1),
  s = 6 + 8 sigmoid(o2),  theta = 0,  nu = o4,  c = o5..o7.
Loss: mean over (scene, primitive, j in {0,1,2,4,5,6,7}) of (o_j - t_j)^2 with
t0 = logit(clip((x-bx)/8)), t1 = logit(clip((y-by)/16)), t2 = logit(clip((s-6)/8)),
clip to [0.02, 0.98]; t4 = nu, t5..7 = c clipped to [-6, 6].
"""
import math

import numpy as np

LAYERS = ((4, 3, 32, 4), (32, 32, 64, 4), (64, 64, 128, 4), (128, 128, 256, 4),
          (256, 256, 256, 4), (256, 256, 64, 1))
LOSS_W = np.array([1, 1, 1, 0, 1, 1, 1, 1], np.float64)


def bf16(x):
    """Round to bfloat16 (nearest even), returned as float64."""
    f = np.ascontiguousarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(theta):
    """Flat parameter vector -> [(W (Cout, K), b (Cout,))] per layer."""
    out, o = [], 0
    for cin_pad, _, cout, k in LAYERS:
        K = k * k * cin_pad
        W = theta[o:o + cout * K].reshape(cout, K)
        o += cout * K
        b = theta[o:o + cout]
        o += cout
        out.append((np.asarray(W, np.float64), np.asarray(b, np.float64)))
    assert o == len(theta)
    return out


def pack_input(images, rnd=True):
    """images (B, 3, 256, 256) in [0, 1] -> (B, 256, 256, 4)."""
    B, _, H, W = images.shape
    X = np.zeros((B, H, W, 4))
    X[..., :3] = (2.0 * (np.asarray(images, np.float32) - np.float32(0.5))).transpose(0, 2, 3, 1)
    return bf16(X) if rnd else X


def im2col(X, k=4, s=2, p=1):
    """(B, H, W, C) -> (B*Ho*Wo, k*k*C), columns ordered (ky, kx, c)."""
    B, H, W, C = X.shape
    Ho, Wo = (H + 2 * p - k) // s + 1, (W + 2 * p - k) // s + 1
    Xp = np.zeros((B, H + 2 * p, W + 2 * p, C))
    Xp[:, p:p + H, p:p + W] = X
    cols = np.empty((B, Ho, Wo, k, k, C))
    for ky in range(k):
        for kx in range(k):
            cols[:, :, :, ky, kx, :] = Xp[:, ky:ky + s * Ho:s, kx:kx + s * Wo:s, :]
    return cols.reshape(B * Ho * Wo, k * k * C), (B, Ho, Wo)


def col2im(dcol, shape, k=4, s=2, p=1):
    """Adjoint of im2col: (B*Ho*Wo, k*k*C) -> (B, H, W, C)."""
    B, H, W, C = shape
    Ho, Wo = (H + 2 * p - k) // s + 1, (W + 2 * p - k) // s + 1
    d = dcol.reshape(B, Ho, Wo, k, k, C)
    dXp = np.zeros((B, H + 2 * p, W + 2 * p, C))
    for ky in range(k):
        for kx in range(k):
            dXp[:, ky:ky + s * Ho:s, kx:kx + s * Wo:s, :] += d[:, :, :, ky, kx, :]
    return dXp[:, p:p + H, p:p + W]


def _mm(acc32):
    """Matrix product with FP64 accumulation, or (acc32 = 1, 2) with the operands and
    the accumulation in float32, the inner dimension summed forwards (1) or backwards
    (2).  The fp32 forms are rounding-sensitivity probes, not the reference: the
    operands are bf16 values, exact in both, so the forms differ only in how the sums
    are rounded, and their difference shows how far a change of accumulation alone
    moves each tensor through the bf16 rounding points."""
    if not acc32:
        return lambda a, b: a @ b
    f = np.float32
    if acc32 == 2:
        return lambda a, b: (np.asarray(a, f)[:, ::-1] @ np.asarray(b, f)[::-1, :]).astype(np.float64)
    return lambda a, b: (np.asarray(a, f) @ np.asarray(b, f)).astype(np.float64)


def forward(theta, images, rnd=True, acc32=False):
    """Returns (outputs O (B*64, 64), cache for backward)."""
    params = unpack(np.asarray(theta, np.float64))
    R = bf16 if rnd else (lambda a: np.asarray(a, np.float64))
    mm = _mm(acc32)
    X = pack_input(images, rnd)
    acts, cols = [X], []
    for (cin_pad, _, cout, k), (W, b) in zip(LAYERS[:-1], params[:-1]):
        col, (B, Ho, Wo) = im2col(X)
        cols.append(col)
        X = R(np.maximum(mm(col, R(W).T) + b, 0.0)).reshape(B, Ho, Wo, cout)
        acts.append(X)
    W6, b6 = params[-1]
    O = mm(X.reshape(-1, 256), R(W6).T) + b6
    return O, dict(params=params, acts=acts, cols=cols, rnd=rnd, acc32=acc32)


def anchor_bases():
    idx = np.arange(512)
    cy, cx, k = idx // 64, (idx // 8) % 8, idx % 8
    return cx * 32 + (k % 4) * 8, cy * 32 + (k // 4) * 16


def _logit(p):
    return np.log(p / (1.0 - p))


def targets(target_params):
    """(B, 512, 8) primitive parameters -> (B, 512, 8) raw network targets."""
    p = np.asarray(target_params, np.float64)
    bx, by = anchor_bases()
    t = np.zeros_like(p)
    t[..., 0] = _logit(np.clip((p[..., 0] - bx) / 8.0, 0.02, 0.98))
    t[..., 1] = _logit(np.clip((p[..., 1] - by) / 16.0, 0.02, 0.98))
    t[..., 2] = _logit(np.clip((p[..., 2] - 6.0) / 8.0, 0.02, 0.98))
    t[..., 4:8] = np.clip(p[..., 4:8], -6.0, 6.0)
    return t


def outputs_by_primitive(O):
    """(B*64, 64) head outputs -> (B, 512, 8): row m = (b, cy, cx), column = slot*8 + j."""
    B = O.shape[0] // 64
    return O.reshape(B, 64, 8, 8).reshape(B, 512, 8)


def loss_and_grad(O, target_params):
    o = outputs_by_primitive(O)
    t = targets(target_params)
    n = o.shape[0] * 512 * 7
    d = (o - t) * LOSS_W
    L = float((d * d).sum() / n)
    dO = (2.0 * d / n).reshape(O.shape)
    return L, dO


def decode(O):
    o = outputs_by_primitive(O)
    bx, by = anchor_bases()
    sig = lambda z: 1.0 / (1.0 + np.exp(-z))
    p = np.zeros_like(o)
    p[..., 0] = bx + 8.0 * sig(o[..., 0])
    p[..., 1] = by + 16.0 * sig(o[..., 1])
    p[..., 2] = 6.0 + 8.0 * sig(o[..., 2])
    p[..., 4:8] = o[..., 4:8]
    return p


def backward(dO, cache):
    """Gradient of the loss w.r.t. the flat parameter vector, same rounding points
    as the GPU: dZ tensors rounded to bf16 before each product."""
    params, acts, cols, rnd = cache["params"], cache["acts"], cache["cols"], cache["rnd"]
    R = bf16 if rnd else (lambda a: np.asarray(a, np.float64))
    mm = _mm(cache.get("acc32", False))
    grads = [None] * len(params)
    W6, _ = params[-1]
    X5 = acts[-1].reshape(-1, 256)
    dZ = R(dO)
    grads[-1] = (mm(dZ.T, X5), dO.sum(0))
    dX = mm(dZ, R(W6)).reshape(acts[-1].shape)
    for li in range(len(LAYERS) - 2, -1, -1):
        X = acts[li + 1]
        dZ = R(np.where(X > 0, dX, 0.0)).reshape(-1, LAYERS[li][2])
        W, _ = params[li]
        grads[li] = (mm(dZ.T, cols[li]), dZ.sum(0))
        if li > 0:
            dX = col2im(mm(dZ, R(W)), acts[li].shape)
    return np.concatenate([np.concatenate([g[0].ravel(), g[1]]) for g in grads])
