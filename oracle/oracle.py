"""ctypes front of the FP64 C oracle, plus the optimiser and loss in numpy FP64.

TEST INFRASTRUCTURE ONLY (tests, smoke check, the benchmark's CPU-baseline leg).

Conventions (shared with the library only through the documented ABI, not code):
  params      float32 (N, 8): x, y, s, theta, nu, c_r, c_g, c_b  (nu and c are logits)
  bitmap_id   int32 (N,)
  atlas       float32 (n_bmp, Hb, Wb), P[v, u] = atlas[b, v, u], values in [0, 1]
  image       (3, H, W) planar;  T_final (H, W);  index 0 = front layer
  background  None (b = 0, Eq. 5), an RGB triple (constant), or a (3, H, W) buffer (Eq. 8)
"""
import ctypes
import math
import os

import numpy as np

from . import build as _build

_lib = None

BG_NONE, BG_CONST, BG_BUFFER = 0, 1, 2

_f32p = ctypes.POINTER(ctypes.c_float)
_f64p = ctypes.POINTER(ctypes.c_double)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.oracle_render.restype = ctypes.c_int64
        L.oracle_render.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _f32p, _i32p,
                                    _f32p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                    ctypes.c_double, ctypes.c_int32, _f64p, _f32p, ctypes.c_double,
                                    ctypes.c_int64, _i32p, _i32p, _f64p, _f64p, _i32p, _i64p]
        L.oracle_grad.restype = None
        L.oracle_grad.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _f32p, _i32p,
                                  _f32p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                  ctypes.c_double, ctypes.c_int32, _f64p, _f32p, ctypes.c_double,
                                  _f64p, _f64p, _f64p]
        L.oracle_grad_rows.restype = None
        L.oracle_grad_rows.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _f32p, _i32p,
                                       _f32p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_double, ctypes.c_int32, _f64p, _f32p,
                                       ctypes.c_double, _f64p, _f64p, ctypes.c_int32,
                                       ctypes.c_int32, _f64p]
        L.oracle_grad_pixels.restype = None
        L.oracle_grad_pixels.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _f32p, _i32p,
                                         _f32p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_double, ctypes.c_int32, _f64p, _f32p,
                                         ctypes.c_double, _f64p, _f64p, ctypes.c_int64, _i32p, _i32p,
                                         _f64p]
        L.oracle_grad_selected.restype = None
        L.oracle_grad_selected.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _f32p,
                                           _i32p, _f32p, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_int32, ctypes.c_double, ctypes.c_int32, _f64p,
                                           _f32p, ctypes.c_double, _f32p, _f32p, ctypes.c_int32,
                                           _i32p, _f64p]
        L.oracle_eq_s5_dalpha.restype = ctypes.c_int32
        L.oracle_eq_s5_dalpha.argtypes = [ctypes.c_int32, _f32p, _i32p, _f32p, ctypes.c_int32,
                                          ctypes.c_int32, ctypes.c_double, ctypes.c_int32,
                                          ctypes.c_int32, _f64p, ctypes.c_double, _f64p, _i32p]
        L.oracle_bin_rects.restype = None
        L.oracle_bin_rects.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_int32, _f32p, _i32p, _f32p, ctypes.c_int32,
                                       ctypes.c_int32, ctypes.c_int32, _i32p, _i64p]
        L.oracle_bin.restype = ctypes.c_int64
        L.oracle_bin.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                 _f32p, _i32p, _f32p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                 _i64p, _i32p, ctypes.c_int64]
        L.oracle_nonzero_boxes.restype = None
        L.oracle_nonzero_boxes.argtypes = [_f32p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _i32p]
        L.oracle_spec_sincos.restype = ctypes.c_int
        L.oracle_spec_sincos.argtypes = [ctypes.c_float, _f32p, _f32p]
        L.oracle_spec_abs_sincos.restype = None
        L.oracle_spec_abs_sincos.argtypes = [ctypes.c_float, _f32p, _f32p]
        L.oracle_num_threads.restype = ctypes.c_int32
        L.oracle_num_threads.argtypes = []
        L.oracle_set_num_threads.restype = None
        L.oracle_set_num_threads.argtypes = [ctypes.c_int32]
        L.oracle_bin_footprint.restype = None
        L.oracle_bin_footprint.argtypes = [ctypes.c_int32, _f32p, ctypes.c_int32, ctypes.c_int32, _f64p]
        L.oracle_local_variance.restype = None
        L.oracle_local_variance.argtypes = [ctypes.c_int32, ctypes.c_int32, _f32p, _f64p]
        L.oracle_structure_init.restype = ctypes.c_int64
        L.oracle_structure_init.argtypes = [ctypes.c_int32, ctypes.c_int32, _f32p, _f32p, ctypes.c_int32, _f64p,
                                            _f64p, _f64p, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_double, _f64p, _f64p, _i32p]
        _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t) if a is not None else None


def _prep(params, bitmap_id, atlas):
    params = np.ascontiguousarray(params, dtype=np.float32).reshape(-1, 8)
    bitmap_id = np.ascontiguousarray(bitmap_id, dtype=np.int32).reshape(-1)
    atlas = np.ascontiguousarray(atlas, dtype=np.float32)
    if atlas.ndim == 2:
        atlas = atlas[None]
    assert params.shape[0] == bitmap_id.shape[0]
    if params.shape[0]:
        assert bitmap_id.min() >= 0 and bitmap_id.max() < atlas.shape[0]
    return params, bitmap_id, atlas


def _bg(background, H, W):
    if background is None:
        return BG_NONE, np.zeros(3), None
    b = np.asarray(background)
    if b.size == 3:
        return BG_CONST, np.ascontiguousarray(b, dtype=np.float64).reshape(3), None
    return BG_BUFFER, np.zeros(3), np.ascontiguousarray(b, dtype=np.float32).reshape(3, H, W)


def num_threads():
    return int(lib().oracle_num_threads())


def set_num_threads(n):
    """Threads of the oracle's later parallel loops (timing only; results unchanged)."""
    lib().oracle_set_num_threads(int(n))


def render(H, W, params, bitmap_id, atlas, alpha_max=1.0, background=(1.0, 1.0, 1.0),
           T_stop=0.0, pixels=None):
    """Forward (Eqs. 1-5, 8) in FP64.

    Returns dict(image (3,H,W) or (3,n), T_final, n_last (index of last contributing
    primitive, -1 if none), pairs (number of sampled (pixel, primitive) pairs),
    contrib (contributing pairs: layers with M > 0 composited while T >= T_stop)).
    `pixels` = (px, py) int arrays renders only those pixels."""
    params, bitmap_id, atlas = _prep(params, bitmap_id, atlas)
    mode, rgb, buf = _bg(background, H, W)
    N = params.shape[0]
    if pixels is None:
        n, px, py = H * W, None, None
    else:
        px = np.ascontiguousarray(pixels[0], dtype=np.int32)
        py = np.ascontiguousarray(pixels[1], dtype=np.int32)
        n = px.shape[0]
    image = np.empty((3, n), np.float64)
    T = np.empty(n, np.float64)
    last = np.empty(n, np.int32)
    contrib = np.zeros(1, np.int64)
    pairs = lib().oracle_render(H, W, N, _p(params, _f32p), _p(bitmap_id, _i32p),
                                _p(atlas, _f32p), atlas.shape[0], atlas.shape[1], atlas.shape[2],
                                float(alpha_max), mode, _p(rgb, _f64p), _p(buf, _f32p),
                                float(T_stop), n, _p(px, _i32p), _p(py, _i32p),
                                _p(image, _f64p), _p(T, _f64p), _p(last, _i32p), _p(contrib, _i64p))
    if pixels is None:
        image, T, last = image.reshape(3, H, W), T.reshape(H, W), last.reshape(H, W)
    return dict(image=image, T_final=T, n_last=last, pairs=int(pairs), contrib=int(contrib[0]))


def grad(H, W, params, bitmap_id, atlas, dL_dimage, dL_dalpha=None, alpha_max=1.0,
         background=(1.0, 1.0, 1.0), T_stop=0.0):
    """dL/dparams (N, 8) float64 for upstream gradients dL/dI (3,H,W) and dL/dI_alpha (H,W)."""
    params, bitmap_id, atlas = _prep(params, bitmap_id, atlas)
    mode, rgb, buf = _bg(background, H, W)
    N = params.shape[0]
    gI = np.ascontiguousarray(dL_dimage, dtype=np.float64).reshape(3, H, W)
    gA = None if dL_dalpha is None else np.ascontiguousarray(dL_dalpha, np.float64).reshape(H, W)
    out = np.zeros((N, 8), np.float64)
    lib().oracle_grad(H, W, N, _p(params, _f32p), _p(bitmap_id, _i32p), _p(atlas, _f32p),
                      atlas.shape[0], atlas.shape[1], atlas.shape[2], float(alpha_max), mode,
                      _p(rgb, _f64p), _p(buf, _f32p), float(T_stop), _p(gI, _f64p),
                      _p(gA, _f64p), _p(out, _f64p))
    return out


def grad_rows(H, W, params, bitmap_id, atlas, dL_dimage, y0, y1, dL_dalpha=None, alpha_max=1.0,
              background=(1.0, 1.0, 1.0), T_stop=0.0):
    """dL/dparams (N, 8) summed over canvas rows y0 <= y < y1 only."""
    params, bitmap_id, atlas = _prep(params, bitmap_id, atlas)
    mode, rgb, buf = _bg(background, H, W)
    N = params.shape[0]
    gI = np.ascontiguousarray(dL_dimage, dtype=np.float64).reshape(3, H, W)
    gA = None if dL_dalpha is None else np.ascontiguousarray(dL_dalpha, np.float64).reshape(H, W)
    out = np.zeros((N, 8), np.float64)
    lib().oracle_grad_rows(H, W, N, _p(params, _f32p), _p(bitmap_id, _i32p), _p(atlas, _f32p),
                           atlas.shape[0], atlas.shape[1], atlas.shape[2], float(alpha_max), mode,
                           _p(rgb, _f64p), _p(buf, _f32p), float(T_stop), _p(gI, _f64p),
                           _p(gA, _f64p), int(y0), int(y1), _p(out, _f64p))
    return out


def grad_pixels(H, W, params, bitmap_id, atlas, dL_dimage, pixels, dL_dalpha=None, alpha_max=1.0,
                background=(1.0, 1.0, 1.0), T_stop=0.0):
    """dL/dparams (N, 8) summed over the pixels (px, py) only (int arrays)."""
    params, bitmap_id, atlas = _prep(params, bitmap_id, atlas)
    mode, rgb, buf = _bg(background, H, W)
    N = params.shape[0]
    gI = np.ascontiguousarray(dL_dimage, dtype=np.float64).reshape(3, H, W)
    gA = None if dL_dalpha is None else np.ascontiguousarray(dL_dalpha, np.float64).reshape(H, W)
    px = np.ascontiguousarray(pixels[0], dtype=np.int32)
    py = np.ascontiguousarray(pixels[1], dtype=np.int32)
    out = np.zeros((N, 8), np.float64)
    lib().oracle_grad_pixels(H, W, N, _p(params, _f32p), _p(bitmap_id, _i32p), _p(atlas, _f32p),
                             atlas.shape[0], atlas.shape[1], atlas.shape[2], float(alpha_max), mode,
                             _p(rgb, _f64p), _p(buf, _f32p), float(T_stop), _p(gI, _f64p), _p(gA, _f64p),
                             px.shape[0], _p(px, _i32p), _p(py, _i32p), _p(out, _f64p))
    return out


def grad_selected(H, W, params, bitmap_id, atlas, dL_dimage, sel, dL_dalpha=None, alpha_max=1.0,
                  background=(1.0, 1.0, 1.0), T_stop=0.0):
    """dL/dparams of the primitives `sel` only ((len(sel), 8) float64)."""
    params, bitmap_id, atlas = _prep(params, bitmap_id, atlas)
    mode, rgb, buf = _bg(background, H, W)
    N = params.shape[0]
    gI = np.ascontiguousarray(dL_dimage, dtype=np.float32).reshape(3, H, W)
    gA = None if dL_dalpha is None else np.ascontiguousarray(dL_dalpha, np.float32).reshape(H, W)
    sel = np.ascontiguousarray(sel, dtype=np.int32)
    out = np.zeros((sel.shape[0], 8), np.float64)
    lib().oracle_grad_selected(H, W, N, _p(params, _f32p), _p(bitmap_id, _i32p),
                               _p(atlas, _f32p), atlas.shape[0], atlas.shape[1], atlas.shape[2],
                               float(alpha_max), mode, _p(rgb, _f64p), _p(buf, _f32p),
                               float(T_stop), _p(gI, _f32p), _p(gA, _f32p), sel.shape[0],
                               _p(sel, _i32p), _p(out, _f64p))
    return out


def eq_s5_dalpha(params, bitmap_id, atlas, x, y, g, gA=0.0, alpha_max=1.0):
    """Eq. S5 as printed (no background term) at one pixel: (dL/dalpha per layer, prim idx)."""
    params, bitmap_id, atlas = _prep(params, bitmap_id, atlas)
    N = params.shape[0]
    out = np.zeros(max(N, 1), np.float64)
    ks = np.zeros(max(N, 1), np.int32)
    g = np.ascontiguousarray(g, np.float64).reshape(3)
    n = lib().oracle_eq_s5_dalpha(N, _p(params, _f32p), _p(bitmap_id, _i32p), _p(atlas, _f32p),
                                  atlas.shape[1], atlas.shape[2], float(alpha_max), int(x), int(y),
                                  _p(g, _f64p), float(gA), _p(out, _f64p), _p(ks, _i32p))
    return out[:n], ks[:n]


def _bin_inputs(params, bitmap_id, atlas):
    params = np.ascontiguousarray(params, dtype=np.float32).reshape(-1, 8)
    bid = np.ascontiguousarray(np.broadcast_to(np.asarray(bitmap_id, np.int32), (params.shape[0],)))
    atlas = np.ascontiguousarray(atlas, dtype=np.float32)
    return params, bid, atlas


def bin_rects(H, W, tile, params, bitmap_id, atlas):
    """Per-primitive tile rectangles (N, 4) {tx0, ty0, tx1, ty1} and tau (N,)."""
    params, bid, atlas = _bin_inputs(params, bitmap_id, atlas)
    N = params.shape[0]
    nb, Hb, Wb = atlas.shape
    rects = np.zeros((max(N, 1), 4), np.int32)
    tau = np.zeros(max(N, 1), np.int64)
    lib().oracle_bin_rects(H, W, tile, N, _p(params, _f32p), _p(bid, _i32p), _p(atlas, _f32p), nb, Hb, Wb,
                           _p(rects, _i32p), _p(tau, _i64p))
    return rects[:N], tau[:N]


def bin(H, W, tile, params, bitmap_id, atlas):
    """Tile lists (Sec. 3.1.1): (offsets (n_tiles+1,) int64, list (K,) int32)."""
    params, bid, atlas = _bin_inputs(params, bitmap_id, atlas)
    N = params.shape[0]
    nb, Hb, Wb = atlas.shape
    ntx, nty = -(-W // tile), -(-H // tile)
    offsets = np.zeros(ntx * nty + 1, np.int64)
    args = (H, W, tile, N, _p(params, _f32p), _p(bid, _i32p), _p(atlas, _f32p), nb, Hb, Wb)
    K = lib().oracle_bin(*args, _p(offsets, _i64p), None, 0)
    lst = np.zeros(max(K, 1), np.int32)
    lib().oracle_bin(*args, _p(offsets, _i64p), _p(lst, _i32p), K)
    return offsets, lst[:K]


def nonzero_boxes(atlas):
    """(n_bmp, 4) {u0, u1, v0, v1}: first and last column and row holding a texel > 0
    ({W_b, -1, H_b, -1} for an all-zero bitmap)."""
    atlas = np.ascontiguousarray(atlas, dtype=np.float32)
    nb, Hb, Wb = atlas.shape
    out = np.zeros((nb, 4), np.int32)
    lib().oracle_nonzero_boxes(_p(atlas, _f32p), nb, Hb, Wb, _p(out, _i32p))
    return out


def spec_abs_sincos(theta):
    a = ctypes.c_float()
    b = ctypes.c_float()
    lib().oracle_spec_abs_sincos(float(np.float32(theta)), ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def spec_sincos(theta):
    """(sin, cos, in range) of the binning specification."""
    a = ctypes.c_float()
    b = ctypes.c_float()
    ok = lib().oracle_spec_sincos(float(np.float32(theta)), ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value, bool(ok)


# ---------------------------------------------------------------------------
# Loss and optimiser (Tab. S1: MSE loss, Adam-like optimiser with per-group gains
# and exponential decay; PSNR of images in [0, 1]).
# ---------------------------------------------------------------------------

#: Tab. S1 learning-rate gains per parameter column: x, y, s (lr_gain_x/y/r = 10),
#: theta (1), nu (lr_gain_v = 1.5), colour (1).
LR_GAINS = (10.0, 10.0, 10.0, 1.0, 1.5, 1.0, 1.0, 1.0)


def mse(image, target):
    d = np.asarray(image, np.float64) - np.asarray(target, np.float64)
    return float(np.mean(d * d))


def mse_grad(image, target):
    """dL/dI of L = mean over 3HW of (I - I*)^2."""
    d = np.asarray(image, np.float64) - np.asarray(target, np.float64)
    return 2.0 * d / d.size


def psnr(image, target):
    m = mse(image, target)
    return float("inf") if m == 0 else 10.0 * math.log10(1.0 / m)


def adam_step(p, g, m, v, t, lr, gains=LR_GAINS, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba) on (N, 8) arrays in FP64, bias-corrected, step t >= 1,
    column j uses learning rate lr * gains[j].  Returns new (p, m, v)."""
    p = np.asarray(p, np.float64)
    g = np.asarray(g, np.float64)
    m = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    lr_col = lr * np.asarray(gains, np.float64)[None, :]
    return p - lr_col * mh / (np.sqrt(vh) + eps), m, v


# ---------------------------------------------------------------------------
# Structure-aware initialisation (Sec. 3.2 "Structure-aware Initialization", Tab. S1)
# ---------------------------------------------------------------------------

def local_variance(image):
    """LV (H, W): per channel the population variance over the 7 x 7 window clipped
    to the canvas, averaged over the three channels.  image (3, H, W)."""
    image = np.ascontiguousarray(image, dtype=np.float32)
    _, H, W = image.shape
    lv = np.zeros((H, W))
    lib().oracle_local_variance(H, W, _p(image, _f32p), _p(lv, _f64p))
    return lv


def structure_init(image, u_pos, u_theta, n_color, s_range, sigma_c=0.02, nu=-2.0, mask=None):
    """Primitive parameters (N, 8) FP64 drawn by the structure-aware initialisation
    from image (3, H, W) with the given random draws (u_pos, u_theta in [0, 1), n_color
    (N, 3) standard normal); mask (H, W): draw only where mask > 0 (an empty mask
    draws nothing: params zero, pixel -1).  Returns (params, NLV (H, W), pixel index
    (N,), Q_total)."""
    image = np.ascontiguousarray(image, dtype=np.float32)
    mask_a = None if mask is None else np.ascontiguousarray(mask, dtype=np.float32)
    _, H, W = image.shape
    u_pos = np.ascontiguousarray(u_pos, dtype=np.float64)
    u_theta = np.ascontiguousarray(u_theta, dtype=np.float64)
    n_color = np.ascontiguousarray(n_color, dtype=np.float64).reshape(-1, 3)
    N = u_pos.shape[0]
    params = np.zeros((N, 8))
    nlv = np.zeros((H, W))
    pix = np.full(max(N, 1), -1, np.int32)
    total = lib().oracle_structure_init(H, W, _p(image, _f32p), _p(mask_a, _f32p), N, _p(u_pos, _f64p),
                                        _p(u_theta, _f64p),
                                        _p(n_color, _f64p), float(s_range[0]), float(s_range[1]),
                                        float(sigma_c), float(nu), _p(params, _f64p), _p(nlv, _f64p),
                                        _p(pix, _i32p))
    return params, nlv, pix[:N], int(total)


# ---------------------------------------------------------------------------
# Gaussian blur of the primitive bitmaps (Sec. 3.2 "Blurring Primitives for
# Enriching Gradients"; Tab. S1 do_gaussian_blur, blur_sigma = 1.0)
# ---------------------------------------------------------------------------

def blur_radius(sigma):
    """Support of the kernel: r = ceil(3 sigma) texels on each side."""
    return int(math.ceil(3.0 * sigma))


def gaussian_blur(texels, sigma):
    """Each bitmap convolved with the 2-D Gaussian exp(-(dy^2 + dx^2) / (2 sigma^2)),
    |dy|, |dx| <= r, normalised to sum 1, texels outside the bitmap zero; FP64,
    the 2-D sum written out.  texels (n_bmp, H_b, W_b) -> same shape."""
    t = np.asarray(texels, np.float64)
    if t.ndim == 2:
        t = t[None]
    r = blur_radius(sigma)
    d = np.arange(-r, r + 1, dtype=np.float64)
    w = np.exp(-(d[:, None] ** 2 + d[None, :] ** 2) / (2.0 * sigma * sigma))
    w /= w.sum()
    n, H, W = t.shape
    pad = np.zeros((n, H + 2 * r, W + 2 * r))
    pad[:, r:r + H, r:r + W] = t
    out = np.zeros_like(t)
    for dy in range(2 * r + 1):
        for dx in range(2 * r + 1):
            out += w[dy, dx] * pad[:, dy:dy + H, dx:dx + W]
    return out


# ---------------------------------------------------------------------------
# Scaling statistics of a binning (Sec. S4: footprint A_i / (H W), tile-hit
# degree tau_i, per-tile density d_t)
# ---------------------------------------------------------------------------

def _log2_bin(v):
    """floor(log2 v) for integers v >= 1."""
    return np.array([int(x).bit_length() - 1 for x in np.asarray(v).ravel()], np.int64)


def bin_stats(H, W, tile, params, bitmap_id, atlas):
    """Histograms of one canvas' binning, 32 bins each: tau_hist[b] = listed primitives
    with floor(log2 tau_i) = b; d_hist[b] = tiles with floor(log2 d_t) = b (empty tiles
    counted apart); foot_hist[b] = listed primitives with A_i / (H W) in
    [2^-(b+1), 2^-b) (b = 0 also takes ratios >= 1; b capped at 31)."""
    params, bitmap_id, atlas = _bin_inputs(params, bitmap_id, atlas)
    N = params.shape[0]
    Hb, Wb = atlas.shape[1:]
    _, tau = bin_rects(H, W, tile, params, bitmap_id, atlas)
    offs, _ = bin(H, W, tile, params, bitmap_id, atlas)
    d = np.diff(offs)
    area = np.zeros(max(N, 1))
    lib().oracle_bin_footprint(N, _p(params, _f32p), Hb, Wb, _p(area, _f64p))
    area = area[:N]
    listed = tau > 0
    out = {"n_listed": int(listed.sum()), "pairs": int(tau.sum()), "tau_max": int(tau.max(initial=0)),
           "d_max": int(d.max(initial=0)), "n_tiles": int(d.size), "empty_tiles": int((d == 0).sum()),
           "tau_hist": np.bincount(_log2_bin(tau[listed]), minlength=32)[:32],
           "d_hist": np.bincount(_log2_bin(d[d > 0]), minlength=32)[:32]}
    fb = []
    for a in area[listed]:
        m, e = math.frexp(a / float(H * W))   # ratio in [2^(e-1), 2^e)
        fb.append(min(31, max(0, -e)))
    out["foot_hist"] = np.bincount(np.array(fb, np.int64), minlength=32)[:32]
    return out



def structure_reinit(params, image, mask, u_pos, u_theta, n_color, s_range, threshold=0.3, sigma_c=0.02,
                     nu=-2.0):
    """Re-initialisation (Sec. 3.3.2; Sec. S3 "Re-initialization Mechanism"): every
    primitive i with sigmoid(nu_i) < threshold takes the structure-aware draw i
    (restricted to mask > 0 when mask is given).  Returns (new params FP64, indices)."""
    p = np.asarray(params, np.float64).reshape(-1, 8).copy()
    drawn, _, pix, total = structure_init(image, u_pos, u_theta, n_color, s_range, sigma_c, nu, mask)
    low = np.nonzero(1.0 / (1.0 + np.exp(-p[:, 4])) < threshold)[0] if total > 0 else np.zeros(0, np.int64)
    p[low] = drawn[low]
    return p, low


# ---------------------------------------------------------------------------
# Spatially constrained loss (Eq. 9, Sec. 3.3.2)
# ---------------------------------------------------------------------------

def alpha_loss(image, T_final, target, target_alpha, lam):
    """L = mean over 3 H W of [alpha* > 0] (I - I*)^2 + lam * mean over H W of
    (I_alpha - alpha*)^2, I_alpha = 1 - T_N (Eq. 9 with both norms read as means).
    Returns (L, dL/dI (3, H, W), dL/dI_alpha (H, W)) in FP64."""
    I = np.asarray(image, np.float64)
    T = np.asarray(T_final, np.float64)
    It = np.asarray(target, np.float64)
    a = np.asarray(target_alpha, np.float64)
    m = (a > 0).astype(np.float64)[None]
    n3, n1 = I.size, T.size
    d = m * (I - It)
    Ia = 1.0 - T
    L = float((d * d).sum() / n3 + lam * ((Ia - a) ** 2).sum() / n1)
    return L, 2.0 * d / n3, 2.0 * lam * (Ia - a) / n1
