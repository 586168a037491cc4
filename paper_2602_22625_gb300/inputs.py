"""Seeded synthetic inputs shaped like DiffBMP's workloads.

This module only draws random numbers and builds bitmaps; it holds none of the
rasterizer's arithmetic, so both the CUDA path and the FP64 oracle can take
their inputs from it.  All randomness comes from numpy's counter-based Philox
generator, so a seed gives the same bytes on every machine.

Stand-ins: the paper optimises photographs, logos, video frames and
CelebAMask-HQ masks with hand-drawn bitmap primitives (fingerprints, flowers,
strokes).  None of those assets are available, so:
  * primitives are procedural bitmaps -- a soft disc (linear 4-texel edge) or a
    cubic Bezier stroke of random width, distance-field rasterised and Gaussian
    blurred (sigma 1, radius 3: the paper's default soft rasterisation, Sec. 3.2.1);
    every bitmap keeps a zero border of at least two texels;
  * target images are renders of other seeded parameter sets.

Parameter convention (per primitive, float32): x, y, s, theta, nu, c_r, c_g, c_b
with s the half-extent in canvas pixels (Eq. 1 maps (x - x_i)/s_i onto [-1, 1]),
nu and c logits.  Workload scales are given as a fraction of the canvas side
(s = s_cfg * W); opacity and colour are drawn in [0, 1] and stored as
logit(clamp(v, 1e-4, 1 - 1e-4)).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(int(seed)))


def _logit(v):
    v = np.clip(np.asarray(v, np.float64), 1e-4, 1.0 - 1e-4)
    return np.log(v / (1.0 - v))


# ---------------------------------------------------------------------------
# Bitmap atlases
# ---------------------------------------------------------------------------

def soft_disc_atlas(seed: int, n: int = 1, size: int = 64, edge: float = 4.0) -> np.ndarray:
    """n soft discs (size x size): radius U[24, 28] texels (scaled with size/64),
    value clip((R - r)/edge, 0, 1), centred at ((size-1)/2, (size-1)/2)."""
    g = rng(seed)
    c = (size - 1) / 2.0
    yy, xx = np.mgrid[0:size, 0:size].astype(np.float64)
    r = np.hypot(xx - c, yy - c)
    out = np.empty((n, size, size), np.float32)
    k = size / 64.0
    for i in range(n):
        R = g.uniform(24.0 * k, 28.0 * k)
        out[i] = np.clip((R - r) / edge, 0.0, 1.0)
        out[i, :2, :] = 0
        out[i, -2:, :] = 0
        out[i, :, :2] = 0
        out[i, :, -2:] = 0
    return out


def _gauss_blur(img: np.ndarray, sigma: float, radius: int) -> np.ndarray:
    k = np.arange(-radius, radius + 1, dtype=np.float64)
    w = np.exp(-0.5 * (k / sigma) ** 2)
    w /= w.sum()
    pad = np.pad(img, radius)
    tmp = sum(w[i] * pad[:, i:i + img.shape[1]] for i in range(2 * radius + 1))
    tmp = tmp[radius:radius + img.shape[0], :]
    pad = np.pad(tmp, ((radius, radius), (0, 0)))
    return sum(w[i] * pad[i:i + img.shape[0], :] for i in range(2 * radius + 1))


def stroke_atlas(seed: int, n: int = 16, size: int = 128, blur_sigma: float = 1.0,
                 n_seg: int = 64) -> np.ndarray:
    """n procedural strokes (size x size): a cubic Bezier curve with control points
    U[12, size-12]^2 and width U[4, 12] texels, rasterised from its distance field
    with a one-texel linear edge, then Gaussian blurred (sigma, radius 3 sigma)."""
    g = rng(seed)
    yy, xx = np.mgrid[0:size, 0:size].astype(np.float64)
    pts = np.stack([xx.ravel(), yy.ravel()], 1)
    t = np.linspace(0.0, 1.0, n_seg + 1)[:, None]
    out = np.empty((n, size, size), np.float32)
    lo, hi = 12.0, size - 12.0
    for i in range(n):
        P = g.uniform(lo, hi, size=(4, 2))
        width = g.uniform(4.0, 12.0)
        curve = ((1 - t) ** 3) * P[0] + 3 * ((1 - t) ** 2) * t * P[1] + \
            3 * (1 - t) * t * t * P[2] + t ** 3 * P[3]
        a, b = curve[:-1], curve[1:]
        ab = b - a
        ap = pts[:, None, :] - a[None]
        tt = np.clip((ap * ab[None]).sum(-1) / np.maximum((ab * ab).sum(-1), 1e-12)[None], 0, 1)
        d = np.linalg.norm(ap - tt[..., None] * ab[None], axis=-1).min(1).reshape(size, size)
        m = np.clip(width / 2.0 - d + 0.5, 0.0, 1.0)
        if blur_sigma > 0:
            m = _gauss_blur(m, blur_sigma, int(math.ceil(3 * blur_sigma)))
        m = np.clip(m, 0.0, 1.0)
        m[:2, :] = 0
        m[-2:, :] = 0
        m[:, :2] = 0
        m[:, -2:] = 0
        out[i] = m.astype(np.float32)
    return out


# ---------------------------------------------------------------------------
# Primitive parameters
# ---------------------------------------------------------------------------

def primitives(seed: int, N: int, H: int, W: int, n_bmp: int, scale: str = "uniform",
               scale_args=(0.1, 0.5), opacity=(0.2, 1.0)) -> tuple[np.ndarray, np.ndarray]:
    """N primitives on an H x W canvas.  x ~ U[0, W), y ~ U[0, H), theta ~ U[0, 2 pi),
    RGB ~ U[0, 1], opacity ~ U[opacity], bitmap id uniform.  Scale law (fraction of W):
      'uniform'   U[a, b]
      'lognormal' LogNormal(mu=a, sigma=b)
      'pareto'    min(x_m U^(-1/alpha), 0.5) with (x_m, alpha) = (a, b)."""
    g = rng(seed)
    p = np.empty((N, 8), np.float64)
    p[:, 0] = g.uniform(0.0, W, N)
    p[:, 1] = g.uniform(0.0, H, N)
    if scale == "uniform":
        sc = g.uniform(scale_args[0], scale_args[1], N)
    elif scale == "lognormal":
        sc = g.lognormal(scale_args[0], scale_args[1], N)
    elif scale == "pareto":
        u = g.uniform(0.0, 1.0, N)
        sc = np.minimum(scale_args[0] * np.maximum(u, 1e-12) ** (-1.0 / scale_args[1]), 0.5)
    else:
        raise ValueError(scale)
    p[:, 2] = sc * W
    p[:, 3] = g.uniform(0.0, 2.0 * math.pi, N)
    p[:, 4] = _logit(g.uniform(opacity[0], opacity[1], N))
    p[:, 5:8] = _logit(g.uniform(0.0, 1.0, (N, 3)))
    bid = g.integers(0, n_bmp, N).astype(np.int32)
    return p.astype(np.float32), bid


# ---------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Scene:
    name: str
    H: int
    W: int
    params: np.ndarray       # (N, 8) float32
    bitmap_id: np.ndarray    # (N,) int32
    atlas: np.ndarray        # (n_bmp, Hb, Wb) float32
    alpha_max: float = 1.0
    background: tuple = (1.0, 1.0, 1.0)
    recipe: str = ""

    @property
    def N(self):
        return self.params.shape[0]


def tiny(seed: int = 1, N: int = 256, H: int = 256, W: int = 256) -> Scene:
    """256^2 canvas, one 64^2 soft disc, 256 primitives, s ~ U[0.1, 0.5] * W."""
    atlas = soft_disc_atlas(seed * 7919 + 1, 1, 64)
    p, b = primitives(seed, N, H, W, 1, "uniform", (0.1, 0.5))
    return Scene("tiny_256sq_256prims", H, W, p, b, atlas,
                 recipe=f"soft disc 64^2 atlas; N={N}; s=U[0.1,0.5]*W; seed={seed}")


_STROKES16 = {}


def strokes16(seed: int = 11) -> np.ndarray:
    if seed not in _STROKES16:
        _STROKES16[seed] = stroke_atlas(seed, 16, 128)
    return _STROKES16[seed]


def main(seed: int = 2, N: int = 20000, H: int = 1024, W: int = 1024, atlas_seed: int = 11) -> Scene:
    """1024^2 canvas, 16 stroke bitmaps 128^2, 20k primitives, s ~ LogNormal(-2, 0.7) * W."""
    atlas = strokes16(atlas_seed)
    p, b = primitives(seed, N, H, W, atlas.shape[0], "lognormal", (-2.0, 0.7))
    return Scene("main_1024sq_20k", H, W, p, b, atlas,
                 recipe=f"16 blurred Bezier strokes 128^2; N={N}; s=LogNormal(-2,0.7)*W; seed={seed}")


def stress(seed: int = 3, N: int = 200000, H: int = 2048, W: int = 2048, x_m: float = 0.035,
           atlas_seed: int = 13) -> Scene:
    """2048^2 canvas, 64 stroke bitmaps, 200k primitives, Pareto(alpha=1.5) scale with
    x_m = 0.035 of the side (the smallest value tried, in steps of 0.005, for which the
    densest tile lists more than 5000 primitives when tiles list only the part of each
    primitive its bitmap's non-zero texels can reach: 5427 at 32^2 tiles, 5069 at 16^2)."""
    atlas = stroke_atlas(atlas_seed, 64, 128)
    p, b = primitives(seed, N, H, W, atlas.shape[0], "pareto", (x_m, 1.5))
    return Scene("stress_2048sq_200k", H, W, p, b, atlas,
                 recipe=f"64 strokes 128^2; N={N}; s=min(x_m U^-1/1.5, 0.5)*W, x_m={x_m}; seed={seed}")


def batched(seed: int = 4, n_canvas: int = 64, side=(256, 1024), nprim=(1000, 50000),
            atlas_seed: int = 11) -> list[Scene]:
    """n_canvas square canvases, side ~ U{256..1024}, N ~ log-uniform[1k, 50k], shared
    16-stroke atlas, s ~ LogNormal(-2, 0.7) * side."""
    g = rng(seed)
    atlas = strokes16(atlas_seed)
    scenes = []
    for c in range(n_canvas):
        S = int(g.integers(side[0], side[1] + 1))
        N = int(round(math.exp(g.uniform(math.log(nprim[0]), math.log(nprim[1])))))
        p, b = primitives(seed * 100003 + c, N, S, S, atlas.shape[0], "lognormal", (-2.0, 0.7))
        scenes.append(Scene(f"batch{c}_{S}sq_{N}", S, S, p, b, atlas))
    return scenes


# ---------------------------------------------------------------------------
# Anchored scenes for the learned proposal network
# ---------------------------------------------------------------------------
#: anchored scene geometry: 8 x 8 cells of 32 px on a 256^2 canvas, 8 slots per cell;
#: slot k sits in sub-cell (k % 4, k // 4) of 8 x 16 px; primitive index
#: (cy * 8 + cx) * 8 + k (cells in raster order, slots in order, index 0 in front)
ANCHOR_CANVAS, ANCHOR_CELLS, ANCHOR_SLOTS = 256, 8, 8
ANCHOR_SCALE = (6.0, 14.0)       # half-extent in pixels
ANCHOR_OPACITY = (0.5, 1.0)


def anchored(seed: int, B: int = 1) -> np.ndarray:
    """B scenes of 512 soft-disc primitives placed by the anchored generator:
    x = cell_x + sub_x + U[0, 8), y = cell_y + sub_y + U[0, 16), s ~ U[6, 14] px,
    theta ~ U[0, 2 pi), opacity ~ U[0.5, 1], RGB ~ U[0, 1] (stored as logits).
    Returns float32 (B, 512, 8)."""
    g = rng(seed)
    C, S = ANCHOR_CELLS, ANCHOR_SLOTS
    cell = ANCHOR_CANVAS // C
    idx = np.arange(C * C * S)
    cy, cx, k = idx // (C * S), (idx // S) % C, idx % S
    base_x = cx * cell + (k % 4) * 8
    base_y = cy * cell + (k // 4) * 16
    p = np.empty((B, C * C * S, 8), np.float64)
    p[..., 0] = base_x[None] + g.uniform(0.0, 8.0, (B, C * C * S))
    p[..., 1] = base_y[None] + g.uniform(0.0, 16.0, (B, C * C * S))
    p[..., 2] = g.uniform(ANCHOR_SCALE[0], ANCHOR_SCALE[1], (B, C * C * S))
    p[..., 3] = g.uniform(0.0, 2.0 * math.pi, (B, C * C * S))
    p[..., 4] = _logit(g.uniform(ANCHOR_OPACITY[0], ANCHOR_OPACITY[1], (B, C * C * S)))
    p[..., 5:8] = _logit(g.uniform(0.0, 1.0, (B, C * C * S, 3)))
    return p.astype(np.float32)


def random_init(seed: int, B: int = 1, N: int = 512, H: int = 256, W: int = 256) -> np.ndarray:
    """The plain method's random initialisation for the same scenes: positions
    uniform over the canvas, scales, opacities and colours from the same ranges."""
    g = rng(seed)
    p = np.empty((B, N, 8), np.float64)
    p[..., 0] = g.uniform(0.0, W, (B, N))
    p[..., 1] = g.uniform(0.0, H, (B, N))
    p[..., 2] = g.uniform(ANCHOR_SCALE[0], ANCHOR_SCALE[1], (B, N))
    p[..., 3] = g.uniform(0.0, 2.0 * math.pi, (B, N))
    p[..., 4] = _logit(g.uniform(ANCHOR_OPACITY[0], ANCHOR_OPACITY[1], (B, N)))
    p[..., 5:8] = _logit(g.uniform(0.0, 1.0, (B, N, 3)))
    return p.astype(np.float32)


def init_draws(seed: int, N: int):
    """The random numbers the structure-aware initialisation consumes for N
    primitives: u_pos, u_theta ~ U[0, 1) (N,), n_color ~ N(0, 1) (N, 3), float64."""
    g = rng(seed)
    return g.uniform(0.0, 1.0, N), g.uniform(0.0, 1.0, N), g.normal(0.0, 1.0, (N, 3))


def cnn_init(seed: int = 0) -> np.ndarray:
    """He-normal initial weights (zero biases) of the proposal network, flattened in
    the library's parameter order: for each layer, W (Cout x K row-major), then b."""
    g = rng(seed)
    chunks = []
    for cin_pad, cin_real, cout, ksz in CNN_LAYERS:
        K = ksz * ksz * cin_pad
        w = g.normal(0.0, math.sqrt(2.0 / (ksz * ksz * cin_real)), (cout, ksz * ksz, cin_pad))
        w[:, :, cin_real:] = 0.0
        if cout == CNN_LAYERS[-1][2]:
            w *= 0.1  # small head: initial proposals near the anchors' centres
        chunks += [w.reshape(cout, K).ravel(), np.zeros(cout)]
    return np.concatenate(chunks).astype(np.float32)


#: (input channels padded, input channels used, output channels, kernel size):
#: five 4x4 stride-2 convolutions with ReLU, then a 1x1 head (8 slots x 8 outputs)
CNN_LAYERS = ((4, 3, 32, 4), (32, 32, 64, 4), (64, 64, 128, 4), (128, 128, 256, 4),
              (256, 256, 256, 4), (256, 256, 64, 1))
