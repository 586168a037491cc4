"""Pins of the FP64 oracle against what the paper and mathematics fix (CPU only).

Each test checks the oracle against something other than itself: a closed form,
a library routine (torch.nn.functional.grid_sample + autograd, torch.optim.Adam),
brute force, finite differences, or a second formula printed in the paper (Eq. S5).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2602_22625_gb300 import inputs

torch = pytest.importorskip("torch")


def sig(z):
    return 1.0 / (1.0 + np.exp(-np.asarray(z, np.float64)))


def logit(p):
    return math.log(p / (1.0 - p))


def disc64():
    return inputs.soft_disc_atlas(5, 1, 64)


def identity_prim(nu=0.3, c=(0.2, -0.5, 1.1), theta=0.0):
    # s = 31.5, centre (31.5, 31.5): pixel (px, py) maps to U = px, V = py (Eqs. 1-2)
    return np.array([[31.5, 31.5, 31.5, theta, nu, *c]], np.float32)


# --------------------------------------------------------------------------
# Closed forms
# --------------------------------------------------------------------------

def test_identity_transform_reproduces_bitmap():
    """Eqs. 1-3 with the identity placement: M = P[py, px]; one layer over a
    constant background gives I = a P chat + (1 - a P) b (Eqs. 4-5, 8)."""
    atlas = np.random.default_rng(0).uniform(0, 1, (1, 64, 64)).astype(np.float32)
    p = identity_prim()
    amax = 0.8
    b = np.array([0.3, 0.6, 0.9])
    out = oracle.render(64, 64, p, [0], atlas, alpha_max=amax, background=b)
    a = amax * sig(p[0, 4])
    P = atlas[0].astype(np.float64)
    chat = sig(p[0, 5:8])
    for j in range(3):
        want = a * P * chat[j] + (1 - a * P) * b[j]
        np.testing.assert_allclose(out["image"][j], want, rtol=0, atol=1e-13)
    np.testing.assert_allclose(out["T_final"], 1 - a * P, atol=1e-13)


def test_two_layer_over_closed_form():
    """Porter-Duff over of two identity-placed layers (index 0 in front)."""
    rng = np.random.default_rng(1)
    atlas = rng.uniform(0, 1, (2, 64, 64)).astype(np.float32)
    p = np.concatenate([identity_prim(0.7, (0.1, 0.2, 0.3)), identity_prim(-0.4, (1.0, -1.0, 0.0))])
    b = np.array([1.0, 0.5, 0.0])
    out = oracle.render(64, 64, p, [0, 1], atlas, alpha_max=1.0, background=b)
    a0 = sig(p[0, 4]) * atlas[0].astype(np.float64)
    a1 = sig(p[1, 4]) * atlas[1].astype(np.float64)
    c0, c1 = sig(p[0, 5:8]), sig(p[1, 5:8])
    for j in range(3):
        want = a0 * c0[j] + (1 - a0) * (a1 * c1[j] + (1 - a1) * b[j])
        np.testing.assert_allclose(out["image"][j], want, atol=1e-13)
    np.testing.assert_allclose(out["T_final"], (1 - a0) * (1 - a1), atol=1e-13)


def test_opaque_front_layer_occludes_everything_behind():
    """A front primitive with alpha_max = 1, nu = +40 over an all-ones interior hides
    every later layer there (1 - sigmoid(40) ~ 4e-18)."""
    rng = np.random.default_rng(2)
    box = np.zeros((1, 64, 64), np.float32)
    box[0, 8:56, 8:56] = 1.0
    front = identity_prim(40.0, (2.0, -2.0, 0.5))
    sc = inputs.tiny(seed=3, N=40, H=64, W=64)
    atlas = np.concatenate([box, sc.atlas])
    params = np.concatenate([front, sc.params])
    bid = np.concatenate([[0], sc.bitmap_id + 1]).astype(np.int32)
    full = oracle.render(64, 64, params, bid, atlas, background=(0.2, 0.4, 0.6))
    alone = oracle.render(64, 64, front, [0], box, background=(0.2, 0.4, 0.6))
    inner = np.zeros((64, 64), bool)
    inner[9:55, 9:55] = True  # taps all inside the ones region
    np.testing.assert_allclose(full["image"][:, inner], alone["image"][:, inner], atol=1e-15)
    # and the interior colour is sigmoid(c) of the front primitive
    want = np.broadcast_to(sig(front[0, 5:8])[:, None], full["image"][:, inner].shape)
    np.testing.assert_allclose(full["image"][:, inner], want, atol=1e-15)
    # but later layers are visible outside the box
    assert np.abs(full["image"][:, ~inner] - alone["image"][:, ~inner]).max() > 1e-2


@pytest.mark.parametrize("how", ["zero_bitmap", "nu_minus_40"])
def test_zero_opacity_is_a_no_op(how):
    sc = inputs.tiny(seed=4, N=30, H=48, W=40)
    zero = np.zeros((1,) + sc.atlas.shape[1:], np.float32)
    atlas = np.concatenate([sc.atlas, zero])
    extra = sc.params[:1].copy()
    extra[0, :3] = [20.0, 24.0, 15.0]
    if how == "nu_minus_40":
        extra[0, 4] = -40.0
        eb = 0
    else:
        eb = 1
    params = np.concatenate([sc.params[:10], extra, sc.params[10:]])
    bid = np.concatenate([sc.bitmap_id[:10], [eb], sc.bitmap_id[10:]]).astype(np.int32)
    a = oracle.render(48, 40, sc.params, sc.bitmap_id, atlas)
    b = oracle.render(48, 40, params, bid, atlas)
    tol = 0.0 if how == "zero_bitmap" else 1e-16
    np.testing.assert_allclose(b["image"], a["image"], atol=tol)
    np.testing.assert_allclose(b["T_final"], a["T_final"], atol=tol)


def test_rotation_by_half_pi_permutes_texels():
    """theta = pi/2 with the identity placement gives u = dy/s, v = -dx/s, so
    M(px, py) = P[63 - px, py] (a texel permutation; float32(pi/2) is within 4.4e-8)."""
    atlas = disc64()
    atlas = atlas * np.linspace(0.2, 1.0, 64, dtype=np.float32)[None, :, None]  # break symmetry
    p = identity_prim(nu=20.0, c=(30.0, 30.0, 30.0), theta=math.pi / 2)
    out = oracle.render(64, 64, p, [0], atlas, alpha_max=1.0, background=(0, 0, 0))
    want = atlas[0].astype(np.float64)[::-1, :].T  # want[py, px] = P[63 - px, py]
    np.testing.assert_allclose(out["image"][0], want, atol=2e-6)
    # the wrong rotation sense would give the mirror image
    assert np.abs(atlas[0][:, ::-1].T - want).max() > 0.1


def test_translation_and_scale_sense():
    """A primitive at (x_i, y_i) = (10, 40) with s = 7: its centre texel
    (U, V) = ((W-1)/2, (H-1)/2) lands on the canvas point (x_i, y_i)."""
    atlas = np.zeros((1, 5, 5), np.float32)
    atlas[0, 2, 2] = 1.0  # single bump at the centre texel
    p = np.array([[10.0, 40.0, 7.0, 0.0, 30.0, 30.0, 30.0, 30.0]], np.float32)
    out = oracle.render(64, 64, p, [0], atlas, background=(0, 0, 0))
    img = out["image"][0]
    assert img[40, 10] == pytest.approx(1.0, abs=1e-12)
    # U = (u+1)/2 * 4 with u = dx/7: one texel is 3.5 canvas pixels
    assert img[40, 10 + 3] == pytest.approx(1.0 - 3.0 / 3.5, abs=1e-12)
    assert img[40 + 2, 10] == pytest.approx(1.0 - 2.0 / 3.5, abs=1e-12)
    # 4 px away is 8/7 texel: the taps then sit on the zero texels next to the bump
    assert img[40, 14] == 0.0 and img[36, 10] == 0.0


# --------------------------------------------------------------------------
# Algorithm S3 in torch float64 (grid_sample + sequential over) with autograd
# --------------------------------------------------------------------------

def torch_naive(H, W, params, bid, atlas, amax, bg):
    """Algorithm S3: meshgrid, per-primitive grid_sample(align_corners=True, zeros),
    sequential over-compositing, then the Eq. 8 background.  float64, autograd."""
    import torch.nn.functional as F
    p = torch.tensor(params.astype(np.float64), requires_grad=True)
    A = torch.tensor(atlas.astype(np.float64))
    Y, X = torch.meshgrid(torch.arange(H, dtype=torch.float64),
                          torch.arange(W, dtype=torch.float64), indexing="ij")
    I = torch.zeros(3, H, W, dtype=torch.float64)
    T = torch.ones(H, W, dtype=torch.float64)
    for i in range(p.shape[0]):
        x, y, s, th, nu = p[i, 0], p[i, 1], p[i, 2], p[i, 3], p[i, 4]
        dx, dy = X - x, Y - y
        u = (torch.cos(th) * dx + torch.sin(th) * dy) / s
        v = (-torch.sin(th) * dx + torch.cos(th) * dy) / s
        grid = torch.stack([u, v], -1)[None]
        m = F.grid_sample(A[int(bid[i])][None, None], grid, mode="bilinear",
                          padding_mode="zeros", align_corners=True)[0, 0]
        a = amax * torch.sigmoid(nu) * m
        c = torch.sigmoid(p[i, 5:8])
        I = I + T[None] * a[None] * c[:, None, None]
        T = T * (1 - a)
    bgt = torch.tensor(np.asarray(bg, np.float64))
    if bgt.numel() == 3:
        bgt = bgt.reshape(3, 1, 1)
    I = I + T[None] * bgt
    return p, I, T


@pytest.mark.parametrize("case", range(6))
def test_oracle_matches_torch_grid_sample_and_autograd(case):
    """Cases 4 and 5 have non-square bitmaps (24 x 40 and 48 x 28), where Eq. 2's
    horizontal and vertical half-widths differ: a swap of the two, or of their ratio in
    the rotation gradient, fails there."""
    rng = np.random.default_rng(100 + case)
    H, W = [(24, 24), (17, 29), (32, 20), (21, 21), (26, 31), (30, 22)][case]
    N = [1, 3, 6, 8, 5, 7][case]
    if case == 4:
        atlas = inputs.stroke_atlas(11, 3, 40, n_seg=16)[:, 6:30, :]
    elif case == 5:
        atlas = inputs.soft_disc_atlas(13, 2, 48)[:, :, 10:38]
    else:
        atlas = inputs.stroke_atlas(7 + case, 3, 24, n_seg=16) if case % 2 else \
            inputs.soft_disc_atlas(9 + case, 2, 32)
    atlas = np.ascontiguousarray(atlas)
    params = np.zeros((N, 8), np.float32)
    params[:, 0] = rng.uniform(0, W, N)
    params[:, 1] = rng.uniform(0, H, N)
    params[:, 2] = rng.uniform(3, 14, N) * rng.choice([1, 1, 1, -1], N)
    params[:, 3] = rng.uniform(-7, 7, N)
    params[:, 4] = rng.uniform(-2, 3, N)
    params[:, 5:8] = rng.uniform(-3, 3, (N, 3))
    bid = rng.integers(0, atlas.shape[0], N).astype(np.int32)
    amax = [1.0, 0.7, 0.9, 1.0, 0.8, 1.0][case]
    bg = [(1.0, 1.0, 1.0), (0.2, 0.5, 0.1), rng.uniform(0, 1, (3, H, W)).astype(np.float32),
          (0.0, 0.0, 0.0), (0.3, 0.3, 0.9), (1.0, 1.0, 1.0)][case]
    p, I, T = torch_naive(H, W, params, bid, atlas, amax, bg)
    out = oracle.render(H, W, params, bid, atlas, alpha_max=amax, background=bg)
    np.testing.assert_allclose(out["image"], I.detach().numpy(), rtol=0, atol=1e-12)
    np.testing.assert_allclose(out["T_final"], T.detach().numpy(), rtol=0, atol=1e-12)
    gI = rng.normal(size=(3, H, W))
    gA = rng.normal(size=(H, W))
    loss = (I * torch.tensor(gI)).sum() + ((1 - T) * torch.tensor(gA)).sum()
    loss.backward()
    g = oracle.grad(H, W, params, bid, atlas, gI, gA, alpha_max=amax, background=bg)
    ref = p.grad.numpy()
    scale = np.abs(ref).max(0) + 1e-30
    np.testing.assert_allclose(g / scale, ref / scale, rtol=0, atol=1e-10)


# --------------------------------------------------------------------------
# Finite differences in FP64
# --------------------------------------------------------------------------

def _loss(H, W, params, bid, atlas, gI, gA, amax, bg):
    o = oracle.render(H, W, params, bid, atlas, alpha_max=amax, background=bg)
    return float((o["image"] * gI).sum() + ((1 - o["T_final"]) * gA).sum())


def test_gradients_match_central_finite_differences():
    """Every gradient column against central differences of the oracle's own forward.
    params are float32, so each FD probe perturbs by an exactly representable step."""
    rng = np.random.default_rng(7)
    H, W, N = 28, 24, 5
    atlas = inputs.stroke_atlas(21, 2, 32, n_seg=16)
    params = np.zeros((N, 8), np.float32)
    params[:, 0] = rng.uniform(4, W - 4, N)
    params[:, 1] = rng.uniform(4, H - 4, N)
    params[:, 2] = rng.uniform(8, 16, N)
    params[:, 3] = rng.uniform(0, 6.28, N)
    params[:, 4] = rng.uniform(-1, 2, N)
    params[:, 5:8] = rng.uniform(-2, 2, (N, 3))
    bid = rng.integers(0, 2, N).astype(np.int32)
    bg = (0.9, 0.3, 0.6)
    amax = 0.85
    gI = rng.normal(size=(3, H, W))
    gA = rng.normal(size=(H, W))
    g = oracle.grad(H, W, params, bid, atlas, gI, gA, alpha_max=amax, background=bg)
    steps = [2 ** -12, 2 ** -12, 2 ** -12, 2 ** -14, 2 ** -12, 2 ** -12, 2 ** -12, 2 ** -12]
    fd = np.zeros_like(g)
    for i in range(N):
        for j in range(8):
            pp = params.copy()
            pm = params.copy()
            pp[i, j] += np.float32(steps[j])
            pm[i, j] -= np.float32(steps[j])
            h = (np.float64(pp[i, j]) - np.float64(pm[i, j]))
            fd[i, j] = (_loss(H, W, pp, bid, atlas, gI, gA, amax, bg) -
                        _loss(H, W, pm, bid, atlas, gI, gA, amax, bg)) / h
    scale = np.abs(g).max(0)
    assert np.all(scale > 0)
    err = np.abs(fd - g) / scale
    assert err.max() < 2e-3, err  # bilinear kinks inside the step bound the agreement
    assert np.median(err) < 1e-5


# --------------------------------------------------------------------------
# Eq. S5 (printed form with suffix sums) against the reverse recursion, b = 0
# --------------------------------------------------------------------------

def test_eq_s5_matches_reverse_recursion_without_background():
    sc = inputs.tiny(seed=8, N=12, H=32, W=32)
    rng = np.random.default_rng(8)
    H, W = 32, 32
    for (x, y) in [(5, 7), (16, 16), (30, 2), (11, 25)]:
        g = rng.normal(size=3)
        gA = rng.normal()
        d_s5, ks = oracle.eq_s5_dalpha(sc.params, sc.bitmap_id, sc.atlas, x, y, g, gA)
        # recursion value of dL/dalpha_k from the opacity-logit gradient at one pixel
        gI = np.zeros((3, H, W))
        gI[:, y, x] = g
        gAm = np.zeros((H, W))
        gAm[y, x] = gA
        G = oracle.grad(H, W, sc.params, sc.bitmap_id, sc.atlas, gI, gAm, background=None)
        o = oracle.render(H, W, sc.params, sc.bitmap_id, sc.atlas, background=None,
                          pixels=(np.array([x]), np.array([y])))
        assert len(ks) >= 1 or o["n_last"][0] == -1
        for d, k in zip(d_s5, ks):
            # dL/dnu = dL/dalpha * alpha_max * M * s(1-s); recover M from a 1-layer render
            solo = oracle.render(H, W, sc.params[k:k + 1], sc.bitmap_id[k:k + 1], sc.atlas,
                                 background=None, pixels=(np.array([x]), np.array([y])))
            s_nu = sig(sc.params[k, 4])
            M = (1 - solo["T_final"][0]) / s_nu
            want = d * M * s_nu * (1 - s_nu)
            assert G[k, 4] == pytest.approx(want, rel=1e-9, abs=1e-14)


# --------------------------------------------------------------------------
# Binning specification
# --------------------------------------------------------------------------

def test_spec_sincos_error_bound():
    th = np.concatenate([np.linspace(-20, 20, 4001), np.random.default_rng(0).uniform(-6e4, 6e4, 2000)])
    th = th.astype(np.float32)
    err = []
    for t in th:
        a, c = oracle.spec_abs_sincos(t)
        err.append(max(abs(a - abs(math.sin(float(t)))), abs(c - abs(math.cos(float(t))))))
    err = np.array(err)
    assert err[:4001].max() < 3e-7
    assert err.max() < 2e-5


def test_spec_signed_sincos_error_bound_and_range():
    """The signed sine and cosine (the tile rectangle's centre offset) carry the
    quadrant's signs: within the same bounds of math.sin / math.cos, their absolute
    values are spec_abs_sincos's, and outside |theta| <= 65536 the call says so."""
    th = np.concatenate([np.linspace(-20, 20, 4001), np.random.default_rng(1).uniform(-6e4, 6e4, 2000)])
    th = th.astype(np.float32)
    err = []
    for t in th:
        sn, cs, ok = oracle.spec_sincos(t)
        assert ok
        assert (abs(sn), abs(cs)) == oracle.spec_abs_sincos(t)
        err.append(max(abs(sn - math.sin(float(t))), abs(cs - math.cos(float(t)))))
    err = np.array(err)
    assert err[:4001].max() < 3e-7
    assert err.max() < 2e-5
    assert not oracle.spec_sincos(np.float32(70000.0))[2]
    assert oracle.spec_abs_sincos(np.float32(70000.0)) == (1.0, 1.0)


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_binning_conservation_order_and_rects(tile):
    sc = inputs.tiny(seed=9, N=300, H=200, W=170)
    offs, lst = oracle.bin(sc.H, sc.W, tile, sc.params, sc.bitmap_id, sc.atlas)
    rects, tau = oracle.bin_rects(sc.H, sc.W, tile, sc.params, sc.bitmap_id, sc.atlas)
    ntx, nty = -(-sc.W // tile), -(-sc.H // tile)
    d = np.diff(offs)
    assert d.sum() == tau.sum() == len(lst)  # sum_i tau_i = sum_t d_t (Sec. S4)
    for t in range(ntx * nty):
        seg = lst[offs[t]:offs[t + 1]]
        assert np.all(np.diff(seg) > 0)  # front-to-back
        tx, ty = t % ntx, t // ntx
        inside = (rects[:, 0] <= tx) & (tx <= rects[:, 2]) & (rects[:, 1] <= ty) & (ty <= rects[:, 3])
        np.testing.assert_array_equal(seg, np.nonzero(inside)[0])


@pytest.mark.parametrize("tile", [8, 32])
def test_lists_from_rects_reproduce_the_oracle_binning(tile):
    """The rectangle expansion + stable sort used as the expected value for binning
    cases too large for the oracle's tile-by-tile definition gives the same lists."""
    from _helpers import lists_from_rects
    sc = inputs.tiny(seed=10, N=500, H=150, W=230)
    sc.params[::7, 2] = 0.0   # unlisted primitives in the mix
    offs, lst = oracle.bin(sc.H, sc.W, tile, sc.params, sc.bitmap_id, sc.atlas)
    rects, _ = oracle.bin_rects(sc.H, sc.W, tile, sc.params, sc.bitmap_id, sc.atlas)
    o2, l2 = lists_from_rects(rects, -(-sc.W // tile), -(-sc.H // tile))
    np.testing.assert_array_equal(o2, offs)
    np.testing.assert_array_equal(l2, lst)


def _offcentre_atlas():
    """Bitmaps whose non-zero texels fill only part of the bitmap, away from its
    centre: a blob in one corner, a thin bar along one edge, a single texel, and
    the soft disc (centred) for reference."""
    a = np.zeros((4, 24, 32), np.float32)
    yy, xx = np.mgrid[0:24, 0:32]
    a[0] = np.clip(1.0 - np.hypot(xx - 25.0, yy - 5.0) / 4.0, 0.0, 1.0)   # corner blob
    a[1, 20:22, 3:29] = 0.7                                                  # bar near the bottom
    a[2, 2, 30] = 1.0                                                        # one texel
    a[3] = inputs.soft_disc_atlas(5, 1, 32)[0, 4:28, :]
    return a


@pytest.mark.parametrize("which", ["disc", "offcentre", "strokes"])
def test_binning_rect_is_tight_and_conservative(which):
    """The fp32 spec box lies between the exact (FP64) box of the pixels within one
    texel of the bitmap's non-zero texels, widened by 0.99 px and by 1.01 px plus the
    margin's |s| 2^-19, and every pixel where a primitive is non-zero lies in one of
    its listed tiles (a solo FP64 render)."""
    tile = 16
    if which == "disc":
        sc = inputs.tiny(seed=10, N=120, H=160, W=144)
    else:
        atlas = _offcentre_atlas() if which == "offcentre" else inputs.stroke_atlas(3, 4, 48)
        p, b = inputs.primitives(17, 96, 160, 144, atlas.shape[0], "uniform", (0.05, 0.3))
        p[::5, 2] *= -1.0   # mirrored primitives: the centre offset changes sign
        sc = inputs.Scene(which, 160, 144, p, b, atlas)
    nb, Hb, Wb = sc.atlas.shape
    rects, tau = oracle.bin_rects(sc.H, sc.W, tile, sc.params, sc.bitmap_id, sc.atlas)
    ntx, nty = -(-sc.W // tile), -(-sc.H // tile)
    kw, kv = (Wb - 1) / 2, (Hb - 1) / 2
    for i, p in enumerate(sc.params.astype(np.float64)):
        ys_, xs_ = np.nonzero(sc.atlas[sc.bitmap_id[i]] > 0)
        # texel box (u0 - 1, u1 + 1) x (v0 - 1, v1 + 1) in normalised coordinates
        u_lo, u_hi = (xs_.min() - 1 - kw) / kw, (xs_.max() + 1 - kw) / kw
        v_lo, v_hi = (ys_.min() - 1 - kv) / kv, (ys_.max() + 1 - kv) / kv
        c, sn = math.cos(p[3]), math.sin(p[3])
        dx = [p[2] * (c * u - sn * v) for u in (u_lo, u_hi) for v in (v_lo, v_hi)]
        dy = [p[2] * (sn * u + c * v) for u in (u_lo, u_hi) for v in (v_lo, v_hi)]
        ext = 1.01 + abs(p[2]) * 2.0 ** -19

        def rect(m):
            r = [math.floor((p[0] + min(dx) - m) / tile), math.floor((p[1] + min(dy) - m) / tile),
                 math.floor((p[0] + max(dx) + m) / tile), math.floor((p[1] + max(dy) + m) / tile)]
            if r[2] < 0 or r[3] < 0 or r[0] > ntx - 1 or r[1] > nty - 1:
                return None
            return [max(r[0], 0), max(r[1], 0), min(r[2], ntx - 1), min(r[3], nty - 1)]
        lo, hi = rect(0.99), rect(ext)
        if tau[i] == 0:
            assert lo is None
            continue
        assert hi is not None
        assert hi[0] <= rects[i, 0] and hi[1] <= rects[i, 1]
        assert rects[i, 2] <= hi[2] and rects[i, 3] <= hi[3]
        if lo:
            assert rects[i, 0] <= lo[0] and rects[i, 1] <= lo[1]
            assert rects[i, 2] >= lo[2] and rects[i, 3] >= lo[3]
        solo = oracle.render(sc.H, sc.W, sc.params[i:i + 1], sc.bitmap_id[i:i + 1], sc.atlas,
                             background=None)
        ys, xs = np.nonzero(solo["T_final"] < 1.0)
        if len(xs):
            assert (xs // tile).min() >= rects[i, 0] and (xs // tile).max() <= rects[i, 2]
            assert (ys // tile).min() >= rects[i, 1] and (ys // tile).max() <= rects[i, 3]


def test_nonzero_boxes_of_the_atlas():
    a = _offcentre_atlas()
    boxes = oracle.nonzero_boxes(np.concatenate([a, np.zeros((1, 24, 32), np.float32)]))
    for b in range(4):
        ys, xs = np.nonzero(a[b] > 0)
        assert list(boxes[b]) == [xs.min(), xs.max(), ys.min(), ys.max()]
    assert list(boxes[2]) == [30, 30, 2, 2]
    assert list(boxes[4]) == [32, -1, 24, -1]   # all zero


def test_binning_skips_invalid_primitives():
    sc = inputs.tiny(seed=11, N=6, H=64, W=64)
    p = sc.params.copy()
    p[1, 2] = 0.0
    p[2, 0] = np.nan
    p[3, 3] = np.inf
    rects, tau = oracle.bin_rects(64, 64, 16, p, sc.bitmap_id, sc.atlas)
    assert tau[1] == tau[2] == tau[3] == 0
    assert tau[0] > 0
    # an all-zero bitmap and a bitmap id outside the atlas list a primitive nowhere
    atlas2 = np.concatenate([sc.atlas, np.zeros_like(sc.atlas)])
    _, tau2 = oracle.bin_rects(64, 64, 16, p[[0, 0, 0]], np.array([0, 1, 2], np.int32), atlas2)
    assert tau2[0] == tau[0] and tau2[1] == 0 and tau2[2] == 0
    out = oracle.render(64, 64, p, sc.bitmap_id, sc.atlas)
    ref = oracle.render(64, 64, p[[0, 4, 5]], sc.bitmap_id[[0, 4, 5]], sc.atlas)
    np.testing.assert_array_equal(out["image"], ref["image"])


# --------------------------------------------------------------------------
# Early termination, loss and optimiser
# --------------------------------------------------------------------------

def test_early_termination_error_is_bounded_by_T_stop():
    sc = inputs.tiny(seed=12, N=400, H=64, W=64)
    exact = oracle.render(64, 64, sc.params, sc.bitmap_id, sc.atlas)
    for ts in [1e-2, 1e-4, 1e-6]:
        trunc = oracle.render(64, 64, sc.params, sc.bitmap_id, sc.atlas, T_stop=ts)
        assert np.abs(trunc["image"] - exact["image"]).max() <= ts
        assert trunc["pairs"] <= exact["pairs"]


def test_mse_psnr_closed_forms():
    a = np.zeros((3, 4, 5))
    b = np.full((3, 4, 5), 0.1)
    assert oracle.mse(a, b) == pytest.approx(0.01)
    assert oracle.psnr(a, b) == pytest.approx(20.0)
    g = oracle.mse_grad(a, b)
    assert g.shape == a.shape and g[0, 0, 0] == pytest.approx(2 * (-0.1) / 60)


def test_adam_matches_torch_optim_adam():
    rng = np.random.default_rng(3)
    N = 7
    p0 = rng.normal(size=(N, 8))
    cols = [torch.tensor(p0[:, j].copy(), requires_grad=True) for j in range(8)]
    lr0 = 0.1
    opt = torch.optim.Adam([{"params": [c], "lr": lr0 * oracle.LR_GAINS[j]} for j, c in enumerate(cols)],
                           betas=(0.9, 0.999), eps=1e-8)
    p, m, v = p0.copy(), np.zeros_like(p0), np.zeros_like(p0)
    gamma = 0.9
    for t in range(1, 6):
        g = rng.normal(size=(N, 8))
        lr = lr0 * gamma ** (t - 1)
        for j, grp in enumerate(opt.param_groups):
            grp["lr"] = lr * oracle.LR_GAINS[j]
        for j, c in enumerate(cols):
            c.grad = torch.tensor(g[:, j].copy())
        opt.step()
        p, m, v = oracle.adam_step(p, g, m, v, t, lr)
    ref = np.stack([c.detach().numpy() for c in cols], 1)
    np.testing.assert_allclose(p, ref, rtol=0, atol=1e-14)


# --------------------------------------------------------------------------
# The contributing-pair count (the work unit of the compositors' roofline)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("T_stop", [0.0, 1e-2])
def test_contributing_pair_count_matches_a_torch_walk(T_stop):
    """Layers with M > 0 that a pixel composites while T >= T_stop, counted by the
    oracle's walk, equal the count of Algorithm S3 in torch (grid_sample per layer,
    a pixel frozen once its T falls below T_stop)."""
    import torch.nn.functional as F
    rng = np.random.default_rng(77)
    H, W, N = 26, 31, 16
    atlas = inputs.soft_disc_atlas(9, 2, 32)   # solid interiors: pixels saturate
    params = np.zeros((N, 8), np.float32)
    params[:, 0] = rng.uniform(0, W, N)
    params[:, 1] = rng.uniform(0, H, N)
    params[:, 2] = rng.uniform(8, 18, N)
    params[:, 3] = rng.uniform(-7, 7, N)
    params[:, 4] = rng.uniform(3, 8, N)
    params[:, 5:8] = rng.uniform(-3, 3, (N, 3))
    bid = rng.integers(0, atlas.shape[0], N).astype(np.int32)
    A = torch.tensor(atlas.astype(np.float64))
    p = torch.tensor(params.astype(np.float64))
    Y, X = torch.meshgrid(torch.arange(H, dtype=torch.float64), torch.arange(W, dtype=torch.float64),
                          indexing="ij")
    T = torch.ones(H, W, dtype=torch.float64)
    count = 0
    for i in range(N):
        x, y, s, th, nu = p[i, 0], p[i, 1], p[i, 2], p[i, 3], p[i, 4]
        u = (torch.cos(th) * (X - x) + torch.sin(th) * (Y - y)) / s
        v = (-torch.sin(th) * (X - x) + torch.cos(th) * (Y - y)) / s
        m = F.grid_sample(A[int(bid[i])][None, None], torch.stack([u, v], -1)[None], mode="bilinear",
                          padding_mode="zeros", align_corners=True)[0, 0]
        a = torch.sigmoid(nu) * m
        alive = T >= T_stop
        count += int(((m > 0) & alive).sum())
        T = torch.where(alive, T * (1 - a), T)
    out = oracle.render(H, W, params, bid, atlas, T_stop=T_stop)
    assert out["contrib"] == count
    assert 0 < count <= out["pairs"]
    if T_stop > 0:   # early termination removes work
        assert count < oracle.render(H, W, params, bid, atlas)["contrib"]


# --------------------------------------------------------------------------
# The sampled gradient (grad_selected) against the full gradient
# --------------------------------------------------------------------------

def _edge_scene(seed):
    """A ragged 37 x 29 canvas of soft discs and edge-to-edge bitmaps plus the
    placements where a support box meets the canvas border or the box rule itself
    matters: primitives centred past the right and bottom edges and across the
    top-left corner, rotated ones, a negative scale, a NaN parameter and a zero scale."""
    H, W = 37, 29
    sc = inputs.tiny(seed=seed, N=24, H=H, W=W)
    extra = np.array([
        [W + 3.0, H / 2, 9.0, 0.4, 0.5, 0.3, -0.2, 1.0],     # past the right edge
        [W / 2, H + 2.5, 7.5, 2.0, 0.2, -1.0, 0.4, 0.1],     # past the bottom edge
        [W - 0.5, H - 0.5, 11.0, 0.9, 1.0, 0.6, 0.6, -0.6],  # bottom-right corner
        [-2.0, -3.0, 8.0, 5.1, 0.7, 0.1, 0.9, -0.3],         # across the top-left corner
        [10.0, 12.0, -6.0, 1.2, 0.4, -0.4, 0.2, 0.8],        # negative scale
        [14.0, 20.0, 5.0, float("nan"), 0.0, 0.0, 0.0, 0.0], # NaN angle: no contribution
        [15.0, 15.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0],          # zero scale: no contribution
        [W - 1.0, 4.0, 3.2, 0.785, 2.0, 1.5, -1.5, 0.0],     # small, at the last column
    ], np.float32)
    params = np.concatenate([sc.params[:12], extra, sc.params[12:]])
    # a second bitmap non-zero up to its edges: its taps in the zero-padding ring
    # (U or V within one texel outside the bitmap) are non-zero, so the support box
    # is exercised to its last row and column
    edge = np.random.default_rng(seed).uniform(0.2, 1.0, (1,) + sc.atlas.shape[1:]).astype(np.float32)
    atlas = np.concatenate([sc.atlas, edge])
    bid = np.zeros(params.shape[0], np.int32)
    bid[::3] = 1
    bid[12:16] = 1
    return H, W, params, bid, atlas


@pytest.mark.parametrize("bg", ["const", "none", "buffer"])
@pytest.mark.parametrize("T_stop", [0.0, 1e-6])
def test_grad_selected_equals_the_rows_of_the_full_gradient(bg, T_stop):
    """grad_selected sums each selected primitive's per-pixel terms over its support
    box clipped to the canvas; every pixel outside the box contributes exactly zero
    (Eq. 6, Eqs. S4-S5), so its rows must equal those of the full gradient, whatever
    the selection order, with repeats, on all three backgrounds (Eq. 8), alpha_max < 1
    and a dL/dI_alpha term."""
    H, W, params, bid, atlas = _edge_scene(7)
    rng = np.random.default_rng(3)
    background = {"const": (0.9, 0.2, 0.5), "none": None,
                  "buffer": rng.uniform(0, 1, (3, H, W)).astype(np.float32)}[bg]
    gI = rng.normal(size=(3, H, W)).astype(np.float32)
    gA = rng.normal(size=(H, W)).astype(np.float32)
    N = params.shape[0]
    sel = np.concatenate([rng.permutation(N), [13, 13, 0, N - 1]]).astype(np.int32)
    for amax, dA in ((1.0, None), (0.65, gA)):
        full = oracle.grad(H, W, params, bid, atlas, gI.astype(np.float64), dL_dalpha=dA, alpha_max=amax,
                           background=background, T_stop=T_stop)
        part = oracle.grad_selected(H, W, params, bid, atlas, gI, sel, dL_dalpha=dA, alpha_max=amax,
                                    background=background, T_stop=T_stop)
        scale = np.abs(full).max()
        assert scale > 0
        np.testing.assert_allclose(part, full[sel], rtol=0, atol=1e-12 * scale)
        # the edge primitives do contribute, so the clipped boxes were exercised
        for i in (12, 13, 14, 15, 16, 19):
            assert np.abs(full[i]).max() > 1e-6 * scale, i
        # invalid primitives: zero rows on both sides
        assert not full[17].any() and not full[18].any()


def test_grad_pixels_equals_rows_and_masked_full_gradients():
    """The gradient restricted to a pixel set equals grad_rows for whole rows, and
    the full gradient (Eq. 6, Eqs. S4-S5) of the upstream gradient masked to the set
    for a scattered set; a listed pixel counts once per listing."""
    H, W, params, bid, atlas = _edge_scene(9)
    rng = np.random.default_rng(12)
    gI = rng.normal(size=(3, H, W))
    gA = rng.normal(size=(H, W))
    for T_stop in (0.0, 1e-6):
        ys, xs = np.mgrid[5:17, 0:W]
        a = oracle.grad_pixels(H, W, params, bid, atlas, gI, (xs.ravel(), ys.ravel()), dL_dalpha=gA,
                               alpha_max=0.8, T_stop=T_stop)
        b = oracle.grad_rows(H, W, params, bid, atlas, gI, 5, 17, dL_dalpha=gA, alpha_max=0.8, T_stop=T_stop)
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-12 * np.abs(b).max())
        mask = rng.uniform(size=(H, W)) < 0.3
        py, px = np.nonzero(mask)
        c = oracle.grad_pixels(H, W, params, bid, atlas, gI, (px, py), dL_dalpha=gA, alpha_max=0.8,
                               T_stop=T_stop)
        d = oracle.grad(H, W, params, bid, atlas, gI * mask, dL_dalpha=gA * mask, alpha_max=0.8, T_stop=T_stop)
        np.testing.assert_allclose(c, d, rtol=0, atol=1e-12 * np.abs(d).max())
    twice = oracle.grad_pixels(H, W, params, bid, atlas, gI, (np.r_[px, px], np.r_[py, py]))
    once = oracle.grad_pixels(H, W, params, bid, atlas, gI, (px, py))
    np.testing.assert_allclose(twice, 2 * once, rtol=1e-13, atol=1e-300)


def test_binning_rect_beyond_the_reduction_range_holds_every_rotation():
    """For |theta| > 65536 the specification's sine and cosine are not computed; the
    box is centred on (x, y) with half-extents |s| (|uc| + eu + |vc| + ev), which holds
    the bitmap's non-zero texels at any rotation: every pixel a solo FP64 render
    leaves with T < 1 lies in a listed tile."""
    atlas = _offcentre_atlas()
    tile = 8
    rng = np.random.default_rng(23)
    for b in range(atlas.shape[0]):
        p = np.zeros((1, 8), np.float32)
        p[0, :3] = (40.0 + rng.uniform(-3, 3), 44.0 + rng.uniform(-3, 3), 14.0)
        p[0, 3] = 1.0e6 + rng.uniform(0, 7)   # beyond 65536
        p[0, 4:] = 2.0
        bid = np.array([b], np.int32)
        rects, tau = oracle.bin_rects(96, 96, tile, p, bid, atlas)
        solo = oracle.render(96, 96, p, bid, atlas, background=None)
        ys, xs = np.nonzero(solo["T_final"] < 1.0)
        assert tau[0] > 0 and len(xs) > 0
        assert (xs // tile).min() >= rects[0, 0] and (xs // tile).max() <= rects[0, 2]
        assert (ys // tile).min() >= rects[0, 1] and (ys // tile).max() <= rects[0, 3]
