"""Batched persistent rendering, every tuning instantiation, CUDA-graph capture of a
whole optimisation step, the autotuner, the loss and Adam kernels, and device-side
error reporting -- all through the C ABI, checked against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2602_22625_gb300 import dbmp as D
from paper_2602_22625_gb300 import inputs
from _helpers import cuda, grad_close, to_dev, torch

pytestmark = pytest.mark.gpu

IMG_TOL = 1e-5
TUNINGS = [(t, b, p) for t in (8, 16, 32) for b in (32, 64) for p in (1, 2, 4) if not (p == 4 and t == 8)]


def small_batch(seed=31, n=5):
    g = np.random.default_rng(seed)
    atlas = inputs.stroke_atlas(5, 4, 32, n_seg=24)
    scenes = []
    sizes = [(70, 53), (33, 90), (64, 64), (17, 21), (48, 100)][:n]
    counts = [40, 0, 25, 7, 60][:n]
    for c, ((H, W), N) in enumerate(zip(sizes, counts)):
        p, b = inputs.primitives(seed * 1000 + c, N, H, W, atlas.shape[0], "uniform", (0.05, 0.3))
        scenes.append(inputs.Scene(f"c{c}", H, W, p, b, atlas))
    return scenes, atlas


def concat(scenes):
    params = np.concatenate([s.params for s in scenes]) if scenes else np.zeros((0, 8), np.float32)
    bid = np.concatenate([s.bitmap_id for s in scenes]).astype(np.int32)
    off = np.concatenate([[0], np.cumsum([s.N for s in scenes])]).astype(np.int64)
    pix = np.concatenate([[0], np.cumsum([s.H * s.W for s in scenes])]).astype(np.int64)
    return params, bid, off, pix


def run_batch(scenes, atlas_np, tuning, gI=None, T_stop=0.0, bg=(1.0, 1.0, 1.0), poison=False):
    cuda()
    params, bid, off, pix = concat(scenes)
    N, P = int(off[-1]), int(pix[-1])
    atlas = D.dbmp_atlas_create(to_dev(atlas_np))
    n_tiles = sum(-(-s.W // 8) * -(-s.H // 8) for s in scenes)
    ws = D.dbmp_workspace_create(max(N, 1), n_tiles, 1 << 24, len(scenes))
    if poison:
        D.dbmp_workspace_poison(ws)
    try:
        D.dbmp_batch_plan(ws, [s.H for s in scenes], [s.W for s in scenes], off.tolist(), *tuning)
        p, b = to_dev(params), to_dev(bid)
        image = torch.full((3 * P,), -7.0, device="cuda")
        T = torch.empty(P, device="cuda")
        nl = torch.empty(P, dtype=torch.int32, device="cuda")
        dparams = torch.zeros(max(N, 1), 8, device="cuda")
        mode = D.BATCH_BIN | D.BATCH_FWD
        gdev = None
        if gI is not None:
            mode |= D.BATCH_BWD
            gdev = to_dev(gI.astype(np.float32))
        bgs = D.make_background(bg)
        D.dbmp_batch_render(ws, p, b, atlas, 1.0, bgs, T_stop, mode, image, T, nl, gdev, dparams)
        st = D.dbmp_status_poll(ws)
        torch.cuda.synchronize()
        return image.cpu().numpy(), T.cpu().numpy(), dparams.cpu().numpy()[:N].astype(np.float64), st
    finally:
        D.dbmp_workspace_destroy(ws)
        D.dbmp_atlas_destroy(atlas)


def split(flat, scenes, pix, channels):
    out = []
    for c, s in enumerate(scenes):
        a = flat[channels * pix[c]: channels * pix[c + 1]]
        out.append(a.reshape((channels, s.H, s.W)) if channels > 1 else a.reshape(s.H, s.W))
    return out


@pytest.mark.parametrize("tuning", TUNINGS, ids=lambda t: f"t{t[0]}b{t[1]}p{t[2]}")
def test_every_tuning_matches_oracle(tuning):
    sc = inputs.tiny(seed=3, N=120, H=72, W=88)
    rng = np.random.default_rng(7)
    gI = rng.normal(size=(3, sc.H, sc.W)).astype(np.float32)
    img, T, g, _ = run_batch([sc], sc.atlas, tuning, gI=gI)
    ref = oracle.render(sc.H, sc.W, sc.params, sc.bitmap_id, sc.atlas, background=sc.background)
    assert np.abs(img.reshape(3, sc.H, sc.W) - ref["image"]).max() <= IMG_TOL
    assert np.abs(T.reshape(sc.H, sc.W) - ref["T_final"]).max() <= IMG_TOL
    gref = oracle.grad(sc.H, sc.W, sc.params, sc.bitmap_id, sc.atlas, gI, background=sc.background)
    grad_close(g, gref, what=str(tuning))


@pytest.mark.parametrize("T_stop", [0.0, 1e-6])
def test_every_tuning_renders_the_same_bits(T_stop):
    """A pixel's composite does not depend on how pixels are grouped into warps: the
    scalar path (1 px/lane) and the packed FP32x2 paths (2 and 4 px/lane, two pixels
    per instruction) round every operation alike, culled primitives are exact no-ops,
    and a pixel stops at T < T_stop whatever its warp does.  So all tunings give the
    same image and transmittance bit for bit, on a ragged multi-canvas batch."""
    scenes, atlas = small_batch(seed=52)
    first = None
    for tuning in TUNINGS:
        img, T, _, st = run_batch(scenes, atlas, tuning, T_stop=T_stop)
        assert st.code == 0
        if first is None:
            first = (tuning, img, T)
            continue
        assert np.array_equal(img, first[1]), f"{tuning} vs {first[0]}"
        assert np.array_equal(T, first[2]), f"{tuning} vs {first[0]}"


def scene_sub_pixel(seed=31, H=48, W=48):
    """Primitives far smaller than a pixel (s = 1e-28 .. 0.2 px; at 1e-28 the transform
    coefficients are ~3e29, within the 2^100 the library accepts) on integer centres at
    rotations 0, 45, 90, 180 and 270 degrees, between two groups of ordinary ones.
    Along the line through a tiny primitive's centre in its u direction, V is within
    the bitmap while |U| reaches ~1e31: those pixels' taps lie far beyond the bitmap's
    columns.  Returns the scene and the indices of the tiny primitives."""
    g = np.random.default_rng(seed)
    tiny = []
    for s in (1e-28, 1e-9, 1e-6, 1e-3, 0.2):
        for th in (0.0, 0.25 * np.pi, 0.5 * np.pi, np.pi, 1.5 * np.pi):
            x, y = g.integers(4, W - 4), g.integers(4, H - 4)
            tiny.append([x, y, s, th, g.normal(), *g.normal(size=3)])
    big = [[g.uniform(0, W), g.uniform(0, H), g.uniform(6, 20), g.uniform(0, 2 * np.pi), g.normal(),
            *g.normal(size=3)] for _ in range(12)]
    p = np.array(big[:6] + tiny + big[6:], np.float32)
    atlas = inputs.tiny(seed=3).atlas[:1]
    sc = inputs.Scene("sub-pixel", H, W, p, np.zeros(len(p), np.int32), atlas)
    return sc, np.arange(6, 6 + len(tiny))


@pytest.mark.parametrize("tuning", [(16, 32, 2), (32, 32, 4), (8, 32, 1)], ids=lambda t: f"t{t[0]}p{t[2]}")
def test_sub_pixel_primitives_sample_nothing_beyond_the_bitmap(tuning):
    """The backward tests only V's range before a gather and relies on the texture's
    border for U: a footprint in columns < 0 or >= W_b reads zeros, however far out
    (here up to |U| ~ 1e31).
    Each tiny primitive composites only at its own centre pixel (where the atlas is
    flat, so its geometric gradients are exactly 0); any texel read beyond the bitmap
    would give it a non-zero geometric gradient, and the deeper layers' recovered
    transmittance would change.  Image and gradients against the oracle."""
    sc, tiny = scene_sub_pixel()
    rng = np.random.default_rng(8)
    gI = rng.normal(size=(3, sc.H, sc.W)).astype(np.float32)
    img, T, g, st = run_batch([sc], sc.atlas, tuning, gI=gI)
    assert st.code == 0
    ref = oracle.render(sc.H, sc.W, sc.params, sc.bitmap_id, sc.atlas, background=sc.background)
    assert np.abs(img.reshape(3, sc.H, sc.W) - ref["image"]).max() <= IMG_TOL
    gref = oracle.grad(sc.H, sc.W, sc.params, sc.bitmap_id, sc.atlas, gI, background=sc.background)
    assert np.all(gref[tiny, :4] == 0.0) and np.abs(gref[tiny, 4:]).max() > 1e-3
    grad_close(g[tiny], gref[tiny], what=f"{tuning} sub-pixel")
    big = np.setdiff1d(np.arange(sc.N), tiny)
    grad_close(g[big], gref[big], what=f"{tuning} ordinary")


@pytest.mark.parametrize("tuning", [(16, 32, 2, 4), (32, 64, 4, 1), (8, 32, 1, 2)],
                         ids=lambda t: f"t{t[0]}b{t[1]}p{t[2]}pb{t[3]}")
def test_forward_and_backward_at_different_ppt_match_oracle(tuning):
    """The backward's regions may differ from the forward's (own pixels per lane)."""
    test_every_tuning_matches_oracle(tuning)


@pytest.mark.parametrize("tuning", [(16, 32, 2), (8, 64, 1), (32, 32, 4)])
def test_multi_canvas_batch_matches_oracle_per_canvas(tuning):
    scenes, atlas = small_batch()
    params, bid, off, pix = concat(scenes)
    rng = np.random.default_rng(9)
    gI = rng.normal(size=3 * int(pix[-1])).astype(np.float32)
    img, T, g, st = run_batch(scenes, atlas, tuning, gI=gI, bg=(0.3, 0.6, 0.9))
    imgs = split(img, scenes, pix, 3)
    gIs = split(gI, scenes, pix, 3)
    for c, s in enumerate(scenes):
        ref = oracle.render(s.H, s.W, s.params, s.bitmap_id, atlas, background=(0.3, 0.6, 0.9))
        assert np.abs(imgs[c] - ref["image"]).max() <= IMG_TOL, c
        if s.N:
            gref = oracle.grad(s.H, s.W, s.params, s.bitmap_id, atlas, gIs[c], background=(0.3, 0.6, 0.9))
            grad_close(g[off[c]:off[c + 1]], gref, what=f"canvas {c}")
    assert st.pairs_required > 0


def scenes_extreme(seed=61):
    """A ragged batch of degenerate canvases and extents: 1 x 1, 1 x 37 and 29 x 1
    canvases, and a 40 x 40 canvas whose primitives include half-extents of 1e3 to
    1e20 px (the bitmap's centre stretched over the canvas), rotations of 1e30 (beyond
    the binning's sine/cosine range: a box holding every rotation), centres 1e9 px
    away with a half-extent that still reaches the canvas, and negative scales; each
    canvas also has a few ordinary primitives."""
    g = np.random.default_rng(seed)
    atlas = inputs.tiny(seed=3).atlas[:1]

    def ordinary(n, H, W):
        return [[g.uniform(-5, W + 5), g.uniform(-5, H + 5), g.uniform(2, 12) * g.choice([-1, 1]),
                 g.uniform(0, 2 * np.pi), g.normal(), *g.normal(size=3)] for _ in range(n)]

    scenes = []
    for H, W in ((1, 1), (1, 37), (29, 1)):
        p = np.array(ordinary(6, H, W), np.float32)
        scenes.append(inputs.Scene(f"{H}x{W}", H, W, p, np.zeros(len(p), np.int32), atlas))
    ext = [[20.0, 20.0, 1e3, 0.3, 0.5, 0.2, -0.4, 0.9],
           [5.0, 33.0, 1e20, 1.1, -0.5, 1.0, 0.3, -0.2],
           [17.0, 9.0, 8.0, 1e30, 0.8, -0.6, 0.1, 0.4],
           [-1e9, 20.0, 1.5e9, 0.0, 0.3, 0.7, -0.9, 0.2],
           [20.0, 1e9, -1.5e9, 0.5 * np.pi, -0.2, -0.3, 0.6, 0.5],
           [30.0, 12.0, -6.0, -1e30, 1.2, 0.4, 0.4, -0.7]]
    p = np.array(ordinary(3, 40, 40) + ext + ordinary(3, 40, 40), np.float32)
    scenes.append(inputs.Scene("extreme", 40, 40, p, np.zeros(len(p), np.int32), atlas))
    return scenes, atlas


@pytest.mark.parametrize("tuning", [(16, 32, 2), (32, 32, 4), (8, 64, 1)], ids=lambda t: f"t{t[0]}p{t[2]}")
def test_degenerate_canvases_and_extents_match_oracle(tuning):
    scenes, atlas = scenes_extreme()
    params, bid, off, pix = concat(scenes)
    rng = np.random.default_rng(10)
    gI = rng.normal(size=3 * int(pix[-1])).astype(np.float32)
    img, T, g, st = run_batch(scenes, atlas, tuning, gI=gI)
    assert st.code == 0
    imgs, Ts, gIs = split(img, scenes, pix, 3), split(T, scenes, pix, 1), split(gI, scenes, pix, 3)
    for c, s in enumerate(scenes):
        ref = oracle.render(s.H, s.W, s.params, s.bitmap_id, atlas, background=s.background)
        assert np.abs(imgs[c] - ref["image"]).max() <= IMG_TOL, s.name
        assert np.abs(Ts[c].reshape(s.H, s.W) - ref["T_final"]).max() <= IMG_TOL, s.name
        gref = oracle.grad(s.H, s.W, s.params, s.bitmap_id, atlas, gIs[c], background=s.background)
        grad_close(g[off[c]:off[c + 1]], gref, what=f"{tuning} {s.name}")


def scene_non_square(seed=71, H=70, W=90):
    """Bitmaps of 24 x 40 texels (H_b != W_b: the horizontal and vertical half-widths
    of Eq. 2 differ, and so do rho and 1/rho in the rotation gradient): two strokes, an
    all-zero bitmap (never listed) and one whose only non-zero texel is its last
    corner (the tight binning box and the zero padding at a corner)."""
    g = np.random.default_rng(seed)
    strokes = inputs.stroke_atlas(17, 2, 40, n_seg=16)[:, 8:32, :]
    corner = np.zeros((1, 24, 40), np.float32)
    corner[0, 23, 39] = 0.9
    atlas = np.ascontiguousarray(np.concatenate([strokes, np.zeros((1, 24, 40), np.float32), corner]))
    N = 90
    p = np.zeros((N, 8), np.float32)
    p[:, 0] = g.uniform(-5, W + 5, N)
    p[:, 1] = g.uniform(-5, H + 5, N)
    p[:, 2] = g.uniform(4, 24, N) * g.choice([1, 1, -1], N)
    p[:, 3] = g.uniform(-4, 4, N)
    p[:, 4] = g.uniform(-1, 2, N)
    p[:, 5:] = g.normal(size=(N, 3))
    bid = g.choice([0, 1, 2, 3], N, p=[0.4, 0.4, 0.1, 0.1]).astype(np.int32)
    return inputs.Scene("non-square", H, W, p, bid, atlas)


@pytest.mark.parametrize("tuning", [(16, 32, 2), (32, 32, 4), (8, 64, 1)], ids=lambda t: f"t{t[0]}p{t[2]}")
def test_non_square_bitmaps_match_oracle(tuning):
    sc = scene_non_square()
    rng = np.random.default_rng(12)
    gI = rng.normal(size=(3, sc.H, sc.W)).astype(np.float32)
    img, T, g, st = run_batch([sc], sc.atlas, tuning, gI=gI, bg=(0.2, 0.4, 0.6))
    assert st.code == 0
    ref = oracle.render(sc.H, sc.W, sc.params, sc.bitmap_id, sc.atlas, background=(0.2, 0.4, 0.6))
    assert np.abs(img.reshape(3, sc.H, sc.W) - ref["image"]).max() <= IMG_TOL
    assert np.abs(T.reshape(sc.H, sc.W) - ref["T_final"]).max() <= IMG_TOL
    gref = oracle.grad(sc.H, sc.W, sc.params, sc.bitmap_id, sc.atlas, gI, background=(0.2, 0.4, 0.6))
    grad_close(g, gref, what=str(tuning))
    assert not g[sc.bitmap_id == 2].any()   # the all-zero bitmap contributes nothing
    corner = np.nonzero(sc.bitmap_id == 3)[0]
    assert np.abs(gref[corner]).max() > 0   # the corner texel is reached


def test_batched_workload_sampled_against_oracle():
    """The 64-canvas workload shape (sides 256..1024, 1k..50k primitives), scaled
    down to 12 canvases so the oracle can check sampled pixels of every canvas."""
    scenes = inputs.batched(seed=4, n_canvas=12, side=(96, 320), nprim=(200, 3000))
    atlas = scenes[0].atlas
    params, bid, off, pix = concat(scenes)
    img, T, _, _ = run_batch(scenes, atlas, (16, 32, 2), T_stop=1e-6)
    imgs = split(img, scenes, pix, 3)
    rng = np.random.default_rng(1)
    for c, s in enumerate(scenes):
        px = rng.integers(0, s.W, 200)
        py = rng.integers(0, s.H, 200)
        ref = oracle.render(s.H, s.W, s.params, s.bitmap_id, atlas, background=s.background,
                            pixels=(px, py))
        assert np.abs(imgs[c][:, py, px] - ref["image"]).max() <= IMG_TOL, c


def test_capacity_overflow_is_reported_and_nothing_is_written():
    cuda()
    sc = inputs.tiny(seed=4, N=200, H=64, W=64)
    atlas = D.dbmp_atlas_create(to_dev(sc.atlas))
    ws = D.dbmp_workspace_create(sc.N, 64, 16, 1)  # room for 16 list entries only
    try:
        D.dbmp_bin(ws, sc.H, sc.W, 16, to_dev(sc.params), to_dev(sc.bitmap_id), sc.N, atlas, 1.0)
        image = torch.full((3, 64, 64), -7.0, device="cuda")
        T = torch.full((64, 64), -7.0, device="cuda")
        nl = torch.zeros(64, 64, dtype=torch.int32, device="cuda")
        D.dbmp_render_fwd(ws, atlas, D.make_background((1, 1, 1)), 0.0, image, T, nl)
        with pytest.raises(D.DbmpError) as e:
            D.dbmp_status_poll(ws)
        assert e.value.code == D.DBMP_ERR_CAPACITY
        st = D.dbmp_status_poll(ws, raise_on_error=False)  # cleared after the first poll
        assert st.code == 0 and st.pairs_required > 16
        assert torch.all(image == -7.0) and torch.all(T == -7.0)
    finally:
        D.dbmp_workspace_destroy(ws)
        D.dbmp_atlas_destroy(atlas)


def test_out_of_range_bitmap_id_is_not_drawn():
    cuda()
    sc = inputs.tiny(seed=6, N=30, H=48, W=48)
    bid = sc.bitmap_id.copy()
    bid[4] = 5   # atlas has one bitmap
    bid[9] = -1
    atlas = D.dbmp_atlas_create(to_dev(sc.atlas))
    ws = D.dbmp_workspace_create(sc.N, 64, 1 << 16, 1)
    try:
        D.dbmp_bin(ws, 48, 48, 16, to_dev(sc.params), to_dev(bid), sc.N, atlas, 1.0)
        image = torch.empty(3, 48, 48, device="cuda")
        T = torch.empty(48, 48, device="cuda")
        nl = torch.empty(48, 48, dtype=torch.int32, device="cuda")
        D.dbmp_render_fwd(ws, atlas, D.make_background((1, 1, 1)), 0.0, image, T, nl)
        st = D.dbmp_status_poll(ws)
        assert st.n_degenerate == 2
        keep = np.setdiff1d(np.arange(sc.N), [4, 9])
        ref = oracle.render(48, 48, sc.params[keep], sc.bitmap_id[keep], sc.atlas)
        assert np.abs(image.cpu().numpy() - ref["image"]).max() <= IMG_TOL
    finally:
        D.dbmp_workspace_destroy(ws)
        D.dbmp_atlas_destroy(atlas)


@pytest.mark.parametrize("offset", [0, 1])
def test_mse_kernel_matches_oracle(offset):
    """offset 0: 16-byte aligned buffers (four elements per load, a 3-element tail);
    offset 1: buffers one float past the boundary (the scalar path)."""
    cuda()
    rng = np.random.default_rng(0)
    a = rng.uniform(0, 1, (3, 77, 45)).astype(np.float32)
    b = rng.uniform(0, 1, (3, 77, 45)).astype(np.float32)
    n = a.size
    ab = torch.zeros(n + 4, device="cuda")
    bb = torch.zeros(n + 4, device="cuda")
    gb = torch.zeros(n + 4, device="cuda")
    ab[offset:offset + n] = to_dev(a).reshape(-1)
    bb[offset:offset + n] = to_dev(b).reshape(-1)
    dL = gb[offset:offset + n].view(3, 77, 45)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    D.dbmp_mse_grad(ab[offset:offset + n], bb[offset:offset + n], dL, loss)
    torch.cuda.synchronize()
    assert float(gb[:offset].abs().sum()) == 0.0 and float(gb[offset + n:].abs().sum()) == 0.0
    # the kernel forms I - I* in float32 (one rounding, relative 6e-8 per element) and
    # squares and sums in float64
    assert loss.item() == pytest.approx(oracle.mse(a, b), rel=2e-7)
    np.testing.assert_allclose(dL.cpu().numpy(), oracle.mse_grad(a, b), rtol=1e-6, atol=1e-12)


@pytest.mark.parametrize("offset", [0, 1], ids=["aligned", "unaligned"])
def test_adam_kernel_matches_oracle(offset):
    """offset 1 shifts every array by one float: the element-wise kernel instead of the
    one with 16-byte vectors."""
    cuda()
    rng = np.random.default_rng(1)
    N = 1000

    def buf(init=None):
        b = torch.zeros(N * 8 + 1, device="cuda")
        t = b[offset:offset + N * 8].view(N, 8)
        if init is not None:
            t.copy_(torch.from_numpy(init))
        return t

    p0 = rng.normal(size=(N, 8)).astype(np.float32)
    p = buf(p0)
    m = buf()
    v = buf()
    step = torch.zeros(1, dtype=torch.int32, device="cuda")
    cfg = D.adam_config(lr=0.1, gamma=0.95, zero_grad=True)
    rp, rm, rv = p0.astype(np.float64), np.zeros((N, 8)), np.zeros((N, 8))
    for t in range(1, 6):
        g = rng.normal(size=(N, 8)).astype(np.float32)
        gd = buf(g)
        D.dbmp_adam_step(p, gd, m, v, step, cfg)
        torch.cuda.synchronize()
        assert torch.all(gd == 0)
        rp, rm, rv = oracle.adam_step(rp, g, rm, rv, t, 0.1 * 0.95 ** (t - 1))
    assert step.item() == 5
    np.testing.assert_allclose(p.cpu().numpy(), rp, rtol=0, atol=2e-5)


def test_cuda_graph_captures_a_whole_optimisation_step():
    """bin + fwd + MSE + bwd captured once in a CUDA graph: replays at fixed
    parameters accumulate exactly the gradient the eager calls accumulate (up to
    atomic summation order).  With the Adam step inside the graph, the device step
    counter advances once per replay and the loss falls."""
    cuda()
    sc = inputs.tiny(seed=8, N=300, H=128, W=128)
    tg = inputs.tiny(seed=9, N=300, H=128, W=128)
    atlas = D.dbmp_atlas_create(to_dev(sc.atlas))
    bg = D.make_background((1, 1, 1))
    ws = D.dbmp_workspace_create(sc.N, 256, 1 << 20, 1)
    D.dbmp_batch_plan(ws, [128], [128], [0, sc.N], 16, 32, 2)
    params = to_dev(sc.params)
    bid = to_dev(sc.bitmap_id)
    target = torch.empty(3, 128, 128, device="cuda")
    T = torch.empty(128, 128, device="cuda")
    nl = torch.empty(128, 128, dtype=torch.int32, device="cuda")
    D.dbmp_batch_render(ws, to_dev(tg.params), to_dev(tg.bitmap_id), atlas, 1.0, bg, 0.0,
                        D.BATCH_BIN | D.BATCH_FWD, target, T, nl)
    image = torch.empty(3, 128, 128, device="cuda")
    dL = torch.empty(3, 128, 128, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    dparams = torch.zeros(sc.N, 8, device="cuda")
    m = torch.zeros(sc.N, 8, device="cuda")
    v = torch.zeros(sc.N, 8, device="cuda")
    step = torch.zeros(1, dtype=torch.int32, device="cuda")
    cfg = D.adam_config(lr=0.02, gamma=0.99, zero_grad=True)

    def grad_only():
        D.dbmp_batch_render(ws, params, bid, atlas, 1.0, bg, 1e-6, D.BATCH_BIN | D.BATCH_FWD, image, T, nl)
        D.dbmp_mse_grad(image, target, dL, loss)
        D.dbmp_batch_render(ws, params, bid, atlas, 1.0, bg, 1e-6, D.BATCH_BWD, image, T, nl, dL, dparams)

    def full_step():
        grad_only()
        D.dbmp_adam_step(params, dparams, m, v, step, cfg)

    try:
        for _ in range(3):
            grad_only()
        torch.cuda.synchronize()
        eager = dparams.clone()
        loss0 = loss.item()
        dparams.zero_()
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            g1 = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g1, stream=s):
                grad_only()
            g2 = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g2, stream=s):
                full_step()
        torch.cuda.synchronize()
        dparams.zero_()
        for _ in range(3):
            g1.replay()
        torch.cuda.synchronize()
        assert loss.item() == pytest.approx(loss0, rel=1e-12)
        grad_close(dparams.cpu().numpy(), eager.cpu().numpy(), rel=1e-4, what="graph vs eager")
        dparams.zero_()
        losses = []
        for _ in range(20):
            g2.replay()
            losses.append(loss.item())
        assert step.item() == 20
        assert losses[-1] < 0.9 * losses[0]
    finally:
        torch.cuda.synchronize()
        D.dbmp_workspace_destroy(ws)
        D.dbmp_atlas_destroy(atlas)


def test_autotune_picks_a_supported_tuning():
    cuda()
    sc = inputs.tiny(seed=10, N=500, H=200, W=160)
    atlas = D.dbmp_atlas_create(to_dev(sc.atlas))
    ws = D.dbmp_workspace_create(sc.N, 25 * 20, 1 << 22, 1)
    try:
        D.dbmp_batch_plan(ws, [sc.H], [sc.W], [0, sc.N])
        p, b = to_dev(sc.params), to_dev(sc.bitmap_id)
        image = torch.empty(3, sc.H, sc.W, device="cuda")
        T = torch.empty(sc.H, sc.W, device="cuda")
        nl = torch.empty(sc.H, sc.W, dtype=torch.int32, device="cuda")
        dL = torch.zeros(3, sc.H, sc.W, device="cuda")
        dp = torch.zeros(sc.N, 8, device="cuda")
        best, ms = D.dbmp_autotune(ws, p, b, atlas, 1.0, D.make_background((1, 1, 1)), 1e-6,
                                   D.BATCH_FWD | D.BATCH_BWD, image, T, nl, dL, dp, reps=1)
        assert tuple(best[:3]) in TUNINGS and (best[0], best[1], best[3]) in TUNINGS and ms > 0
        D.dbmp_batch_render(ws, p, b, atlas, 1.0, D.make_background((1, 1, 1)), 0.0,
                            D.BATCH_BIN | D.BATCH_FWD, image, T, nl)
        ref = oracle.render(sc.H, sc.W, sc.params, sc.bitmap_id, sc.atlas)
        assert np.abs(image.cpu().numpy() - ref["image"]).max() <= IMG_TOL
    finally:
        D.dbmp_workspace_destroy(ws)
        D.dbmp_atlas_destroy(atlas)


@pytest.mark.parametrize("which", ["main", "tiny_prims"])
def test_density_guided_autotune_agrees_with_the_exhaustive_search(which):
    """The tile-density statistics (Sec. S4) feeding the search: with tile sizes that
    list more than 2x the entries of the sparsest one left untimed, the autotuner picks
    the exhaustive search's tile size, at a time within noise of its best.  The main
    workload's primitives span many tiles (the search keeps tile 32 only); primitives
    of a few pixels hit one tile at any size, so there every tile size is timed."""
    cuda()
    if which == "main":
        sc = inputs.main()
    else:
        p, b = inputs.primitives(77, 20000, 1024, 1024, 16, "uniform", (0.002, 0.004))
        sc = inputs.Scene("tiny_prims", 1024, 1024, p, b, inputs.strokes16())
    atlas = D.dbmp_atlas_create(to_dev(sc.atlas))
    ws = D.dbmp_workspace_create(sc.N, (sc.H // 8) * (sc.W // 8), 64 << 20, 1)
    try:
        p, b = to_dev(sc.params), to_dev(sc.bitmap_id)
        image = torch.empty(3, sc.H, sc.W, device="cuda")
        T = torch.empty(sc.H, sc.W, device="cuda")
        nl = torch.empty(sc.H, sc.W, dtype=torch.int32, device="cuda")
        dL = torch.full((3, sc.H, sc.W), 1e-6, device="cuda")
        dp = torch.zeros(sc.N, 8, device="cuda")
        picks = {}
        for ratio in (0.0, 2.0, 0.0, 2.0):
            D.dbmp_batch_plan(ws, [sc.H], [sc.W], [0, sc.N])
            D.dbmp_autotune_set_prune(ws, ratio)
            best, ms = D.dbmp_autotune(ws, p, b, atlas, 1.0, D.make_background((1, 1, 1)), 1e-6,
                                       D.BATCH_FWD | D.BATCH_BWD, image, T, nl, dL, dp, reps=3)
            picks.setdefault(ratio, []).append((tuple(best), ms))
        print(which, picks)
        ex_tiles = {t[0] for t, _ in picks[0.0]}
        pr_tiles = {t[0] for t, _ in picks[2.0]}
        best_ex = min(ms for _, ms in picks[0.0])
        best_pr = min(ms for _, ms in picks[2.0])
        assert pr_tiles & ex_tiles, picks
        assert best_pr <= 1.05 * best_ex, picks
        with pytest.raises(D.DbmpError):
            D.dbmp_autotune_set_prune(ws, -1.0)
    finally:
        D.dbmp_workspace_destroy(ws)
        D.dbmp_atlas_destroy(atlas)


@pytest.mark.parametrize("tuning", [(16, 32, 4), (8, 64, 1), (32, 32, 2)], ids=lambda t: f"t{t[0]}b{t[1]}p{t[2]}")
def test_poisoned_workspace_changes_nothing(tuning):
    """Every scratch buffer of the workspace filled with NaN / -1 before planning:
    binning, forward and backward must read nothing they did not write, so the images
    are bit-identical to a clean workspace's and the gradients equal up to the order of
    their float atomics."""
    scenes, atlas = small_batch(seed=37)
    params, bid, off, pix = concat(scenes)
    rng = np.random.default_rng(5)
    gI = rng.normal(size=3 * int(pix[-1])).astype(np.float32)
    img0, T0, g0, _ = run_batch(scenes, atlas, tuning, gI=gI)
    img1, T1, g1, st = run_batch(scenes, atlas, tuning, gI=gI, poison=True)
    assert st.code == 0
    assert np.array_equal(img0, img1) and np.array_equal(T0, T1)
    assert np.all(np.isfinite(g1))
    grad_close(g1, g0, rel=1e-5, what="poisoned")


def test_poisoned_single_canvas_workspace_matches_oracle():
    cuda()
    sc = inputs.tiny(seed=8, N=70, H=61, W=83)
    atlas = D.dbmp_atlas_create(to_dev(sc.atlas))
    ws = D.dbmp_workspace_create(sc.N, 16 * 16, 1 << 20, 1)
    D.dbmp_workspace_poison(ws)
    try:
        bg = D.make_background(sc.background)
        params, bid = to_dev(sc.params), to_dev(sc.bitmap_id)   # the backward reads params again
        D.dbmp_bin(ws, sc.H, sc.W, 16, params, bid, sc.N, atlas, 1.0)
        image = torch.empty(3, sc.H, sc.W, device="cuda")
        T = torch.empty(sc.H, sc.W, device="cuda")
        nl = torch.empty(sc.H, sc.W, dtype=torch.int32, device="cuda")
        D.dbmp_render_fwd(ws, atlas, bg, 0.0, image, T, nl)
        gI = np.random.default_rng(6).normal(size=(3, sc.H, sc.W)).astype(np.float32)
        dp = torch.zeros(sc.N, 8, device="cuda")
        D.dbmp_render_bwd(ws, atlas, bg, 0.0, to_dev(gI), None, T, nl, dp)
        st = D.dbmp_status_poll(ws)
        assert st.code == 0
        ref = oracle.render(sc.H, sc.W, sc.params, sc.bitmap_id, sc.atlas, background=sc.background)
        assert np.abs(image.cpu().numpy() - ref["image"]).max() <= IMG_TOL
        gref = oracle.grad(sc.H, sc.W, sc.params, sc.bitmap_id, sc.atlas, gI, background=sc.background)
        grad_close(dp.cpu().numpy().astype(np.float64), gref, what="poisoned single")
    finally:
        D.dbmp_workspace_destroy(ws)
        D.dbmp_atlas_destroy(atlas)


def test_gpu_optimisation_resumes_from_a_checkpoint(tmp_path):
    """Six optimisation steps in one go against three, a checkpoint (parameters, Adam
    moments, step counter) written and read back into fresh device buffers, and three
    more.  The file is exact; the gradients' float atomics sum in any order, so the
    resumed run agrees with the uninterrupted one as closely as two uninterrupted runs
    agree with each other, not bit for bit."""
    from paper_2602_22625_gb300 import checkpoint
    cuda()
    sc = inputs.tiny(seed=9, N=60, H=64, W=64)
    tg = inputs.tiny(seed=10, N=60, H=64, W=64)
    atlas = D.dbmp_atlas_create(to_dev(sc.atlas))
    ws = D.dbmp_workspace_create(sc.N, 64, 1 << 20, 1)
    try:
        D.dbmp_batch_plan(ws, [sc.H], [sc.W], [0, sc.N], tile=16, batch=32, ppt=2)
        bg = D.make_background(sc.background)
        bid = to_dev(sc.bitmap_id)
        image = torch.empty(3, sc.H, sc.W, device="cuda")
        T = torch.empty(sc.H, sc.W, device="cuda")
        nl = torch.empty(sc.H, sc.W, dtype=torch.int32, device="cuda")
        target = torch.empty(3, sc.H, sc.W, device="cuda")
        D.dbmp_batch_render(ws, to_dev(tg.params), to_dev(tg.bitmap_id), atlas, 1.0, bg, 0.0,
                            D.BATCH_BIN | D.BATCH_FWD, target, T, nl)
        dL = torch.empty(3, sc.H, sc.W, device="cuda")
        loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        dp = torch.zeros(sc.N, 8, device="cuda")
        cfg = D.adam_config(lr=0.05, gamma=0.99, zero_grad=True)

        def steps(p, m, v, step, n):
            for _ in range(n):
                D.dbmp_batch_render(ws, p, bid, atlas, 1.0, bg, 0.0, D.BATCH_BIN | D.BATCH_FWD, image, T, nl)
                D.dbmp_mse_grad(image, target, dL, loss)
                D.dbmp_batch_render(ws, p, bid, atlas, 1.0, bg, 0.0, D.BATCH_BWD, image, T, nl, dL, dp)
                D.dbmp_adam_step(p, dp, m, v, step, cfg)

        def fresh():
            return (to_dev(sc.params), torch.zeros(sc.N, 8, device="cuda"), torch.zeros(sc.N, 8, device="cuda"),
                    torch.zeros(1, dtype=torch.int32, device="cuda"))

        p, m, v, step = fresh()
        steps(p, m, v, step, 6)
        ref = p.cpu().numpy()
        p, m, v, step = fresh()
        steps(p, m, v, step, 6)
        noise = np.abs(p.cpu().numpy() - ref).max()   # two uninterrupted runs (atomics' order)
        p, m, v, step = fresh()
        steps(p, m, v, step, 3)
        ck = tmp_path / "gpu.ckpt"
        checkpoint.save(ck, {"params": p, "m": m, "v": v, "step": step}, step=int(step.item()))
        a, s, _ = checkpoint.load(ck)
        assert s == 3 and np.array_equal(a["params"], p.cpu().numpy())
        p2, m2, v2, step2 = (to_dev(a["params"]), to_dev(a["m"]), to_dev(a["v"]), to_dev(a["step"]))
        steps(p2, m2, v2, step2, 3)
        assert int(step2.item()) == 6
        got = p2.cpu().numpy()
        # Adam divides by sqrt(v), so on parameters with near-zero gradients the
        # atomics' rounding can move a step by a visible amount; a broken resume
        # (moments, step or parameters not restored) moves every parameter by about
        # the learning rate instead
        d = np.abs(got - ref)
        assert d.max() <= max(20 * noise, 1e-3 * np.abs(ref).max()), (d.max(), noise)
        assert d.mean() <= 1e-3, d.mean()
    finally:
        D.dbmp_workspace_destroy(ws)
        D.dbmp_atlas_destroy(atlas)


@pytest.mark.parametrize("tuning", [(16, 32, 4), (32, 32, 4), (8, 32, 1)], ids=lambda t: f"t{t[0]}b{t[1]}p{t[2]}")
def test_fused_mse_matches_the_separate_passes(tuning):
    """dbmp_batch_render_mse (the loss in the forward's epilogue) against the forward,
    dbmp_mse_grad and the backward run one after another on a ragged multi-canvas
    batch: images and dL/dI bit for bit, the loss to FP64 rounding (summation order),
    the gradients to float32 atomics' rounding; and the loss against the oracle's."""
    cuda()
    scenes, atlas_np = small_batch(seed=41)
    params, bid, off, pix = concat(scenes)
    N, P = int(off[-1]), int(pix[-1])
    target = to_dev(np.random.default_rng(8).uniform(0, 1, 3 * P).astype(np.float32))
    atlas = D.dbmp_atlas_create(to_dev(atlas_np))
    n_tiles = sum(-(-s.W // 8) * -(-s.H // 8) for s in scenes)
    ws = D.dbmp_workspace_create(max(N, 1), n_tiles, 1 << 24, len(scenes))
    try:
        D.dbmp_batch_plan(ws, [s.H for s in scenes], [s.W for s in scenes], off.tolist(), *tuning)
        p, b = to_dev(params), to_dev(bid)
        bg = D.make_background((1.0, 1.0, 1.0))
        out = []
        for fused in (False, True):
            image = torch.empty(3 * P, device="cuda")
            T = torch.empty(P, device="cuda")
            nl = torch.empty(P, dtype=torch.int32, device="cuda")
            dL = torch.empty(3 * P, device="cuda")
            loss = torch.full((1,), 7.0, dtype=torch.float64, device="cuda")
            dp = torch.zeros(max(N, 1), 8, device="cuda")
            mode = D.BATCH_BIN | D.BATCH_FWD | D.BATCH_BWD
            if fused:
                D.dbmp_batch_render_mse(ws, p, b, atlas, 1.0, bg, 0.0, mode, target, image, T, nl, dL, loss, dp)
            else:
                D.dbmp_batch_render(ws, p, b, atlas, 1.0, bg, 0.0, D.BATCH_BIN | D.BATCH_FWD, image, T, nl)
                D.dbmp_mse_grad(image, target, dL, loss)
                D.dbmp_batch_render(ws, p, b, atlas, 1.0, bg, 0.0, D.BATCH_BWD, image, T, nl, dL, dp)
            assert D.dbmp_status_poll(ws).code == 0
            torch.cuda.synchronize()
            out.append([x.cpu().numpy() for x in (image, T, nl, dL, loss, dp)])
        (i0, t0, n0, d0, l0, g0), (i1, t1, n1, d1, l1, g1) = out
        assert np.array_equal(i0, i1) and np.array_equal(t0, t1) and np.array_equal(n0, n1)
        assert np.array_equal(d0, d1)
        assert abs(l1[0] - l0[0]) <= 1e-12 * abs(l0[0])
        grad_close(g1[:N].astype(np.float64), g0[:N].astype(np.float64), rel=1e-5, what="fused mse")
        ref = oracle.mse(i0, target.cpu().numpy())
        assert abs(l1[0] - ref) <= 1e-9 * ref
    finally:
        D.dbmp_workspace_destroy(ws)
        D.dbmp_atlas_destroy(atlas)


def test_batched_64_canvases_in_the_benchmarked_configuration():
    """The 64-canvas batch the benchmark times (sides 256..1024, 1k..50k primitives per
    canvas, 1.03 M in all), planned at tile 32, batch 32, 4 px/lane, T_stop 1e-6, in one
    binning, one forward and one backward launch.  Four canvases (the cheapest two, the
    median and the largest) against the oracle: every pixel and T, and the gradients of
    primitives sampled from each canvas' front quarter and from its back half under a
    random upstream gradient (together, and the back half on its own scale wherever its
    reference is not negligible)."""
    cuda()
    scenes = inputs.batched(seed=4)
    atlas_np = scenes[0].atlas
    params, bid, off, pix = concat(scenes)
    N, P = int(off[-1]), int(pix[-1])
    rng = np.random.default_rng(64)
    gI = rng.normal(size=3 * P).astype(np.float32) * 1e-3
    atlas = D.dbmp_atlas_create(to_dev(atlas_np))
    n_tiles = sum((s.W // 8) * (s.H // 8) for s in scenes)
    ws = D.dbmp_workspace_create(N, n_tiles, 400 << 20, len(scenes))
    try:
        D.dbmp_batch_plan(ws, [s.H for s in scenes], [s.W for s in scenes], off.tolist(), tile=32, batch=32,
                          ppt=4, ppt_bwd=4)
        p, b = to_dev(params), to_dev(bid)
        image = torch.empty(3 * P, device="cuda")
        T = torch.empty(P, device="cuda")
        nl = torch.empty(P, dtype=torch.int32, device="cuda")
        dp = torch.zeros(N, 8, device="cuda")
        D.dbmp_batch_render(ws, p, b, atlas, 1.0, D.make_background((1.0, 1.0, 1.0)), 1e-6,
                            D.BATCH_BIN | D.BATCH_FWD | D.BATCH_BWD, image, T, nl, to_dev(gI), dp)
        assert D.dbmp_status_poll(ws).code == 0
        torch.cuda.synchronize()
        img, Tf, g = image.cpu().numpy(), T.cpu().numpy(), dp.cpu().numpy().astype(np.float64)
    finally:
        D.dbmp_workspace_destroy(ws)
        D.dbmp_atlas_destroy(atlas)
    cost = sorted(range(len(scenes)), key=lambda c: scenes[c].H * scenes[c].W * scenes[c].N)
    for c in (cost[0], cost[1], cost[len(cost) // 2], cost[-1]):
        s = scenes[c]
        ref = oracle.render(s.H, s.W, s.params, s.bitmap_id, atlas_np, background=(1.0, 1.0, 1.0), T_stop=1e-6)
        got = img[3 * pix[c]: 3 * pix[c + 1]].reshape(3, s.H, s.W)
        assert np.abs(got - ref["image"]).max() <= IMG_TOL, f"canvas {c}"
        assert np.abs(Tf[pix[c]: pix[c + 1]].reshape(s.H, s.W) - ref["T_final"]).max() <= IMG_TOL
        gIc = gI[3 * pix[c]: 3 * pix[c + 1]].reshape(3, s.H, s.W)
        front = rng.choice(max(4, s.N // 4), 4, replace=False)            # front quarter: visible layers
        back = s.N // 2 + rng.choice(s.N - s.N // 2, 4, replace=False)    # back half: deep in the lists
        sel = np.sort(np.concatenate([front, back]))
        gref = oracle.grad_selected(s.H, s.W, s.params, s.bitmap_id, atlas_np, gIc, sel,
                                    background=(1.0, 1.0, 1.0), T_stop=1e-6)
        grad_close(g[off[c] + sel], gref, what=f"canvas {c}")
        isb = sel >= s.N // 2
        gb, rb = g[off[c] + sel[isb]], gref[isb]
        scale = np.abs(gref).max(axis=0)
        for j in range(8):   # back rows on their own scale, where they carry gradient
            if np.abs(rb[:, j]).max() > 1e-3 * scale[j]:
                assert np.abs(gb[:, j] - rb[:, j]).max() <= 1e-2 * np.abs(rb[:, j]).max(), (c, j)
