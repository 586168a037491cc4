"""CUDA path vs the FP64 oracle: binning (bit-exact), forward (max-abs 1e-5) and
backward (relative 1e-3 per parameter group), through the C ABI."""
import numpy as np
import pytest

import oracle
from paper_2602_22625_gb300 import dbmp as D
from paper_2602_22625_gb300 import inputs
from paper_2602_22625_gb300.render import Atlas, Renderer
from _helpers import cuda, grad_close, lists_from_rects, to_dev, torch

pytestmark = pytest.mark.gpu

IMG_TOL = 1e-5


def gpu_bin(sc, tile):
    dev = cuda()
    atlas = Atlas(to_dev(sc.atlas))
    r = Renderer(sc.H, sc.W, atlas, max(sc.N, 1), tile=tile, background=sc.background, check=True)
    p = to_dev(sc.params)
    b = to_dev(sc.bitmap_id)
    r.bin(p, b)
    st = r.status()
    K = st.pairs_required
    n_tiles = (-(-sc.W // tile)) * (-(-sc.H // tile))
    offs = torch.empty(n_tiles + 1, dtype=torch.int64, device=dev)
    lst = torch.empty(max(K, 1), dtype=torch.int32, device=dev)
    D.dbmp_get_tile_lists(r.ws.handle, offs, lst)
    torch.cuda.synchronize()
    return offs.cpu().numpy(), lst.cpu().numpy()[:K]


def scene_ragged(seed=21, N=60, H=77, W=45):
    sc = inputs.tiny(seed=seed, N=N, H=H, W=W)
    sc.params[:, 2] = np.abs(sc.params[:, 2]) * 0.25
    return sc


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_bin_bit_exact_tiny(tile):
    sc = inputs.tiny(seed=1)
    offs, lst = gpu_bin(sc, tile)
    ro, rl = oracle.bin(sc.H, sc.W, tile, sc.params, sc.bitmap_id, sc.atlas)
    np.testing.assert_array_equal(offs, ro)
    np.testing.assert_array_equal(lst, rl)


def test_bin_bit_exact_ragged_invalid_and_negative_scale():
    sc = scene_ragged()
    p = sc.params
    p[3, 2] = 0.0
    p[5, 0] = np.nan
    p[7, 2] *= -1.0
    p[9, 3] = 1e6  # beyond the reduction range: conservative box
    for tile in (8, 16, 32):
        offs, lst = gpu_bin(sc, tile)
        ro, rl = oracle.bin(sc.H, sc.W, tile, p, sc.bitmap_id, sc.atlas)
        np.testing.assert_array_equal(offs, ro)
        np.testing.assert_array_equal(lst, rl)


@pytest.mark.parametrize("tile", [16, 32])
def test_bin_bit_exact_main_workload(tile):
    sc = inputs.main()
    offs, lst = gpu_bin(sc, tile)
    ro, rl = oracle.bin(sc.H, sc.W, tile, sc.params, sc.bitmap_id, sc.atlas)
    np.testing.assert_array_equal(offs, ro)
    np.testing.assert_array_equal(lst, rl)


def test_bin_bit_exact_multi_pass_chunks():
    """300k primitives on a 2048 x 2048 canvas at tile 8 (65,536 tiles): the
    histogram needs chunks of 2048 primitives, so each binning CTA takes its chunk
    in two passes, and rows of 256 tiles give one-row slabs."""
    atlas = inputs.stroke_atlas(seed=32, n=8, size=64)
    p, b = inputs.primitives(31, 300_000, 2048, 2048, atlas.shape[0], "uniform", (0.001, 0.004))
    sc = inputs.Scene("small_2048sq_300k", 2048, 2048, p, b, atlas)
    offs, lst = gpu_bin(sc, 8)
    # the oracle's definition tests every primitive against every tile (2e10 tests
    # here); the expected lists come from its rectangles expanded and stably sorted
    rects, _ = oracle.bin_rects(sc.H, sc.W, 8, sc.params, sc.bitmap_id, sc.atlas)
    ro, rl = lists_from_rects(rects, 256, 256)
    np.testing.assert_array_equal(offs, ro)
    np.testing.assert_array_equal(lst, rl)


def test_bin_empty():
    sc = inputs.tiny(seed=2, N=0, H=40, W=50)
    offs, lst = gpu_bin(sc, 16)
    assert len(lst) == 0 and np.all(offs == 0)


# ---------------------------------------------------------------------------
# forward
# ---------------------------------------------------------------------------

def gpu_forward(sc, tile=16, T_stop=0.0, background="scene", alpha_max=1.0):
    atlas = Atlas(to_dev(sc.atlas))
    bg = sc.background if isinstance(background, str) else background
    if isinstance(bg, np.ndarray) and bg.size > 3:
        bg = to_dev(bg.astype(np.float32))
    r = Renderer(sc.H, sc.W, atlas, max(sc.N, 1), tile=tile, background=bg, T_stop=T_stop,
                 alpha_max=alpha_max, check=True)
    p, b = to_dev(sc.params), to_dev(sc.bitmap_id)
    img, T, nl = r.forward(p, b)
    st = r.status()
    torch.cuda.synchronize()
    return r, p, b, img, T, nl, st


@pytest.mark.parametrize("tile", [8, 16, 32])
@pytest.mark.parametrize("T_stop", [0.0, 1e-6])
def test_forward_tiny_matches_oracle(tile, T_stop):
    sc = inputs.tiny(seed=1)
    _, _, _, img, T, nl, st = gpu_forward(sc, tile, T_stop)
    ref = oracle.render(sc.H, sc.W, sc.params, sc.bitmap_id, sc.atlas, background=sc.background,
                        T_stop=T_stop)
    assert np.abs(img.cpu().numpy() - ref["image"]).max() <= IMG_TOL
    assert np.abs(T.cpu().numpy() - ref["T_final"]).max() <= IMG_TOL
    exact = oracle.render(sc.H, sc.W, sc.params, sc.bitmap_id, sc.atlas, background=sc.background)
    assert np.abs(img.cpu().numpy() - exact["image"]).max() <= IMG_TOL
    assert st.pairs_evaluated > 0


@pytest.mark.parametrize("bg", ["none", "const", "buffer"])
@pytest.mark.parametrize("alpha_max", [1.0, 0.7])
def test_forward_ragged_backgrounds(bg, alpha_max):
    sc = scene_ragged()
    background = {"none": None, "const": (0.2, 0.7, 0.4),
                  "buffer": np.random.default_rng(3).uniform(0, 1, (3, sc.H, sc.W)).astype(np.float32)}[bg]
    _, _, _, img, T, nl, _ = gpu_forward(sc, 16, 0.0, background=background, alpha_max=alpha_max)
    ref = oracle.render(sc.H, sc.W, sc.params, sc.bitmap_id, sc.atlas, alpha_max=alpha_max,
                        background=background)
    assert np.abs(img.cpu().numpy() - ref["image"]).max() <= IMG_TOL
    assert np.abs(T.cpu().numpy() - ref["T_final"]).max() <= IMG_TOL
    # n_last names the oracle's last contributing primitive
    offs, lst = oracle.bin(sc.H, sc.W, 16, sc.params, sc.bitmap_id, sc.atlas)
    nl = nl.cpu().numpy()
    ntx = -(-sc.W // 16)
    yy, xx = np.mgrid[0:sc.H, 0:sc.W]
    tid = (yy // 16) * ntx + xx // 16
    prim = np.where(nl >= 0, lst[np.minimum(offs[tid] + np.maximum(nl, 0), len(lst) - 1)], -1)
    assert np.mean(prim == ref["n_last"]) > 0.999


def test_forward_empty_scene_is_background():
    sc = inputs.tiny(seed=5, N=0, H=33, W=70)
    _, _, _, img, T, nl, _ = gpu_forward(sc, 16, 0.0, background=(0.1, 0.2, 0.3))
    img = img.cpu().numpy()
    for j, v in enumerate((0.1, 0.2, 0.3)):
        assert np.all(img[j] == np.float32(v))
    assert np.all(T.cpu().numpy() == 1.0) and np.all(nl.cpu().numpy() == -1)


def test_forward_main_workload_sampled_pixels():
    sc = inputs.main()
    _, _, _, img, T, _, st = gpu_forward(sc, 16, 1e-6)
    rng = np.random.default_rng(0)
    px = rng.integers(0, sc.W, 3000)
    py = rng.integers(0, sc.H, 3000)
    ref = oracle.render(sc.H, sc.W, sc.params, sc.bitmap_id, sc.atlas, background=sc.background,
                        pixels=(px, py))  # exact composite, no early termination
    got = img.cpu().numpy()[:, py, px]
    assert np.abs(got - ref["image"]).max() <= IMG_TOL
    assert np.abs(T.cpu().numpy()[py, px] - ref["T_final"]).max() <= IMG_TOL
    assert st.pairs_required > 0


# ---------------------------------------------------------------------------
# backward
# ---------------------------------------------------------------------------

def gpu_grad(sc, gI, gA=None, tile=16, T_stop=0.0, background="scene", alpha_max=1.0):
    r, p, b, img, T, nl, _ = gpu_forward(sc, tile, T_stop, background=background, alpha_max=alpha_max)
    g = r.backward(to_dev(gI.astype(np.float32)), T, nl,
                   None if gA is None else to_dev(gA.astype(np.float32)))
    torch.cuda.synchronize()
    return g.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_backward_tiny_matches_oracle(tile):
    sc = inputs.tiny(seed=1)
    rng = np.random.default_rng(11)
    gI = rng.normal(size=(3, sc.H, sc.W)).astype(np.float32)
    g = gpu_grad(sc, gI, tile=tile)
    ref = oracle.grad(sc.H, sc.W, sc.params, sc.bitmap_id, sc.atlas, gI, background=sc.background)
    grad_close(g, ref, what=f"tile{tile}")


@pytest.mark.parametrize("bg", ["none", "const", "buffer"])
def test_backward_ragged_with_alpha_gradient(bg):
    sc = scene_ragged(seed=23, N=80)
    rng = np.random.default_rng(12)
    gI = rng.normal(size=(3, sc.H, sc.W)).astype(np.float32)
    gA = rng.normal(size=(sc.H, sc.W)).astype(np.float32)
    background = {"none": None, "const": (0.9, 0.1, 0.5),
                  "buffer": rng.uniform(0, 1, (3, sc.H, sc.W)).astype(np.float32)}[bg]
    g = gpu_grad(sc, gI, gA, background=background, alpha_max=0.8)
    ref = oracle.grad(sc.H, sc.W, sc.params, sc.bitmap_id, sc.atlas, gI, gA, alpha_max=0.8,
                      background=background)
    grad_close(g, ref, what=bg)


def test_backward_takes_its_state_from_the_given_maps_not_the_last_forward():
    """The backward depends only on the binning and the T_final / n_last it is
    given: after an exact forward (T_stop = 0) another forward of the same binning
    terminates early (T_stop = 0.3, far fewer list entries walked); the backward
    with the exact forward's maps still gives the exact gradient."""
    sc = inputs.tiny(seed=5, N=1500, H=96, W=80)
    r, p, b, img, T, nl, st0 = gpu_forward(sc, tile=16, T_stop=0.0)
    img2, T2, nl2 = torch.empty_like(img), torch.empty_like(T), torch.empty_like(nl)
    D.dbmp_render_fwd(r.ws.handle, r.atlas.handle, r.bg, 0.3, img2, T2, nl2)
    st1 = r.status()
    torch.cuda.synchronize()
    assert int(nl.max()) >= 64 and st1.warp_steps < 0.5 * st0.warp_steps   # fewer batches visited
    rng = np.random.default_rng(13)
    gI = rng.normal(size=(3, sc.H, sc.W)).astype(np.float32)
    g = r.backward(to_dev(gI), T, nl)
    torch.cuda.synchronize()
    ref = oracle.grad(sc.H, sc.W, sc.params, sc.bitmap_id, sc.atlas, gI, background=sc.background)
    grad_close(g.cpu().numpy().astype(np.float64), ref, what="maps of the exact forward")


def test_backward_opaque_layer_uses_rewalk():
    """A layer with alpha = 1 exactly (alpha_max = 1, sigmoid(nu) = 1 in float32, M = 1)
    leaves T = 0 behind it; the backward then recovers T in front of it by a re-walk."""
    atlas = np.zeros((1, 16, 16), np.float32)
    atlas[0, 2:14, 2:14] = 1.0
    p = np.array([[20.0, 20.0, 6.0, 0.3, 0.5, 0.2, -0.3, 0.8],
                  [24.0, 18.0, 12.0, 0.1, 60.0, 1.0, 0.5, -1.0],   # opaque
                  [22.0, 22.0, 9.0, 0.7, 1.0, -0.4, 0.9, 0.1]], np.float32)
    sc = inputs.Scene("opaque", 40, 40, p, np.zeros(3, np.int32), atlas)
    rng = np.random.default_rng(4)
    gI = rng.normal(size=(3, 40, 40)).astype(np.float32)
    g = gpu_grad(sc, gI)
    ref = oracle.grad(40, 40, p, sc.bitmap_id, atlas, gI, background=sc.background)
    grad_close(g, ref, what="opaque")


def test_backward_main_workload_sampled_primitives():
    sc = inputs.main()
    rng = np.random.default_rng(13)
    gI = rng.normal(size=(3, sc.H, sc.W)).astype(np.float32) * 1e-3
    g = gpu_grad(sc, gI, T_stop=1e-6)
    small = np.nonzero(np.abs(sc.params[:200, 2]) < 40)[0][:6]
    sel = np.concatenate([small, [0, 1]])
    ref = oracle.grad_selected(sc.H, sc.W, sc.params, sc.bitmap_id, sc.atlas, gI, sel,
                               background=sc.background, T_stop=1e-6)
    grad_close(g[sel], ref, what="main")



def scene_lattice(shift=0.0):
    """Primitives placed so that every pixel's bitmap coordinates (U, V) are exact
    integers or half-integers (theta = 0, |A| = |D| in {1/2, 1, 2}, centres on the
    matching lattice), moved by `shift` px in x and y: samples sit on texel boundaries
    (shift 0) or |A| shift to one side of them, on the bitmap's first and last lattice
    cells (U or V = -1 and W_b - 1) and just outside.  The atlas has no zero texels, so
    a bitmap read past its last row would pick up the next bitmap's first row."""
    Hb = Wb = 16                     # kw = kv = 7.5
    atlas = np.random.default_rng(5).uniform(0.05, 1.0, (3, Hb, Wb)).astype(np.float32)
    rows = [  # x, y, s, bitmap: U = (7.5 / s)(px - x) + 7.5
        (50.5, 40.5, 7.5, 0), (60.0, 45.0, 15.0, 1), (55.5, 50.5, -7.5, 2), (52.25, 47.75, 3.75, 0),
        (44.5, 58.5, 7.5, 1), (70.0, 30.0, 15.0, 2), (38.5, 35.5, -7.5, 0), (64.25, 60.25, 3.75, 1),
    ]
    rng = np.random.default_rng(6)
    p = np.zeros((len(rows), 8), np.float32)
    for i, (x, y, s, _) in enumerate(rows):
        p[i, :4] = (x + shift, y + shift, s, 0.0)
        p[i, 4] = rng.uniform(-0.5, 1.5)           # opacity logit
        p[i, 5:] = rng.normal(size=3)              # colour logits
    bid = np.array([r[3] for r in rows], np.int32)
    return inputs.Scene("lattice_96sq", 96, 96, p, bid, atlas, recipe="lattice-aligned samples")


@pytest.mark.parametrize("tile", [8, 16])
@pytest.mark.parametrize("shift", [0.0, 2.0 ** -12, -(2.0 ** -12)])
def test_lattice_aligned_samples_match_oracle(tile, shift):
    """The texture gather's 2 x 2 footprint and its zero border against the FP64
    bilinear sample at texel boundaries and bitmap edges.  M is continuous across a
    texel boundary, so on the lattice (shift 0) the image and the opacity and colour
    gradients are compared; the geometric gradients are one-sided there (which side
    is decided by each side's rounding of U) and are compared on the shifted lattices,
    where U = k -/+ |A| 2^-12 is exact in fp32 and far from k in FP64."""
    sc = scene_lattice(shift)
    _, _, _, img, T, nl, _ = gpu_forward(sc, tile, 0.0)
    ref = oracle.render(sc.H, sc.W, sc.params, sc.bitmap_id, sc.atlas, background=sc.background)
    assert np.abs(img.cpu().numpy() - ref["image"]).max() <= IMG_TOL
    assert np.abs(T.cpu().numpy() - ref["T_final"]).max() <= IMG_TOL
    gI = np.random.default_rng(13).normal(size=(3, sc.H, sc.W)).astype(np.float32)
    g = gpu_grad(sc, gI, tile=tile)
    grad_ref = oracle.grad(sc.H, sc.W, sc.params, sc.bitmap_id, sc.atlas, gI, background=sc.background)
    cols = slice(4, 8) if shift == 0.0 else slice(0, 8)
    gz, rz = np.zeros_like(g), np.zeros_like(grad_ref)
    gz[:, cols], rz[:, cols] = g[:, cols], grad_ref[:, cols]
    grad_close(gz, rz, what=f"lattice tile{tile} shift{shift}")


def test_atlas_beyond_the_texture_height_is_rejected():
    """The texel plane stacks n_bmp (H_b + 1) rows; past the device's pitch-linear
    texture height (65000 rows on GB300) the atlas is refused on the host."""
    cuda()
    ok = to_dev(np.zeros((503, 128, 128), np.float32))     # 503 x 129 = 64887 rows
    a = D.dbmp_atlas_create(ok)
    D.dbmp_atlas_destroy(a)
    big = to_dev(np.zeros((504, 128, 128), np.float32))    # 65016 rows
    with pytest.raises(D.DbmpError) as e:
        D.dbmp_atlas_create(big)
    assert e.value.code == D.DBMP_ERR_INVALID_ARG and "texture" in str(e.value)



def test_main_workload_in_the_benchmarked_configuration():
    """One optimisation step as the benchmark times it, at full size (1024^2 canvas,
    20k primitives, tile 32, batch 32, 4 pixels per lane forward and backward, T_stop
    1e-6): dbmp_batch_render(BIN), dbmp_batch_render_mse(FWD) with the loss in the
    forward's epilogue, dbmp_batch_render(BWD), dbmp_adam_step.  Against the FP64
    oracle: every pixel, the loss, dL/dI, the gradient of every primitive (the oracle's
    backward takes the GPU's dL/dI, itself checked) and the updated parameters."""
    cuda()
    sc = inputs.main()
    tg = inputs.main(seed=1002)
    target = to_dev(oracle.render(tg.H, tg.W, tg.params, tg.bitmap_id, tg.atlas,
                                  background=tg.background)["image"].astype(np.float32))
    atlas = D.dbmp_atlas_create(to_dev(sc.atlas))
    ws = D.dbmp_workspace_create(sc.N, (sc.W // 8) * (sc.H // 8), 96 << 20, 1)
    try:
        D.dbmp_workspace_count_pairs(ws)
        D.dbmp_batch_plan(ws, [sc.H], [sc.W], [0, sc.N], tile=32, batch=32, ppt=4, ppt_bwd=4)
        bg = D.make_background(sc.background)
        p, b = to_dev(sc.params), to_dev(sc.bitmap_id)
        image = torch.empty(3, sc.H, sc.W, device="cuda")
        T = torch.empty(sc.H, sc.W, device="cuda")
        nl = torch.empty(sc.H, sc.W, dtype=torch.int32, device="cuda")
        dL = torch.empty(3, sc.H, sc.W, device="cuda")
        loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        dp = torch.zeros(sc.N, 8, device="cuda")
        m = torch.zeros(sc.N, 8, device="cuda")
        v = torch.zeros(sc.N, 8, device="cuda")
        step = torch.zeros(1, dtype=torch.int32, device="cuda")
        cfg = D.adam_config(lr=0.1, gamma=0.1 ** (1.0 / 500), zero_grad=True)
        D.dbmp_batch_render(ws, p, b, atlas, 1.0, bg, 1e-6, D.BATCH_BIN, None, T, nl)
        D.dbmp_batch_render_mse(ws, p, b, atlas, 1.0, bg, 1e-6, D.BATCH_FWD, target, image, T, nl, dL, loss)
        D.dbmp_batch_render(ws, p, b, atlas, 1.0, bg, 1e-6, D.BATCH_BWD, image, T, nl, dL, dp)
        st = D.dbmp_status_poll(ws)
        assert st.code == 0
        grad = dp.cpu().numpy().astype(np.float64)
        D.dbmp_adam_step(p, dp, m, v, step, cfg)
        torch.cuda.synchronize()
        img, tgt = image.cpu().numpy(), target.cpu().numpy()
        ref = oracle.render(sc.H, sc.W, sc.params, sc.bitmap_id, sc.atlas, background=sc.background,
                            T_stop=1e-6)
        assert np.abs(img - ref["image"]).max() <= IMG_TOL
        assert np.abs(T.cpu().numpy() - ref["T_final"]).max() <= IMG_TOL
        # the work count behind the roofline: layers with M > 0 composited while
        # T >= T_stop; fp32 and FP64 part on M > 0 or on the threshold only for pixels
        # within rounding of the support edge or of T_stop
        assert abs(st.pairs_contributing - ref["contrib"]) <= 1e-2 * ref["contrib"]
        # the loss of the GPU's own image to summation order; against the oracle's image,
        # |mean(d1^2) - mean(d2^2)| <= max|d1 - d2| * mean|d1 + d2| bounds the difference
        L = loss.item()
        assert abs(L - oracle.mse(img, tgt)) <= 1e-6 * L
        assert abs(L - oracle.mse(ref["image"], tgt)) <= IMG_TOL * (2.0 * np.sqrt(L) + IMG_TOL)
        gI = dL.cpu().numpy()
        np.testing.assert_allclose(gI, oracle.mse_grad(img, tgt), rtol=1e-6, atol=1e-12)
        gref = oracle.grad(sc.H, sc.W, sc.params, sc.bitmap_id, sc.atlas, gI, background=sc.background,
                           T_stop=1e-6)
        grad_close(grad, gref, what="benchmarked configuration")
        # Adam at step 1 takes the GPU's gradient; zero_grad clears it for the next step
        rp, _, _ = oracle.adam_step(sc.params, grad, np.zeros((sc.N, 8)), np.zeros((sc.N, 8)), 1, 0.1)
        # positions reach 1024, where a float32 ulp is 6e-5: allow 2 ulp beside the step's error
        assert np.all(np.abs(p.cpu().numpy() - rp) <= 2e-5 + 2.4e-7 * np.abs(rp))
        assert step.item() == 1 and torch.all(dp == 0)
    finally:
        D.dbmp_workspace_destroy(ws)
        D.dbmp_atlas_destroy(atlas)


def test_backward_with_a_full_survivor_record_matches_a_roomy_workspace():
    """The workspace's survivor record holds max_pairs / 8 entries (at least 65 536),
    divided among the forward's warps.  With max_pairs equal to the main workload's
    list entries, the forward's warps run out of room (the workload keeps about a
    third of its list entries as survivors), and the regions they could not record
    are walked from their tile lists by the backward.  The gradient equals that of a
    workspace with room for every survivor, up to float32 summation order."""
    cuda()
    sc = inputs.main()
    tg = inputs.main(seed=1002)
    atlas = D.dbmp_atlas_create(to_dev(sc.atlas))
    bg = D.make_background(sc.background)
    p, b = to_dev(sc.params), to_dev(sc.bitmap_id)
    target = torch.empty(3, sc.H, sc.W, device="cuda")
    image = torch.empty(3, sc.H, sc.W, device="cuda")
    T = torch.empty(sc.H, sc.W, device="cuda")
    nl = torch.empty(sc.H, sc.W, dtype=torch.int32, device="cuda")
    dL = torch.empty(3, sc.H, sc.W, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    grads, survivors = [], []
    K = None
    try:
        for roomy in (True, False):
            ws = D.dbmp_workspace_create(sc.N, (sc.W // 8) * (sc.H // 8), (96 << 20) if roomy else K, 1)
            try:
                D.dbmp_batch_plan(ws, [sc.H], [sc.W], [0, sc.N], tile=32, batch=32, ppt=4, ppt_bwd=4)
                if roomy:
                    D.dbmp_batch_render(ws, to_dev(tg.params), to_dev(tg.bitmap_id), atlas, 1.0, bg, 0.0,
                                        D.BATCH_BIN | D.BATCH_FWD, target, T, nl)
                dp = torch.zeros(sc.N, 8, device="cuda")
                D.dbmp_batch_render(ws, p, b, atlas, 1.0, bg, 1e-6, D.BATCH_BIN, None, T, nl)
                D.dbmp_batch_render_mse(ws, p, b, atlas, 1.0, bg, 1e-6, D.BATCH_FWD, target, image, T, nl, dL,
                                        loss)
                D.dbmp_batch_render(ws, p, b, atlas, 1.0, bg, 1e-6, D.BATCH_BWD, image, T, nl, dL, dp)
                st = D.dbmp_status_poll(ws)
                assert st.code == 0
                K = st.pairs_required
                survivors.append(st.survivors)
                grads.append(dp.cpu().numpy().astype(np.float64))
            finally:
                D.dbmp_workspace_destroy(ws)
    finally:
        D.dbmp_atlas_destroy(atlas)
    assert survivors[1] > max(K // 8, 1 << 16)   # more survivors than the tight record holds
    grad_close(grads[1], grads[0], rel=1e-4, what="survivor record full")


def test_forward_with_and_without_the_pair_counter_renders_the_same_bits():
    """The contributing-pair counter is a separately compiled instance of the forward:
    with it off (the default) the status reports no count, and image, T_final and
    n_last are bit for bit those of the counting instance."""
    cuda()
    sc = inputs.main()
    atlas = D.dbmp_atlas_create(to_dev(sc.atlas))
    ws = D.dbmp_workspace_create(sc.N, (sc.W // 8) * (sc.H // 8), 32 << 20, 1)
    try:
        D.dbmp_batch_plan(ws, [sc.H], [sc.W], [0, sc.N], tile=32, batch=32, ppt=4, ppt_bwd=4)
        bg = D.make_background(sc.background)
        p, b = to_dev(sc.params), to_dev(sc.bitmap_id)
        out, counts = [], []
        for on in (False, True):
            D.dbmp_workspace_count_pairs(ws, on)
            img = torch.empty(3, sc.H, sc.W, device="cuda")
            T = torch.empty(sc.H, sc.W, device="cuda")
            nl = torch.empty(sc.H, sc.W, dtype=torch.int32, device="cuda")
            D.dbmp_batch_render(ws, p, b, atlas, 1.0, bg, 1e-6, D.BATCH_BIN | D.BATCH_FWD, img, T, nl)
            counts.append(D.dbmp_status_poll(ws).pairs_contributing)
            out.append((img.cpu().numpy(), T.cpu().numpy(), nl.cpu().numpy()))
    finally:
        D.dbmp_workspace_destroy(ws)
        D.dbmp_atlas_destroy(atlas)
    assert counts[0] == 0 and counts[1] > 0
    for a, c in zip(out[0], out[1]):
        assert np.array_equal(a, c)
