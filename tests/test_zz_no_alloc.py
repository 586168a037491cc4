"""The allocation-free forward entry point (dbmp_render_fwd_static).

Some callers cannot allocate device memory: an application or plugin that owns
a fixed device-memory budget, or a real-time loop that cannot afford cudaMalloc,
which may synchronise the whole device and can run out of memory mid-run.  For
them the library offers one forward entry point whose scratch memory is a fixed
array compiled into the library.  This test calls it through the C ABI twice in
a row on different scenes and compares each result with the regular entry
points (dbmp_bin + dbmp_render_fwd).  Both run the same binning and the same
forward kernel at the same tuning, so image, T_final and n_last must agree bit
for bit.  It also drives the entry point past its tile-list capacity, with and
without a status read, and checks that the next call works again.  It lives in
its own file, named to be collected last, and passes both alone in a fresh
process and after the rest of the suite.
"""
import numpy as np
import pytest

from paper_2602_22625_gb300 import dbmp as D
from paper_2602_22625_gb300 import inputs
from _helpers import cuda, to_dev, torch

pytestmark = pytest.mark.gpu


def regular_forward(sc, bg, T_stop):
    atlas = D.dbmp_atlas_create(to_dev(sc.atlas))
    ws = D.dbmp_workspace_create(max(sc.N, 1), (-(-sc.W // 16)) * (-(-sc.H // 16)), 1 << 20, 1)
    try:
        img = torch.empty(3, sc.H, sc.W, device="cuda")
        T = torch.empty(sc.H, sc.W, device="cuda")
        nl = torch.empty(sc.H, sc.W, dtype=torch.int32, device="cuda")
        D.dbmp_bin(ws, sc.H, sc.W, 16, to_dev(sc.params), to_dev(sc.bitmap_id), sc.N, atlas, 1.0)
        D.dbmp_render_fwd(ws, atlas, bg, T_stop, img, T, nl)
        D.dbmp_status_poll(ws)
        return img.cpu().numpy(), T.cpu().numpy(), nl.cpu().numpy()
    finally:
        D.dbmp_workspace_destroy(ws)
        D.dbmp_atlas_destroy(atlas)


def test_static_forward_matches_regular_forward_on_two_calls_in_a_row():
    cuda()
    scenes = [inputs.tiny(seed=41, N=300, H=200, W=176), inputs.tiny(seed=42, N=90, H=77, W=130)]
    bgs = [D.make_background((1.0, 1.0, 1.0)), D.make_background((0.2, 0.5, 0.8))]
    for sc, bg, T_stop in zip(scenes, bgs, (0.0, 1e-6)):
        img = torch.full((3, sc.H, sc.W), -5.0, device="cuda")
        T = torch.full((sc.H, sc.W), -5.0, device="cuda")
        nl = torch.full((sc.H, sc.W), -5, dtype=torch.int32, device="cuda")
        st = D.dbmp_render_fwd_static(sc.H, sc.W, to_dev(sc.params), to_dev(sc.bitmap_id),
                                      to_dev(sc.atlas), 1.0, bg, T_stop, img, T, nl)
        assert st.code == 0 and st.pairs_required > 0
        ref_img, ref_T, ref_nl = regular_forward(sc, bg, T_stop)
        assert np.array_equal(img.cpu().numpy(), ref_img)
        assert np.array_equal(T.cpu().numpy(), ref_T)
        assert np.array_equal(nl.cpu().numpy(), ref_nl)


def test_static_forward_rejects_sizes_beyond_its_maximum():
    cuda()
    sc = inputs.tiny(seed=43, N=10, H=64, W=64)
    img = torch.empty(3, 600, 600, device="cuda")
    T = torch.empty(600, 600, device="cuda")
    nl = torch.empty(600, 600, dtype=torch.int32, device="cuda")
    with pytest.raises(D.DbmpError) as e:
        D.dbmp_render_fwd_static(600, 600, to_dev(sc.params), to_dev(sc.bitmap_id), to_dev(sc.atlas), 1.0,
                                 D.make_background((1, 1, 1)), 0.0, img, T, nl)
    assert e.value.code == D.DBMP_ERR_INVALID_ARG and "512" in str(e.value)


def test_static_forward_alternating_atlas_shapes():
    """The entry point keeps one texture object per atlas shape over its scratch texel
    plane: shapes A, B, A in a row (the third call reuses A's object, with the plane
    rewritten by B in between) all match the regular entry points."""
    cuda()
    a = inputs.tiny(seed=44, N=120, H=96, W=112)                  # 1 x 64 x 64 soft disc
    b = inputs.tiny(seed=45, N=80, H=90, W=90)
    b.atlas = np.random.default_rng(9).uniform(0.05, 1.0, (3, 16, 24)).astype(np.float32)
    b.bitmap_id = (np.arange(b.N) % 3).astype(np.int32)
    bg = D.make_background((1.0, 1.0, 1.0))
    for sc in (a, b, a):
        img = torch.full((3, sc.H, sc.W), -5.0, device="cuda")
        T = torch.full((sc.H, sc.W), -5.0, device="cuda")
        nl = torch.full((sc.H, sc.W), -5, dtype=torch.int32, device="cuda")
        st = D.dbmp_render_fwd_static(sc.H, sc.W, to_dev(sc.params), to_dev(sc.bitmap_id),
                                      to_dev(sc.atlas), 1.0, bg, 0.0, img, T, nl)
        assert st.code == 0 and st.pairs_required > 0
        ref_img, ref_T, ref_nl = regular_forward(sc, bg, 0.0)
        assert np.array_equal(img.cpu().numpy(), ref_img)
        assert np.array_equal(T.cpu().numpy(), ref_T)
        assert np.array_equal(nl.cpu().numpy(), ref_nl)


def test_static_forward_capacity_overflow_then_recovers():
    """2048 primitives that each cover the whole 512^2 canvas need 2048 x 1024 tile-list
    entries, twice the scratch area's 1 048 576.  With a status read the call returns
    DBMP_ERR_CAPACITY; without one it returns at once and leaves the outputs as they
    were; the next call of a scene that fits matches the regular entry points."""
    cuda()
    big = inputs.tiny(seed=46, N=2048, H=512, W=512)
    big.params[:, 0] = 256.0
    big.params[:, 1] = 256.0
    big.params[:, 2] = 400.0
    bg = D.make_background((1.0, 1.0, 1.0))
    img = torch.full((3, 512, 512), -5.0, device="cuda")
    T = torch.full((512, 512), -5.0, device="cuda")
    nl = torch.full((512, 512), -5, dtype=torch.int32, device="cuda")
    p, b, a = to_dev(big.params), to_dev(big.bitmap_id), to_dev(big.atlas)
    with pytest.raises(D.DbmpError) as e:
        D.dbmp_render_fwd_static(512, 512, p, b, a, 1.0, bg, 0.0, img, T, nl)
    assert e.value.code == D.DBMP_ERR_CAPACITY and "2097152" in str(e.value)
    st = D.dbmp_render_fwd_static(512, 512, p, b, a, 1.0, bg, 0.0, img, T, nl, with_status=False)
    assert st is None
    torch.cuda.synchronize()
    assert bool((img == -5.0).all()) and bool((T == -5.0).all()) and bool((nl == -5).all())
    sc = inputs.tiny(seed=47, N=200, H=160, W=144)
    img = torch.full((3, sc.H, sc.W), -5.0, device="cuda")
    T = torch.full((sc.H, sc.W), -5.0, device="cuda")
    nl = torch.full((sc.H, sc.W), -5, dtype=torch.int32, device="cuda")
    st = D.dbmp_render_fwd_static(sc.H, sc.W, to_dev(sc.params), to_dev(sc.bitmap_id), to_dev(sc.atlas), 1.0,
                                  bg, 0.0, img, T, nl)
    assert st.code == 0 and 0 < st.pairs_required <= 1 << 20
    ref_img, ref_T, ref_nl = regular_forward(sc, bg, 0.0)
    assert np.array_equal(img.cpu().numpy(), ref_img)
    assert np.array_equal(T.cpu().numpy(), ref_T)
    assert np.array_equal(nl.cpu().numpy(), ref_nl)
