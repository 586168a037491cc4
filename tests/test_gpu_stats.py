"""Scaling statistics of a binning on the GPU (Sec. S4) against the oracle, through the
C ABI: every count and histogram bin exactly."""
import numpy as np
import pytest

import oracle
from paper_2602_22625_gb300 import dbmp as D
from paper_2602_22625_gb300 import inputs
from _helpers import cuda, to_dev, torch

pytestmark = pytest.mark.gpu


def compare(got, ref):
    for k in ("n_listed", "pairs", "tau_max", "d_max", "n_tiles", "empty_tiles"):
        assert got[k] == ref[k], k
    for k in ("tau_hist", "d_hist", "foot_hist"):
        np.testing.assert_array_equal(np.array(got[k]), np.asarray(ref[k]), err_msg=k)


@pytest.mark.parametrize("tile", [16, 32])
def test_stats_main_workload(tile):
    cuda()
    sc = inputs.main()
    atlas = D.dbmp_atlas_create(to_dev(sc.atlas))
    ws = D.dbmp_workspace_create(sc.N, (sc.W // 8) * (sc.H // 8), 64 << 20, 1)
    try:
        p, b = to_dev(sc.params), to_dev(sc.bitmap_id)
        D.dbmp_bin(ws, sc.H, sc.W, tile, p, b, sc.N, atlas, 1.0)
        got = D.dbmp_bin_stats(ws)
    finally:
        D.dbmp_workspace_destroy(ws)
        D.dbmp_atlas_destroy(atlas)
    compare(got, oracle.bin_stats(sc.H, sc.W, tile, sc.params, sc.bitmap_id, sc.atlas))


def test_stats_of_a_multi_canvas_plan_sum_the_canvases():
    cuda()
    scenes = inputs.batched(seed=4, n_canvas=6, side=(96, 320), nprim=(200, 3000))
    atlas_np = scenes[0].atlas
    params = np.concatenate([s.params for s in scenes])
    bid = np.concatenate([s.bitmap_id for s in scenes]).astype(np.int32)
    off = np.concatenate([[0], np.cumsum([s.N for s in scenes])]).tolist()
    atlas = D.dbmp_atlas_create(to_dev(atlas_np))
    n_tiles = sum(-(-s.W // 8) * -(-s.H // 8) for s in scenes)
    ws = D.dbmp_workspace_create(len(params), n_tiles, 1 << 24, len(scenes))
    try:
        D.dbmp_batch_plan(ws, [s.H for s in scenes], [s.W for s in scenes], off, 16, 32, 2)
        P = sum(s.H * s.W for s in scenes)
        T = torch.empty(P, device="cuda")
        nl = torch.empty(P, dtype=torch.int32, device="cuda")
        D.dbmp_batch_render(ws, to_dev(params), to_dev(bid), atlas, 1.0, D.make_background((1, 1, 1)), 0.0,
                            D.BATCH_BIN, None, T, nl)
        got = D.dbmp_bin_stats(ws)
    finally:
        D.dbmp_workspace_destroy(ws)
        D.dbmp_atlas_destroy(atlas)
    refs = [oracle.bin_stats(s.H, s.W, 16, s.params, s.bitmap_id, atlas_np) for s in scenes]
    ref = {k: sum(r[k] for r in refs) for k in ("n_listed", "pairs", "n_tiles", "empty_tiles",
                                                "tau_hist", "d_hist", "foot_hist")}
    ref["tau_max"] = max(r["tau_max"] for r in refs)
    ref["d_max"] = max(r["d_max"] for r in refs)
    compare(got, ref)


def test_stats_need_a_binning():
    cuda()
    ws = D.dbmp_workspace_create(10, 16, 1024, 1)
    try:
        with pytest.raises(D.DbmpError):
            D.dbmp_bin_stats(ws)
    finally:
        D.dbmp_workspace_destroy(ws)
