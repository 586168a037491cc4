"""One canvas shared by ranks holding the same parameters (sharded.py), on one GPU:
each band of tile rows is rendered and differentiated through dbmp_batch_set_rows in
turn, as its rank would.  Every pixel of a band equals the whole canvas' render bit for
bit, and the bands' losses and parameter gradients (Eq. 6, summed over the band's
pixels) add up to the whole canvas' (the float atomics sum in another order)."""
import numpy as np
import pytest

from paper_2602_22625_gb300 import dbmp as D
from paper_2602_22625_gb300 import inputs, sharded
from _helpers import cuda, grad_close, to_dev, torch

pytestmark = pytest.mark.gpu


def step(ws, p, b, atlas, bg, target, image, T, nl, dL):
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    dp = torch.zeros(p.shape[0], 8, device="cuda")
    D.dbmp_batch_render_mse(ws, p, b, atlas, 1.0, bg, 1e-6, D.BATCH_BIN | D.BATCH_FWD | D.BATCH_BWD, target,
                            image, T, nl, dL, loss, dp)
    assert D.dbmp_status_poll(ws).code == 0
    return float(loss.item()), dp.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("tile", [16, 32])
def test_bands_sum_to_the_whole_canvas(tile):
    cuda()
    sc = inputs.main(seed=8, N=3000, H=288, W=256)
    tg = inputs.main(seed=9, N=3000, H=288, W=256)
    atlas = D.dbmp_atlas_create(to_dev(sc.atlas))
    ws = D.dbmp_workspace_create(sc.N, (sc.W // 8) * (sc.H // 8), 16 << 20, 1)
    bg = D.make_background(sc.background)
    shape = (3, sc.H, sc.W)
    try:
        D.dbmp_batch_plan(ws, [sc.H], [sc.W], [0, sc.N], tile=tile, batch=32, ppt=4, ppt_bwd=4)
        target = torch.empty(shape, device="cuda")
        T = torch.empty(sc.H, sc.W, device="cuda")
        nl = torch.empty(sc.H, sc.W, dtype=torch.int32, device="cuda")
        D.dbmp_batch_render(ws, to_dev(tg.params), to_dev(tg.bitmap_id), atlas, 1.0, bg, 0.0,
                            D.BATCH_BIN | D.BATCH_FWD, target, T, nl)
        p, b = to_dev(sc.params), to_dev(sc.bitmap_id)
        image, dL = torch.empty(shape, device="cuda"), torch.empty(shape, device="cuda")
        loss_full, g_full = step(ws, p, b, atlas, bg, target, image, T, nl, dL)
        ref = (image.cpu().numpy(), T.cpu().numpy(), nl.cpu().numpy())
        for world in (2, 3, 5):
            image.fill_(-7.0)
            T.fill_(-7.0)
            nl.fill_(-7)
            loss, g = 0.0, np.zeros_like(g_full)
            rows = []
            for r in range(world):
                rows.append(sharded.select_band(ws, sc.H, world, r, tile))
                l_r, g_r = step(ws, p, b, atlas, bg, target, image, T, nl, dL)
                assert 0.0 < l_r < loss_full
                loss += l_r
                g += g_r
            D.dbmp_batch_set_rows(ws, 0, 0)
            assert rows[0][0] == 0 and rows[-1][1] >= sc.H
            got = (image.cpu().numpy(), T.cpu().numpy(), nl.cpu().numpy())
            for a, e in zip(got, ref):   # every band wrote exactly its own rows
                assert np.array_equal(a, e), world
            assert abs(loss - loss_full) <= 1e-12 * loss_full
            grad_close(g, g_full, rel=1e-5, what=f"{world} bands")
        with pytest.raises(D.DbmpError):
            D.dbmp_batch_set_rows(ws, 8 if tile > 8 else 4, 64)   # not on the tile grid
    finally:
        D.dbmp_workspace_destroy(ws)
        D.dbmp_atlas_destroy(atlas)
