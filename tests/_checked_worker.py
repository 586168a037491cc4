"""Body of the index-check test, run in a subprocess with DBMP_LIBRARY=checked (the
build with device-side index checks).  Prints one JSON line of results."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def main():
    import numpy as np
    import torch
    import oracle
    from paper_2602_22625_gb300 import dbmp as D
    from paper_2602_22625_gb300 import inputs

    dev = torch.device("cuda")
    H, W, tile, N = 96, 80, 16, 90
    full = inputs.tiny(seed=13, N=N + 40, H=H, W=W)
    atlas_np = inputs.stroke_atlas(17, 3, 32, n_seg=24)          # 3 bitmaps: row 5 is inside the plane
    bid = (np.arange(N + 40) % 3).astype(np.int32)
    params = full.params.copy()
    params[:, 2] = np.abs(params[:, 2]) * 0.5
    bg = (1.0, 1.0, 1.0)
    atlas = D.dbmp_atlas_create(torch.from_numpy(atlas_np).to(dev))
    n_tiles = (-(-W // tile)) * (-(-H // tile))
    ws = D.dbmp_workspace_create(N + 64, n_tiles, 1 << 20, 1)
    out = {"checks": D.dbmp_index_checks()}
    img = torch.empty(3, H, W, device=dev)
    T = torch.empty(H, W, device=dev)
    nl = torch.empty(H, W, dtype=torch.int32, device=dev)
    bgd = D.make_background(bg)

    def bin_(n):
        D.dbmp_batch_plan(ws, [H], [W], [0, n], tile=tile, batch=32, ppt=2)
        D.dbmp_batch_render(ws, torch.from_numpy(params[:n]).to(dev), torch.from_numpy(bid[:n]).to(dev), atlas,
                            1.0, bgd, 0.0, D.BATCH_BIN, None, T, nl)

    def fwd():
        D.dbmp_batch_render(ws, None, None, atlas, 1.0, bgd, 0.0, D.BATCH_FWD, img, T, nl)
        st = D.dbmp_status_poll(ws, raise_on_error=False)
        return img.cpu().numpy().astype(np.float64), st

    def lists():
        K = D.dbmp_status_poll(ws, raise_on_error=False).pairs_required
        offs = torch.empty(n_tiles + 1, dtype=torch.int64, device=dev)
        lst = torch.empty(K, dtype=torch.int32, device=dev)
        D.dbmp_get_tile_lists(ws, offs, lst)
        return offs.cpu().numpy(), lst.cpu().numpy(), K

    def ref(drop=None, pixels=None):
        p = params[:N].copy()
        if drop is not None:
            p[drop, 4] = -100.0           # opacity 4e-44: the primitive is absent
        return oracle.render(H, W, p, bid[:N], atlas_np, background=bg)["image"]

    def err(a, b, mask=None):
        d = np.abs(a - b)
        return float(d.max() if mask is None else d[:, mask].max(initial=0.0))

    try:
        bin_(N + 40)                      # records N .. N+39 hold valid primitives afterwards
        bin_(N)
        base = ref()
        im, st = fwd()
        out["clean"] = {"bad_kind": st.bad_kind, "err": err(im, base)}
        # 1) a list entry naming a stale record past N (inside the record array)
        offs, lst, K = lists()
        t = int(np.argmax(np.diff(offs)))
        pos = int(offs[t] + (offs[t + 1] - offs[t]) // 2)
        dropped = int(lst[pos])
        D.dbmp_workspace_debug_set(ws, 1, pos, N + 5)
        im, st = fwd()
        ty, tx = divmod(t, -(-W // tile))
        in_t = np.zeros((H, W), bool)
        in_t[ty * tile:(ty + 1) * tile, tx * tile:(tx + 1) * tile] = True
        out["list_entry"] = {"bad_kind": st.bad_kind, "bad_index": st.bad_index, "want_index": pos,
                             "err_other": err(im, base, ~in_t), "err_tile": err(im, ref(drop=dropped), in_t)}
        # 2) the last tile's range ending past K, over entries that name primitive 0
        bin_(N)
        offs, lst, K = lists()
        for k in range(8):
            D.dbmp_workspace_debug_set(ws, 1, K + k, 0)
        D.dbmp_workspace_debug_set(ws, 0, n_tiles, K + 8)
        im, st = fwd()
        out["tile_range"] = {"bad_kind": st.bad_kind, "bad_index": st.bad_index, "want_index": n_tiles - 1,
                             "err": err(im, base)}
        # 3) a record whose bitmap row is not the first row of a bitmap
        bin_(N)
        victim = int(lst[offs[t]])
        D.dbmp_workspace_debug_set(ws, 2, victim, 5)
        im, st = fwd()
        out["bitmap_row"] = {"bad_kind": st.bad_kind, "bad_index": st.bad_index, "want_index": victim,
                             "err": err(im, ref(drop=victim))}
    finally:
        D.dbmp_workspace_destroy(ws)
        D.dbmp_atlas_destroy(atlas)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
