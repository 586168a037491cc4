"""Shared helpers of the test suite (no method arithmetic here)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

GROUPS = ("x", "y", "s", "theta", "nu", "c_r", "c_g", "c_b")


def cuda():
    if not torch.cuda.is_available():
        pytest.skip("CUDA not available")
    return torch.device("cuda")


def to_dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def grad_close(g, ref, rel=1e-3, what=""):
    """Per parameter group: ||g - ref||_2 <= rel ||ref||_2 and |g - ref| <= rel max|ref|
    (groups whose reference is identically zero must come out zero up to 1e-12)."""
    g = np.asarray(g, np.float64)
    ref = np.asarray(ref, np.float64)
    assert g.shape == ref.shape
    for j, name in enumerate(GROUPS):
        r = ref[:, j]
        d = g[:, j] - r
        nr = np.linalg.norm(r)
        if nr == 0:
            assert np.abs(g[:, j]).max(initial=0) <= 1e-12, (what, name)
            continue
        rel_l2 = np.linalg.norm(d) / nr
        rel_max = np.abs(d).max() / np.abs(r).max()
        assert rel_l2 <= rel and rel_max <= rel, f"{what} {name}: rel_l2={rel_l2:.3g} rel_max={rel_max:.3g}"


def lists_from_rects(rects, ntx, nty):
    """Tile lists from per-primitive inclusive tile rectangles (N, 4) {tx0, ty0, tx1,
    ty1}: every (tile, primitive) pair, sorted by tile with a stable sort so that the
    primitive index stays increasing inside a tile.  Returns (offsets, list)."""
    rects = np.asarray(rects, np.int64)
    w = np.maximum(rects[:, 2] - rects[:, 0] + 1, 0)
    h = np.maximum(rects[:, 3] - rects[:, 1] + 1, 0)
    n = w * h
    prim = np.repeat(np.arange(len(rects)), n)
    k = np.arange(n.sum()) - np.repeat(np.cumsum(n) - n, n)
    wr = np.repeat(w, n)
    tile = (np.repeat(rects[:, 1], n) + k // np.maximum(wr, 1)) * ntx + np.repeat(rects[:, 0], n) + k % np.maximum(wr, 1)
    order = np.argsort(tile, kind="stable")
    offs = np.zeros(ntx * nty + 1, np.int64)
    np.cumsum(np.bincount(tile, minlength=ntx * nty), out=offs[1:])
    return offs, prim[order].astype(np.int32)
