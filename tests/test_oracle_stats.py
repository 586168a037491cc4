"""Pins of the oracle's scaling statistics of a binning (Sec. S4: footprint A_i/(HW),
tile-hit degree tau_i, per-tile density d_t), CPU only: the conservation identity,
brute-force histograms, and the footprint of an axis-aligned primitive."""
import math

import numpy as np

import oracle
from paper_2602_22625_gb300 import inputs


def test_conservation_and_brute_force_histograms():
    sc = inputs.tiny(seed=12, N=400, H=150, W=190)
    st = oracle.bin_stats(sc.H, sc.W, 16, sc.params, sc.bitmap_id, sc.atlas)
    rects, tau = oracle.bin_rects(sc.H, sc.W, 16, sc.params, sc.bitmap_id, sc.atlas)
    offs, lst = oracle.bin(sc.H, sc.W, 16, sc.params, sc.bitmap_id, sc.atlas)
    d = np.diff(offs)
    assert st["pairs"] == tau.sum() == d.sum() == len(lst)          # sum tau = sum d (Sec. S4)
    assert st["tau_hist"].sum() == st["n_listed"] == (tau > 0).sum()
    assert st["d_hist"].sum() + st["empty_tiles"] == st["n_tiles"] == d.size
    for b in range(32):
        assert st["tau_hist"][b] == sum(1 for t in tau if t > 0 and 2 ** b <= t < 2 ** (b + 1))
        assert st["d_hist"][b] == sum(1 for x in d if x > 0 and 2 ** b <= x < 2 ** (b + 1))
    assert st["tau_max"] == tau.max() and st["d_max"] == d.max()


def test_footprint_of_axis_aligned_primitives():
    """theta = 0: hx = s e_u, hy = s e_v (e = 1 + 2/(size-1)), A = (2 hx + 2)(2 hy + 2):
    the footprint is the whole bitmap's padded box, whatever part of it is non-zero."""
    H = W = 256
    Hb = Wb = 64
    e = 1.0 + 2.0 / 63.0
    s_vals = [0.4, 3.0, 10.0, 40.0, 300.0]
    p = np.zeros((len(s_vals), 8), np.float32)
    p[:, 0] = 128.0
    p[:, 1] = 128.0
    p[:, 2] = s_vals
    atlas = np.zeros((1, Hb, Wb), np.float32)
    atlas[0, 20:40, 30:34] = 1.0   # a small non-zero part: the binning box shrinks, the footprint does not
    st = oracle.bin_stats(H, W, 16, p, np.zeros(len(s_vals), np.int32), atlas)
    want = np.zeros(32, np.int64)
    for s in s_vals:
        a = (2 * s * e + 2) ** 2 / (H * W)
        want[0 if a >= 1 else min(31, int(math.floor(-math.log2(a))))] += 1
    np.testing.assert_array_equal(st["foot_hist"], want)
    assert st["n_listed"] == len(s_vals)
