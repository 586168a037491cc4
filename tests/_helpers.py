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
