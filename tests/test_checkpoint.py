"""Checkpoint / resume: the file format round-trips bit for bit, and an optimisation
resumed from a checkpoint continues exactly as the uninterrupted one (FP64 oracle
forward, backward and Adam on one thread on a tiny scene, so the comparison is exact;
the GPU continuation, whose gradient atomics sum in any order, is checked in
test_gpu_batch.py)."""
import numpy as np
import pytest

import oracle
from paper_2602_22625_gb300 import checkpoint, inputs


def test_round_trip_is_bit_exact(tmp_path):
    rng = np.random.default_rng(1)
    arrays = {"params": rng.normal(size=(37, 8)).astype(np.float32),
              "m": rng.normal(size=(37, 8)), "v": np.abs(rng.normal(size=(37, 8))),
              "ids": rng.integers(-5, 5, 37).astype(np.int32), "empty": np.zeros((0, 8), np.float32)}
    p = tmp_path / "a.ckpt"
    checkpoint.save(p, arrays, step=12, meta={"lr": 0.1, "seed": 3})
    back, step, meta = checkpoint.load(p)
    assert step == 12 and meta == {"lr": 0.1, "seed": 3}
    for k, a in arrays.items():
        assert back[k].dtype == a.dtype and back[k].shape == a.shape
        assert back[k].tobytes() == a.tobytes()


def test_bad_files_are_rejected(tmp_path):
    p = tmp_path / "b.ckpt"
    p.write_bytes(b"NOTACKPT" + b"\0" * 16)
    with pytest.raises(ValueError):
        checkpoint.load(p)
    checkpoint.save(p, {"x": np.arange(10, dtype=np.int64)}, step=0)
    p.write_bytes(p.read_bytes()[:-8])
    with pytest.raises(ValueError):
        checkpoint.load(p)


def _steps(sc, target, p, m, v, t0, n):
    for t in range(t0 + 1, t0 + n + 1):
        img = oracle.render(sc.H, sc.W, p, sc.bitmap_id, sc.atlas, background=sc.background)["image"]
        g = oracle.grad(sc.H, sc.W, p, sc.bitmap_id, sc.atlas, oracle.mse_grad(img, target),
                        background=sc.background)
        p, m, v = oracle.adam_step(p, g, m, v, t, 0.01)
    return p, m, v


@pytest.fixture
def one_thread():
    """The oracle's parallel gradient sums are order-dependent; one thread makes the
    FP64 run reproducible bit for bit."""
    n = oracle.num_threads()
    oracle.set_num_threads(1)
    yield
    oracle.set_num_threads(n)


def test_resume_continues_exactly(tmp_path, one_thread):
    sc = inputs.tiny(seed=5, N=12, H=24, W=24)
    tg = inputs.tiny(seed=6, N=12, H=24, W=24)
    target = oracle.render(tg.H, tg.W, tg.params, tg.bitmap_id, tg.atlas, background=tg.background)["image"]
    p0 = sc.params.astype(np.float64)
    z = np.zeros_like(p0)
    p_ref, m_ref, v_ref = _steps(sc, target, p0, z, z, 0, 4)
    p, m, v = _steps(sc, target, p0, z, z, 0, 2)
    ck = tmp_path / "run.ckpt"
    checkpoint.save(ck, {"params": p, "m": m, "v": v}, step=2)
    a, step, _ = checkpoint.load(ck)
    p2, m2, v2 = _steps(sc, target, a["params"], a["m"], a["v"], step, 2)
    assert np.array_equal(p2, p_ref) and np.array_equal(m2, m_ref) and np.array_equal(v2, v_ref)
