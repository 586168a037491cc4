"""Defaults of the oracle and the library against the paper's table of common
hyperparameters (tests/golden/tab_s1_common_hyperparams.txt, Tab. S1).  Where the
value is an algorithmic constant (the variance window, the base probability), it is
checked through the oracle's behaviour, not by reading a constant."""
import inspect
import pathlib

import numpy as np

import oracle
from paper_2602_22625_gb300 import dbmp as D
from paper_2602_22625_gb300 import inputs, proposer

GOLD = pathlib.Path(__file__).parent / "golden" / "tab_s1_common_hyperparams.txt"


def table():
    out = {}
    for line in GOLD.read_text().splitlines():
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = (s.strip() for s in line.split("="))
            out[k] = float(v)
    return out


def test_learning_rate_and_gains():
    t = table()
    # parameter columns: x, y, s (the table's r), theta, nu (the table's v), c_r, c_g, c_b
    want = (t["lr_gain_x"], t["lr_gain_y"], t["lr_gain_r"], t["lr_gain_theta"], t["lr_gain_v"],
            t["lr_gain_c"], t["lr_gain_c"], t["lr_gain_c"])
    assert tuple(oracle.LR_GAINS) == want
    cfg = D.adam_config()
    assert tuple(cfg.gains) == want
    assert np.float32(cfg.lr) == np.float32(t["learning_rate.default"])


def test_colour_noise_and_blur_defaults():
    t = table()
    for fn in (oracle.structure_init, oracle.structure_reinit, proposer.structure_init):
        assert inspect.signature(fn).parameters["sigma_c"].default == t["std_c_init"]
    assert inspect.signature(inputs.stroke_atlas).parameters["blur_sigma"].default == t["blur_sigma"]
    assert inspect.signature(oracle.render).parameters["alpha_max"].default == t["alpha_upper_bound"]


def test_variance_window_is_the_tables():
    """One bright pixel: the local variance is non-zero exactly within the window."""
    w = int(table()["variance_window_size"])
    img = np.zeros((3, 31, 31), np.float32)
    img[:, 15, 15] = 1.0
    lv = oracle.local_variance(img)
    ys, xs = np.nonzero(lv > 0)
    assert ys.min() == 15 - w // 2 and ys.max() == 15 + w // 2
    assert xs.min() == 15 - w // 2 and xs.max() == 15 + w // 2


def test_variance_base_probability_is_the_tables():
    """The draws' total mass is sum_p floor((b + (1 - b) NLV_p) 2^20) with b the table's
    base probability; a flat region (NLV = 0) keeps weight b."""
    b = table()["variance_base_prob"]
    rng = np.random.default_rng(3)
    img = np.zeros((3, 24, 24), np.float32)
    img[:, 8:16, 8:16] = rng.uniform(0, 1, (3, 8, 8))
    n = 16
    _, nlv, _, total = oracle.structure_init(img, rng.uniform(0, 1, n), rng.uniform(0, 1, n),
                                             rng.normal(size=(n, 3)), (2.0, 6.0))
    assert nlv.min() == 0.0 and np.isclose(nlv.max(), 1.0)
    assert total == int(np.floor((b + (1.0 - b) * nlv) * 2.0 ** 20).sum())
