"""The oracle's pins must catch plausible mistakes (CPU only).

Each case plants one mistake in a copy of the oracle's C source (a wrong sign,
swapped taps, a dropped term, a wrong index or scale), builds it in a temporary
directory and runs the pin tests against it; at least one pin must fail.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTANTS = {
    "rotation_sense": ("L->u = (q->cs * dx + q->sn * dy) / q->s;",
                       "L->u = (q->cs * dx - q->sn * dy) / q->s;"),
    "taps_transposed": ("L->p01 = tap(q->bmp, Hb, Wb, iv, iu + 1);\n    L->p10 = tap(q->bmp, Hb, Wb, iv + 1, iu);",
                        "L->p10 = tap(q->bmp, Hb, Wb, iv, iu + 1);\n    L->p01 = tap(q->bmp, Hb, Wb, iv + 1, iu);"),
    "background_dropped_in_backward": ("double R[3] = {b[0], b[1], b[2]};", "double R[3] = {0, 0, 0};"),
    "sigmoid_derivative_dropped": ("q->chat[j] * (1.0 - q->chat[j]);", "q->chat[j];"),
    "theta_gradient_sign": ("Gk[3] += gu * L->v + gv * (-L->u);", "Gk[3] += gu * L->v + gv * (L->u);"),
    "bitmap_scale_W_not_W_minus_1": ("double U = (L->u + 1.0) / 2.0 * (double)(Wb - 1);",
                                     "double U = (L->u + 1.0) / 2.0 * (double)(Wb);"),
    "bitmap_V_scale_uses_width": ("double V = (L->v + 1.0) / 2.0 * (double)(Hb - 1);",
                                  "double V = (L->v + 1.0) / 2.0 * (double)(Wb - 1);"),
    "half_widths_swapped_in_backward": ("double gu = dM * dMdU * kw, gv = dM * dMdV * kv;",
                                        "double gu = dM * dMdU * kv, gv = dM * dMdV * kw;"),
    "early_termination_dropped": ("        if (T < T_stop) break;\n        orc_layer L;", "        orc_layer L;"),
    "zero_samples_counted_as_layers": ("        if (L.M == 0.0) continue;\n        L.k = k;", "        L.k = k;"),
    "back_product_not_updated": ("B *= (1.0 - L->alpha);\n    }\n}", "}\n}"),
    "transmittance_update": ("T *= (1.0 - L.alpha);", "T *= (1.0 - 0.5 * L.alpha);"),
    "bin_margin_sign": ("float fx0 = floorf(((cx - hx) - m) * inv_t);",
                        "float fx0 = floorf(((cx - hx) + m) * inv_t);"),
    "bin_support_ring_dropped": ("float hu = (float)(box[1] - box[0] + 2) * 0.5f;",
                                 "float hu = (float)(box[1] - box[0]) * 0.5f;"),
    "bin_half_widths_swapped": ("float uc = cu / kw, eu = hu / kw, vc = cv / kv, ev = hv / kv;",
                                "float uc = cu / kv, eu = hu / kv, vc = cv / kw, ev = hv / kw;"),
    "bin_centre_offset_sign": ("dxc = s * (cs * uc - sn * vc);", "dxc = s * (cs * uc + sn * vc);"),
    "bin_centre_offset_dropped": ("float cx = p[0] + dxc, cy = p[1] + dyc;", "float cx = p[0], cy = p[1] + dyc;"),
    "bin_quadrant_sign": ("        *sn = cr;\n        *cs = -sr;", "        *sn = cr;\n        *cs = sr;"),
    "bin_nonzero_box_row_col_swapped": ("if (u < box[0]) box[0] = u;", "if (v < box[0]) box[0] = v;"),
    "variance_window_5_wide": ("const int32_t x0 = x - 3 < 0 ? 0 : x - 3, x1 = x + 3 > W - 1 ? W - 1 : x + 3;",
                               "const int32_t x0 = x - 2 < 0 ? 0 : x - 2, x1 = x + 2 > W - 1 ? W - 1 : x + 2;"),
    "variance_not_centred": ("const double d = (double)P[(size_t)yy * W + xx] - mean;",
                             "const double d = (double)P[(size_t)yy * W + xx];"),
    "base_probability_dropped": ("const double w = 0.1 + 0.9 * lv[p];", "const double w = lv[p];"),
    "scale_rule_reversed": ("o[2] = s_max - (s_max - s_min) * lv[p];", "o[2] = s_min + (s_max - s_min) * lv[p];"),
    "grad_selected_clip_off_by_one": ("if (x1 > W - 1) x1 = W - 1;", "if (x1 > W - 2) x1 = W - 2;"),
    # the support box has a pixel of slack beyond the padding ring, so a box shorter by
    # one or two rows is still exact (an equivalent mutant); three rows cut into it
    "grad_selected_box_short_by_three_rows": ("y1 = (long)ceil(q->yhi);", "y1 = (long)ceil(q->yhi) - 3;"),
    "grad_selected_row_index": ("pixel_grad(P, Hb, Wb, Ls, n, g, gA, b, Gl, sel[t]);",
                                "pixel_grad(P, Hb, Wb, Ls, n, g, gA, b, Gl, t);"),
    "grad_pixels_index_transposed": ("size_t pix = (size_t)py[i] * (size_t)W + (size_t)px[i];",
                                     "size_t pix = (size_t)px[i] * (size_t)W + (size_t)py[i];"),
    "mask_ignored": ("Q[p + 1] = Q[p] + (mask && !(mask[p] > 0.0f) ? 0 : (int64_t)floor(w * 1048576.0));",
                     "Q[p + 1] = Q[p] + (int64_t)floor(w * 1048576.0);"),
}


# mistakes planted in the oracle's Python half (oracle/oracle.py)
PY_MUTANTS = {
    "adam_bias_correction_dropped": ("    mh = m / (1.0 - beta1 ** t)\n", "    mh = m\n"),
    "adam_second_moment_not_squared": ("(1.0 - beta2) * g * g", "(1.0 - beta2) * np.abs(g)"),
    "mse_grad_factor_two_dropped": ("    return 2.0 * d / d.size", "    return d / d.size"),
}


# mistakes planted in the proposal network's oracle (oracle/cnn.py), against its pins
CNN_MUTANTS = {
    "col2im_taps_transposed": ("+= d[:, :, :, ky, kx, :]", "+= d[:, :, :, kx, ky, :]"),
    "relu_mask_dropped_in_backward": ("dZ = R(np.where(X > 0, dX, 0.0))", "dZ = R(dX)"),
    "bias_gradient_dropped": ("grads[li] = (mm(dZ.T, cols[li]), dZ.sum(0))",
                              "grads[li] = (mm(dZ.T, cols[li]), 0.0 * dZ.sum(0))"),
    "im2col_padding_misplaced": ("Xp[:, p:p + H, p:p + W] = X", "Xp[:, :H, :W] = X"),
}

PIN_FILES = ("tests/test_oracle_pins.py", "tests/test_oracle_init.py")


def run_pins(tmp_path, src, pysrc=None, files=None, pins=PIN_FILES):
    """Runs the pin tests `pins` against a copy of the oracle built from `src` (and, if
    given, `pysrc` as its oracle.py and `files` {name: text} for other oracle files), with
    the test files and the helpers they import copied beside it; returns the pytest result."""
    shutil.copytree(os.path.join(ROOT, "oracle"), tmp_path / "oracle",
                    ignore=shutil.ignore_patterns("_lib", "__pycache__"))
    (tmp_path / "oracle" / "dbmp_oracle.c").write_text(src)
    if pysrc is not None:
        (tmp_path / "oracle" / "oracle.py").write_text(pysrc)
    for name, text in (files or {}).items():
        (tmp_path / "oracle" / name).write_text(text)
    (tmp_path / "tests").mkdir()
    for f in [os.path.basename(p) for p in pins] + ["conftest.py", "_helpers.py"]:
        shutil.copy(os.path.join(ROOT, "tests", f), tmp_path / "tests" / f)
    os.symlink(os.path.join(ROOT, "paper_2602_22625_gb300"), tmp_path / "paper_2602_22625_gb300")
    return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *pins],
                          cwd=tmp_path, capture_output=True, text=True, timeout=300)


def assert_caught(r):
    """A pin failed on an assertion (not on an import or another error)."""
    assert r.returncode == 1, r.stdout[-2000:] + r.stderr[-2000:]
    assert "failed" in r.stdout and "Error" not in r.stdout.replace("AssertionError", ""), r.stdout[-2000:]


def test_unmutated_copy_passes_the_pins(tmp_path):
    """The control: the copied oracle and pins pass as they stand, so a failure
    below comes from the planted mistake, not from the copy (a missing helper module
    would make every mutant look caught)."""
    r = run_pins(tmp_path, open(os.path.join(ROOT, "oracle", "dbmp_oracle.c")).read())
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    src = open(os.path.join(ROOT, "oracle", "dbmp_oracle.c")).read()
    a, b = MUTANTS[name]
    assert a in src
    r = run_pins(tmp_path, src.replace(a, b, 1))
    assert_caught(r)


@pytest.mark.parametrize("name", sorted(PY_MUTANTS))
def test_pins_catch_planted_mistake_in_the_python_half(name, tmp_path):
    src = open(os.path.join(ROOT, "oracle", "dbmp_oracle.c")).read()
    py = open(os.path.join(ROOT, "oracle", "oracle.py")).read()
    a, b = PY_MUTANTS[name]
    assert a in py
    r = run_pins(tmp_path, src, py.replace(a, b, 1))
    assert_caught(r)


def test_unmutated_network_oracle_passes_its_pins(tmp_path):
    r = run_pins(tmp_path, open(os.path.join(ROOT, "oracle", "dbmp_oracle.c")).read(),
                 pins=("tests/test_oracle_cnn.py",))
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]


@pytest.mark.parametrize("name", sorted(CNN_MUTANTS))
def test_network_pins_catch_planted_mistake(name, tmp_path):
    src = open(os.path.join(ROOT, "oracle", "dbmp_oracle.c")).read()
    cnn = open(os.path.join(ROOT, "oracle", "cnn.py")).read()
    a, b = CNN_MUTANTS[name]
    assert a in cnn
    r = run_pins(tmp_path, src, files={"cnn.py": cnn.replace(a, b, 1)}, pins=("tests/test_oracle_cnn.py",))
    assert_caught(r)
