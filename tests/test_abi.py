"""The C-ABI library builds, loads without a GPU, exports every entry point that
include/dbmp.h declares, and rejects bad arguments on the host (CPU only: no
call here reaches a CUDA kernel or allocation)."""
import ctypes
import os
import re

import pytest

from paper_2602_22625_gb300 import _build
from paper_2602_22625_gb300 import dbmp as D

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(dbmp_\w+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return D.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 18
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing
    assert set(D.EXPORTS) <= names


def test_abi_version(lib):
    assert lib.dbmp_abi_version() == 1


def test_host_argument_validation(lib):
    out = ctypes.c_void_p()
    assert lib.dbmp_workspace_create(None, ctypes.byref(out)) == D.DBMP_ERR_INVALID_ARG
    assert b"limits" in lib.dbmp_last_error()
    bad = D.DbmpLimits(-1, 1, 1, 1)
    assert lib.dbmp_workspace_create(ctypes.byref(bad), ctypes.byref(out)) == D.DBMP_ERR_INVALID_ARG
    huge = D.DbmpLimits(1, 1, 1 << 40, 1)
    assert lib.dbmp_workspace_create(ctypes.byref(huge), ctypes.byref(out)) == D.DBMP_ERR_INVALID_ARG
    n = ctypes.c_size_t()
    ok = D.DbmpLimits(1000, 64, 1 << 20, 1)
    assert lib.dbmp_workspace_bytes(ctypes.byref(ok), ctypes.byref(n)) == D.DBMP_OK
    assert n.value > 4 * (1 << 20)
    assert lib.dbmp_atlas_create(None, 1, 8, 8, None, ctypes.byref(out)) == D.DBMP_ERR_INVALID_ARG
    assert lib.dbmp_atlas_create(ctypes.c_void_p(16), 0, 8, 8, None, ctypes.byref(out)) == D.DBMP_ERR_INVALID_ARG
    assert lib.dbmp_atlas_create(ctypes.c_void_p(16), 1, 1, 8, None, ctypes.byref(out)) == D.DBMP_ERR_INVALID_ARG
    assert lib.dbmp_bin(None, 8, 8, 16, None, None, 0, None, 1.0, None) == D.DBMP_ERR_INVALID_ARG
    bg = D.DbmpBackground()
    assert lib.dbmp_render_fwd(None, None, ctypes.byref(bg), 0.0, None, None, None, None) == \
        D.DBMP_ERR_INVALID_ARG
    assert lib.dbmp_mse_grad(None, None, -1, None, None, None) == D.DBMP_ERR_INVALID_ARG
    cfg = D.adam_config()
    assert lib.dbmp_adam_step(None, None, None, None, -1, ctypes.c_void_p(16), ctypes.byref(cfg),
                              None) == D.DBMP_ERR_INVALID_ARG
    cfg.beta1 = 1.5
    assert lib.dbmp_adam_step(None, None, None, None, 0, ctypes.c_void_p(16), ctypes.byref(cfg),
                              None) == D.DBMP_ERR_INVALID_ARG


def test_errors_raise_in_python(lib):
    with pytest.raises(D.DbmpError) as e:
        D._check(lib.dbmp_bin(None, 8, 8, 16, None, None, 0, None, 1.0, None))
    assert e.value.code == D.DBMP_ERR_INVALID_ARG
