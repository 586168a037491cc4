"""Python binding of libdbmp (include/dbmp.h): argument marshalling only.

Every function named dbmp_* here calls the C entry point of the same name with
raw device pointers taken from torch tensors; all computation runs in the
library's CUDA kernels.  There is no CPU fallback: if the library cannot be
loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import _build

DBMP_OK = 0
DBMP_ERR_INVALID_ARG = -1
DBMP_ERR_CAPACITY = -2
DBMP_ERR_CUDA = -3
DBMP_ERR_TIMEOUT = -4
DBMP_ERR_NOT_READY = -5
DBMP_ERR_NO_MEMORY = -6

BG_NONE, BG_CONST, BG_BUFFER = 0, 1, 2
BATCH_BIN, BATCH_FWD, BATCH_BWD = 1, 2, 4

#: every entry point include/dbmp.h declares
EXPORTS = (
    "dbmp_last_error", "dbmp_abi_version", "dbmp_atlas_create", "dbmp_atlas_destroy",
    "dbmp_atlas_update", "dbmp_workspace_bytes", "dbmp_workspace_create", "dbmp_workspace_destroy",
    "dbmp_status_poll", "dbmp_bin", "dbmp_get_tile_lists", "dbmp_render_fwd", "dbmp_render_bwd",
    "dbmp_mse_grad", "dbmp_adam_step", "dbmp_batch_plan", "dbmp_batch_render", "dbmp_autotune",
    "dbmp_autotune_set_prune",
    "dbmp_render_fwd_static", "dbmp_gemm_bf16", "dbmp_proposer_num_params", "dbmp_proposer_create",
    "dbmp_proposer_destroy", "dbmp_proposer_set_params", "dbmp_proposer_get", "dbmp_propose",
    "dbmp_proposer_train_step", "dbmp_structure_init_scratch_bytes", "dbmp_structure_init",
    "dbmp_blur_bitmaps", "dbmp_bin_stats", "dbmp_structure_reinit", "dbmp_alpha_loss_grad",
    "dbmp_workspace_poison", "dbmp_batch_render_mse", "dbmp_fp32_peak", "dbmp_render_alpha", "dbmp_proposer_activations",
    "dbmp_batch_set_rows", "dbmp_index_checks", "dbmp_workspace_debug_set", "dbmp_workspace_count_pairs",
)


class DbmpBinStats(ctypes.Structure):
    _fields_ = [("n_listed", ctypes.c_int64), ("pairs", ctypes.c_int64), ("tau_max", ctypes.c_int64),
                ("d_max", ctypes.c_int64), ("n_tiles", ctypes.c_int64), ("empty_tiles", ctypes.c_int64),
                ("tau_hist", ctypes.c_int64 * 32), ("d_hist", ctypes.c_int64 * 32),
                ("foot_hist", ctypes.c_int64 * 32)]


class DbmpError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libdbmp error {code}: {msg}")
        self.code = code


class DbmpBackground(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("rgb", ctypes.c_float * 3), ("buf_dev", ctypes.c_void_p)]


class DbmpLimits(ctypes.Structure):
    _fields_ = [("max_prims", ctypes.c_int32), ("max_tiles", ctypes.c_int32),
                ("max_pairs", ctypes.c_int64), ("max_canvases", ctypes.c_int32)]


class DbmpDeviceStatus(ctypes.Structure):
    _fields_ = [("code", ctypes.c_int32), ("n_degenerate", ctypes.c_int32),
                ("pairs_required", ctypes.c_int64), ("pairs_evaluated", ctypes.c_int64),
                ("pairs_evaluated_bwd", ctypes.c_int64), ("pairs_contributing", ctypes.c_int64),
                ("warp_steps", ctypes.c_int64), ("warp_steps_bwd", ctypes.c_int64),
                ("survivors", ctypes.c_int64), ("survivors_bwd", ctypes.c_int64),
                ("bad_kind", ctypes.c_int32), ("bad_pad", ctypes.c_int32), ("bad_index", ctypes.c_int64)]


class DbmpAdamConfig(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_float), ("gamma", ctypes.c_float), ("beta1", ctypes.c_float),
                ("beta2", ctypes.c_float), ("eps", ctypes.c_float), ("gains", ctypes.c_float * 8),
                ("zero_grad", ctypes.c_int32)]


class DbmpProposerAdam(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float)]


class DbmpTuning(ctypes.Structure):
    _fields_ = [("tile", ctypes.c_int32), ("batch", ctypes.c_int32), ("ppt", ctypes.c_int32),
                ("ppt_bwd", ctypes.c_int32)]


_lib = None
_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_f32 = ctypes.c_float


def library_path() -> str:
    """libdbmp.so, or with DBMP_LIBRARY=checked in the environment the build with
    device-side index checks (libdbmp_checked.so)."""
    return _build.LIB_CHECKED if os.environ.get("DBMP_LIBRARY") == "checked" else _build.LIB


def load(build_if_missing: bool = True):
    """Loads libdbmp.so (building it with nvcc if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and not _build.up_to_date():
        _build.build()
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"libdbmp.so not found at {path}; run paper_2602_22625_gb300._build.build()")
    L = ctypes.CDLL(path)
    sig = {
        "dbmp_last_error": (ctypes.c_char_p, []),
        "dbmp_abi_version": (_i32, []),
        "dbmp_atlas_create": (_i32, [_vp, _i32, _i32, _i32, _vp, ctypes.POINTER(_vp)]),
        "dbmp_atlas_destroy": (_i32, [_vp]),
        "dbmp_atlas_update": (_i32, [_vp, _vp, _vp]),
        "dbmp_workspace_bytes": (_i32, [ctypes.POINTER(DbmpLimits), ctypes.POINTER(ctypes.c_size_t)]),
        "dbmp_workspace_create": (_i32, [ctypes.POINTER(DbmpLimits), ctypes.POINTER(_vp)]),
        "dbmp_workspace_destroy": (_i32, [_vp]),
        "dbmp_workspace_poison": (_i32, [_vp, _vp]),
        "dbmp_workspace_count_pairs": (_i32, [_vp, _i32]),
        "dbmp_status_poll": (_i32, [_vp, _vp, ctypes.POINTER(DbmpDeviceStatus)]),
        "dbmp_bin": (_i32, [_vp, _i32, _i32, _i32, _vp, _vp, _i32, _vp, _f32, _vp]),
        "dbmp_get_tile_lists": (_i32, [_vp, _vp, _vp, _i64, ctypes.POINTER(_i32), _vp]),
        "dbmp_render_fwd": (_i32, [_vp, _vp, ctypes.POINTER(DbmpBackground), _f32, _vp, _vp, _vp, _vp]),
        "dbmp_render_bwd": (_i32, [_vp, _vp, ctypes.POINTER(DbmpBackground), _f32, _vp, _vp, _vp, _vp,
                                   _vp, _vp]),
        "dbmp_mse_grad": (_i32, [_vp, _vp, _i64, _vp, _vp, _vp]),
        "dbmp_adam_step": (_i32, [_vp, _vp, _vp, _vp, _i32, _vp, ctypes.POINTER(DbmpAdamConfig), _vp]),
        "dbmp_batch_plan": (_i32, [_vp, _i32, _vp, _vp, _vp, ctypes.POINTER(DbmpTuning), _vp]),
        "dbmp_batch_render": (_i32, [_vp, _vp, _vp, _vp, _f32, ctypes.POINTER(DbmpBackground), _f32,
                                     _i32, _vp, _vp, _vp, _vp, _vp, _vp]),
        "dbmp_batch_render_mse": (_i32, [_vp, _vp, _vp, _vp, _f32, ctypes.POINTER(DbmpBackground), _f32,
                                         _i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
        "dbmp_autotune_set_prune": (_i32, [_vp, _f32]),
        "dbmp_autotune": (_i32, [_vp, _vp, _vp, _vp, _f32, ctypes.POINTER(DbmpBackground), _f32, _i32,
                                 _vp, _vp, _vp, _vp, _vp, _i32, ctypes.POINTER(DbmpTuning),
                                 ctypes.POINTER(_f32), _vp]),
        "dbmp_render_alpha": (_i32, [_vp, _vp, _i64, _vp]),
        "dbmp_batch_set_rows": (_i32, [_vp, _i32, _i32]),
        "dbmp_index_checks": (_i32, []),
        "dbmp_workspace_debug_set": (_i32, [_vp, _i32, _i64, _i64, _vp]),
        "dbmp_proposer_activations": (_i32, [_vp, _i32, _vp, _i64]),
        "dbmp_fp32_peak": (_i32, [_i32, _i32, _vp, _i64, ctypes.POINTER(ctypes.c_double), _vp]),
        "dbmp_gemm_bf16": (_i32, [_vp, _i32, _vp, _i32, _i32, _i32, _i32, _i32, _vp, _vp, _i32, _vp, _i32,
                                  _vp, _vp]),
        "dbmp_proposer_num_params": (_i64, []),
        "dbmp_proposer_create": (_i32, [_i32, ctypes.POINTER(_vp)]),
        "dbmp_proposer_destroy": (_i32, [_vp]),
        "dbmp_proposer_set_params": (_i32, [_vp, _vp, _i64]),
        "dbmp_proposer_get": (_i32, [_vp, _i32, _vp, _i64]),
        "dbmp_propose": (_i32, [_vp, _vp, _i32, _vp, _vp]),
        "dbmp_proposer_train_step": (_i32, [_vp, _vp, _vp, _i32, ctypes.POINTER(DbmpProposerAdam), _vp, _vp]),
        "dbmp_blur_bitmaps": (_i32, [_vp, _i32, _i32, _i32, _f32, _vp, _vp]),
        "dbmp_bin_stats": (_i32, [_vp, _vp, ctypes.POINTER(DbmpBinStats)]),
        "dbmp_structure_init_scratch_bytes": (_i32, [_i32, _i32, ctypes.POINTER(ctypes.c_size_t)]),
        "dbmp_structure_init": (_i32, [_vp, _vp, _i32, _i32, _i32, _vp, _vp, _vp, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, _vp, _vp, _vp, _vp]),
        "dbmp_structure_reinit": (_i32, [_vp, _vp, _i32, _i32, _i32, _vp, _vp, _vp, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, _vp,
                                         _vp, _vp, _vp, _vp, _vp]),
        "dbmp_alpha_loss_grad": (_i32, [_vp, _vp, _vp, _vp, _i64, _f32, _vp, _vp, _vp, _vp]),
        "dbmp_render_fwd_static": (_i32, [_i32, _i32, _vp, _vp, _i32, _vp, _i32, _i32, _i32, _f32,
                                          ctypes.POINTER(DbmpBackground), _f32, _vp, _vp, _vp, _vp,
                                          ctypes.POINTER(DbmpDeviceStatus)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(code):
    if code != DBMP_OK:
        msg = load().dbmp_last_error().decode(errors="replace")
        raise DbmpError(code, msg)
    return code


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def make_background(background, H=None, W=None):
    """None -> no background (Eq. 5); 3 numbers -> constant; (3,H,W) CUDA tensor -> buffer."""
    bg = DbmpBackground()
    if background is None:
        bg.mode = BG_NONE
    elif isinstance(background, torch.Tensor) and background.numel() > 3:
        bg.mode = BG_BUFFER
        bg.buf_dev = _ptr(background)
    else:
        vals = [float(v) for v in (background.tolist() if isinstance(background, torch.Tensor) else background)]
        bg.mode = BG_CONST
        for j in range(3):
            bg.rgb[j] = vals[j]
    return bg


# ----------------------------------------------------------------------------
# Entry points (same names as the C ABI)
# ----------------------------------------------------------------------------

def dbmp_abi_version():
    return load().dbmp_abi_version()


def dbmp_atlas_create(texels, stream=None):
    assert texels.dtype == torch.float32 and texels.dim() == 3
    out = _vp()
    _check(load().dbmp_atlas_create(_ptr(texels), texels.shape[0], texels.shape[1], texels.shape[2],
                                    _stream(stream), ctypes.byref(out)))
    return out.value


def dbmp_atlas_update(atlas, texels, stream=None):
    _check(load().dbmp_atlas_update(atlas, _ptr(texels), _stream(stream)))


def dbmp_atlas_destroy(atlas):
    _check(load().dbmp_atlas_destroy(atlas))


def dbmp_workspace_bytes(max_prims, max_tiles, max_pairs, max_canvases=1):
    lim = DbmpLimits(max_prims, max_tiles, max_pairs, max_canvases)
    n = ctypes.c_size_t()
    _check(load().dbmp_workspace_bytes(ctypes.byref(lim), ctypes.byref(n)))
    return n.value


def dbmp_workspace_create(max_prims, max_tiles, max_pairs, max_canvases=1):
    lim = DbmpLimits(max_prims, max_tiles, max_pairs, max_canvases)
    out = _vp()
    _check(load().dbmp_workspace_create(ctypes.byref(lim), ctypes.byref(out)))
    return out.value


def dbmp_workspace_destroy(ws):
    _check(load().dbmp_workspace_destroy(ws))


def dbmp_workspace_poison(ws, stream=None):
    _check(load().dbmp_workspace_poison(ws, _stream(stream)))


def dbmp_workspace_count_pairs(ws, on=True):
    """Forwards of `ws` count the contributing pairs into the status (off by default)."""
    _check(load().dbmp_workspace_count_pairs(ws, 1 if on else 0))


def dbmp_status_poll(ws, stream=None, raise_on_error=True):
    st = DbmpDeviceStatus()
    code = load().dbmp_status_poll(ws, _stream(stream), ctypes.byref(st))
    if raise_on_error:
        _check(code)
    return st


def dbmp_bin(ws, H, W, tile, params, bitmap_id, N, atlas, alpha_max, stream=None):
    _check(load().dbmp_bin(ws, H, W, tile, _ptr(params), _ptr(bitmap_id), N, atlas, alpha_max,
                           _stream(stream)))


def dbmp_get_tile_lists(ws, offsets, lst, stream=None):
    n = _i32()
    _check(load().dbmp_get_tile_lists(ws, _ptr(offsets), _ptr(lst), lst.numel(), ctypes.byref(n),
                                      _stream(stream)))
    return n.value


def dbmp_render_fwd(ws, atlas, bg, T_stop, image, T_final, n_last, stream=None):
    _check(load().dbmp_render_fwd(ws, atlas, ctypes.byref(bg), T_stop, _ptr(image), _ptr(T_final),
                                  _ptr(n_last), _stream(stream)))


def dbmp_render_bwd(ws, atlas, bg, T_stop, dL_dimage, dL_dalpha, T_final, n_last, dparams, stream=None):
    _check(load().dbmp_render_bwd(ws, atlas, ctypes.byref(bg), T_stop, _ptr(dL_dimage), _ptr(dL_dalpha),
                                  _ptr(T_final), _ptr(n_last), _ptr(dparams), _stream(stream)))


def dbmp_mse_grad(image, target, dL_dI, loss, stream=None):
    _check(load().dbmp_mse_grad(_ptr(image), _ptr(target), image.numel(), _ptr(dL_dI), _ptr(loss),
                                _stream(stream)))


def adam_config(lr=0.1, gamma=1.0, beta1=0.9, beta2=0.999, eps=1e-8,
                gains=(10.0, 10.0, 10.0, 1.0, 1.5, 1.0, 1.0, 1.0), zero_grad=False):
    c = DbmpAdamConfig()
    c.lr, c.gamma, c.beta1, c.beta2, c.eps = lr, gamma, beta1, beta2, eps
    c.zero_grad = 1 if zero_grad else 0
    for j in range(8):
        c.gains[j] = gains[j]
    return c


def dbmp_adam_step(params, grad, m, v, step, cfg, stream=None):
    _check(load().dbmp_adam_step(_ptr(params), _ptr(grad), _ptr(m), _ptr(v), params.shape[0], _ptr(step),
                                 ctypes.byref(cfg), _stream(stream)))


def dbmp_batch_plan(ws, H, W, prim_offset, tile=16, batch=32, ppt=2, ppt_bwd=0, stream=None):
    n = len(H)
    Ha = (_i32 * n)(*H)
    Wa = (_i32 * n)(*W)
    Oa = (_i32 * (n + 1))(*prim_offset)
    t = DbmpTuning(tile, batch, ppt, ppt_bwd)
    _check(load().dbmp_batch_plan(ws, n, Ha, Wa, Oa, ctypes.byref(t), _stream(stream)))


BAD_NONE, BAD_TILE_RANGE, BAD_LIST_ENTRY, BAD_BITMAP_ROW, BAD_LIST_WRITE = 0, 1, 2, 3, 4


def dbmp_index_checks():
    """True if the loaded library is the index-checked build."""
    return bool(load().dbmp_index_checks())


def dbmp_workspace_debug_set(ws, what, index, value, stream=None):
    """Testing aid: overwrites a tile offset (0), list entry (1) or record bitmap row (2)."""
    _check(load().dbmp_workspace_debug_set(ws, int(what), int(index), int(value), _stream(stream)))


def dbmp_batch_set_rows(ws, y0, y1):
    """Restricts the plan's renders to canvas rows [y0, y1) (0, 0: all rows)."""
    _check(load().dbmp_batch_set_rows(ws, int(y0), int(y1)))


def dbmp_batch_render(ws, params, bitmap_id, atlas, alpha_max, bg, T_stop, mode, image=None, T_final=None,
                      n_last=None, dL_dimage=None, dparams=None, stream=None):
    _check(load().dbmp_batch_render(ws, _ptr(params), _ptr(bitmap_id), atlas, alpha_max, ctypes.byref(bg),
                                    T_stop, mode, _ptr(image), _ptr(T_final), _ptr(n_last),
                                    _ptr(dL_dimage), _ptr(dparams), _stream(stream)))


def dbmp_batch_render_mse(ws, params, bitmap_id, atlas, alpha_max, bg, T_stop, mode, target, image, T_final,
                          n_last, dL_dimage, loss, dparams=None, stream=None):
    """dbmp_batch_render with the MSE loss fused into the forward: dL/dI into dL_dimage
    and the loss into loss (float64 [1]); mode must include BATCH_FWD."""
    _check(load().dbmp_batch_render_mse(ws, _ptr(params), _ptr(bitmap_id), atlas, alpha_max, ctypes.byref(bg),
                                        T_stop, mode, _ptr(target), _ptr(image), _ptr(T_final), _ptr(n_last),
                                        _ptr(dL_dimage), _ptr(dparams), _ptr(loss), _stream(stream)))


def dbmp_autotune_set_prune(ws, max_pairs_ratio):
    """0: dbmp_autotune times every tile size; r > 0: only those whose binning lists at
    most r x the entries of the sparsest size, in increasing order of entries."""
    _check(load().dbmp_autotune_set_prune(ws, float(max_pairs_ratio)))


def dbmp_autotune(ws, params, bitmap_id, atlas, alpha_max, bg, T_stop, mode, image, T_final, n_last,
                  dL_dimage=None, dparams=None, reps=3, stream=None):
    best = DbmpTuning()
    ms = _f32()
    _check(load().dbmp_autotune(ws, _ptr(params), _ptr(bitmap_id), atlas, alpha_max, ctypes.byref(bg),
                                T_stop, mode, _ptr(image), _ptr(T_final), _ptr(n_last), _ptr(dL_dimage),
                                _ptr(dparams), reps, ctypes.byref(best), ctypes.byref(ms),
                                _stream(stream)))
    return (best.tile, best.batch, best.ppt, best.ppt_bwd), ms.value


def dbmp_render_fwd_static(H, W, params, bitmap_id, texels, alpha_max, bg, T_stop, image, T_final, n_last,
                           stream=None, with_status=True):
    """Forward render from the library's built-in scratch area (no device allocation).
    Returns the device status when with_status (the call then synchronises)."""
    st = DbmpDeviceStatus() if with_status else None
    _check(load().dbmp_render_fwd_static(H, W, _ptr(params), _ptr(bitmap_id), params.shape[0], _ptr(texels),
                                         texels.shape[0], texels.shape[1], texels.shape[2], alpha_max,
                                         ctypes.byref(bg), T_stop, _ptr(image), _ptr(T_final), _ptr(n_last),
                                         _stream(stream), ctypes.byref(st) if st is not None else None))
    return st


def dbmp_gemm_bf16(A, B, M, N, K, mode, Cf=None, Cb=None, ldc=None, bias=None, split_k=1, status=None,
                   stream=None):
    _check(load().dbmp_gemm_bf16(_ptr(A), A.shape[-1], _ptr(B), B.shape[-1], M, N, K, mode, _ptr(Cf), _ptr(Cb),
                                 N if ldc is None else ldc, _ptr(bias), split_k, _ptr(status), _stream(stream)))


def dbmp_fp32_peak(packed, iters, sink, stream=None):
    """Queues the FP32 issue-rate microbenchmark (one float per thread of `sink`);
    returns the launch's floating-point operations."""
    fl = ctypes.c_double()
    _check(load().dbmp_fp32_peak(int(packed), int(iters), _ptr(sink), sink.numel(), ctypes.byref(fl),
                                 _stream(stream)))
    return fl.value


def dbmp_proposer_num_params():
    return int(load().dbmp_proposer_num_params())


def dbmp_proposer_create(max_batch):
    out = _vp()
    _check(load().dbmp_proposer_create(max_batch, ctypes.byref(out)))
    return out.value


def dbmp_proposer_destroy(p):
    _check(load().dbmp_proposer_destroy(p))


def dbmp_proposer_set_params(p, theta):
    import numpy as np
    theta = np.ascontiguousarray(theta, dtype=np.float32)
    _check(load().dbmp_proposer_set_params(p, theta.ctypes.data, theta.size))


def dbmp_proposer_get(p, which):
    import numpy as np
    out = np.empty(dbmp_proposer_num_params(), np.float32)
    _check(load().dbmp_proposer_get(p, which, out.ctypes.data, out.size))
    return out


def dbmp_proposer_activations(p, layer, batch):
    """Activations of layer 0..6 of the last forward (float32 numpy array)."""
    import numpy as np
    sides = (256, 128, 64, 32, 16, 8)
    chans = (4, 32, 64, 128, 256, 256)
    shape = (batch * 64, 64) if layer == 6 else (batch, sides[layer], sides[layer], chans[layer])
    out = np.empty(shape, np.float32)
    _check(load().dbmp_proposer_activations(p, int(layer), out.ctypes.data, out.size))
    return out


def dbmp_propose(p, images, params_out, stream=None):
    _check(load().dbmp_propose(p, _ptr(images), images.shape[0], _ptr(params_out), _stream(stream)))


def dbmp_proposer_train_step(p, images, target_params, loss, adam=None, stream=None):
    cfg = None
    if adam is not None:
        cfg = DbmpProposerAdam(*adam)
    _check(load().dbmp_proposer_train_step(p, _ptr(images), _ptr(target_params), images.shape[0],
                                           ctypes.byref(cfg) if cfg is not None else None, _ptr(loss),
                                           _stream(stream)))


def dbmp_structure_init_scratch_bytes(H, W):
    n = ctypes.c_size_t()
    _check(load().dbmp_structure_init_scratch_bytes(H, W, ctypes.byref(n)))
    return n.value


def dbmp_structure_init(image, u_pos, u_theta, n_color, s_min, s_max, sigma_c, nu, params, nlv=None,
                        scratch=None, mask=None, stream=None):
    """Structure-aware initialisation of params (N, 8) from image (3, H, W) with the
    given random draws (float64 device tensors); mask (H, W) restricts the draws.
    scratch: a uint8 device tensor of dbmp_structure_init_scratch_bytes(H, W) bytes
    (allocated here when None)."""
    _, H, W = image.shape
    if scratch is None:
        scratch = torch.empty(dbmp_structure_init_scratch_bytes(H, W), dtype=torch.uint8, device=image.device)
    _check(load().dbmp_structure_init(_ptr(image), _ptr(mask), H, W, params.shape[0], _ptr(u_pos), _ptr(u_theta),
                                      _ptr(n_color), float(s_min), float(s_max), float(sigma_c), float(nu),
                                      _ptr(scratch), _ptr(params), _ptr(nlv), _stream(stream)))


def dbmp_structure_reinit(image, u_pos, u_theta, n_color, s_min, s_max, sigma_c, nu, threshold, params,
                          adam_m=None, adam_v=None, count=None, scratch=None, mask=None, stream=None):
    """Redraws every primitive of params (N, 8, in place) whose sigmoid(nu) < threshold."""
    _, H, W = image.shape
    if scratch is None:
        scratch = torch.empty(dbmp_structure_init_scratch_bytes(H, W), dtype=torch.uint8, device=image.device)
    _check(load().dbmp_structure_reinit(_ptr(image), _ptr(mask), H, W, params.shape[0], _ptr(u_pos), _ptr(u_theta),
                                        _ptr(n_color), float(s_min), float(s_max), float(sigma_c), float(nu),
                                        float(threshold), _ptr(scratch), _ptr(params), _ptr(adam_m), _ptr(adam_v),
                                        _ptr(count), _stream(stream)))


def dbmp_render_alpha(T_final, alpha, stream=None):
    """alpha = 1 - T_final (the rendered alpha channel), in the library."""
    if T_final.numel() != alpha.numel():
        raise ValueError("T_final and alpha differ in size")
    _check(load().dbmp_render_alpha(_ptr(T_final), _ptr(alpha), T_final.numel(), _stream(stream)))
    return alpha


def dbmp_alpha_loss_grad(image, T_final, target, target_alpha, lambda_alpha, dL_dimage, dL_dalpha, loss,
                         stream=None):
    _check(load().dbmp_alpha_loss_grad(_ptr(image), _ptr(T_final), _ptr(target), _ptr(target_alpha),
                                       T_final.numel(), float(lambda_alpha), _ptr(dL_dimage), _ptr(dL_dalpha),
                                       _ptr(loss), _stream(stream)))


def dbmp_blur_bitmaps(texels, sigma, out=None, stream=None):
    """Gaussian blur (radius ceil(3 sigma), zero padding) of every bitmap of
    texels (n_bmp, H_b, W_b) float32 CUDA; returns out."""
    if texels.dim() == 2:
        texels = texels[None]
    if out is None:
        out = torch.empty_like(texels)
    n, H, W = texels.shape
    _check(load().dbmp_blur_bitmaps(_ptr(texels), n, H, W, float(sigma), _ptr(out), _stream(stream)))
    return out


def dbmp_bin_stats(ws, stream=None):
    """Scaling statistics of the workspace's last binning as a dict (histograms as lists)."""
    st = DbmpBinStats()
    _check(load().dbmp_bin_stats(ws, _stream(stream), ctypes.byref(st)))
    out = {f: getattr(st, f) for f in ("n_listed", "pairs", "tau_max", "d_max", "n_tiles", "empty_tiles")}
    for f in ("tau_hist", "d_hist", "foot_hist"):
        out[f] = list(getattr(st, f))
    return out
