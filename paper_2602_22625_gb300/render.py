"""Renderer objects and the autograd wrapper over the libdbmp C ABI.

Everything here manages handles and tensors and calls the ABI; the compositing,
its gradient, the loss and the optimiser all run in libdbmp's kernels.
"""
from __future__ import annotations

import torch

from . import dbmp as D


class Atlas:
    """Device sampling layout of a bitmap atlas (float32 [n_bmp, H_b, W_b], values in [0, 1])."""

    def __init__(self, texels: torch.Tensor):
        if texels.dim() == 2:
            texels = texels[None]
        texels = texels.to(device="cuda", dtype=torch.float32).contiguous()
        self.n_bmp, self.Hb, self.Wb = texels.shape
        self.handle = D.dbmp_atlas_create(texels)

    def update(self, texels: torch.Tensor):
        D.dbmp_atlas_update(self.handle, texels.to(device="cuda", dtype=torch.float32).contiguous())

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            try:
                D.dbmp_atlas_destroy(h)
            except Exception:
                pass
            self.handle = None


class Workspace:
    def __init__(self, max_prims: int, max_tiles: int, max_pairs: int, max_canvases: int = 1):
        self.limits = (int(max_prims), int(max_tiles), int(max_pairs), int(max_canvases))
        self.handle = D.dbmp_workspace_create(*self.limits)
        self.generation = 0

    def status(self, raise_on_error=True):
        return D.dbmp_status_poll(self.handle, raise_on_error=raise_on_error)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            try:
                torch.cuda.synchronize()
                D.dbmp_workspace_destroy(h)
            except Exception:
                pass
            self.handle = None


def tiles_of(H, W, tile):
    return (-(-W // tile)) * (-(-H // tile))


class Renderer:
    """Renders one H x W canvas of bitmap primitives (forward + backward).

    background: None (Eq. 5), an RGB triple, or a (3, H, W) CUDA tensor (Eq. 8).
    T_stop: early-termination threshold (image error <= T_stop; 0 = exact).
    check: False (default) queues work only, so forward and backward never
    synchronise the host and can be captured in a CUDA graph; a tile-list capacity
    overflow then leaves the outputs unwritten and is reported by status().  True:
    poll the device status after every binning (one synchronisation) and grow the
    tile-list capacity when it overflowed.
    """

    def __init__(self, H, W, atlas: Atlas, max_prims, tile=16, alpha_max=1.0,
                 background=(1.0, 1.0, 1.0), T_stop=1e-6, max_pairs=None, check=False):
        self.H, self.W, self.tile = int(H), int(W), int(tile)
        self.atlas = atlas
        self.alpha_max = float(alpha_max)
        self.background = background
        self.bg = D.make_background(background, H, W)
        self.T_stop = float(T_stop)
        self.check = check
        self.max_prims = int(max_prims)
        n_tiles = tiles_of(H, W, tile)
        if max_pairs is None:
            max_pairs = max(1 << 20, 32 * self.max_prims)
        self.ws = Workspace(self.max_prims, n_tiles, max_pairs)
        self._binned = None

    @property
    def generation(self):
        return self.ws.generation

    def bin(self, params: torch.Tensor, bitmap_id: torch.Tensor):
        N = params.shape[0]
        if N > self.max_prims:
            raise ValueError(f"{N} primitives > max_prims {self.max_prims}")
        D.dbmp_bin(self.ws.handle, self.H, self.W, self.tile, params, bitmap_id, N, self.atlas.handle,
                   self.alpha_max)
        self.ws.generation += 1
        if self.check:
            st = D.dbmp_status_poll(self.ws.handle, raise_on_error=False)
            if st.code == D.DBMP_ERR_CAPACITY:
                need = int(st.pairs_required * 1.25) + 1024
                lim = self.ws.limits
                self.ws = Workspace(lim[0], lim[1], need, lim[3])
                D.dbmp_bin(self.ws.handle, self.H, self.W, self.tile, params, bitmap_id, N,
                           self.atlas.handle, self.alpha_max)
                self.ws.generation += 1
                D.dbmp_status_poll(self.ws.handle)
            elif st.code != D.DBMP_OK:
                D._check(st.code)
        self._binned = (params, bitmap_id)
        return self.ws.generation

    def forward(self, params, bitmap_id, out=None):
        params = params.contiguous()
        bitmap_id = bitmap_id.to(torch.int32).contiguous()
        self.bin(params, bitmap_id)
        if out is None:
            dev = params.device
            out = (torch.empty(3, self.H, self.W, device=dev), torch.empty(self.H, self.W, device=dev),
                   torch.empty(self.H, self.W, device=dev, dtype=torch.int32))
        image, T_final, n_last = out
        D.dbmp_render_fwd(self.ws.handle, self.atlas.handle, self.bg, self.T_stop, image, T_final, n_last)
        return image, T_final, n_last

    def backward(self, dL_dimage, T_final, n_last, dL_dalpha=None, dparams=None):
        N = self._binned[0].shape[0]
        if dparams is None:
            dparams = torch.zeros(N, 8, device=dL_dimage.device)
        D.dbmp_render_bwd(self.ws.handle, self.atlas.handle, self.bg, self.T_stop, dL_dimage.contiguous(),
                          None if dL_dalpha is None else dL_dalpha.contiguous(), T_final, n_last, dparams)
        return dparams

    def status(self):
        return self.ws.status()


class RenderFunction(torch.autograd.Function):
    """image (3,H,W), alpha (H,W) = render(params (N,8)); gradients w.r.t. params.

    The forward saves T_final and n_last only; the backward recovers per-layer
    transmittance on the fly.  If the renderer's workspace was re-binned in between
    (another forward), the backward re-bins the saved parameters first (binning is
    deterministic, so the lists are identical)."""

    @staticmethod
    def forward(ctx, params, bitmap_id, renderer: Renderer):
        image, T_final, n_last = renderer.forward(params.detach(), bitmap_id)
        ctx.renderer = renderer
        ctx.gen = renderer.generation
        ctx.save_for_backward(params.detach(), bitmap_id, T_final, n_last)
        alpha = D.dbmp_render_alpha(T_final, torch.empty_like(T_final))
        return image, alpha

    @staticmethod
    def backward(ctx, g_image, g_alpha):
        params, bitmap_id, T_final, n_last = ctx.saved_tensors
        r = ctx.renderer
        if r.generation != ctx.gen or r._binned is None or r._binned[0].data_ptr() != params.data_ptr():
            r.bin(params, bitmap_id)
        if g_image is None:
            g_image = torch.zeros(3, r.H, r.W, device=params.device)
        dparams = r.backward(g_image, T_final, n_last, g_alpha)
        return dparams, None, None


def render(params, bitmap_id, renderer: Renderer):
    """Differentiable render: returns (image (3,H,W), alpha (H,W) = 1 - T_final)."""
    return RenderFunction.apply(params, bitmap_id.to(torch.int32), renderer)
