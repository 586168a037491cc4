"""Learned proposal network (training, inference) and the refinement that follows
it, over the libdbmp C ABI.  Training pairs are rendered on the fly by the
batched rasterizer from seeded anchored parameter sets (100k pairs would be ~79 GB
of images if stored)."""
from __future__ import annotations

import json
import math
import time

import numpy as np
import torch

from . import dbmp as D
from . import inputs

SIDE = 256
N_PRIMS = 512


class SceneRenderer:
    """Renders batches of 256 x 256 anchored scenes (512 soft discs each) with one
    batched plan: bin + persistent forward for all canvases in a few launches."""

    def __init__(self, max_batch, atlas_np=None, background=(1.0, 1.0, 1.0)):
        self.atlas_np = inputs.soft_disc_atlas(7, 1, 64) if atlas_np is None else atlas_np
        self.atlas = D.dbmp_atlas_create(torch.from_numpy(self.atlas_np).cuda())
        self.max_batch = max_batch
        n_tiles = max_batch * (SIDE // 8) ** 2
        self.ws = D.dbmp_workspace_create(max_batch * N_PRIMS, n_tiles, max_batch * N_PRIMS * 64, max_batch)
        self.bg = D.make_background(background)
        self.bid = torch.zeros(max_batch * N_PRIMS, dtype=torch.int32, device="cuda")
        self.T = torch.empty(max_batch * SIDE * SIDE, device="cuda")
        self.nl = torch.empty(max_batch * SIDE * SIDE, dtype=torch.int32, device="cuda")
        self.B = None

    def render(self, params, out):
        """params: (B, 512, 8) CUDA float32 -> out: (B, 3, 256, 256) CUDA float32."""
        B = params.shape[0]
        if B != self.B:
            D.dbmp_batch_plan(self.ws, [SIDE] * B, [SIDE] * B, [N_PRIMS * b for b in range(B + 1)], 16, 32, 2)
            self.B = B
        D.dbmp_batch_render(self.ws, params.reshape(-1, 8), self.bid[:B * N_PRIMS], self.atlas, 1.0, self.bg,
                            1e-6, D.BATCH_BIN | D.BATCH_FWD, out, self.T[:B * SIDE * SIDE],
                            self.nl[:B * SIDE * SIDE])
        return out

    def close(self):
        torch.cuda.synchronize()
        D.dbmp_workspace_destroy(self.ws)
        D.dbmp_atlas_destroy(self.atlas)


class Proposer:
    def __init__(self, max_batch=64, seed=0):
        self.handle = D.dbmp_proposer_create(max_batch)
        self.max_batch = max_batch
        D.dbmp_proposer_set_params(self.handle, inputs.cnn_init(seed))
        self.loss = torch.zeros(1, dtype=torch.float64, device="cuda")

    def set_params(self, theta):
        D.dbmp_proposer_set_params(self.handle, theta)

    def params(self):
        return D.dbmp_proposer_get(self.handle, 0)

    def grads(self):
        return D.dbmp_proposer_get(self.handle, 1)

    def activations(self, layer, batch):
        """Layer 0..6 activations of the last forward of `batch` images (testing aid)."""
        return D.dbmp_proposer_activations(self.handle, layer, batch)

    def propose(self, images):
        out = torch.empty(images.shape[0], N_PRIMS, 8, device="cuda")
        D.dbmp_propose(self.handle, images.contiguous(), out)
        return out

    def train_step(self, images, target_params, lr=None):
        adam = None if lr is None else (lr, 0.9, 0.999, 1e-8)
        D.dbmp_proposer_train_step(self.handle, images.contiguous(), target_params.contiguous(), self.loss, adam)
        return self.loss

    def close(self):
        if self.handle:
            torch.cuda.synchronize()
            D.dbmp_proposer_destroy(self.handle)
            self.handle = None


def train(prop: Proposer, scenes: SceneRenderer, n_pairs, batch, seed=1000, lr=1e-3, lr_end=1e-4, log_every=0):
    """Trains on n_pairs freshly rendered (image, parameters) pairs; returns the
    per-step losses (synchronised every log_every steps, 0 = only at the end)."""
    steps = max(1, n_pairs // batch)
    img = torch.empty(batch, 3, SIDE, SIDE, device="cuda")
    losses = []
    pinned = torch.empty(batch, N_PRIMS, 8).pin_memory()
    for t in range(steps):
        pinned.copy_(torch.from_numpy(inputs.anchored(seed + t, batch)))
        tp = pinned.cuda(non_blocking=True)
        scenes.render(tp, img)
        a = t / max(steps - 1, 1)
        cur_lr = lr * (lr_end / lr) ** a
        loss = prop.train_step(img, tp, cur_lr)
        if log_every and (t % log_every == 0 or t == steps - 1):
            losses.append(float(loss.item()))
    torch.cuda.synchronize()
    if not losses:
        losses.append(float(prop.loss.item()))
    return losses


def time_to(psnrs, times, goal):
    for p, t in zip(psnrs, times):
        if p >= goal:
            return t
    return None


def refine(init_params, target_image, atlas, steps=200, lr=0.1, background=(1.0, 1.0, 1.0), t0=None,
           psnr_goal=30.0, bitmap_id=None, log=None, stop_at=None):
    """The plain method: Adam on all primitive parameters of one 256^2 canvas against
    target_image (3, 256, 256).  Returns (psnr per step, seconds per step since t0,
    seconds to reach psnr_goal or None, final params).  With `log` (a writable text
    file) each step appends one JSON line {"step", "loss", "psnr", "s"}.  With
    `stop_at` the run ends at the first step whose PSNR reaches it."""
    params = init_params.reshape(N_PRIMS, 8).contiguous().clone()
    bid = torch.zeros(N_PRIMS, dtype=torch.int32, device="cuda") if bitmap_id is None else bitmap_id
    ws = D.dbmp_workspace_create(N_PRIMS, (SIDE // 16) ** 2, N_PRIMS * 256, 1)
    bg = D.make_background(background)
    image = torch.empty(3, SIDE, SIDE, device="cuda")
    T = torch.empty(SIDE, SIDE, device="cuda")
    nl = torch.empty(SIDE, SIDE, dtype=torch.int32, device="cuda")
    dL = torch.empty_like(image)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    g = torch.zeros(N_PRIMS, 8, device="cuda")
    m = torch.zeros_like(g)
    v = torch.zeros_like(g)
    step = torch.zeros(1, dtype=torch.int32, device="cuda")
    cfg = D.adam_config(lr=lr, gamma=0.1 ** (1.0 / steps), zero_grad=True)
    psnrs, times, hit = [], [], None
    t0 = time.perf_counter() if t0 is None else t0
    try:
        for _ in range(steps + 1):
            D.dbmp_bin(ws, SIDE, SIDE, 16, params, bid, N_PRIMS, atlas, 1.0)
            D.dbmp_render_fwd(ws, atlas, bg, 1e-6, image, T, nl)
            D.dbmp_mse_grad(image, target_image, dL, loss)
            mse = loss.item()
            ps = 10.0 * math.log10(1.0 / max(mse, 1e-30))
            psnrs.append(ps)
            times.append(time.perf_counter() - t0)
            if log is not None:
                log.write(json.dumps({"step": len(psnrs) - 1, "loss": mse, "psnr": ps, "s": times[-1]}) + "\n")
            if hit is None and ps >= psnr_goal:
                hit = times[-1]
            if len(psnrs) > steps or (stop_at is not None and ps >= stop_at):
                break
            D.dbmp_render_bwd(ws, atlas, bg, 1e-6, dL, None, T, nl, g)
            D.dbmp_adam_step(params, g, m, v, step, cfg)
    finally:
        torch.cuda.synchronize()
        D.dbmp_workspace_destroy(ws)
    return psnrs, times, hit, params


def structure_init(target, seed, N=N_PRIMS, s_range=inputs.ANCHOR_SCALE, sigma_c=0.02, nu=-2.0, scratch=None):
    """The paper's structure-aware initialisation of N primitives from target
    (3, H, W) on the GPU (Sec. 3.2; Tab. S1 window 7, base probability 0.1,
    colour std 0.02; nu = -2 as in the text), with seeded random draws."""
    u, ut, nc = inputs.init_draws(seed, N)
    dev = target.device
    params = torch.empty(N, 8, device=dev)
    D.dbmp_structure_init(target.contiguous(), torch.from_numpy(u).to(dev), torch.from_numpy(ut).to(dev),
                          torch.from_numpy(nc).to(dev), s_range[0], s_range[1], sigma_c, nu, params,
                          scratch=scratch)
    return params


def cnn_train_flops(batch):
    """Algorithmic FLOPs of one training step of the network (forward, input and
    weight gradients; no input gradient for the first layer), with the 3 real
    input channels of the first layer."""
    f = 0
    side = 256
    for li, (cin_pad, cin, cout, k) in enumerate(inputs.CNN_LAYERS):
        so = side // 2 if k == 4 else side
        macs = batch * so * so * cout * k * k * cin
        f += 2 * macs * (2 if li == 0 else 3)
        side = so
    return f
