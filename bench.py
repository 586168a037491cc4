#!/usr/bin/env python
"""Benchmark of one optimisation step of the bitmap-primitive rasterizer.

Workload: 1024 x 1024 FP32 canvas, 20 000 primitives over 16 procedural stroke
bitmaps of 128 x 128 (seeded Bezier strokes, Gaussian-blurred), scale
LogNormal(-2, 0.7) of the canvas side, uniform rotation and colour, opacity
U[0.2, 1], fixed depth order, MSE against a seeded target render.

One step = the whole hot path: binning (preprocess, tile lists), forward
composite, MSE gradient, backward composite, Adam update.  Prints ONE JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl dbmp|reference]

--impl reference times the FP64 CPU oracle (the correctness reference) on the
host cores, one bounded sample of rows per step, scaled to the full canvas.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+bwd ms/step at 1024^2 x 20k prims"
WORKLOAD = "main_1024sq_20k"
L2_FLUSH_BYTES = 512 << 20
T_STOP = 1e-6

# Algorithmic FP32 operations (FMA = 2) per contributing (pixel, primitive) pair, the
# unit of work: a pair with alpha > 0 composited before the pixel saturated.  Pairs
# whose bitmap sample is zero change nothing and are not counted.
FLOPS_SAMPLE = 21       # Eqs. 1-2 and the bilinear sample (Eqs. S1-S3)
FLOPS_COMPOSITE = 10    # Eqs. 3-5 (alpha, over, transmittance)
FLOPS_GRAD = 44         # Eq. 6, S4, S5 terms and the reverse recursion
FLOPS_FWD_PAIR = FLOPS_SAMPLE + FLOPS_COMPOSITE
FLOPS_BWD_PAIR = FLOPS_SAMPLE + FLOPS_GRAD
FP32_LANES = 128        # FP32 multiply-add lanes per SM (4 sub-partitions x 32)

# kernels one step launches (bin: prep, count, colscan, tilescan with the tile ordering, scatter;
# fwd with the MSE loss in its epilogue; bwd, finalize; adam, step counter)
LAUNCHES_PER_STEP = 10


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="dbmp", choices=["dbmp", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-ablation", action="store_true",
                    help="skip the soft-rasterisation ablation and the spatial-constraint comparison")
    ap.add_argument("--learned-pairs", type=int, default=100_000)
    ap.add_argument("--tile", type=int, default=16)
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--ppt", type=int, default=2)
    ap.add_argument("--ppt-bwd", type=int, default=0, help="pixels per lane of the backward (0: --ppt)")
    ap.add_argument("--shard", default="replicas", choices=["replicas", "bands"],
                    help="N > 1: replicas = one canvas per rank (weak scaling, no exchange); bands = one canvas "
                         "split into bands of tile rows, the gradient summed by one all-reduce per step "
                         "(strong scaling)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_seeds(rank):
    """Seeds of a rank's own canvas and target: every rank renders a workload of the
    same shape and distribution (weak scaling, no exchange)."""
    return 2 + rank, 1002 + rank


def max_over_ranks(values, device, world):
    """Element-wise maximum of `values` (floats) over all ranks (the slowest rank's
    time); a plain copy when world == 1."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], device=device, dtype=torch.float64)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def config(extra=None):
    c = {"workload": WORKLOAD, "H": 1024, "W": 1024, "N": 20000, "atlas": "16 strokes 128x128",
         "scale": "LogNormal(-2,0.7)*W", "T_stop": T_STOP, "background": "white",
         "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MB memset, outside the timed region)"}
    if extra:
        c.update(extra)
    return c


# ---------------------------------------------------------------------------
# CPU oracle leg
# ---------------------------------------------------------------------------

def oracle_band_step(sc, target, y0, y1):
    """FP64 oracle forward + backward of the rows y0..y1 of the workload (MSE vs target)."""
    import numpy as np
    import oracle
    ys, xs = np.mgrid[y0:y1, 0:sc.W]
    out = oracle.render(sc.H, sc.W, sc.params, sc.bitmap_id, sc.atlas, background=sc.background,
                        T_stop=T_STOP, pixels=(xs.ravel(), ys.ravel()))
    img = out["image"].reshape(3, y1 - y0, sc.W)
    gI = np.zeros((3, sc.H, sc.W))
    gI[:, y0:y1] = 2.0 * (img - target[:, y0:y1]) / (3 * sc.H * sc.W)
    oracle.grad_rows(sc.H, sc.W, sc.params, sc.bitmap_id, sc.atlas, gI, y0, y1,
                     background=sc.background, T_stop=T_STOP)


def oracle_target(sc_t):
    import numpy as np  # noqa: F401
    import oracle
    return oracle.render(sc_t.H, sc_t.W, sc_t.params, sc_t.bitmap_id, sc_t.atlas,
                         background=sc_t.background)["image"]


def cpu_baseline(min_s=10.0, max_reps=40):
    """The oracle as it stands on the host cores: fwd + bwd of the whole canvas in
    FP64, repeated until at least min_s seconds of CPU work (bounded sample)."""
    import oracle
    from paper_2602_22625_gb300 import inputs
    sc = inputs.main(seed=2)
    ts = inputs.main(seed=1002)
    tgt = oracle.render(ts.H, ts.W, ts.params, ts.bitmap_id, ts.atlas, background=ts.background,
                        T_stop=T_STOP)["image"]   # input data only: not timed
    times = []
    while sum(times) < min_s and len(times) < max_reps:
        t0 = time.perf_counter()
        oracle_band_step(sc, tgt, 0, sc.H)
        times.append(time.perf_counter() - t0)
    cores = oracle.num_threads()
    # one core: a band of rows through the canvas centre, scaled to the whole canvas
    rows = 32
    y0 = sc.H // 2 - rows // 2
    oracle.set_num_threads(1)
    try:
        t0 = time.perf_counter()
        oracle_band_step(sc, tgt, y0, y0 + rows)
        one = (time.perf_counter() - t0) * sc.H / rows
    finally:
        oracle.set_num_threads(cores)
    return {"value": statistics.mean(times) * 1e3, "unit": "ms", "cores": cores, "kind": "oracle",
            "sample": f"the whole {sc.H}x{sc.W} canvas, fwd+bwd in FP64 (T_stop={T_STOP}), {len(times)} "
                      f"repetitions, {sum(times):.1f} s of CPU work",
            "one_core": {"value": one * 1e3, "unit": "ms", "cores": 1,
                         "sample": f"rows {y0}..{y0 + rows} of {sc.H}, fwd+bwd in FP64, scaled x{sc.H // rows} "
                                   f"to the whole canvas"}}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import numpy as np
    import oracle
    from paper_2602_22625_gb300 import inputs
    sc = inputs.main(seed=2)
    tgt_sc = inputs.main(seed=1002)
    rows = 16
    y0 = sc.H // 2 - rows // 2
    ys, xs = np.mgrid[y0:y0 + rows, 0:sc.W]
    tgt = np.zeros((3, sc.H, sc.W))
    tgt[:, y0:y0 + rows] = oracle.render(tgt_sc.H, tgt_sc.W, tgt_sc.params, tgt_sc.bitmap_id,
                                         tgt_sc.atlas, background=tgt_sc.background,
                                         pixels=(xs.ravel(), ys.ravel()))["image"].reshape(3, rows, sc.W)
    for _ in range(args.warmup):
        oracle_band_step(sc, tgt, y0, y0 + rows)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle_band_step(sc, tgt, y0, y0 + rows)
        times.append((time.perf_counter() - t0) * 1e3 * sc.H / rows)
    v = statistics.mean(times)
    cores = oracle.num_threads()
    line = {"metric": METRIC, "value": v, "unit": "ms", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": v, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": config({"tile": None}),
            "cpu_baseline": {"value": v, "unit": "ms", "cores": cores, "kind": "oracle",
                             "sample": f"each step: rows {y0}..{y0 + rows} of 1024, fwd+bwd FP64, "
                                       f"scaled x{sc.H // rows} to the full canvas"},
            "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU leg
# ---------------------------------------------------------------------------

class Clocks:
    """Samples SM clock and throttle reasons with nvidia-smi while the timed loop runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        busy = [s for s in sm if mx and s > 0.5 * mx] or sm
        return {"sm_mhz": statistics.median(busy) if busy else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def binning_hbm(N, K, n_tiles, bin_ms):
    """The binning pass against the HBM roofline: its algorithmic bytes are the
    parameters and bitmap ids read (36 B per primitive), the records written for the
    compositors (48 B per primitive), the tile lists (4 B per entry) and the tile
    offsets (8 B per tile)."""
    peak, source = hbm_peak_gbs()
    nbytes = 36 * N + 48 * N + 4 * K + 8 * (n_tiles + 1)
    achieved = nbytes / (bin_ms * 1e-3) / 1e9
    return {"bytes": nbytes, "ms": bin_ms, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_source": source}


def hbm_peak_gbs():
    """(GB/s, where it comes from): the measured copy bandwidth, else the fallback."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (copy, measured)"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback: 6.8 TB/s, one earlier copy measurement on a GB300"   # no measured file


def fp32_peak(local):
    """The FP32 rate the compositors' ALU roofline divides by, measured on this GPU:
    dbmp_fp32_peak's independent multiply-add chains with scalar FFMA and with packed
    FP32x2 FMA instructions, clocks sampled meanwhile.  peak = the faster form.  Also
    the figure derived from the queried SM count, 128 FP32 lanes and the maximum SM
    clock, for comparison."""
    import torch
    from paper_2602_22625_gb300 import microbench
    with Clocks(local) as clk:
        r = microbench.fp32(iters=20000, reps=25)
    c = clk.summary()
    mx = c.get("sm_max_mhz") or 2070.0
    derived = r["sms"] * FP32_LANES * 2 * mx * 1e6 / 1e12
    best = "ffma2" if r["ffma2_tflops"] > r["ffma_tflops"] else "ffma"
    return {"peak": r[f"{best}_tflops"], "ffma_tflops": r["ffma_tflops"], "ffma2_tflops": r["ffma2_tflops"],
            "sms": r["sms"], "sm_mhz": c.get("sm_mhz"), "sm_max_mhz": mx, "reasons": c.get("reasons"),
            "derived_tflops": derived,
            "source": f"measured: dbmp_fp32_peak ({best}), {r['sms']} SMs x 8 CTAs x 256 threads x 16 "
                      f"independent chains, median SM clock {c.get('sm_mhz')} MHz",
            "device": torch.cuda.get_device_name(local)}


def traffic_for(kernel_key, tile, batch, ppt):
    """DRAM bytes per launch from the committed ncu summary, if it still matches the
    source and was taken at this tuning (tile, batch, the pass' pixels per lane)."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p))
        e = d.get(kernel_key)
        if not e or (e.get("tile"), e.get("batch"), e.get("ppt")) != (tile, batch, ppt):
            return None
        # the kernel's source files (the compositors and the header of their device definitions)
        names = e.get("sources") or [e["source"]]
        src = b"".join(open(os.path.join(ROOT, "paper_2602_22625_gb300", "csrc", n), "rb").read() for n in names)
        if hashlib.sha256(src).hexdigest() != e["sha256"]:
            return None
        return e["bytes_per_launch"]
    except Exception:
        return None


def c1_style_targets(seed, n):
    """Out-of-distribution targets for the learned initialiser: C1-style scenes (256
    soft discs with scale U[0.1, 0.5] of the side, i.e. 26-128 px against the 6-14 px
    the network was trained on, uniform positions, heavy overlap), padded to 512
    primitives with invisible ones (opacity logit -30)."""
    import numpy as np
    from paper_2602_22625_gb300 import inputs
    out = np.zeros((n, 512, 8), np.float32)
    for i in range(n):
        p, _ = inputs.primitives(seed + i, 256, 256, 256, 1, "uniform", (0.1, 0.5))
        out[i, :256] = p
        out[i, 256:, 2] = 1.0
        out[i, 256:, 4] = -30.0
    return out


def learned_vs_plain(n_pairs, batch=64, n_targets=8, steps=3000, n_ood=4):
    """Trains the proposal network on n_pairs freshly rendered anchored scenes, then
    on held-out targets times each arm to 30 dB (and 25, 20 dB): learned = propose +
    refinement, plain = random init + refinement, structure = the paper's
    structure-aware initialisation + refinement, with nu = -2 (the text) and nu = -4
    (Tab. S1 v_init_bias), scale range [6, 14] px (the targets' scale law).  Every arm
    has the same budget of `steps` refinement steps and stops at 30 dB.  The same arms
    run on n_ood out-of-distribution C1-style targets.  Also times the network's
    training step on the tensor cores and the initialisation kernels."""
    import numpy as np
    import torch
    from paper_2602_22625_gb300 import dbmp as D
    from paper_2602_22625_gb300 import inputs, proposer

    scenes = proposer.SceneRenderer(max_batch=batch)
    P = proposer.Proposer(max_batch=batch, seed=0)
    try:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        losses = proposer.train(P, scenes, n_pairs, batch, seed=10_000, lr=5e-4, lr_end=5e-5,
                                log_every=max(1, n_pairs // batch // 8))
        train_s = time.perf_counter() - t0
        # tensor-core training step alone (images already rendered)
        imgs = torch.empty(batch, 3, 256, 256, device="cuda")
        tp = torch.from_numpy(inputs.anchored(123, batch)).cuda()
        scenes.render(tp, imgs)
        for _ in range(3):
            P.train_step(imgs, tp, 1e-6)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        reps = 20
        for _ in range(reps):
            P.train_step(imgs, tp, 1e-6)
        e1.record()
        e1.synchronize()
        step_ms = e0.elapsed_time(e1) / reps
        flops = proposer.cnn_train_flops(batch)
        # the structure-aware initialisation kernels alone (one 256^2 target, 512 draws)
        held = torch.from_numpy(inputs.anchored(777_001, n_targets)).cuda()
        targets = torch.empty(n_targets, 3, 256, 256, device="cuda")
        scenes.render(held, targets)
        scratch = torch.empty(D.dbmp_structure_init_scratch_bytes(256, 256), dtype=torch.uint8, device="cuda")
        for _ in range(3):
            proposer.structure_init(targets[0], 1, scratch=scratch)
        e0.record()
        for _ in range(reps):
            proposer.structure_init(targets[0], 1, scratch=scratch)
        e1.record()
        e1.synchronize()
        init_ms = e0.elapsed_time(e1) / reps

        def run_arms(tgts, rand, seed0):
            arms = {"learned": [], "plain": [], "structure_nu-2": [], "structure_nu-4": []}
            for i in range(tgts.shape[0]):
                runs = (("learned", lambda: P.propose(tgts[i:i + 1])[0]), ("plain", lambda: rand[i]),
                        ("structure_nu-2", lambda: proposer.structure_init(tgts[i], seed0 + i, nu=-2.0)),
                        ("structure_nu-4", lambda: proposer.structure_init(tgts[i], seed0 + i, nu=-4.0)))
                for arm, init_fn in runs:
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()   # the clock includes the initialisation
                    init = init_fn()
                    arms[arm].append(proposer.refine(init, tgts[i], scenes.atlas, steps, t0=t0, stop_at=30.0)[:2])
            res = {}
            for arm, rs in arms.items():
                for goal in (20.0, 25.0, 30.0):
                    ts = [proposer.time_to(ps, tm, goal) for ps, tm in rs]
                    hit = [t for t in ts if t is not None]
                    res[f"{arm}_reached_{int(goal)}db"] = f"{len(hit)}/{len(ts)}"
                    res[f"{arm}_median_s_to_{int(goal)}db"] = float(np.median(hit)) if len(hit) == len(ts) else None
                    res[f"{arm}_median_steps_to_{int(goal)}db"] = (
                        float(np.median([next(k for k, p in enumerate(ps) if p >= goal) for ps, _ in rs]))
                        if len(hit) == len(ts) else None)
                res[f"{arm}_psnr_start"] = float(np.median([ps[0] for ps, _ in rs]))
                res[f"{arm}_psnr_best"] = float(np.median([max(ps) for ps, _ in rs]))
            a, b = res["learned_median_s_to_30db"], res["plain_median_s_to_30db"]
            res["plain_over_learned_s_to_30db"] = (b / a) if a and b else None
            return res

        rand = torch.from_numpy(inputs.random_init(777_002, n_targets)).cuda()
        out = {"pairs": n_pairs, "batch": batch, "train_s": train_s, "train_loss": [losses[0], losses[-1]],
               "targets": n_targets, "refine_steps_budget": steps, "stop": "at 30 dB",
               "cnn_train_step_ms": step_ms, "cnn_train_tflops": flops / (step_ms * 1e-3) / 1e12,
               "cnn_train_frac_of_bf16_peak": flops / (step_ms * 1e-3) / 1e12 / bf16_peak_tflops()[0],
               "structure_init_ms": init_ms,
               "structure_init": "Sec. 3.2 structure-aware: 7x7 local variance, draws ~ 0.1 + 0.9 NLV, "
                                 "s in [6, 14] by NLV, nu = -2 (text) or -4 (Tab. S1), colour std 0.02 "
                                 "(includes the draws' upload)"}
        out.update(run_arms(targets, rand, 777_100))
        if n_ood:
            ood = torch.from_numpy(c1_style_targets(888_000, n_ood)).cuda()
            tg = torch.empty(n_ood, 3, 256, 256, device="cuda")
            scenes.render(ood, tg)
            rand2 = torch.from_numpy(inputs.random_init(888_100, n_ood)).cuda()
            out["out_of_distribution"] = dict(run_arms(tg, rand2, 888_200), targets=n_ood,
                                              scenes="C1-style: 256 soft discs, scale U[0.1, 0.5] x 256 px, "
                                                     "uniform positions (the network saw 6-14 px anchored discs)")
        return out
    finally:
        P.close()
        scenes.close()


def bf16_peak_tflops():
    """(TFLOP/s, where it comes from): the measured cuBLAS bf16 burst rate, else the fallback."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["bf16_tflops"]), "MEASURED_PEAKS.json bf16_tflops (burst, measured)"
    except (OSError, ValueError, KeyError):
        return 1900.0, "fallback: 1.9 PFLOP/s bf16 burst, one earlier measurement on a GB300"


def other_workload(name, peak_tflops, steps=5, warmup=3):
    """One optimisation step (bin, forward with the fused MSE, backward, Adam) of the
    batched workload (64 canvases, side U{256..1024}, N log-uniform [1k, 50k], one
    plan and one persistent launch per pass) or the stress workload (2048^2, 200k
    primitives, Pareto scales), autotuned, L2 flushed between timed steps; the target
    is a render of other seeds.  Returns ms per step, the phases, the work and the
    backward against the derived FP32 peak."""
    import numpy as np
    import torch
    from paper_2602_22625_gb300 import dbmp as D
    from paper_2602_22625_gb300 import inputs
    dev = torch.device("cuda")
    if name == "batched":
        scenes = inputs.batched(seed=4)
        # targets: the same canvases and primitive counts, other seeds (so one plan serves both)
        tparts = [inputs.primitives(7000 + c, s.N, s.H, s.W, s.atlas.shape[0], "lognormal", (-2.0, 0.7))
                  for c, s in enumerate(scenes)]
    else:
        scenes = [inputs.stress(seed=3)]
        t = inputs.stress(seed=1003)
        tparts = [(t.params, t.bitmap_id)]
    atlas_np = scenes[0].atlas
    P = np.concatenate([s.params for s in scenes])
    B = np.concatenate([s.bitmap_id for s in scenes]).astype(np.int32)
    tP = np.concatenate([p for p, _ in tparts])
    tB = np.concatenate([b for _, b in tparts]).astype(np.int32)
    off = [0] + [int(v) for v in np.cumsum([s.N for s in scenes])]
    Hs, Ws = [s.H for s in scenes], [s.W for s in scenes]
    N, pix = off[-1], sum(h * w for h, w in zip(Hs, Ws))
    atlas = D.dbmp_atlas_create(torch.from_numpy(atlas_np).to(dev))
    ws = D.dbmp_workspace_create(N, sum((h // 8) * (w // 8) for h, w in zip(Hs, Ws)), 400 << 20, len(Hs))
    try:
        bg = D.make_background((1.0, 1.0, 1.0))
        image = torch.empty(3 * pix, device=dev)
        T = torch.empty(pix, device=dev)
        nl = torch.empty(pix, dtype=torch.int32, device=dev)
        target = torch.empty(3 * pix, device=dev)
        dL = torch.empty(3 * pix, device=dev)
        loss = torch.zeros(1, dtype=torch.float64, device=dev)
        D.dbmp_batch_plan(ws, Hs, Ws, off, tile=32, batch=32, ppt=4)
        D.dbmp_batch_render(ws, torch.from_numpy(tP).to(dev), torch.from_numpy(tB).to(dev), atlas, 1.0, bg, 0.0,
                            D.BATCH_BIN | D.BATCH_FWD, target, T, nl)
        params = torch.from_numpy(P).to(dev)
        bid = torch.from_numpy(B).to(dev)
        dp = torch.zeros(N, 8, device=dev)
        m = torch.zeros_like(dp)
        v = torch.zeros_like(dp)
        step = torch.zeros(1, dtype=torch.int32, device=dev)
        D.dbmp_batch_render_mse(ws, params, bid, atlas, 1.0, bg, T_STOP, D.BATCH_BIN | D.BATCH_FWD, target, image,
                                T, nl, dL, loss)
        (t, b, pp, pb), _ = D.dbmp_autotune(ws, params, bid, atlas, 1.0, bg, T_STOP, D.BATCH_FWD | D.BATCH_BWD,
                                            image, T, nl, dL, dp, reps=3)
        dp.zero_()
        adam = D.adam_config(lr=0.1, gamma=0.1 ** (1.0 / 500), zero_grad=True)
        flush = torch.empty(L2_FLUSH_BYTES // 4, device=dev)
        st = torch.cuda.current_stream()

        def one(ev=None):
            if ev:
                ev[0].record(st)
            D.dbmp_batch_render(ws, params, bid, atlas, 1.0, bg, T_STOP, D.BATCH_BIN, None, T, nl)
            if ev:
                ev[1].record(st)
            D.dbmp_batch_render_mse(ws, params, bid, atlas, 1.0, bg, T_STOP, D.BATCH_FWD, target, image, T, nl,
                                    dL, loss)
            if ev:
                ev[2].record(st)
            D.dbmp_batch_render(ws, params, bid, atlas, 1.0, bg, T_STOP, D.BATCH_BWD, image, T, nl, dL, dp)
            if ev:
                ev[3].record(st)
            D.dbmp_adam_step(params, dp, m, v, step, adam)
            if ev:
                ev[4].record(st)

        for _ in range(warmup):
            one()
        # whole steps timed alone, then as many with an event between phases
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(steps)]
        evp = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(steps)]
        torch.cuda.synchronize()
        for k in range(steps):
            flush.zero_()
            evs[k][0].record(st)
            one()
            evs[k][1].record(st)
        for k in range(steps):
            flush.zero_()
            one(evp[k])
        torch.cuda.synchronize()
        step_ms = np.array([evs[k][0].elapsed_time(evs[k][1]) for k in range(steps)])
        ph = np.array([[evp[k][i].elapsed_time(evp[k][i + 1]) for i in range(4)] for k in range(steps)])
        s_ = D.dbmp_status_poll(ws)
        D.dbmp_workspace_count_pairs(ws, True)   # one counting forward for the work unit
        D.dbmp_batch_render(ws, params, bid, atlas, 1.0, bg, T_STOP, D.BATCH_BIN | D.BATCH_FWD, image, T, nl)
        s_ = D.dbmp_status_poll(ws)
        bwd = float(ph[:, 2].mean())
        bwd_tf = FLOPS_BWD_PAIR * s_.pairs_contributing / (bwd * 1e-3) / 1e12
        return {"workload": "batched_64_canvases" if name == "batched" else "stress_2048sq_200k",
                "canvases": len(Hs), "pixels": pix, "primitives": N, "tuning": [t, b, pp, pb],
                "ms_per_step": float(step_ms.mean()),
                "breakdown_ms": {"bin": float(ph[:, 0].mean()), "fwd_with_mse": float(ph[:, 1].mean()),
                                 "bwd": bwd, "adam": float(ph[:, 3].mean())},
                "pairs_contributing": s_.pairs_contributing, "tile_list_entries": s_.pairs_required,
                "bwd_tflops": bwd_tf, "bwd_frac_of_fp32_peak": bwd_tf / peak_tflops,
                "steps": steps, "l2": "flushed between timed steps"}
    finally:
        D.dbmp_workspace_destroy(ws)
        D.dbmp_atlas_destroy(atlas)


def blur_ablation(n_targets=4, steps=300, sigma=1.0):
    """Soft rasterisation (Sec. 3.2, Tab. S1 blur_sigma 1.0) on and off: targets are
    256^2 renders of 512 primitives with 16 hard-edged stroke bitmaps; the same random
    initialisation is refined against them with the hard atlas and with the atlas
    blurred on the GPU.  Reports the final PSNR of both arms and the blur kernel time."""
    import numpy as np
    import torch
    from paper_2602_22625_gb300 import dbmp as D
    from paper_2602_22625_gb300 import inputs, proposer

    hard_np = inputs.stroke_atlas(21, 16, 128, blur_sigma=0.0)
    hard_dev = torch.from_numpy(hard_np).cuda()
    soft_dev = D.dbmp_blur_bitmaps(hard_dev, sigma)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(20):
        D.dbmp_blur_bitmaps(hard_dev, sigma, out=soft_dev)
    e1.record()
    e1.synchronize()
    blur_ms = e0.elapsed_time(e1) / 20
    hard = D.dbmp_atlas_create(hard_dev)
    soft = D.dbmp_atlas_create(soft_dev)
    N, S = proposer.N_PRIMS, proposer.SIDE
    ws = D.dbmp_workspace_create(N, (S // 16) ** 2, N * 256, 1)
    bg = D.make_background((1.0, 1.0, 1.0))
    res = {"hard": [], "blurred": []}
    try:
        for k in range(n_targets):
            tp, tb = inputs.primitives(31_000 + k, N, S, S, 16, "uniform", (0.03, 0.08))
            tbid = torch.from_numpy(tb).cuda()
            tgt = torch.empty(3, S, S, device="cuda")
            T = torch.empty(S, S, device="cuda")
            nl = torch.empty(S, S, dtype=torch.int32, device="cuda")
            D.dbmp_bin(ws, S, S, 16, torch.from_numpy(tp).cuda(), tbid, N, hard, 1.0)
            D.dbmp_render_fwd(ws, hard, bg, 1e-6, tgt, T, nl)
            init = torch.from_numpy(inputs.random_init(32_000 + k, 1, N, S, S)[0]).cuda()
            bid = torch.from_numpy(inputs.rng(33_000 + k).integers(0, 16, N).astype(np.int32)).cuda()
            for arm, atlas in (("hard", hard), ("blurred", soft)):
                ps = proposer.refine(init, tgt, atlas, steps, bitmap_id=bid)[0]
                res[arm].append(ps[-1])
    finally:
        torch.cuda.synchronize()
        D.dbmp_workspace_destroy(ws)
        D.dbmp_atlas_destroy(hard)
        D.dbmp_atlas_destroy(soft)
    return {"targets": n_targets, "steps": steps, "sigma": sigma, "blur_ms_16x128sq": blur_ms,
            "psnr_final_hard": res["hard"], "psnr_final_blurred": res["blurred"],
            "median_gain_db": float(np.median(np.array(res["blurred"]) - np.array(res["hard"])))}


def spatial_constraint(steps=300, N=512, side=256, seed=41):
    """Spatially constrained rendering (Sec. 3.3.2, Sec. S3): an object (a 256^2 render
    of 512 opaque primitives placed inside a disc, its alpha 1 - T of that render) is
    fitted from the spatially constrained initialisation over a fresh uniform-noise
    background every iteration (Eq. 8).  Arms as in the paper's ablation: (a) masked
    MSE only, (b) + opacity loss (weight 0.3), (c) + re-initialisation of primitives
    with sigmoid(nu) < 0.3 every 50 iterations after a 199-iteration warm-up; all with
    the opacity learning-rate gain 5.  Reports the final PSNR over the object
    (alpha* > 0) and the mean |I_alpha - alpha*| over the canvas."""
    import numpy as np
    import torch
    from paper_2602_22625_gb300 import dbmp as D
    from paper_2602_22625_gb300 import inputs

    g = inputs.rng(seed)
    S = side
    atlas_np = inputs.soft_disc_atlas(7, 1, 64)
    atlas = D.dbmp_atlas_create(torch.from_numpy(atlas_np).cuda())
    ws = D.dbmp_workspace_create(N, (S // 8) ** 2, N * 512, 1)
    bid = torch.zeros(N, dtype=torch.int32, device="cuda")
    T = torch.empty(S, S, device="cuda")
    nl = torch.empty(S, S, dtype=torch.int32, device="cuda")
    out = {"steps": steps, "primitives": N, "canvas": S, "opacity_loss_weight": 0.3, "reinit": "sigmoid(nu) < 0.3 "
           "every 50 iterations after 199", "background": "U[0,1]^3 per pixel, redrawn every iteration"}
    try:
        # the object: primitives inside a disc of radius 0.32 S, opaque
        r = 0.32 * S * np.sqrt(g.uniform(0, 1, N))
        ph = g.uniform(0, 2 * np.pi, N)
        tp = np.zeros((N, 8), np.float32)
        tp[:, 0] = S / 2 + r * np.cos(ph)
        tp[:, 1] = S / 2 + r * np.sin(ph)
        tp[:, 2] = g.uniform(6, 14, N)
        tp[:, 3] = g.uniform(0, 2 * np.pi, N)
        tp[:, 4] = 6.0
        tp[:, 5:8] = np.log((c := g.uniform(0.05, 0.95, (N, 3))) / (1 - c))
        target = torch.empty(3, S, S, device="cuda")
        D.dbmp_bin(ws, S, S, 16, torch.from_numpy(tp).cuda(), bid, N, atlas, 1.0)
        D.dbmp_render_fwd(ws, atlas, D.make_background(None), 0.0, target, T, nl)
        alpha_t = (1.0 - T).clone()
        inside = alpha_t > 0
        u, ut, nc = (torch.from_numpy(a).cuda() for a in inputs.init_draws(seed + 1, N))
        init = torch.empty(N, 8, device="cuda")
        D.dbmp_structure_init(target, u, ut, nc, 6.0, 14.0, 0.02, -2.0, init, mask=alpha_t)
        gen = torch.Generator(device="cuda")
        for arm, lam, reinit in (("mse", 0.0, False), ("mse_opacity", 0.3, False),
                                 ("mse_opacity_reinit", 0.3, True)):
            gen.manual_seed(seed + 2)
            params = init.clone()
            grad = torch.zeros(N, 8, device="cuda")
            m = torch.zeros_like(grad)
            v = torch.zeros_like(grad)
            step = torch.zeros(1, dtype=torch.int32, device="cuda")
            cfg = D.adam_config(lr=0.1, gamma=0.1 ** (1.0 / steps), zero_grad=True,
                                gains=(10.0, 10.0, 10.0, 1.0, 5.0, 1.0, 1.0, 1.0))
            img = torch.empty(3, S, S, device="cuda")
            dI = torch.empty_like(img)
            dA = torch.empty(S, S, device="cuda")
            loss = torch.zeros(1, dtype=torch.float64, device="cuda")
            bgbuf = torch.empty(3, S, S, device="cuda")
            count = torch.zeros(1, dtype=torch.int32, device="cuda")
            for it in range(steps):
                if reinit and it >= 199 and it % 50 == 0:
                    ru, rut, rnc = (torch.from_numpy(a).cuda() for a in inputs.init_draws(seed + 100 + it, N))
                    D.dbmp_structure_reinit(target, ru, rut, rnc, 6.0, 14.0, 0.02, -2.0, 0.3, params, m, v, count,
                                            mask=alpha_t)
                torch.rand(3, S, S, generator=gen, device="cuda", out=bgbuf)
                bg = D.make_background(bgbuf)
                D.dbmp_bin(ws, S, S, 16, params, bid, N, atlas, 1.0)
                D.dbmp_render_fwd(ws, atlas, bg, 1e-6, img, T, nl)
                D.dbmp_alpha_loss_grad(img, T, target, alpha_t, lam, dI, dA, loss)
                D.dbmp_render_bwd(ws, atlas, bg, 1e-6, dI, dA, T, nl, grad)
                D.dbmp_adam_step(params, grad, m, v, step, cfg)
            # final state, judged over a fresh noise background
            torch.rand(3, S, S, generator=gen, device="cuda", out=bgbuf)
            bg = D.make_background(bgbuf)
            D.dbmp_bin(ws, S, S, 16, params, bid, N, atlas, 1.0)
            D.dbmp_render_fwd(ws, atlas, bg, 1e-6, img, T, nl)
            mse_in = float(((img - target) ** 2)[:, inside].mean())
            out[arm] = {"psnr_object": 10 * np.log10(1.0 / max(mse_in, 1e-30)),
                        "alpha_mae": float(((1.0 - T) - alpha_t).abs().mean()),
                        "transparent_fraction": float((torch.sigmoid(params[:, 4]) < 0.3).float().mean()),
                        "reinitialised": int(count.item())}
    finally:
        torch.cuda.synchronize()
        D.dbmp_workspace_destroy(ws)
        D.dbmp_atlas_destroy(atlas)
    return out


def run_dbmp(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2602_22625_gb300 import dbmp as D
    from paper_2602_22625_gb300 import inputs

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    D.load()
    peak = fp32_peak(local)

    # inputs: each rank renders its own workload (weak scaling: no exchange), or with
    # --shard bands every rank holds the same canvas and renders its band of it
    bands = args.shard == "bands" and world > 1
    seed, tgt_seed = rank_seeds(0 if bands else rank)
    sc = inputs.main(seed=seed)
    tgt = inputs.main(seed=tgt_seed)
    atlas_t = torch.from_numpy(sc.atlas).to(dev)
    atlas = D.dbmp_atlas_create(atlas_t)
    N, H, W = sc.N, sc.H, sc.W
    params0 = torch.from_numpy(sc.params).to(dev)
    params = params0.clone()
    bid = torch.from_numpy(sc.bitmap_id).to(dev)
    image = torch.empty(3, H, W, device=dev)
    T_final = torch.empty(H, W, device=dev)
    n_last = torch.empty(H, W, device=dev, dtype=torch.int32)
    target = torch.empty(3, H, W, device=dev)
    dL = torch.empty(3, H, W, device=dev)
    loss = torch.zeros(1, device=dev, dtype=torch.float64)
    dparams = torch.zeros(N, 8, device=dev)
    m = torch.zeros(N, 8, device=dev)
    v = torch.zeros(N, 8, device=dev)
    step = torch.zeros(1, device=dev, dtype=torch.int32)
    bg = D.make_background(sc.background)
    max_pairs = 96 << 20
    ws = D.dbmp_workspace_create(N, (W // 8) * (H // 8), max_pairs, 1)
    D.dbmp_batch_plan(ws, [H], [W], [0, N], tile=args.tile, batch=args.batch, ppt=args.ppt,
                      ppt_bwd=args.ppt_bwd)

    # target image: render of the target parameter set
    tgt_p = torch.from_numpy(tgt.params).to(dev)
    tgt_b = torch.from_numpy(tgt.bitmap_id).to(dev)
    D.dbmp_batch_render(ws, tgt_p, tgt_b, atlas, 1.0, bg, 0.0, D.BATCH_BIN | D.BATCH_FWD, target, T_final,
                        n_last)
    D.dbmp_status_poll(ws)

    # a real upstream gradient for the autotuner's backward
    D.dbmp_batch_render(ws, params, bid, atlas, 1.0, bg, T_STOP, D.BATCH_BIN | D.BATCH_FWD, image, T_final,
                        n_last)
    D.dbmp_mse_grad(image, target, dL, loss)
    D.dbmp_status_poll(ws)
    tuning = {"tile": args.tile, "batch": args.batch, "ppt": args.ppt, "ppt_bwd": args.ppt_bwd or args.ppt,
              "autotuned": False}
    if not args.no_autotune:
        # five renders per candidate and phase: steps vary by a few per cent, about the
        # margin between the best two tile sizes
        (t, b, pp, pb), ms = D.dbmp_autotune(ws, params, bid, atlas, 1.0, bg, T_STOP,
                                         D.BATCH_FWD | D.BATCH_BWD, image, T_final, n_last, dL, dparams,
                                         reps=5)
        tuning = {"tile": t, "batch": b, "ppt": pp, "ppt_bwd": pb, "autotuned": True,
                  "autotune_ms_bin_fwd_bwd": ms}
        dparams.zero_()
    if bands:
        from paper_2602_22625_gb300 import sharded
        band = sharded.select_band(ws, H, world, rank, tuning["tile"])
    adam = D.adam_config(lr=0.1, gamma=0.1 ** (1.0 / 500), zero_grad=True)

    flush = torch.empty(L2_FLUSH_BYTES // 4, device=dev)
    stream = torch.cuda.current_stream()

    def one_step(ev=None):
        if ev:
            ev[0].record(stream)
        D.dbmp_batch_render(ws, params, bid, atlas, 1.0, bg, T_STOP, D.BATCH_BIN, None, T_final, n_last)
        if ev:
            ev[1].record(stream)
        # the MSE loss and dL/dI in the forward's epilogue (no separate pass)
        D.dbmp_batch_render_mse(ws, params, bid, atlas, 1.0, bg, T_STOP, D.BATCH_FWD, target, image, T_final,
                                n_last, dL, loss)
        if ev:
            ev[2].record(stream)
            ev[3].record(stream)
        D.dbmp_batch_render(ws, params, bid, atlas, 1.0, bg, T_STOP, D.BATCH_BWD, image, T_final, n_last,
                            dL, dparams)
        if bands:   # the step's one exchange: the bands' gradients summed
            sharded.sum_gradient_(dparams, world)
        if ev:
            ev[4].record(stream)
        D.dbmp_adam_step(params, dparams, m, v, step, adam)
        if ev:
            ev[5].record(stream)

    # the warm-up steps count the contributing pairs (the work unit; the count is a
    # separately compiled instance of the forward), the timed steps do not
    D.dbmp_workspace_count_pairs(ws, True)
    for _ in range(max(args.warmup, 3)):
        one_step()
    st = D.dbmp_status_poll(ws)
    pairs = (st.pairs_evaluated, st.pairs_evaluated_bwd, st.pairs_contributing, st.pairs_required)
    D.dbmp_workspace_count_pairs(ws, False)

    # ---- device-timed steps (inputs resident in HBM) ----
    # Each step is timed by events around it alone (an event between two kernels would
    # keep the second from starting as the first one's programmatic dependent); as many
    # steps again, with an event between phases, give the phase breakdown.
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
    evp = [[torch.cuda.Event(enable_timing=True) for _ in range(6)] for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        for k in range(args.steps):
            flush.zero_()
            evs[k][0].record(stream)
            one_step()
            evs[k][1].record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms = np.array([evs[k][0].elapsed_time(evs[k][1]) for k in range(args.steps)])
    ms = float(step_ms.mean())
    st = D.dbmp_status_poll(ws)
    for k in range(args.steps):
        flush.zero_()
        one_step(evp[k])
    torch.cuda.synchronize()
    phase = np.array([[evp[k][i].elapsed_time(evp[k][i + 1]) for i in range(5)] for k in range(args.steps)])
    # the contributing pairs of the state the timed steps end in: one counting forward
    D.dbmp_workspace_count_pairs(ws, True)
    D.dbmp_batch_render(ws, params, bid, atlas, 1.0, bg, T_STOP, D.BATCH_BIN | D.BATCH_FWD, image, T_final, n_last)
    stc = D.dbmp_status_poll(ws)
    D.dbmp_workspace_count_pairs(ws, False)
    pairs_end = (st.pairs_evaluated, st.pairs_evaluated_bwd, stc.pairs_contributing, st.pairs_required)

    # ---- the same step captured once as a CUDA graph and replayed ----
    graph_ms = None
    try:
        if bands:   # no capture of the NCCL exchange
            raise RuntimeError("the banded step's all-reduce is not captured")
        cap = torch.cuda.Stream(device=dev)
        cap.wait_stream(stream)
        with torch.cuda.stream(cap):
            g_step = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g_step, stream=cap):
                one_step()
        torch.cuda.synchronize()
        for _ in range(3):
            g_step.replay()
        gts = []
        for k in range(args.steps):
            flush.zero_()
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            g_step.replay()
            a1.record(stream)
            torch.cuda.synchronize()
            gts.append(a0.elapsed_time(a1))
        graph_ms = float(np.mean(gts))
    except RuntimeError as e:   # capture refused: report the eager step only
        print(f"graph capture: {e}", file=sys.stderr)
    # Sec. S4 scaling statistics of the last step's binning (histograms: log2 bins)
    sstats = D.dbmp_bin_stats(ws)
    for k in ("tau_hist", "d_hist", "foot_hist"):
        h = sstats[k]
        nz = [i for i, v in enumerate(h) if v]
        sstats[k] = {"first_bin": nz[0], "counts": h[nz[0]:nz[-1] + 1]} if nz else {"first_bin": 0, "counts": []}

    # ---- end to end through the C ABI with host buffers ----
    h_params = params0.cpu().pin_memory()
    h_bid = bid.cpu().pin_memory()
    h_target = target.cpu().pin_memory()
    h_loss = torch.zeros(1, dtype=torch.float64).pin_memory()
    e2e_ms = []
    for k in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        params.copy_(h_params, non_blocking=True)
        bid.copy_(h_bid, non_blocking=True)
        target.copy_(h_target, non_blocking=True)
        one_step()
        h_loss.copy_(loss, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    h2d = h_params.numel() * 4 + h_bid.numel() * 4 + h_target.numel() * 4
    d2h = 8

    # ---- max over ranks ----
    ms, e2e = max_over_ranks([ms, float(np.mean(e2e_ms))], dev, world)

    fwd_ms = float(phase[:, 1].mean())
    bwd_ms = float(phase[:, 3].mean())
    ev_f, ev_b, contrib = pairs_end[0], pairs_end[1], pairs_end[2]
    flops_f = FLOPS_FWD_PAIR * contrib
    flops_b = FLOPS_BWD_PAIR * contrib
    if bwd_ms >= fwd_ms:
        dom, flops, dms, key, kppt = "k_bwd (backward compositor)", flops_b, bwd_ms, "bwd", tuning["ppt_bwd"]
    else:
        dom, flops, dms, key, kppt = "k_fwd (forward compositor)", flops_f, fwd_ms, "fwd", tuning["ppt"]
    achieved = flops / (dms * 1e-3) / 1e12
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline()
    learned = None
    if rank == 0 and world == 1 and not args.no_learned:
        learned = learned_vs_plain(args.learned_pairs)
    ablation = constrained = None
    others = None
    if rank == 0 and world == 1 and not args.no_ablation:
        ablation = blur_ablation()
        constrained = spatial_constraint()
        others = [other_workload("batched", peak["peak"]), other_workload("stress", peak["peak"])]
    if world > 1:
        dist.barrier()
    if rank != 0:
        dist.destroy_process_group()
        return
    line = {
        "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": False,
        "scaling": "strong" if bands else "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config({"tile": tuning["tile"], "batch": tuning["batch"], "ppt": tuning["ppt"],
                          "ppt_bwd": tuning["ppt_bwd"],
                          "autotuned": tuning["autotuned"],
                          "autotune_ms_bin_fwd_bwd": tuning.get("autotune_ms_bin_fwd_bwd"),
                          "loss": "MSE over 3HW, fused into the forward's epilogue (fwd includes it; mse ~ 0)",
                          "parallelism": (f"bands x{world} (one canvas, rows {band[0]}..{band[1]} on rank 0; one sum "
                                          f"all-reduce of the {N}x8 gradient per step)") if bands else
                                         f"replicas x{world} (one canvas per GPU, no exchange)"}),
        "breakdown_ms": {"bin": float(phase[:, 0].mean()), "fwd": fwd_ms, "mse": float(phase[:, 2].mean()),
                         "bwd": bwd_ms, "adam": float(phase[:, 4].mean()),
                         "step_min": float(step_ms.min()), "step_max": float(step_ms.max()),
                         "note": "phases from as many steps again with an event between phases (an event "
                                 "keeps the next kernel from starting as a programmatic dependent, so the "
                                 "phases add up to a little more than the step)"},
        "work": {"pairs_contributing": contrib, "pairs_in_walk_fwd": ev_f, "pairs_in_walk_bwd": ev_b,
                 "tile_list_entries": pairs_end[3], "warp_steps_fwd": st.warp_steps,
                 "warp_steps_bwd": st.warp_steps_bwd, "survivors_fwd": st.survivors,
                 "survivors_bwd": st.survivors_bwd, "at_warmup_end": list(pairs)},
        "roofline": {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak["peak"],
                     "unit": "TFLOP/s", "frac": achieved / peak["peak"],
                     "peak_source": peak["source"], "fp32_peak": peak,
                     "unit_of_work": "contributing (pixel, primitive) pair",
                     "flops_per_unit": FLOPS_BWD_PAIR if key == "bwd" else FLOPS_FWD_PAIR,
                     "algorithmic_flops_per_launch": flops, "kernel_ms": dms,
                     "traffic": traffic_for(key, tuning["tile"], tuning["batch"], kppt)},
        "binning_hbm": binning_hbm(N, pairs_end[3], (H // tuning["tile"]) * (W // tuning["tile"]),
                                   float(phase[:, 0].mean())),
        "e2e": {"value": e2e, "unit": "ms", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "graph_ms_per_step": graph_ms,
        "gpu_launches": LAUNCHES_PER_STEP * args.steps,
        "clocks": clk.summary(),
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if learned is not None:
        line["time_to_30db"] = learned
    if ablation is not None:
        line["blur_ablation"] = ablation
    if constrained is not None:
        line["spatial_constraint"] = constrained
    if others is not None:
        line["other_workloads"] = others
    line["scaling_stats"] = dict(sstats, note="tau: tiles per primitive, d: primitives per tile, foot: padded "
                                              "box area / canvas area; bin b = [2^b, 2^(b+1)) (foot: "
                                              "[2^-(b+1), 2^-b))")
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_dbmp(args)


if __name__ == "__main__":
    main()
