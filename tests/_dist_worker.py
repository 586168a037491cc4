"""Rank body of the world-size-2 gloo tests (spawned processes; CPU only)."""
import json
import os
import sys


def run(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import torch
    import torch.distributed as dist
    import bench
    from paper_2602_22625_gb300 import inputs

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, local = bench.dist_env()
        seed, tgt_seed = bench.rank_seeds(r)
        sc = inputs.main(seed=seed, N=200)
        # each rank reports a different time; every rank must see the slowest
        mx = bench.max_over_ranks([1.0 + r, 10.0 - r], torch.device("cpu"), w)
        dist.barrier()
        res = {"world": w, "rank": r, "local": local, "seed": seed, "tgt_seed": tgt_seed, "max": mx,
               "shape": [sc.N, sc.H, sc.W], "param_sum": float(sc.params.sum())}
        with open(os.path.join(out_dir, f"rank{r}.json"), "w") as f:
            json.dump(res, f)
    finally:
        dist.destroy_process_group()


def reference_arm(rank, world, out_dir):
    """bench.py --impl reference under a 2-rank launch: rank 0 alone prints the line."""
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import contextlib
    import io
    import types
    import bench
    buf = io.StringIO()
    t0 = __import__("time").perf_counter()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(types.SimpleNamespace(steps=1, warmup=1, gpus=world))
    with open(os.path.join(out_dir, f"ref{rank}.txt"), "w") as f:
        f.write(buf.getvalue())
    with open(os.path.join(out_dir, f"ref{rank}.time"), "w") as f:
        f.write(str(__import__("time").perf_counter() - t0))


def sharded(rank, world, port, out_dir):
    """One canvas shared by the ranks: each rank's FP64 oracle gradient over its band
    of rows (the loss normalised over the whole canvas), summed by the all-reduce of
    sharded.sum_gradient_, must equal the whole canvas' gradient."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import numpy as np
    import torch
    import torch.distributed as dist
    import oracle
    from paper_2602_22625_gb300 import inputs, sharded as S

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sc = inputs.tiny(seed=5, N=80, H=70, W=52)   # 5 tile rows of 16: bands of 3 and 2
        tg = inputs.tiny(seed=6, N=80, H=70, W=52)
        img = oracle.render(sc.H, sc.W, sc.params, sc.bitmap_id, sc.atlas, background=sc.background)["image"]
        tgt = oracle.render(tg.H, tg.W, tg.params, tg.bitmap_id, tg.atlas, background=tg.background)["image"]
        gI = 2.0 * (img - tgt) / img.size                 # MSE over the whole canvas
        y0, y1 = S.band_rows(sc.H, world, rank, tile=16)
        g = oracle.grad_rows(sc.H, sc.W, sc.params, sc.bitmap_id, sc.atlas, gI, y0, min(y1, sc.H),
                             background=sc.background)
        t = torch.from_numpy(g.copy())
        S.sum_gradient_(t, world)
        full = oracle.grad(sc.H, sc.W, sc.params, sc.bitmap_id, sc.atlas, gI, background=sc.background)
        res = {"rows": [y0, y1], "err": float(np.abs(t.numpy() - full).max() / np.abs(full).max()),
               "own": float(np.abs(g).max() / np.abs(full).max())}
        with open(os.path.join(out_dir, f"shard{rank}.json"), "w") as f:
            json.dump(res, f)
    finally:
        dist.destroy_process_group()
