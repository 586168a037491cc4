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
