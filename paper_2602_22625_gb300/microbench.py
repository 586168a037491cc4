"""Microbenchmarks of the library's tensor-core kernels, runnable on their own:

    python -m paper_2602_22625_gb300.microbench gemm 4096     # bf16 GEMM M = N = K = 4096
    python -m paper_2602_22625_gb300.microbench cnn 64        # proposal-network training steps

Each runs a few warm-up launches, then times repetitions with CUDA events and prints
one line of JSON (the GEMM also times torch.matmul on the same operands)."""
import json
import sys

import torch

from . import dbmp as D


def _time(fn, reps):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def gemm(n, reps=10):
    A = (torch.randn(n, n, device="cuda") * 0.1).to(torch.bfloat16)
    B = (torch.randn(n, n, device="cuda") * 0.1).to(torch.bfloat16)
    C = torch.zeros(n, n, device="cuda")
    ours = lambda: D.dbmp_gemm_bf16(A.view(torch.int16), B.view(torch.int16), n, n, n, 0, Cf=C)
    for _ in range(2):
        ours()
    ms = _time(ours, reps)
    ref = lambda: torch.matmul(A, B.t())
    for _ in range(2):
        ref()
    tms = _time(ref, reps)
    flop = 2.0 * n ** 3
    return {"gemm": n, "ms": ms, "tflops": flop / ms / 1e9, "torch_ms": tms, "torch_tflops": flop / tms / 1e9}


def cnn(batch, reps=10):
    from . import inputs, proposer
    scenes = proposer.SceneRenderer(max_batch=batch)
    P = proposer.Proposer(max_batch=batch, seed=0)
    try:
        imgs = torch.empty(batch, 3, 256, 256, device="cuda")
        tp = torch.from_numpy(inputs.anchored(123, batch)).cuda()
        scenes.render(tp, imgs)
        step = lambda: P.train_step(imgs, tp, 1e-6)
        for _ in range(2):
            step()
        ms = _time(step, reps)
    finally:
        P.close()
        scenes.close()
    return {"cnn_train_batch": batch, "ms": ms, "tflops": proposer.cnn_train_flops(batch) / ms / 1e9}


if __name__ == "__main__":
    what, size = sys.argv[1], int(sys.argv[2])
    print(json.dumps(gemm(size) if what == "gemm" else cnn(size)))
