"""Microbenchmarks of the library's tensor-core kernels, runnable on their own:

    python -m paper_2602_22625_gb300.microbench gemm 4096     # bf16 GEMM M = N = K = 4096
    python -m paper_2602_22625_gb300.microbench cnn 64        # proposal-network training steps
    python -m paper_2602_22625_gb300.microbench fp32 20000    # FP32 multiply-add issue rate

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


def fp32(iters=20000, reps=20, blocks_per_sm=8):
    """FP32 multiply-add rate of the whole GPU with scalar FFMA and with packed FP32x2
    FMA instructions (dbmp_fp32_peak): 8 blocks of 256 threads per SM, 16 independent
    chains per thread, timed over `reps` launches with CUDA events.  Returns TFLOP/s
    (2 per multiply-add) of each form and the SM count."""
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    sink = torch.empty(sms * blocks_per_sm * 256, device="cuda")
    out = {"sms": sms, "threads": sink.numel(), "iters": iters, "reps": reps}
    for packed, name in ((0, "ffma"), (1, "ffma2")):
        fl = D.dbmp_fp32_peak(packed, iters, sink)
        for _ in range(3):
            D.dbmp_fp32_peak(packed, iters, sink)
        ms = _time(lambda: D.dbmp_fp32_peak(packed, iters, sink), reps)
        out[f"{name}_ms"] = ms
        out[f"{name}_tflops"] = fl / (ms * 1e-3) / 1e12
    return out


if __name__ == "__main__":
    what, size = sys.argv[1], int(sys.argv[2])
    fn = {"gemm": gemm, "cnn": cnn, "fp32": fp32}[what]
    print(json.dumps(fn(size)))
