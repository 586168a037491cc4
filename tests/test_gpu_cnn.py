"""The proposal network on the tensor cores against its FP64 oracle (same bfloat16
rounding points), and what a briefly trained network gains over random
initialisation before and after the plain refinement."""
import io
import json

import numpy as np
import pytest

from oracle import cnn
from paper_2602_22625_gb300 import dbmp as D
from paper_2602_22625_gb300 import inputs, proposer
from _helpers import cuda, to_dev, torch

pytestmark = pytest.mark.gpu


def layer_slices():
    out, o = [], 0
    for cin_pad, _, cout, k in cnn.LAYERS:
        nw = cout * k * k * cin_pad
        out.append((slice(o, o + nw), slice(o + nw, o + nw + cout)))
        o += nw + cout
    return out


@pytest.fixture(scope="module", params=[2, 3])
def case(request):
    """Two images, and three: an odd batch, where a tensor copy of the 8 x 8 layer's
    128 pixel rows (two whole images) reaches past the last image."""
    B = request.param
    rng = np.random.default_rng(B - 2)
    theta = inputs.cnn_init(1)
    # positive biases keep most units active; random ones exercise both ReLU sides
    for w, b in layer_slices():
        theta[b] = rng.normal(0.05, 0.05, theta[b].shape[0])
    images = rng.uniform(0, 1, (B, 3, 256, 256)).astype(np.float32)
    tp = inputs.anchored(11, B)
    return theta, images, tp


def test_proposer_gradient_matches_oracle(case):
    """Every element of every activation (the five bf16 convolution outputs and the
    head's fp32 outputs) and of every weight and bias gradient against the FP64
    oracle with the same bf16 rounding points.

    Derivation of the bounds.  Both sides round inputs, weights, post-ReLU activations
    and the backward's dZ tensors to bf16 at the same points; they differ only in how
    the products are accumulated (FP64 in the oracle, FP32 in TMEM on the GPU).  A sum
    that lands near a bf16 rounding boundary then rounds to the neighbouring value, and
    such one-ulp flips (2^-8 relative) propagate along the chain.  The oracle measures
    this effect on itself: rerun with FP32 accumulation, the inner dimension summed
    forwards and backwards (cnn.forward(acc32=1, 2)), it moves each tensor element-wise
    by probe = max over the two of max|d| / max|ref|.  The tensor cores
    accumulate in FP32 too, in another order, so they move each tensor by an amount of
    the same kind; the bound is 8 x probe (the tensor cores were seen at 1.4-5.4 x on a
    GB300, element-wise) plus a floor for tensors the probe barely moves (5e-4 for gradients and head
    outputs, one bf16 ulp, 2^-8, for activations).  A wrong index, operand or swizzle
    atom gives errors of order max|ref|.  The norm-wise 2% check stays as a second line."""
    cuda()
    theta, images, tp = case
    B = images.shape[0]
    P = proposer.Proposer(max_batch=B)
    try:
        P.set_params(theta)
        loss = P.train_step(to_dev(images), to_dev(tp))
        g = P.grads()
        L = loss.item()
        acts = [P.activations(l, B).astype(np.float64) for l in range(7)]
    finally:
        P.close()
    O, cache = cnn.forward(theta.astype(np.float64), images)
    Lr, dO = cnn.loss_and_grad(O, tp)
    gr = cnn.backward(dO, cache)
    probes = []
    for order in (1, 2):
        O32, cache32 = cnn.forward(theta.astype(np.float64), images, acc32=order)
        probes.append((O32, cache32, cnn.backward(cnn.loss_and_grad(O32, tp)[1], cache32)))
    assert L == pytest.approx(Lr, rel=1e-4)

    def probe_of(get, ref):
        return max(np.abs(get(p) - ref).max() for p in probes) / np.abs(ref).max()

    # forward: the packed input exactly, then each layer element-wise
    assert np.array_equal(acts[0], cache["acts"][0])
    for l in range(1, 6):
        ref = cache["acts"][l]
        probe = probe_of(lambda p: p[1]["acts"][l], ref)
        err = np.abs(acts[l] - ref).max() / np.abs(ref).max()
        assert err <= 8 * probe + 2.0 ** -8, (l, err, probe)
        flips = (acts[l] != ref).mean()
        assert flips <= 10 * max((p[1]["acts"][l] != ref).mean() for p in probes) + 1e-3, (l, flips)
    probe = probe_of(lambda p: p[0], O)
    err = np.abs(acts[6] - O).max() / np.abs(O).max()
    assert err <= 8 * probe + 5e-4, ("head", err, probe)
    # backward: every element of each weight and bias gradient
    errs = {}
    for li, (w, b) in enumerate(layer_slices()):
        for sl, what in ((w, "W"), (b, "b")):
            ref = gr[sl]
            scale = np.abs(ref).max()
            probe = probe_of(lambda p: p[2][sl], ref)
            err = np.abs(g[sl] - ref).max() / scale
            errs[f"{li}{what}"] = (err, probe)
            assert err <= 8 * probe + 5e-4, (f"{li}{what}", err, probe)
            assert np.linalg.norm(g[sl] - ref) / np.linalg.norm(ref) < 2e-2, f"{li}{what}"
    print(errs)


def test_propose_matches_oracle_decode(case):
    cuda()
    theta, images, _ = case
    P = proposer.Proposer(max_batch=images.shape[0])
    try:
        P.set_params(theta)
        got = P.propose(to_dev(images)).cpu().numpy()
    finally:
        P.close()
    O, _ = cnn.forward(theta.astype(np.float64), images)
    ref = cnn.decode(O)
    assert np.abs(got - ref).max() <= 2e-3 * max(1.0, np.abs(ref).max())


def test_trained_proposals_beat_random_init():
    """Train on 16384 freshly rendered pairs, then compare on held-out scenes: PSNR
    of the proposal itself, and after 60 steps of the plain refinement.  (The loss
    has a floor: colours and opacities of slots hidden behind others cannot be
    read from the image.)"""
    cuda()
    scenes = proposer.SceneRenderer(max_batch=64)
    P = proposer.Proposer(max_batch=64, seed=2)
    try:
        losses = proposer.train(P, scenes, n_pairs=16384, batch=64, seed=5000, lr=2e-3, lr_end=2e-4,
                                log_every=32)
        print("training loss", losses)
        assert losses[-1] < 0.8 * losses[0], losses
        held = torch.from_numpy(inputs.anchored(999_001, 4)).cuda()
        targets = torch.empty(4, 3, 256, 256, device="cuda")
        scenes.render(held, targets)
        learned = P.propose(targets)
        rand = torch.from_numpy(inputs.random_init(999_002, 4)).cuda()
        gains0, gains60 = [], []
        for i in range(4):
            log = io.StringIO()
            pl, _, _, _ = proposer.refine(learned[i], targets[i], scenes.atlas, steps=60, log=log)
            rows = [json.loads(r) for r in log.getvalue().splitlines()]   # one JSON line per step
            assert [r["step"] for r in rows] == list(range(61)) and [r["psnr"] for r in rows] == pl
            pr, _, _, _ = proposer.refine(rand[i], targets[i], scenes.atlas, steps=60)
            gains0.append(pl[0] - pr[0])
            gains60.append(pl[-1] - pr[-1])
        print("PSNR gain of the learned init at step 0:", gains0, "after 60 steps:", gains60)
        assert min(gains0) > 1.0, gains0
        assert np.mean(gains60) > 0.0, gains60
    finally:
        P.close()
        scenes.close()
