"""Uneven batches: frames of different sizes through one grouped launch per
layer (net_forward_uneven), each frame checked against the FP64 oracle, and
each result identical alone and in the mix."""
import numpy as np
import pytest

import oracle
from paper_1811_03882_gb300 import synth
from helpers import default_precs, make_net

pytestmark = pytest.mark.gpu
TOL = {"bf16": 2e-2, "fp32": 1e-4}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1811_03882_gb300 import build
    build.build()
    oracle.build()


def _uneven(net, frames):
    import torch
    d_in = [torch.from_numpy(f).cuda() for f in frames]
    outs = []
    for f in frames:
        c, ho, wo = net.output_shape(f.shape[2], f.shape[3])
        outs.append(torch.full((1, c, ho, wo), float("nan"), device="cuda"))
    net.forward_uneven(d_in, [f.shape[2] for f in frames], outs)
    torch.cuda.synchronize()
    return [o.cpu().numpy() for o in outs]


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
def test_uneven_small_frames_vs_oracle_and_alone(prec):
    spec = synth.net_9conv()
    blob = synth.weights_for(spec, 51)
    sides = [64, 32, 96, 64, 128, 32]
    frames = [synth.frame_for(51, i, s) for i, s in enumerate(sides)]
    with make_net(spec, prec=prec, max_batch=1, max_side=128) as net:
        net.load_weights(blob)
        mix = _uneven(net, frames)
        mix_again = _uneven(net, frames)            # graph replay of the same batch
        alone = [_uneven(net, [f])[0] for f in frames]
    precs = default_precs(spec, prec)
    for i, (f, y) in enumerate(zip(frames, mix)):
        ex = oracle.forward(spec.layers, 3, f, blob)
        e = oracle.normwise_rel_err(y, ex)
        print("%s frame %d side %d: err %.3e" % (prec, i, sides[i], e))
        assert y.shape == ex.shape and e <= TOL[prec]
        np.testing.assert_array_equal(y, mix_again[i])
        # no reduction spans frames: alone and in the mix agree bit for bit
        np.testing.assert_array_equal(y, alone[i])
        if prec == "bf16":
            qa = oracle.forward_quant(spec.layers, 3, f, blob, precs)
            assert oracle.rms_rel_err(y, qa) <= 1.2e-2


def test_uneven_64_frames_full_size():
    """64 frames with sides drawn from {320, 416, 512, 608}, 9-conv BF16,
    one grouped launch per layer; sampled frames recomputed by the oracle."""
    spec = synth.net_9conv()
    blob = synth.weights_for(spec, synth.SEED_UNEVEN)
    sides = synth.uneven_sides()
    frames = [synth.frame_for(synth.SEED_UNEVEN, i, int(s)) for i, s in enumerate(sides)]
    with make_net(spec, prec="bf16", max_batch=1, max_side=608) as net:
        net.load_weights(blob)
        ys = _uneven(net, frames)
    for i in (0, int(np.argmax(sides)), 63):
        ex = oracle.forward(spec.layers, 3, frames[i], blob)
        e = oracle.normwise_rel_err(ys[i], ex)
        agree, _, _ = oracle.argmax_agreement(ys[i], ex, 2e-2)
        print("uneven frame %d side %d: err %.3e argmax %.4f" % (i, sides[i], e, agree))
        assert e <= 2e-2 and agree >= 0.99
    assert all(np.isfinite(y).all() for y in ys)


def test_uneven_tuned_grouped_plan():
    """The genetic search over the grouped launches (N tile, CTAs per SM,
    ring stage cap per layer): every plan computes the same sums in the same
    order, so the tuned batch is bit-identical to the analytic one and each
    frame to its own pass; the frames also meet the oracle."""
    import torch
    spec = synth.net_9conv()
    blob = synth.weights_for(spec, 52)
    sides = [96, 64, 160, 32, 128, 64, 96]
    frames = [synth.frame_for(52, i, s) for i, s in enumerate(sides)]
    with make_net(spec, prec="bf16", max_batch=1, max_side=160) as net:
        net.load_weights(blob)
        before = _uneven(net, frames)
        d_in = [torch.from_numpy(f).cuda() for f in frames]
        d_out = [torch.empty((1,) + net.output_shape(s, s), device="cuda") for s in sides]
        plan, res = net.tune_uneven(d_in, sides, d_out, population=8, generations=4, reps=2, seed=3)
        print("grouped plan", plan, res)
        assert res["ms"] <= res["ms_analytic"] and res["evaluations"] >= 1
        assert net.plan_grouped() == plan
        after = _uneven(net, frames)
        alone = [_uneven(net, [f])[0] for f in frames]
    for i, f in enumerate(frames):
        np.testing.assert_array_equal(after[i], before[i])
        np.testing.assert_array_equal(after[i], alone[i])
        assert oracle.normwise_rel_err(after[i], oracle.forward(spec.layers, 3, f, blob)) <= 2e-2
