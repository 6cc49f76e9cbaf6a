"""Genetic FP8/BF16 plan search (net_tune_precision): the tuned plan meets
the FP8 error budget against the FP64 oracle on frames it was not tuned on,
and it is never slower than the all-BF16 plan by more than noise."""
import numpy as np
import pytest

import oracle
from paper_1811_03882_gb300 import synth
from helpers import default_precs, make_net

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1811_03882_gb300 import build
    build.build()
    oracle.build()


def test_tuned_fp8_plan_meets_budget_on_unseen_frames():
    import torch
    spec = synth.net_19conv()
    side = 96
    blob = synth.weights_for(spec, 81)
    xc = synth.make_frames(synth.Stream(synth.SEED_CALIB), 2, 3, side, side)
    x = synth.make_frames(synth.Stream(82), 2, 3, side, side)
    with make_net(spec, prec="fp8", max_batch=2, max_side=side) as net:
        net.load_weights(blob)
        d_c = torch.from_numpy(xc).cuda()
        net.calibrate(d_c, 2, side, side)
        plan, res = net.tune_precision(d_c, 2, side, side, max_err=0.05, population=10,
                                       generations=6, reps=2, seed=7)
        print("plan", plan, res)
        assert res["err"] <= 0.05 and res["fp8_layers"] >= 0
        assert res["evaluations"] + res["memo_hits"] >= 10 * 6
        assert net.layer_prec() == plan
        assert plan[0] == "bf16"            # the 3-channel layer never runs in FP8
        y = net.forward(x)
    ex = oracle.forward(spec.layers, 3, x, blob)
    e = oracle.normwise_rel_err(y, ex)
    agree, _, _ = oracle.argmax_agreement(y, ex, 8e-2)
    print("tuned plan on unseen frames: err %.3e argmax %.4f" % (e, agree))
    assert e <= 8e-2 and agree >= 0.99


def test_layer_precision_switching_round_trip():
    import torch
    spec = synth.net_9conv()
    blob = synth.weights_for(spec, 83)
    x = synth.frame_for(83, 0, 64)
    xc = synth.make_frames(synth.Stream(synth.SEED_CALIB), 1, 3, 64, 64)
    with make_net(spec, prec="fp8", max_side=64) as net:
        net.load_weights(blob)
        sc = oracle.act_scales_from(spec.layers, 3, xc, blob)
        net.set_act_scales(np.asarray(sc, np.float32))
        y8 = net.forward(x)
        net.set_layer_prec(["bf16"] * 9)
        ybf = net.forward(x)
        net.set_layer_prec(["bf16"] + ["fp8"] * 8)
        y8b = net.forward(x)
    np.testing.assert_array_equal(y8, y8b)
    qa = oracle.forward_quant(spec.layers, 3, x, blob, ["bf16"] * 9)
    assert oracle.rms_rel_err(ybf, qa) <= 1.2e-2
    assert oracle.normwise_rel_err(ybf, oracle.forward(spec.layers, 3, x, blob)) <= 2e-2


def test_tile_plan_overrides_and_search():
    """Per-layer (N tile, split-K) overrides and the genetic tile-plan search
    (net_set_layer_tiles / net_plan_tiles / net_tune_tiles): overrides show in
    the plan, bad values are refused, every plan stays within the BF16 budget
    of the oracle, and the search never returns a plan slower than the
    analytic one it starts from."""
    import torch
    from paper_1811_03882_gb300 import binding
    spec = synth.net_19conv()
    side, batch = 160, 2
    _, x, blob = synth.workload_net(spec, 85, batch, side, side)
    ex = oracle.forward(spec.layers, 3, x, blob)
    with make_net(spec, prec="bf16", max_batch=batch, max_side=side) as net:
        net.load_weights(blob)
        d_x = torch.from_numpy(x).cuda()
        base = net.plan_tiles(batch, side, side)
        assert all(bn in (64, 128, 256) and ks in (1, 2, 4, 8, 16) for bn, ks in base)
        # layer 13 (3x3, 512 -> 1024): a different N tile and split
        bn13, ks13 = base[13]
        alt = (128 if bn13 != 128 else 256, 1 if ks13 != 1 else 2)
        net.set_layer_tiles(13, *alt)
        assert net.plan_tiles(batch, side, side)[13] == alt
        y = net.forward(x)
        assert oracle.normwise_rel_err(y, ex) <= 2e-2
        with pytest.raises(binding.NetError) as e:
            net.set_layer_tiles(13, 96, 1)
        assert e.value.status == binding.NET_E_INVAL
        with pytest.raises(binding.NetError) as e:
            net.set_layer_tiles(0, 64, 4)        # the im2col first layer has one K step
        assert e.value.status == binding.NET_E_INVAL
        net.set_layer_tiles(13, 0, 0)
        assert net.plan_tiles(batch, side, side) == base
        # CTAs per SM: layer 3 (1x1, 64 outputs) forced to each value
        for mb in (1, 2):
            net.set_layer_ctas(3, mb)
            assert net.plan_ctas(batch, side, side)[3] == mb
            assert oracle.normwise_rel_err(net.forward(x), ex) <= 2e-2
        net.set_layer_ctas(3, 0)
        with pytest.raises(binding.NetError) as e:
            net.set_layer_ctas(3, 3)
        assert e.value.status == binding.NET_E_INVAL
        plan, res = net.tune_tiles(d_x, batch, side, side, population=6, generations=3, reps=2, seed=11)
        print("tile plan", plan, res)
        assert res["ms"] <= res["ms_analytic"] and res["evaluations"] >= 1
        assert net.plan_tiles(batch, side, side) == plan
        y = net.forward(x)
    assert oracle.normwise_rel_err(y, ex) <= 2e-2
