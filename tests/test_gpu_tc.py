"""Tensor-core paths (BF16, FP8 E4M3) on the GPU against the oracle.

Two references: the exact FP64 oracle (the stated budgets: BF16 <= 2e-2,
FP8 <= 8e-2 normwise max relative error on the final map, argmax agreement
>= 99%) and the quantisation-aware oracle, which rounds weights and
activations exactly as the library stores them, so a kernel bug cannot hide
inside the rounding budget.
"""
import numpy as np
import pytest

import oracle
from paper_1811_03882_gb300 import synth
from helpers import default_precs, make_net, run_device

pytestmark = pytest.mark.gpu
TOL = {"bf16": 2e-2, "fp8": 8e-2}
# Against the quantisation-aware oracle.  A single layer (output stored in
# FP32) differs from it only by FP32 vs FP64 accumulation: ~1e-6.  The first
# tensor-core layer of a deep network matches it exactly too; after that,
# BF16 products (16 significant bits) summed in the tensor core's FP32
# accumulator round differently from FP64 and flip a stored BF16 activation
# by one unit in the last place (2^-8) now and then; each flip perturbs the
# next layer's sums and the flips cascade (0.01% of elements at layer 2,
# about half by layer 9), so the RMS gap settles at BF16's own noise level
# (~7e-3).  E4M3 products sum exactly in FP32, so an all-FP8 network
# matches to ~1e-7; in a mixed plan the BF16 flips reach FP8 layers, where a
# moved rounding is one E4M3 step (2^-3), and the RMS gap settles near 4e-2.
# A wrong tap, channel or scale gives an O(1) RMS gap.
QRMS = {"bf16": 1.2e-2, "fp8": 6e-2}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1811_03882_gb300 import build
    build.build()
    oracle.build()


def _check(spec, x, blob, prec, max_batch, max_side, scales=None, tight=None, layer_prec=None,
           budget=None, qrms=None):
    precs = default_precs(spec, prec, layer_prec)
    ex = oracle.forward(spec.layers, spec.in_c, x, blob)
    qa = oracle.forward_quant(spec.layers, spec.in_c, x, blob, precs, scales)
    with make_net(spec, prec=prec, max_batch=max_batch, max_side=max_side, layer_prec=layer_prec) as net:
        net.load_weights(blob)
        if scales is not None:
            net.set_act_scales(np.asarray(scales, np.float32))
        y = run_device(net, x)
    e_q = oracle.normwise_rel_err(y, qa)
    r_q = oracle.rms_rel_err(y, qa)
    e_x = oracle.normwise_rel_err(y, ex)
    agree, npos, ties = oracle.argmax_agreement(y, ex, TOL[prec])
    print("%s %s: vs quant-aware max %.3e rms %.3e, vs exact %.3e, argmax %.4f (%d pos, %d ties)"
          % (spec.name, prec, e_q, r_q, e_x, agree, npos, ties))
    assert np.isfinite(y).all()
    if tight is not None:
        assert e_q <= tight, e_q
    assert r_q <= (qrms if qrms is not None else QRMS[prec]), r_q
    assert e_x <= (budget if budget is not None else TOL[prec]), e_x
    if budget is None:
        assert agree >= 0.99
    return y


def test_bf16_single_tc_layer():
    # 16 input channels: the conv itself runs on the tensor cores (32-byte K chunks)
    spec, x, blob = synth.workload_single()
    _check(spec, x, blob, "bf16", 1, 32, tight=1e-4)


@pytest.mark.parametrize("cin,cout,k,pool,hw", [
    (32, 64, 3, synth.POOL_2X2S2, (24, 40)),     # 64-byte chunks, pool tiles, ragged
    (64, 128, 3, synth.POOL_NONE, (13, 13)),    # 128-byte chunks, odd map
    (128, 64, 1, synth.POOL_NONE, (28, 28)),    # 1x1
    (256, 256, 3, synth.POOL_2X2S2, (16, 16)),  # two K chunks per tap, BN 256 region
    (96, 1000, 1, synth.POOL_NONE, (14, 14)),   # N tail: 1000 outputs
    # first layers over few channels: two taps per MMA (8-channel pixels)
    (3, 128, 3, synth.POOL_2X2S2, (40, 56)),    # one 128-column N tile, pool, ragged x
    (3, 256, 3, synth.POOL_NONE, (20, 36)),     # N tile widened to 256, 16 x 8 tiles on a 20-wide map
    (5, 48, 3, synth.POOL_NONE, (17, 23)),      # five channels, odd map
])
def test_bf16_layer_shapes(cin, cout, k, pool, hw):
    L = synth.Layer
    spec = synth.NetSpec("layer", cin, [L(k, cout, True, synth.ACT_LEAKY, pool)])
    s = synth.Stream(cin * 7 + cout)
    x = synth.make_frames(s, 2, cin, hw[0], hw[1], -1, 1)
    blob = synth.pack_blob(spec, synth.make_params(s, spec))
    _check(spec, x, blob, "bf16", 2, max(hw), tight=1e-4)


def test_bf16_9conv_small_ragged():
    spec = synth.net_9conv()
    s = synth.Stream(41)
    x = synth.make_frames(s, 2, 3, 96, 160)
    blob = synth.pack_blob(spec, synth.make_params(s, spec))
    _check(spec, x, blob, "bf16", 2, 160)


def test_bf16_19conv_small():
    spec = synth.net_19conv()
    s = synth.Stream(42)
    x = synth.make_frames(s, 2, 3, 64, 96)
    blob = synth.pack_blob(spec, synth.make_params(s, spec))
    _check(spec, x, blob, "bf16", 2, 96)


def _fp8_scales(spec, blob, side):
    s = synth.Stream(synth.SEED_CALIB)
    xc = synth.make_frames(s, 1, spec.in_c, side, side)
    return oracle.act_scales_from(spec.layers, spec.in_c, xc, blob)


def test_fp8_single_tc_layer():
    spec = synth.net_single_conv()
    s = synth.Stream(43)
    x = synth.make_frames(s, 1, 16, 32, 32, -1, 1)
    blob = synth.pack_blob(spec, synth.make_params(s, spec))
    sc = oracle.act_scales_from(spec.layers, 16, x, blob)
    _check(spec, x, blob, "fp8", 1, 32, scales=sc, tight=2e-3)


def test_fp8_all_layers_9conv_small():
    """Every layer with >= 16 input channels in E4M3.  Each such layer adds
    2-5% normwise error (3 significant bits), so the all-FP8 network is held
    to the quantisation-aware oracle: E4M3 products sum exactly in the FP32
    accumulator and the epilogue rounds once in FP32, so the stored codes
    match the oracle's and only the FP32 epilogue and the final map differ
    (~1e-7 RMS).  The 8e-2 budget against the exact oracle binds the mixed
    plans below."""
    spec = synth.net_9conv()
    s = synth.Stream(44)
    x = synth.make_frames(s, 2, 3, 64, 64)
    blob = synth.pack_blob(spec, synth.make_params(s, spec))
    _check(spec, x, blob, "fp8", 2, 64, scales=_fp8_scales(spec, blob, 64), budget=0.25, qrms=1e-5)


# FP8 on the 3x3 layers with the most FLOPs, BF16 elsewhere
MIX9 = ["bf16"] * 6 + ["fp8", "fp8"] + ["bf16"]
MIX19 = ["bf16"] * 13 + ["fp8", "bf16", "fp8", "bf16", "bf16", "bf16"]


@pytest.mark.parametrize("name,mix,hw", [("9-conv", MIX9, (64, 96)), ("19-conv", MIX19, (64, 64))])
def test_fp8_mixed_plan_meets_budget(name, mix, hw):
    spec = synth.NETS[name]()
    s = synth.Stream(46)
    x = synth.make_frames(s, 2, 3, *hw)
    blob = synth.pack_blob(spec, synth.make_params(s, spec))
    _check(spec, x, blob, "fp8", 2, max(hw), scales=_fp8_scales(spec, blob, 64), layer_prec=mix)


def _full_size(netfn, seed, batch, side, prec, frames, layer_prec=None, tuned=False):
    """Full-size batch on the GPU (the launch configuration bench.py times);
    the oracle recomputes the sampled frames one by one.  tuned: the plans the
    bench runs, found the same way (genetic FP8/BF16 precision search on the
    calibration frame, then the genetic tile search on the batch)."""
    import torch
    spec = netfn()
    _, x, blob = synth.workload_net(spec, seed, batch, side, side)
    sc = _fp8_scales(spec, blob, side) if prec == "fp8" else None
    with make_net(spec, prec=prec, max_batch=batch, max_side=side, layer_prec=layer_prec) as net:
        net.load_weights(blob)
        if sc is not None:
            net.set_act_scales(np.asarray(sc, np.float32))
        if tuned:
            if prec == "fp8":
                xc = synth.make_frames(synth.Stream(synth.SEED_CALIB), 1, 3, side, side)
                plan, ga = net.tune_precision(torch.from_numpy(xc).cuda(), 1, side, side, max_err=0.05,
                                              population=12, generations=8, reps=2, seed=3)
                print("precision plan", plan, ga)
            tiles, tr = net.tune_tiles(torch.from_numpy(x).cuda(), batch, side, side, population=12,
                                       generations=8, reps=3, seed=5)
            print("tile plan", tiles, tr)
        y = run_device(net, x)
        precs = net.layer_prec()
    assert np.isfinite(y).all()
    for f in frames:
        ex = oracle.forward(spec.layers, 3, x[f:f + 1], blob)
        qa = oracle.forward_quant(spec.layers, 3, x[f:f + 1], blob, precs, sc)
        e_x = oracle.normwise_rel_err(y[f:f + 1], ex)
        r_q = oracle.rms_rel_err(y[f:f + 1], qa)
        agree, npos, ties = oracle.argmax_agreement(y[f:f + 1], ex, TOL[prec])
        print("%s %s frame %d: vs exact %.3e, rms vs quant-aware %.3e, argmax %.4f (%d ties)"
              % (spec.name, prec, f, e_x, r_q, agree, ties))
        assert e_x <= TOL[prec] and r_q <= QRMS[prec] and agree >= 0.99


def test_19conv_448_b8_bf16_full_size():
    _full_size(synth.net_19conv, synth.SEED_19CONV, 8, 448, "bf16", [0, 7])


def test_19conv_448_b8_bf16_full_size_tuned_tiles():
    _full_size(synth.net_19conv, synth.SEED_19CONV, 8, 448, "bf16", [0, 7], tuned=True)


def test_19conv_448_b8_fp8_full_size_tuned_plans():
    _full_size(synth.net_19conv, synth.SEED_19CONV, 8, 448, "fp8", [0, 7], tuned=True)


def test_19conv_448_b8_fp8_full_size_mixed():
    _full_size(synth.net_19conv, synth.SEED_19CONV, 8, 448, "fp8", [3], layer_prec=MIX19)


def test_9conv_416_bf16_full_size():
    _full_size(synth.net_9conv, synth.SEED_9CONV, 1, 416, "bf16", [0])


def _step(r, prec, scale):
    """Spacing of the storage format at each reference value: a value the
    GPU rounded the other way differs from the oracle's by one such step."""
    a = np.abs(r)
    if prec == "bf16":
        return np.exp2(np.floor(np.log2(np.maximum(a, 2.0 ** -126))) - 7)
    v = a / scale   # E4M3: 3 fraction bits, subnormal spacing 2^-9
    return np.exp2(np.floor(np.log2(np.maximum(v, 2.0 ** -6))) - 3) * scale


@pytest.mark.parametrize("prec,mix", [("bf16", None), ("fp8", None), ("fp8", MIX19)])
def test_per_layer_error_report(prec, mix):
    """Every layer checked on its own: the quantisation-aware oracle's layer l
    applied to the GPU's own (stored) layer l-1 output, so no earlier
    layer's rounding flips reach it.  A stored output may differ from the
    oracle only where the FP32 accumulator and FP64 round to neighbouring
    values of the storage format: by at most one step, in few elements.  The
    final FP32 map matches to 1e-5.  The end-to-end error of every layer
    against both oracles is printed beside it."""
    import torch
    spec = synth.net_19conv()
    s = synth.Stream(45)
    x = synth.make_frames(s, 1, 3, 64, 64)
    blob = synth.pack_blob(spec, synth.make_params(s, spec))
    params = synth.unpack_blob(spec, blob)
    precs = default_precs(spec, prec, mix)
    sc = _fp8_scales(spec, blob, 64) if prec == "fp8" else np.ones(len(spec.layers))
    exs = oracle.forward(spec.layers, 3, x, blob, keep_all=True)
    qas = oracle.forward_quant(spec.layers, 3, x, blob, precs, sc, keep_all=True)
    with make_net(spec, prec=prec, max_batch=1, max_side=64, layer_prec=mix) as net:
        net.load_weights(blob)
        if prec == "fp8":
            net.set_act_scales(np.asarray(sc, np.float32))
        outs = [torch.full(r.shape, float("nan"), device="cuda") for r in exs]
        net.forward_trace(torch.from_numpy(x).cuda(), 1, 64, 64, outs)
        torch.cuda.synchronize()
    outs = [o.cpu().numpy() for o in outs]
    n, a, cin = len(spec.layers), x, 3
    for l, (layer, p) in enumerate(zip(spec.layers, params)):
        o = outs[l]
        assert np.isfinite(o).all(), l
        one = synth.NetSpec("one", cin, [layer])
        last = l + 1 == n
        store = None if last else (precs[l + 1], sc[l + 1] if precs[l + 1] == "fp8" else 1.0)
        loc = oracle.forward_quant(one.layers, cin, a, synth.pack_blob(one, [p]), [precs[l]], [sc[l]],
                                   out_store=store)
        d = np.abs(o - loc)
        e_loc = oracle.normwise_rel_err(o, loc)
        r_loc = oracle.rms_rel_err(o, loc)
        flips = float((d > 1e-5 * np.abs(loc).max()).mean())   # stored values that moved
        print("layer %2d %s: local max %.3e rms %.3e, %.4f%% elements moved | end to end: vs exact %.3e, "
              "vs quant-aware %.3e (rms %.3e)"
              % (l, precs[l], e_loc, r_loc, 100.0 * flips, oracle.normwise_rel_err(o, exs[l]),
                 oracle.normwise_rel_err(o, qas[l]), oracle.rms_rel_err(o, qas[l])))
        if last:
            assert e_loc <= 1e-5, (l, e_loc)
        else:
            # each side rounds its own sum (FP32 accumulator / FP64) to the
            # nearest stored value: |g - r| <= half a step at g + half a step
            # at r + the accumulators' difference, at most 1e-5 of the layer's
            # largest value (which also covers the FP32 product code * scale
            # the trace writes for an FP8 value)
            eps = 1e-5 * np.abs(loc).max()
            bound = 0.5 * (_step(loc, store[0], store[1]) + _step(o, store[0], store[1])) + eps
            assert (d <= bound).all(), (l, float((d / bound).max()))
            assert flips <= 1e-2, (l, flips)
            assert r_loc <= 2e-3, (l, r_loc)
        a, cin = o, layer.cout


@pytest.mark.parametrize("cin,cout,k,pool,hw,bn", [
    (64, 256, 3, synth.POOL_NONE, (56, 40), 64),     # 4 N tiles, tap-merged stages
    (64, 128, 3, synth.POOL_2X2S2, (48, 64), 64),    # 2 N tiles, pooled
    (512, 256, 1, synth.POOL_NONE, (28, 28), 64),    # 1x1, 4 N tiles, 8 K chunks resident
])
def test_resident_weights_several_n_tiles(cin, cout, k, pool, hw, bn):
    """Weights resident in shared memory with several N tiles: the grid is a
    multiple of the N tile count and every CTA keeps its own tile's weights
    (forced through the tile override).  Checked against the
    quantisation-aware oracle like the other single layers."""
    L = synth.Layer
    spec = synth.NetSpec("layer", cin, [L(k, cout, True, synth.ACT_LEAKY, pool)])
    s = synth.Stream(cin * 3 + cout + bn)
    x = synth.make_frames(s, 2, cin, hw[0], hw[1], -1, 1)
    blob = synth.pack_blob(spec, synth.make_params(s, spec))
    precs = default_precs(spec, "bf16")
    qa = oracle.forward_quant(spec.layers, cin, x, blob, precs)
    with make_net(spec, prec="bf16", max_batch=2, max_side=max(hw)) as net:
        net.load_weights(blob)
        net.set_layer_tiles(0, bn, 1)
        assert net.plan_tiles(2, hw[0], hw[1])[0] == (bn, 1)
        y = run_device(net, x)
    e = oracle.normwise_rel_err(y, qa)
    print("resident %d N tiles: err %.3e" % (-(-cout // bn), e))
    assert np.isfinite(y).all() and e <= 1e-4
