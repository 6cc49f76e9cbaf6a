"""Pins of the quantisation-aware oracle (``oracle.forward_quant``) and of
the FP8 activation scales (``oracle.act_scales_from``).

The reference here is an independent float64 composition written with torch
library routines: the batchnorm fold in float64, ``F.conv2d``, the roundings
done by torch's own ``bfloat16`` / ``float8_e4m3fn`` casts, per-output-channel
weight scales, the activation re-rounded before every layer, the bias kept in
FP32, the final map in FP32.  torch casts a float64 tensor to those formats
through float32, which would round twice; the composition therefore first
rounds to float32 *to odd* (truncate, then set the last bit when the value was
inexact; Boldo and Melquiond, "Emulation of FMA and correctly rounded sums:
proved algorithms using rounding to odd", IEEE TC 2008), after which one
round-to-nearest-even cast to a format of at most 22 significant bits equals
a single rounding of the float64 value.

Every layer's output must match to 1e-12 (both sides compute in float64 and
differ only in summation order).  ``test_pins_catch_plausible_slips`` shows
the comparison binds: each slip a reduced-precision oracle could plausibly
contain, planted in the composition, moves the result far past that bound.
"""
import numpy as np
import pytest
import torch
import torch.nn.functional as F

from paper_1811_03882_gb300 import synth
from helpers import default_precs

FP8_MAX = 448.0
TOL = 1e-12


# ------------------------------------------------------------- roundings
def _f32_odd(t):
    """float64 -> float32 rounded to odd (see module docstring)."""
    f = t.to(torch.float32)
    over = f.to(torch.float64).abs() > t.abs()                      # RNE went away from zero
    f = torch.where(over, torch.nextafter(f, torch.zeros_like(f)), f)   # now truncated
    inexact = f.to(torch.float64) != t
    bits = f.view(torch.int32)
    return torch.where(inexact, bits | 1, bits).view(torch.float32)


def _bf16(t):
    return _f32_odd(t).to(torch.bfloat16).to(torch.float64)


def _e4m3_sat(t):
    # satfinite: values beyond the largest finite E4M3 value clamp to +-448
    return _f32_odd(t.clamp(-FP8_MAX, FP8_MAX)).to(torch.float8_e4m3fn).to(torch.float64)


def _store(t, prec, scale, slip):
    if prec == "fp32":
        return t.to(torch.float32).to(torch.float64)
    if prec == "bf16":
        return t if slip == "no_reround" else _bf16(t)
    if slip == "scale_once":
        return _e4m3_sat(t / scale)
    return _e4m3_sat(t / scale) * scale


# ---------------------------------------------------- float64 compositions
def _fold(l, p):
    w = torch.from_numpy(p.w.astype(np.float64))
    if l.bn:
        s = torch.from_numpy(p.gamma.astype(np.float64)) / torch.sqrt(
            torch.from_numpy(p.var.astype(np.float64)) + 1e-5)
        b = torch.from_numpy(p.beta.astype(np.float64)) - torch.from_numpy(p.mean.astype(np.float64)) * s
        return w * s[:, None, None, None], b, w
    return w, torch.from_numpy(p.bias.astype(np.float64)), w


def _epilogue(l, y):
    if l.act == synth.ACT_LEAKY:
        y = F.leaky_relu(y, 0.1)
    if l.pool == synth.POOL_2X2S2:
        y = F.max_pool2d(y, 2, 2)
    elif l.pool == synth.POOL_2X2S1_SAME:
        y = F.max_pool2d(F.pad(y, (0, 1, 0, 1), value=-float("inf")), 2, 1)
    return y


def torch_forward_quant(spec, x, blob, precs, scales, slip=None):
    """Every layer's output of the reduced-precision pass (list)."""
    ps = synth.unpack_blob(spec, blob)
    n = len(spec.layers)
    a = _store(torch.from_numpy(x.astype(np.float64)), precs[0], scales[0] if precs[0] == "fp8" else 1.0, slip)
    outs = []
    for i, (l, p) in enumerate(zip(spec.layers, ps)):
        wf, bf, wraw = _fold(l, p)
        if precs[i] == "fp8":
            src = wraw if slip == "scale_before_fold" else wf
            sw = torch.clamp(src.abs().reshape(src.shape[0], -1).amax(dim=1), min=1e-30) / FP8_MAX
            wq = _e4m3_sat(wf / sw[:, None, None, None]) * sw[:, None, None, None]
        elif precs[i] == "bf16":
            wq = wf if slip == "weights_unrounded" else _bf16(wf)
        else:
            wq = wf.to(torch.float32).to(torch.float64)
        y = F.conv2d(a, wq, padding=l.k // 2)
        b = _bf16(bf) if slip == "bias_bf16" else bf.to(torch.float32).to(torch.float64)
        y = _epilogue(l, y + b[None, :, None, None])
        if i + 1 < n:
            nxt = precs[i + 1]
            a = _store(y, nxt, scales[i + 1] if nxt == "fp8" else 1.0, slip)
        else:
            a = y.to(torch.float32).to(torch.float64)
        outs.append(a.numpy())
    return outs


def torch_layer_inputs(spec, x, blob):
    """Exact float64 pass: the input of every layer (batchnorm unfolded)."""
    ps = synth.unpack_blob(spec, blob)
    a = torch.from_numpy(x.astype(np.float64))
    ins = []
    for l, p in zip(spec.layers, ps):
        ins.append(a.numpy())
        y = F.conv2d(a, torch.from_numpy(p.w.astype(np.float64)), padding=l.k // 2)
        if l.bn:
            y = F.batch_norm(y, torch.from_numpy(p.mean.astype(np.float64)),
                             torch.from_numpy(p.var.astype(np.float64)),
                             torch.from_numpy(p.gamma.astype(np.float64)),
                             torch.from_numpy(p.beta.astype(np.float64)), False, 0.0, 1e-5)
        else:
            y = y + torch.from_numpy(p.bias.astype(np.float64))[None, :, None, None]
        a = _epilogue(l, y)
    return ins


def _nerr(y, r):
    return float(np.abs(y - r).max() / max(np.abs(r).max(), 1e-300))


# ----------------------------------------------------------------- tests
def test_round_to_odd_cast_is_one_rounding(orc):
    """The composition's roundings of float64 values (random, near format
    midpoints, saturating, E4M3 subnormal) equal the oracle's direct ones;
    a plain cast through float32 rounds some near-midpoint values twice."""
    rng = np.random.default_rng(5)
    v = rng.standard_normal(20000) * np.exp2(rng.integers(-12, 12, 20000))
    # just above a BF16 midpoint by less than half a float32 ulp: float32 RNE
    # lands on the midpoint and a second RNE goes to even, i.e. down
    m = (1.0 + np.arange(1, 200) * 2.0 ** -7) + 2.0 ** -8
    near = m + 2.0 ** -30
    vv = np.concatenate([v, near, -near])
    got = _bf16(torch.from_numpy(vv)).numpy()
    np.testing.assert_array_equal(got, orc.round_bf16(vv))
    naive = torch.from_numpy(near).to(torch.bfloat16).to(torch.float64).numpy()
    assert (naive != orc.round_bf16(near)).any()
    e = np.concatenate([rng.standard_normal(20000) * 100.0, [500.0, -1000.0, 464.0, 2.0 ** -8, 3 * 2.0 ** -10],
                        (1.0 + np.arange(1, 8) * 2.0 ** -3 + 2.0 ** -4) + 2.0 ** -30])
    np.testing.assert_array_equal(_e4m3_sat(torch.from_numpy(e)).numpy(), orc.round_e4m3_sat(e))


MIX9 = ["bf16"] * 6 + ["fp8", "fp8"] + ["bf16"]
MIX19 = ["bf16"] * 13 + ["fp8", "bf16", "fp8", "bf16", "bf16", "bf16"]
PLANS = [("9-conv", "bf16", None, 64), ("9-conv", "fp8", None, 64), ("9-conv", "fp8", MIX9, 32),
         ("19-conv", "bf16", None, 64), ("19-conv", "fp8", None, 64), ("19-conv", "fp8", MIX19, 32)]


def _case(name, side, seed=91):
    spec = synth.NETS[name]()
    s = synth.Stream(seed)
    x = synth.make_frames(s, 2, 3, side, side)
    blob = synth.pack_blob(spec, synth.make_params(s, spec))
    return spec, x, blob


@pytest.mark.parametrize("name,prec,mix,side", PLANS)
def test_forward_quant_vs_torch_composition(orc, name, prec, mix, side):
    spec, x, blob = _case(name, side)
    precs = default_precs(spec, prec, mix)
    sc = orc.act_scales_from(spec.layers, 3, x[:1], blob)
    got = orc.forward_quant(spec.layers, 3, x, blob, precs, sc, keep_all=True)
    ref = torch_forward_quant(spec, x, blob, precs, sc)
    for l, (g, r) in enumerate(zip(got, ref)):
        assert g.shape == r.shape
        assert _nerr(g, r) <= TOL, (l, _nerr(g, r))


@pytest.mark.parametrize("name,side", [("9-conv", 64), ("19-conv", 64)])
def test_act_scales_every_layer(orc, name, side):
    spec, x, blob = _case(name, side, seed=92)
    sc = orc.act_scales_from(spec.layers, 3, x, blob)
    ins = torch_layer_inputs(spec, x, blob)
    assert len(sc) == len(ins) == len(spec.layers)
    for l, t in enumerate(ins):
        assert sc[l] == pytest.approx(np.abs(t).max() / FP8_MAX, rel=TOL), l


@pytest.mark.parametrize("slip", ["bias_bf16", "no_reround", "scale_once", "scale_before_fold",
                                  "weights_unrounded"])
def test_pins_catch_plausible_slips(orc, slip):
    """Each slip, planted in the composition, leaves the oracle far outside
    the 1e-12 bound on the final map; so an oracle containing it would fail
    test_forward_quant_vs_torch_composition."""
    spec, x, blob = _case("9-conv", 32, seed=93)
    precs = default_precs(spec, "fp8", MIX9)
    sc = orc.act_scales_from(spec.layers, 3, x[:1], blob)
    got = orc.forward_quant(spec.layers, 3, x, blob, precs, sc)
    good = torch_forward_quant(spec, x, blob, precs, sc)[-1]
    bad = torch_forward_quant(spec, x, blob, precs, sc, slip=slip)[-1]
    assert _nerr(got, good) <= TOL
    assert _nerr(got, bad) > 1e-4, slip


def test_single_layer_chain_equals_whole_pass(orc):
    """forward_quant over one layer with out_store (the next layer's format
    and scale), chained layer by layer, reproduces the whole pass's stored
    layer outputs exactly: the form the GPU tests use to check one layer on
    the GPU's own input."""
    spec, x, blob = _case("19-conv", 32, seed=94)
    precs = default_precs(spec, "fp8", MIX19)
    sc = orc.act_scales_from(spec.layers, 3, x[:1], blob)
    whole = orc.forward_quant(spec.layers, 3, x, blob, precs, sc, keep_all=True)
    params = synth.unpack_blob(spec, blob)
    a, cin, n = x, 3, len(spec.layers)
    for l, (layer, p) in enumerate(zip(spec.layers, params)):
        one = synth.NetSpec("one", cin, [layer])
        out = (precs[l + 1], sc[l + 1] if precs[l + 1] == "fp8" else 1.0) if l + 1 < n else None
        a = orc.forward_quant(one.layers, cin, a, synth.pack_blob(one, [p]), [precs[l]],
                              [sc[l]], out_store=out)
        np.testing.assert_array_equal(a, whole[l])
        cin = layer.cout
