"""Pins of the FP64 oracle against facts that do not come from the oracle.

Each test checks one layer function (or the whole pass) against a
hand-computed example, a closed form, an invariant, brute force in plain
Python, or an independent library routine (torch CPU, float64).  A dropped
term, a wrong sign, an index slip or a transposed operand in oracle.c fails
at least one of them.
"""
import itertools
import os

import numpy as np
import pytest
import torch
import torch.nn.functional as F

from paper_1811_03882_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _blocks(path):
    """Parses a golden file: a '# name' line (one token) opens a block of
    numeric rows; '#' lines with more words are commentary."""
    out, name = {}, None
    for line in open(path):
        line = line.strip()
        if not line:
            continue
        if line.startswith("#"):
            tag = line[1:].split()
            name = tag[0] if len(tag) == 1 else None
            if name:
                out[name] = []
            continue
        if name is not None:
            out[name].append([float(t) for t in line.split()])
    return {k: np.array(v) for k, v in out.items()}


def _rng(seed):
    return np.random.default_rng(seed)


# ------------------------------------------------------------------ conv
def test_conv_hand_examples(orc):
    g = _blocks(os.path.join(GOLD, "conv_3x3_hand.txt"))
    for case in "AB":
        x = g[case + ".input"][None, None]
        w = g[case + ".kernel"][None, None]
        y = orc.conv2d(x, w)[0, 0]
        np.testing.assert_array_equal(y, g[case + ".output"])


def _brute_conv(x, w):
    """Pure-Python loops over the definition (tiny inputs only)."""
    N, C, H, W = x.shape
    O, _, k, _ = w.shape
    p = (k - 1) // 2
    y = np.zeros((N, O, H, W))
    for n, o, i, j in itertools.product(range(N), range(O), range(H), range(W)):
        s = 0.0
        for c, kh, kw in itertools.product(range(C), range(k), range(k)):
            ii, jj = i + kh - p, j + kw - p
            if 0 <= ii < H and 0 <= jj < W:
                s += x[n, c, ii, jj] * w[o, c, kh, kw]
        y[n, o, i, j] = s
    return y


@pytest.mark.parametrize("shape", [(1, 2, 3, 4, 3, 3), (2, 3, 5, 2, 2, 1), (1, 1, 1, 1, 2, 3)])
def test_conv_brute_force(orc, shape):
    N, C, H, W, O, k = shape
    r = _rng(1)
    x = r.standard_normal((N, C, H, W))
    w = r.standard_normal((O, C, k, k))
    np.testing.assert_allclose(orc.conv2d(x, w), _brute_conv(x, w), rtol=0, atol=1e-12)


@pytest.mark.parametrize("k", [1, 3])
@pytest.mark.parametrize("hw", [(7, 9), (16, 16), (1, 5)])
def test_conv_vs_torch(orc, k, hw):
    r = _rng(2)
    x = r.standard_normal((2, 5, *hw))
    w = r.standard_normal((6, 5, k, k))
    ref = F.conv2d(torch.from_numpy(x), torch.from_numpy(w), padding=k // 2).numpy()
    np.testing.assert_allclose(orc.conv2d(x, w), ref, rtol=0, atol=1e-11)


def test_conv1x1_is_matmul(orc):
    r = _rng(3)
    x = r.standard_normal((2, 7, 5, 6))
    w = r.standard_normal((4, 7, 1, 1))
    ref = np.einsum("nchw,oc->nohw", x, w[:, :, 0, 0])
    np.testing.assert_allclose(orc.conv2d(x, w), ref, rtol=0, atol=1e-12)


def test_conv_delta_kernel_is_identity(orc):
    r = _rng(4)
    x = r.standard_normal((1, 4, 6, 5))
    w = np.zeros((4, 4, 3, 3))
    for c in range(4):
        w[c, c, 1, 1] = 1.0
    np.testing.assert_array_equal(orc.conv2d(x, w), x)


def test_conv_linear_in_x(orc):
    r = _rng(5)
    x1, x2 = r.standard_normal((2, 1, 3, 8, 8))
    w = r.standard_normal((5, 3, 3, 3))
    a, b = 0.75, -2.5
    lhs = orc.conv2d(a * x1 + b * x2, w)
    rhs = a * orc.conv2d(x1, w) + b * orc.conv2d(x2, w)
    np.testing.assert_allclose(lhs, rhs, rtol=0, atol=1e-12)


def test_conv_translation_equivariance_interior(orc):
    r = _rng(6)
    x = r.standard_normal((1, 2, 10, 10))
    w = r.standard_normal((3, 2, 3, 3))
    y = orc.conv2d(x, w)
    xs = np.roll(x, (1, 2), axis=(2, 3))
    ys = orc.conv2d(xs, w)
    # interior outputs whose receptive field avoids the wrapped rows/cols
    np.testing.assert_allclose(ys[..., 3:9, 4:9], y[..., 2:8, 2:7], rtol=0, atol=1e-12)


# ------------------------------------------------------------ bn / bias
def test_batchnorm_hand_value(orc):
    y = np.full((1, 1, 1, 1), 2.0)
    # gamma*(y-mean)/sqrt(var+eps)+beta = 3*(2-1)/2 + 0.5 = 2.0
    out = orc.batchnorm(y, [3.0], [0.5], [1.0], [4.0 - orc.BN_EPS])
    assert out[0, 0, 0, 0] == pytest.approx(2.0, abs=1e-15)


def test_batchnorm_vs_torch(orc):
    r = _rng(7)
    y = r.standard_normal((2, 4, 3, 3))
    g, b, m = r.uniform(0.5, 1.5, 4), r.uniform(-.1, .1, 4), r.uniform(-.1, .1, 4)
    v = r.uniform(0.5, 1.5, 4)
    ref = F.batch_norm(torch.from_numpy(y), torch.from_numpy(m), torch.from_numpy(v),
                       torch.from_numpy(g), torch.from_numpy(b), False, 0.0, orc.BN_EPS).numpy()
    np.testing.assert_allclose(orc.batchnorm(y, g, b, m, v), ref, rtol=0, atol=1e-13)


def test_bn_then_conv_equals_folded_conv(orc):
    """conv -> BN (unfolded) == conv with W*s plus b' (algebraic identity)."""
    r = _rng(8)
    x = r.standard_normal((1, 3, 6, 6))
    p = {"w": r.standard_normal((4, 3, 3, 3)), "gamma": r.uniform(.5, 1.5, 4),
         "beta": r.uniform(-.1, .1, 4), "mean": r.uniform(-.1, .1, 4), "var": r.uniform(.5, 1.5, 4)}
    unf = orc.batchnorm(orc.conv2d(x, p["w"]), p["gamma"], p["beta"], p["mean"], p["var"])
    wf, bf = orc.fold(p)
    fol = orc.add_bias(orc.conv2d(x, wf), bf)
    np.testing.assert_allclose(unf, fol, rtol=0, atol=1e-12)


def test_bias(orc):
    y = np.zeros((1, 2, 2, 2))
    out = orc.add_bias(y, [1.5, -2.0])
    assert (out[0, 0] == 1.5).all() and (out[0, 1] == -2.0).all()


# ---------------------------------------------------------------- leaky
def test_leaky_piecewise_linear(orc):
    v = np.array([-3.0, -1e-300, 0.0, 1e-300, 2.5, -0.0])
    out = orc.leaky(v)
    np.testing.assert_array_equal(out, np.where(v > 0, v, 0.1 * v))
    assert out[2] == 0.0


def test_leaky_positively_homogeneous_and_torch(orc):
    r = _rng(9)
    v = r.standard_normal(1000)
    for a in (0.5, 3.0):
        np.testing.assert_allclose(orc.leaky(a * v), a * orc.leaky(v), rtol=1e-15, atol=0)
    ref = F.leaky_relu(torch.from_numpy(v), 0.1).numpy()
    np.testing.assert_allclose(orc.leaky(v), ref, rtol=1e-15, atol=0)


# ----------------------------------------------------------------- pool
def test_maxpool_s2_vs_torch_and_const(orc):
    r = _rng(10)
    x = r.standard_normal((2, 3, 6, 8))
    ref = F.max_pool2d(torch.from_numpy(x), 2, 2).numpy()
    np.testing.assert_array_equal(orc.maxpool2_s2(x), ref)
    c = np.full((1, 2, 4, 4), -1.25)
    np.testing.assert_array_equal(orc.maxpool2_s2(c), np.full((1, 2, 2, 2), -1.25))


def test_maxpool_commutes_with_leaky(orc):
    r = _rng(11)
    x = r.standard_normal((1, 3, 8, 8))
    np.testing.assert_array_equal(orc.maxpool2_s2(orc.leaky(x)), orc.leaky(orc.maxpool2_s2(x)))
    np.testing.assert_array_equal(orc.maxpool2_s1_same(orc.leaky(x)),
                                  orc.leaky(orc.maxpool2_s1_same(x)))


def test_maxpool_s1_same_hand_example(orc):
    g = _blocks(os.path.join(GOLD, "maxpool_2x2_s1_same_3x3.txt"))
    y = orc.maxpool2_s1_same(g["input"][None, None])[0, 0]
    np.testing.assert_array_equal(y, g["output"])


def test_maxpool_s1_same_vs_padded_torch(orc):
    r = _rng(12)
    x = r.standard_normal((2, 3, 13, 13))
    xp = F.pad(torch.from_numpy(x), (0, 1, 0, 1), value=-np.inf)
    ref = F.max_pool2d(xp, 2, 1).numpy()
    np.testing.assert_array_equal(orc.maxpool2_s1_same(x), ref)
    c = np.full((1, 1, 5, 5), 0.5)
    np.testing.assert_array_equal(orc.maxpool2_s1_same(c), c)


# ------------------------------------------------------------- rounding
def test_round_bf16_vs_torch(orc):
    r = _rng(13)
    v = np.concatenate([r.standard_normal(20000) * 10.0 ** r.integers(-30, 30, 20000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.01171875, 3.0e38]]).astype(np.float32)
    ref = torch.from_numpy(v).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(orc.round_bf16(v.astype(np.float64)), ref)


def test_round_e4m3_hand_cases(orc):
    rows = [l.split() for l in open(os.path.join(GOLD, "e4m3_cases.txt"))
            if l.strip() and not l.startswith("#")]
    v = np.array([float(a) for a, _ in rows])
    e = np.array([float(b) for _, b in rows])
    np.testing.assert_array_equal(orc.round_e4m3_sat(v), e)


def test_round_e4m3_vs_torch_in_range(orc):
    r = _rng(14)
    v = (r.standard_normal(20000) * 2.0 ** r.integers(-12, 8, 20000)).astype(np.float32)
    v = np.clip(v, -448, 448)
    ref = torch.from_numpy(v).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    np.testing.assert_array_equal(orc.round_e4m3_sat(v.astype(np.float64)), ref)


# ---------------------------------------------------------- whole pass
def _torch_forward(spec, x, blob):
    """Independent float64 composition from torch library routines."""
    ps = synth.unpack_blob(spec, blob)
    a = torch.from_numpy(x.astype(np.float64))
    for l, p in zip(spec.layers, ps):
        y = F.conv2d(a, torch.from_numpy(p.w.astype(np.float64)), padding=l.k // 2)
        if l.bn:
            y = F.batch_norm(y, torch.from_numpy(p.mean.astype(np.float64)),
                             torch.from_numpy(p.var.astype(np.float64)),
                             torch.from_numpy(p.gamma.astype(np.float64)),
                             torch.from_numpy(p.beta.astype(np.float64)), False, 0.0, 1e-5)
        else:
            y = y + torch.from_numpy(p.bias.astype(np.float64))[None, :, None, None]
        if l.act == synth.ACT_LEAKY:
            y = F.leaky_relu(y, 0.1)
        if l.pool == synth.POOL_2X2S2:
            y = F.max_pool2d(y, 2, 2)
        elif l.pool == synth.POOL_2X2S1_SAME:
            y = F.max_pool2d(F.pad(y, (0, 1, 0, 1), value=-float("inf")), 2, 1)
        a = y
    return a.numpy()


@pytest.mark.parametrize("name,hw", [("single-conv", 32), ("9-conv", 64), ("19-conv", 64)])
def test_forward_vs_torch_composition(orc, name, hw):
    spec = synth.NETS[name]()
    s = synth.Stream(77)
    x = synth.make_frames(s, 2, spec.in_c, hw, hw, -1.0, 1.0)
    blob = synth.pack_blob(spec, synth.make_params(s, spec))
    got = orc.forward(spec.layers, spec.in_c, x, blob)
    ref = _torch_forward(spec, x, blob)
    assert got.shape == ref.shape
    assert orc.normwise_rel_err(got, ref) < 1e-12


def test_forward_quant_fp32_close_to_exact(orc):
    spec = synth.net_9conv()
    s = synth.Stream(78)
    x = synth.make_frames(s, 1, 3, 64, 64)
    blob = synth.pack_blob(spec, synth.make_params(s, spec))
    ex = orc.forward(spec.layers, 3, x, blob)
    q32 = orc.forward_quant(spec.layers, 3, x, blob, ["fp32"] * len(spec.layers))
    assert orc.normwise_rel_err(q32, ex) < 1e-6
    qbf = orc.forward_quant(spec.layers, 3, x, blob, ["bf16"] * len(spec.layers))
    e = orc.normwise_rel_err(qbf, ex)
    assert 1e-4 < e < 2e-2   # BF16 storage is visible but within its budget


def test_forward_quant_fp8_scales(orc):
    spec = synth.net_single_conv()
    s = synth.Stream(79)
    x = synth.make_frames(s, 1, 16, 16, 16, -1.0, 1.0)
    blob = synth.pack_blob(spec, synth.make_params(s, spec))
    sc = orc.act_scales_from(spec.layers, 16, x, blob)
    assert sc[0] == pytest.approx(np.abs(x).max() / 448.0)
    ex = orc.forward(spec.layers, 16, x, blob)
    q8 = orc.forward_quant(spec.layers, 16, x, blob, ["fp8"], sc)
    e = orc.normwise_rel_err(q8, ex)
    assert 1e-3 < e < 8e-2


def test_weight_scale_fp8(orc):
    w = np.zeros((2, 1, 1, 3))
    w[0, 0, 0] = [1.0, -8.96, 2.0]
    w[1, 0, 0] = [0.5, 0.25, -0.125]
    np.testing.assert_allclose(orc.weight_scales_fp8(w), [8.96 / 448, 0.5 / 448])


def test_metrics(orc):
    r = np.array([[1.0, -4.0], [2.0, 0.0]])
    y = r + np.array([[0.0, 0.2], [0.0, 0.0]])
    assert orc.normwise_rel_err(y, r) == pytest.approx(0.05)
    assert orc.rms_rel_err(y, r) == pytest.approx(0.2 / np.sqrt(21.0))
    ref = np.zeros((1, 3, 1, 2))
    ref[0, :, 0, 0] = [1.0, 3.0, 2.0]
    ref[0, :, 0, 1] = [1.0, 1.0005, 0.0]   # near-tie at position 1
    got = ref.copy()
    got[0, :, 0, 1] = [1.0005, 1.0, 0.0]
    agree, n, ties = orc.argmax_agreement(got, ref, 1e-3)
    assert (agree, n, ties) == (1.0, 2, 1)


def test_parse_blob_length_check(orc):
    spec = synth.net_single_conv()
    blob = synth.workload_single()[2]
    orc.parse_blob(spec.layers, 16, blob)
    with pytest.raises(ValueError):
        orc.parse_blob(spec.layers, 16, blob[:-1])
