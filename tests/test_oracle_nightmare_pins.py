"""Pins of the nightmare oracle (oracle.conv2d_bwd_data, oracle/nightmare.py)
against facts that do not come from it: the adjoint identity
<conv(x), y> = <x, conv_bwd(y)>, torch autograd in float64 (conv, leaky,
both max pools, whole networks with batchnorm unfolded), brute force on a
tiny case, hand-worked max-pool ties (tests/golden/maxpool_bwd_ties.txt)
and a finite difference of the objective."""
import os

import numpy as np
import pytest
import torch
import torch.nn.functional as F

import oracle
from oracle import nightmare
from paper_1811_03882_gb300 import synth
from test_oracle_pins import _blocks

GOLD = os.path.join(os.path.dirname(__file__), "golden", "maxpool_bwd_ties.txt")


@pytest.mark.parametrize("k,shape", [(3, (2, 3, 5, 7)), (1, (1, 4, 3, 3)), (3, (1, 2, 1, 1))])
def test_conv_bwd_data_adjoint_and_autograd(orc, k, shape):
    rng = np.random.default_rng(k + shape[1])
    N, C, H, W = shape
    O = 5
    x = rng.standard_normal(shape)
    w = rng.standard_normal((O, C, k, k))
    y = rng.standard_normal((N, O, H, W))
    dx = orc.conv2d_bwd_data(y, w)
    assert np.sum(orc.conv2d(x, w) * y) == pytest.approx(np.sum(x * dx), rel=1e-12)
    xt = torch.from_numpy(x).requires_grad_(True)
    (F.conv2d(xt, torch.from_numpy(w), padding=k // 2) * torch.from_numpy(y)).sum().backward()
    np.testing.assert_allclose(dx, xt.grad.numpy(), rtol=1e-12, atol=1e-12)


def test_conv_bwd_data_brute_force(orc):
    rng = np.random.default_rng(9)
    dy = rng.standard_normal((1, 2, 3, 4))
    w = rng.standard_normal((2, 3, 3, 3))
    dx = orc.conv2d_bwd_data(dy, w)
    ref = np.zeros((1, 3, 3, 4))
    for c in range(3):
        for i in range(3):
            for j in range(4):
                for o in range(2):
                    for kh in range(3):
                        for kw in range(3):
                            a, b = i - kh + 1, j - kw + 1
                            if 0 <= a < 3 and 0 <= b < 4:
                                ref[0, c, i, j] += dy[0, o, a, b] * w[o, c, kh, kw]
    np.testing.assert_allclose(dx, ref, rtol=1e-13, atol=1e-13)


def test_pool_and_leaky_bwd_vs_autograd():
    rng = np.random.default_rng(4)
    h = rng.standard_normal((2, 3, 6, 8))
    g2 = rng.standard_normal((2, 3, 3, 4))
    ht = torch.from_numpy(h).requires_grad_(True)
    (F.max_pool2d(ht, 2, 2) * torch.from_numpy(g2)).sum().backward()
    np.testing.assert_allclose(nightmare.maxpool2_s2_bwd(g2, h), ht.grad.numpy(), rtol=0, atol=1e-15)
    h1 = rng.standard_normal((1, 2, 5, 7))
    g1 = rng.standard_normal(h1.shape)
    ht = torch.from_numpy(h1).requires_grad_(True)
    (F.max_pool2d(F.pad(ht, (0, 1, 0, 1), value=-float("inf")), 2, 1) * torch.from_numpy(g1)).sum().backward()
    np.testing.assert_allclose(nightmare.maxpool2_s1_same_bwd(g1, h1), ht.grad.numpy(), rtol=0, atol=1e-14)
    z = rng.standard_normal((2, 3, 4, 4))
    gz = rng.standard_normal(z.shape)
    zt = torch.from_numpy(z).requires_grad_(True)
    (F.leaky_relu(zt, 0.1) * torch.from_numpy(gz)).sum().backward()
    np.testing.assert_allclose(nightmare.leaky_bwd(gz, z), zt.grad.numpy(), rtol=1e-15, atol=0)


def test_pool_bwd_ties_by_hand():
    g = _blocks(GOLD)
    d = nightmare.maxpool2_s2_bwd(g["g_s2"][None, None], g["h_s2"][None, None])
    np.testing.assert_array_equal(d[0, 0], g["d_s2"])
    d = nightmare.maxpool2_s1_same_bwd(g["g_s1"][None, None], g["h_s1"][None, None])
    np.testing.assert_array_equal(d[0, 0], g["d_s1"])


def _torch_grad(spec, x, blob, layer):
    """Independent float64 composition with torch autograd."""
    ps = synth.unpack_blob(spec, blob)
    xt = torch.from_numpy(x.astype(np.float64)).requires_grad_(True)
    a = xt
    for l, p in list(zip(spec.layers, ps))[:layer + 1]:
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
    J = 0.5 * (a * a).sum()
    J.backward()
    return xt.grad.numpy(), float(J.detach())


@pytest.mark.parametrize("layer", [0, 3, 5, 6, 8])
def test_input_grad_vs_autograd(orc, layer):
    spec = synth.net_9conv()
    s = synth.Stream(95)
    x = synth.make_frames(s, 1, 3, 32, 32)
    blob = synth.pack_blob(spec, synth.make_params(s, spec))
    g, J = nightmare.input_grad(spec.layers, 3, x, blob, layer)
    gt, Jt = _torch_grad(spec, x, blob, layer)
    assert J == pytest.approx(Jt, rel=1e-12)
    assert np.abs(g - gt).max() <= 1e-10 * np.abs(gt).max()


def test_input_grad_finite_difference(orc):
    spec = synth.NetSpec("two", 3, [synth.leaky_bn(3, 8, synth.POOL_2X2S2), synth.leaky_bn(3, 6)])
    s = synth.Stream(96)
    x = synth.make_frames(s, 1, 3, 8, 8).astype(np.float64)
    blob = synth.pack_blob(spec, synth.make_params(s, spec))
    g, J = nightmare.input_grad(spec.layers, 3, x, blob, 1)
    rng = np.random.default_rng(0)
    for _ in range(5):
        idx = tuple(int(rng.integers(0, n)) for n in x.shape)
        e = 1e-6
        xp, xm = x.copy(), x.copy()
        xp[idx] += e
        xm[idx] -= e
        fd = (nightmare.input_grad(spec.layers, 3, xp, blob, 1)[1] - nightmare.input_grad(spec.layers, 3, xm, blob, 1)[1]) / (2 * e)
        assert fd == pytest.approx(g[idx], rel=1e-5, abs=1e-7)


def test_ascent_step_closed_form():
    x = np.ones((2, 1, 2, 2))
    g = np.array([[[[1.0, -1.0], [2.0, 0.0]]], [[[0.5, 0.5], [0.5, 0.5]]]])
    y = nightmare.ascent_step(x, g, 0.1)
    np.testing.assert_allclose(y[0, 0], 1 + 0.1 * g[0, 0] / 1.0)
    np.testing.assert_allclose(y[1, 0], 1 + 0.1 * 1.0)
