"""net_conv2d_f32_noalloc: the conv-layer entry point for callers that cannot
allocate device memory when they call (graph capture in progress, real-time
loops, fixed memory budgets).  Its output must match the network path
(net_forward_device on a one-layer network) within the FP32 tolerance the
other tests use, on consecutive calls that reuse the shared static scratch.

Kept in a file collected last so that a stop-at-first-failure run has
already run every other test.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1811_03882_gb300 import synth
from helpers import make_net, run_device

pytestmark = pytest.mark.gpu
TOL32 = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1811_03882_gb300 import build
    build.build()
    oracle.build()


def _layer_case(seed, n, cin, h, w, cout, k, act, pool):
    spec = synth.NetSpec("one", cin, [synth.Layer(k, cout, False, act, pool)])
    s = synth.Stream(seed)
    x = synth.make_frames(s, n, cin, h, w, -1.0, 1.0)
    p = synth.make_params(s, spec)[0]
    return spec, x, p


def _free_bytes():
    from paper_1811_03882_gb300 import binding  # noqa: F401  (library loaded)
    import torch
    free, _ = torch.cuda.mem_get_info()
    return free


def _noalloc(x, p, cout, k, act, pool, free_delta=None):
    import torch
    from paper_1811_03882_gb300 import binding
    n, cin, h, w = x.shape
    ho, wo = (h // 2, w // 2) if pool == synth.POOL_2X2S2 else (h, w)
    d_x = torch.from_numpy(x).cuda()
    d_w = torch.from_numpy(np.ascontiguousarray(p.w)).cuda()
    d_b = torch.from_numpy(p.bias).cuda()
    d_y = torch.full((n, cout, ho, wo), float("nan"), device="cuda")
    torch.cuda.synchronize()
    free0 = _free_bytes()
    binding.conv2d_f32_noalloc(d_x, n, cin, h, w, d_w, d_b, cout, k, act, pool, d_y, None)
    torch.cuda.synchronize()
    if free_delta is not None:
        free_delta.append(free0 - _free_bytes())
    return d_y.cpu().numpy()


CASES = [
    # split-K active (few output tiles, K = 9 * 64): partial sums in the static scratch
    (71, 1, 64, 26, 26, 128, 3, synth.ACT_LEAKY, synth.POOL_2X2S2),
    # a different layer right after it: 1x1, linear, no pool, batch 2
    (72, 2, 256, 13, 13, 64, 1, synth.ACT_LINEAR, synth.POOL_NONE),
    # 20 outputs (not a multiple of 8: the reduction's 4-wide path, padded
    # weight rows) over 37 inputs (odd, padded to 40), split in two along K
    (73, 1, 37, 20, 22, 20, 3, synth.ACT_LEAKY, synth.POOL_2X2S2),
    # scratch within 11 KB of the array's end: 796 -> 72 channels on 42 x 46,
    # K split 17 ways on 148 to 152 SMs, so the partial sums fill the tail
    (74, 1, 796, 42, 46, 72, 3, synth.ACT_LEAKY, synth.POOL_NONE),
    # the packed input alone nearly fills the array (1440 x 1440 x 4 floats)
    (75, 1, 4, 1440, 1440, 8, 3, synth.ACT_LINEAR, synth.POOL_NONE),
]


def test_noalloc_matches_network_path_on_consecutive_calls():
    outs = []
    for case in CASES:
        seed, n, cin, h, w, cout, k, act, pool = case
        spec, x, p = _layer_case(seed, n, cin, h, w, cout, k, act, pool)
        blob = synth.pack_blob(spec, [p])
        with make_net(spec, max_batch=n, max_side=max(h, w)) as net:
            net.load_weights(blob)
            ref_path = run_device(net, x)
        y = _noalloc(x, p, cout, k, act, pool)
        assert y.shape == ref_path.shape
        assert np.isfinite(y).all()
        assert oracle.normwise_rel_err(y, ref_path) <= TOL32
        assert oracle.normwise_rel_err(y, oracle.forward(spec.layers, cin, x, blob)) <= TOL32
        outs.append(y)
    # the second call left the first layer's scratch contents behind; running
    # the first case again must still give its own result
    seed, n, cin, h, w, cout, k, act, pool = CASES[0]
    _, x, p = _layer_case(seed, n, cin, h, w, cout, k, act, pool)
    delta = []
    again = _noalloc(x, p, cout, k, act, pool, free_delta=delta)
    assert delta[0] <= 0                   # the call itself allocated no device memory
    assert oracle.normwise_rel_err(again, outs[0]) <= TOL32


def test_noalloc_rejects_layers_beyond_the_scratch():
    import torch
    from paper_1811_03882_gb300 import binding
    d = torch.zeros(16, device="cuda")
    # 8 x 512 x 448 x 448 float32 input alone is 3.3 GB of scratch
    with pytest.raises(binding.NetError) as e:
        binding.conv2d_f32_noalloc(d, 8, 512, 448, 448, d, d, 64, 3, 1, 0, d, None)
    assert e.value.status == binding.NET_E_INVAL
    assert "scratch" in str(e.value)
    with pytest.raises(binding.NetError) as e:   # stride-1 pool is not offered here
        binding.conv2d_f32_noalloc(d, 1, 4, 8, 8, d, d, 4, 3, 1, 2, d, None)
    assert e.value.status == binding.NET_E_INVAL
