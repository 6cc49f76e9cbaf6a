"""FP32 path on the GPU against the FP64 oracle (normwise max relative error
<= 1e-4 on the final map), through the C ABI."""
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


def test_single_conv_layer():
    spec, x, blob = synth.workload_single()
    ref = oracle.forward(spec.layers, spec.in_c, x, blob)
    with make_net(spec, max_side=32) as net:
        net.load_weights(blob)
        y = run_device(net, x)
        assert y.shape == ref.shape == (1, 32, 16, 16)
        assert oracle.normwise_rel_err(y, ref) <= TOL32
        # host API: 1 H2D + 1 D2H, identical result
        np.testing.assert_array_equal(net.forward(x), y)


def test_9conv_416_fp32_full_size():
    spec, x, blob = synth.workload_net(synth.net_9conv(), synth.SEED_9CONV, 1, 416, 416)
    ref = oracle.forward(spec.layers, 3, x, blob)
    with make_net(spec, max_side=416) as net:
        net.load_weights(blob)
        y = run_device(net, x)
    err = oracle.normwise_rel_err(y, ref)
    agree, _, _ = oracle.argmax_agreement(y, ref, TOL32)
    assert err <= TOL32, err
    assert agree >= 0.99


@pytest.mark.parametrize("n,h,w", [(2, 96, 160), (3, 64, 32), (1, 32, 32)])
def test_9conv_ragged_tiles(n, h, w):
    spec = synth.net_9conv()
    s = synth.Stream(1000 + h + w)
    x = synth.make_frames(s, n, 3, h, w)
    blob = synth.pack_blob(spec, synth.make_params(s, spec))
    ref = oracle.forward(spec.layers, 3, x, blob)
    with make_net(spec, max_batch=4, max_side=160) as net:
        net.load_weights(blob)
        y = run_device(net, x)
    assert oracle.normwise_rel_err(y, ref) <= TOL32


def test_9conv_per_layer_trace():
    import torch
    spec = synth.net_9conv()
    s = synth.Stream(31)
    x = synth.make_frames(s, 2, 3, 64, 96)
    blob = synth.pack_blob(spec, synth.make_params(s, spec))
    refs = oracle.forward(spec.layers, 3, x, blob, keep_all=True)
    with make_net(spec, max_batch=2, max_side=96) as net:
        net.load_weights(blob)
        outs = [torch.full(r.shape, float("nan"), device="cuda") for r in refs]
        net.forward_trace(torch.from_numpy(x).cuda(), 2, 64, 96, outs)
        torch.cuda.synchronize()
        for l, (o, r) in enumerate(zip(outs, refs)):
            assert oracle.normwise_rel_err(o.cpu().numpy(), r) <= TOL32, l


def test_19conv_fp32_small():
    spec = synth.net_19conv()
    s = synth.Stream(32)
    x = synth.make_frames(s, 2, 3, 64, 64)
    blob = synth.pack_blob(spec, synth.make_params(s, spec))
    ref = oracle.forward(spec.layers, 3, x, blob)
    with make_net(spec, max_batch=2, max_side=64) as net:
        net.load_weights(blob)
        y = run_device(net, x)
    assert oracle.normwise_rel_err(y, ref) <= TOL32


def test_s1_same_pool_odd_sizes_and_last_layer():
    L = synth.Layer
    spec = synth.NetSpec("s1", 5, [L(3, 24, True, synth.ACT_LEAKY, synth.POOL_2X2S1_SAME),
                                   L(1, 7, False, synth.ACT_LINEAR, synth.POOL_2X2S1_SAME)])
    s = synth.Stream(33)
    x = synth.make_frames(s, 2, 5, 13, 11, -1, 1)
    blob = synth.pack_blob(spec, synth.make_params(s, spec))
    ref = oracle.forward(spec.layers, 5, x, blob)
    with make_net(spec, max_batch=2, max_side=13) as net:
        net.load_weights(blob)
        y = run_device(net, x)
    assert y.shape == (2, 7, 13, 11)
    assert oracle.normwise_rel_err(y, ref) <= TOL32


def test_error_statuses():
    from paper_1811_03882_gb300 import binding
    spec, x, blob = synth.workload_single()
    with make_net(spec, max_side=32) as net:
        with pytest.raises(binding.NetError) as e:
            net.forward(x)
        assert e.value.status == binding.NET_E_WEIGHTS
        with pytest.raises(binding.NetError) as e:
            net.load_weights(blob[:-3])
        assert e.value.status == binding.NET_E_WEIGHTS
        net.load_weights(blob)
        with pytest.raises(binding.NetError) as e:
            net.forward(np.zeros((1, 16, 31, 32), np.float32))   # odd size before a s2 pool
        assert e.value.status == binding.NET_E_SHAPE
        with pytest.raises(binding.NetError) as e:
            net.forward(np.zeros((2, 16, 32, 32), np.float32))   # batch > max_batch
        assert e.value.status == binding.NET_E_SHAPE
        with pytest.raises(binding.NetError) as e:
            net.forward(np.zeros((1, 16, 64, 64), np.float32))   # side > max_side
        assert e.value.status == binding.NET_E_SHAPE
        with pytest.raises(binding.NetError) as e:
            net.forward(x, out=np.zeros(10, np.float32))
        assert e.value.status == binding.NET_E_INVAL
        # the handle still works after the rejected calls
        ref = oracle.forward(spec.layers, spec.in_c, x, blob)
        assert oracle.normwise_rel_err(net.forward(x), ref) <= TOL32
