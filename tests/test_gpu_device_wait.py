"""Failure detection on the device, without a GPU fault: every wait inside
the tensor-core conv kernel is bounded.  net_inject_device_fault makes one
layer of the next pass run with a ~1 ms bound while one of its K steps is
never loaded, so the MMA issuer's wait for it expires.  The kernel must
record the failure in the host-mapped flag, drain its copies and MMAs, free
its tensor memory and return: the pass reports NET_E_DEVICE_WAIT, the CUDA
context stays usable, and the next pass on the same handle is correct."""
import numpy as np
import pytest

import oracle
from paper_1811_03882_gb300 import synth
from helpers import make_net

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1811_03882_gb300 import build
    build.build()
    oracle.build()


@pytest.mark.parametrize("layer", [13, 2])
def test_expired_device_wait_is_reported_and_handle_recovers(layer):
    import torch
    from paper_1811_03882_gb300 import binding
    spec = synth.net_19conv()
    _, x, blob = synth.workload_net(spec, 61, 2, 64, 64)
    ref = oracle.forward(spec.layers, 3, x, blob)
    with make_net(spec, prec="bf16", max_batch=2, max_side=64) as net:
        net.load_weights(blob)
        y0 = net.forward(x)
        assert oracle.normwise_rel_err(y0, ref) <= 2e-2
        net.inject_device_fault(layer)
        with pytest.raises(binding.NetError) as e:
            net.forward(x)
        assert e.value.status == binding.NET_E_DEVICE_WAIT
        assert "expired" in str(e.value)
        torch.cuda.synchronize()                 # the context is still usable
        y1 = net.forward(x)
        np.testing.assert_array_equal(y1, y0)    # the next pass is unaffected
        y2 = net.forward(x)
        np.testing.assert_array_equal(y2, y0)
    with make_net(spec, prec="fp32", max_batch=1, max_side=64) as n32:
        with pytest.raises(binding.NetError) as e:
            n32.inject_device_fault(layer)       # CUDA-core layers have no such waits
        assert e.value.status == binding.NET_E_INVAL


def test_expired_band_wait_is_reported_and_pass_ends_at_once():
    """A layer on the row-band dataflow whose band wait expires (a count the
    previous layer never reaches, ~1 ms bound) aborts like any other wait;
    the layers after it, which wait on its bands, are released by its
    finished-warp count instead of waiting out their own bounds, so the pass
    ends within a fraction of a second; the next passes are unaffected."""
    import time
    import torch
    from paper_1811_03882_gb300 import binding
    spec = synth.net_19conv()
    _, x, blob = synth.workload_net(spec, 62, 2, 64, 64)
    with make_net(spec, prec="bf16", max_batch=2, max_side=64) as net:
        net.load_weights(blob)
        y0 = net.forward(x)
        flow = net.plan_flow(2, 64, 64)
        layers = [l for l, f in enumerate(flow) if f]
        assert layers, flow
        with pytest.raises(binding.NetError):
            net.inject_flow_fault(0, 2, 64, 64)   # the first layer never waits on bands
        for layer in (layers[0], layers[-1]):
            net.inject_flow_fault(layer, 2, 64, 64)
            t0 = time.perf_counter()
            with pytest.raises(binding.NetError) as e:
                net.forward(x)
            assert time.perf_counter() - t0 < 0.5, layer
            assert e.value.status == binding.NET_E_DEVICE_WAIT
            torch.cuda.synchronize()
            np.testing.assert_array_equal(net.forward(x), y0)
            np.testing.assert_array_equal(net.forward(x), y0)

