"""net_forward_async / net_forward_wait: stream-ordered host API with two
staging slots.  Results must equal the synchronous net_forward bit for bit,
across slot reuse (more calls in flight than slots) and mixed with
synchronous calls; bad arguments fail on the host."""
import numpy as np
import pytest

from paper_1811_03882_gb300 import synth
from helpers import make_net

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1811_03882_gb300 import build
    build.build()


def test_async_matches_sync_across_slot_reuse():
    import torch
    from paper_1811_03882_gb300 import binding
    spec = synth.net_9conv()
    blob = synth.weights_for(spec, 81)
    xs = [synth.make_frames(synth.Stream(81 + i), 2, 3, 128, 128) for i in range(5)]
    with make_net(spec, prec="bf16", max_batch=2, max_side=128) as net:
        net.load_weights(blob)
        c, ho, wo = net.output_shape(128, 128)
        ref = [net.forward(x) for x in xs]
        # pinned host buffers, five calls in flight over two slots
        hin = [torch.from_numpy(x).pin_memory() for x in xs]
        hout = [torch.full((2, c, ho, wo), float("nan")).pin_memory() for _ in xs]
        for a, b in zip(hin, hout):
            net.forward_async(a.numpy(), b.numpy())
        net.forward_wait()
        for r, b in zip(ref, hout):
            np.testing.assert_array_equal(b.numpy(), r)
        # a synchronous call between asynchronous ones
        o = np.full((2, c, ho, wo), np.nan, np.float32)
        net.forward_async(hin[1].numpy(), hout[0].numpy())
        np.testing.assert_array_equal(net.forward(xs[3]), ref[3])
        net.forward_async(hin[2].numpy(), o)
        net.forward_wait()
        np.testing.assert_array_equal(hout[0].numpy(), ref[1])
        np.testing.assert_array_equal(o, ref[2])
        with pytest.raises(binding.NetError) as e:
            net.forward_async(hin[0].numpy(), np.zeros(4, np.float32))   # too small for the result
        assert e.value.status == binding.NET_E_INVAL
        net.forward_wait()
