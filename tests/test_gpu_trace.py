"""Phase trace of the tensor-core launches (net_trace / net_trace_read).

The trace must not change what a pass computes, every CTA of every
tensor-core layer must leave its stamps in program order, and the
dependency wait must hold: no CTA of a layer that waits for the whole
previous kernel gets past that wait before the last CTA of the previous
layer has finished.  Layers on the row-band dataflow (net_plan_flow) start
earlier by design; at least one layer of this pass must be one, and at
least one must still wait for the whole previous kernel.
"""
import numpy as np
import pytest

import oracle
from paper_1811_03882_gb300 import synth
from helpers import make_net, run_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1811_03882_gb300 import build
    build.build()
    oracle.build()


def test_trace_stamps_are_ordered_and_change_nothing():
    spec = synth.net_19conv()
    _, x, blob = synth.workload_net(spec, 23, 2, 160, 160)
    with make_net(spec, prec="bf16", max_batch=2, max_side=160) as net:
        net.load_weights(blob)
        y0 = run_device(net, x)
        with pytest.raises(Exception):
            net.trace_read()                     # never enabled: NET_E_STATE
        net.trace(True)
        y1 = run_device(net, x)
        y2 = run_device(net, x)                  # a graph captured with the trace pointer
        buf = net.trace_read().astype(np.int64)
        net.trace(False)
        y3 = run_device(net, x)
        flow = net.plan_flow(2, 160, 160)
    assert any(flow) and not all(flow), flow
    np.testing.assert_array_equal(y1, y0)
    np.testing.assert_array_equal(y2, y0)
    np.testing.assert_array_equal(y3, y0)
    prev_end = None
    for l in range(len(spec.layers)):
        ran = buf[l, :, 0] > 0
        n = int(ran.sum())
        assert n > 0, l                          # every layer of this network runs on the tensor cores
        assert not buf[l, ~ran].any(), l         # CTAs beyond the grid wrote nothing
        assert ran[:n].all(), l                  # the grid's CTAs are 0 .. n - 1
        B = buf[l, :n]
        assert (B[:, :9] > 0).all(), l
        # thread 0: start, prologue, past the dependency wait; the first MMA
        # issuer: first K step, last MMA; warp 2: epilogue start and end
        assert (B[:, 0] <= B[:, 1]).all() and (B[:, 1] <= B[:, 2]).all(), l
        assert (B[:, 3] <= B[:, 4]).all() and (B[:, 5] <= B[:, 6]).all(), l
        # the closing barrier comes after every role's last stamp; warp 2's
        # last accumulator is ready between its start and its end
        assert (B[:, 8] >= B[:, [1, 2, 4, 6, 7]].max(axis=1)).all(), l
        if B[:, 9].any():                       # (the tap-pair first layer leaves it out)
            assert (B[:, 9] >= B[:, 5]).all() and (B[:, 6] >= B[:, 9]).all(), l
        if prev_end is not None and not flow[l]:
            assert B[:, 2].min() >= prev_end, l  # programmatic launch waited for the whole previous grid
        prev_end = int(B[:, 8].max())
