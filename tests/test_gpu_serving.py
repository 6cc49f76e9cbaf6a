"""Request queue with continuous batching (net_submit / net_poll / net_wait /
net_stats): results against the oracle, identical alone and in the mix,
admission by the activation budget, and host-side failure paths."""
import os
import subprocess
import sys
import time

import numpy as np
import pytest

import oracle
from paper_1811_03882_gb300 import synth
from helpers import make_net

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1811_03882_gb300 import build
    build.build()
    oracle.build()


def _uneven_alone(net, f):
    import torch
    c, ho, wo = net.output_shape(f.shape[2], f.shape[3])
    out = torch.full((1, c, ho, wo), float("nan"), device="cuda")
    net.forward_uneven([torch.from_numpy(f).cuda()], [f.shape[2]], [out])
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_serving_results_match_oracle_and_alone():
    spec = synth.net_9conv()
    blob = synth.weights_for(spec, 61)
    sides = [64, 96, 32, 128, 64, 96, 32, 64, 128, 96]
    frames = [synth.frame_for(61, i, s) for i, s in enumerate(sides)]
    with make_net(spec, prec="bf16", max_side=128) as net:
        net.load_weights(blob)
        ids = [net.submit(f) for f in frames]          # all in flight together
        outs = []
        for f, rid in zip(frames, ids):
            c, ho, wo = net.output_shape(f.shape[2], f.shape[3])
            y = np.full((1, c, ho, wo), np.nan, np.float32)
            net.wait(rid, y, 20000)
            outs.append(y)
        fps, p50, p99 = net.stats()
        assert fps > 0 and 0 < p50 <= p99
        # the same frame submitted alone
        rid = net.submit(frames[3])
        alone = np.full_like(outs[3], np.nan)
        net.wait(rid, alone, 20000)
        np.testing.assert_array_equal(alone, outs[3])
        for i in (0, 3, 8):
            np.testing.assert_array_equal(outs[i], _uneven_alone(net, frames[i]))
    for i, (f, y) in enumerate(zip(frames, outs)):
        ex = oracle.forward(spec.layers, 3, f, blob)
        e = oracle.normwise_rel_err(y, ex)
        assert e <= 2e-2, (i, e)


def test_serving_budget_queueing_and_rejection():
    from paper_1811_03882_gb300 import binding
    spec = synth.net_9conv()
    blob = synth.weights_for(spec, 62)
    # room for about two 96x96 requests at a time: the rest must queue
    with make_net(spec, prec="bf16", max_side=416, budget=2 * (1 << 20)) as net:
        net.load_weights(blob)
        frames = [synth.frame_for(62, i, 96) for i in range(6)]
        ids = [net.submit(f) for f in frames]
        c, ho, wo = net.output_shape(96, 96)
        res = []
        for rid in ids:
            y = np.zeros((1, c, ho, wo), np.float32)
            net.wait(rid, y, 20000)
            res.append(y)
        for f, y in zip(frames, res):
            assert oracle.normwise_rel_err(y, oracle.forward(spec.layers, 3, f, blob)) <= 2e-2
        with pytest.raises(binding.NetError) as e:
            net.submit(synth.frame_for(62, 9, 416))   # needs more than the whole budget
        assert e.value.status == binding.NET_E_BUDGET
        with pytest.raises(binding.NetError) as e:
            net.wait(123456, np.zeros(4, np.float32), 10)
        assert e.value.status == binding.NET_E_INVAL


def test_serving_wait_timeout_with_a_slow_step():
    """A slow scheduler step is injected on the host (environment knob read
    when the queue starts); net_wait must time out, then finish normally.
    Runs in a child process so the knob does not leak into other tests."""
    code = r'''
import sys, numpy as np
sys.path.insert(0, %r); sys.path.insert(0, %r)
from paper_1811_03882_gb300 import synth, binding
from helpers import make_net
spec = synth.net_9conv()
with make_net(spec, prec="bf16", max_side=64) as net:
    net.load_weights(synth.weights_for(spec, 63))
    f = synth.frame_for(63, 0, 64)
    rid = net.submit(f)
    c, ho, wo = net.output_shape(64, 64)
    y = np.zeros((1, c, ho, wo), np.float32)
    try:
        net.wait(rid, y, 5)
        print("NO-TIMEOUT")
    except binding.NetError as e:
        assert e.status == binding.NET_E_TIMEOUT, e
    if not net.poll(rid, y):
        net.wait(rid, y, 60000)
    assert np.isfinite(y).all()
    print("OK")
''' % (ROOT, os.path.join(ROOT, "tests"))
    env = dict(os.environ, NET_SERVE_STEP_DELAY_US="20000")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert "OK" in r.stdout and "NO-TIMEOUT" not in r.stdout


def test_serving_in_flight_cap_queues_and_completes():
    """With at most 2 requests on the device (NET_SERVE_MAX_ACTIVE, read when
    the queue starts) a burst of 12 frames still completes, in a child
    process so the knob stays local."""
    code = r'''
import sys, numpy as np
sys.path.insert(0, %r); sys.path.insert(0, %r)
import oracle
from paper_1811_03882_gb300 import synth
from helpers import make_net
spec = synth.net_9conv()
blob = synth.weights_for(spec, 64)
frames = [synth.frame_for(64, i, 32 * (1 + i %% 3)) for i in range(12)]
with make_net(spec, prec="bf16", max_side=96) as net:
    net.load_weights(blob)
    ids = [net.submit(f) for f in frames]
    for f, rid in zip(frames, ids):
        c, ho, wo = net.output_shape(f.shape[2], f.shape[3])
        y = np.zeros((1, c, ho, wo), np.float32)
        net.wait(rid, y, 60000)
        assert oracle.normwise_rel_err(y, oracle.forward(spec.layers, 3, f, blob)) <= 2e-2
print("OK")
''' % (ROOT, os.path.join(ROOT, "tests"))
    env = dict(os.environ, NET_SERVE_MAX_ACTIVE="2")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert "OK" in r.stdout


def test_serving_concurrent_submitters_and_full_steps():
    """Four threads submit at once into a fresh queue (one queue must start),
    and a slow first step lets a burst pile up so that the next steps carry
    up to the in-flight cap: 19 layers x 128 requests of problem tables in
    one step.  Every result is checked against the same frame alone."""
    code = r'''
import sys, threading, numpy as np
sys.path.insert(0, %r); sys.path.insert(0, %r)
import oracle
from paper_1811_03882_gb300 import synth
from helpers import make_net
spec = synth.net_19conv()
blob = synth.weights_for(spec, 65)
frames = [synth.frame_for(65, i, 32 * (1 + i %% 3)) for i in range(160)]
with make_net(spec, prec="bf16", max_side=96) as net:
    net.load_weights(blob)
    ids = [None] * len(frames)
    def sub(k):
        for i in range(k, len(frames), 4):
            ids[i] = net.submit(frames[i])
    ths = [threading.Thread(target=sub, args=(k,)) for k in range(4)]
    for t in ths: t.start()
    for t in ths: t.join()
    assert len(set(ids)) == len(frames)
    outs = []
    for f, rid in zip(frames, ids):
        c, ho, wo = net.output_shape(f.shape[2], f.shape[3])
        y = np.full((1, c, ho, wo), np.nan, np.float32)
        net.wait(rid, y, 120000)
        outs.append(y)
    for i in (0, 1, 2, 77, 159):
        rid = net.submit(frames[i])
        alone = np.full_like(outs[i], np.nan)
        net.wait(rid, alone, 60000)
        assert np.array_equal(alone, outs[i]), i
    for i in (0, 2, 100):
        e = oracle.normwise_rel_err(outs[i], oracle.forward(spec.layers, 3, frames[i], blob))
        assert e <= 2e-2, (i, e)
print("OK")
''' % (ROOT, os.path.join(ROOT, "tests"))
    env = dict(os.environ, NET_SERVE_STEP_DELAY_US="20000")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    assert "OK" in r.stdout
