"""Split-K reduced inside a thread-block cluster (BF16 tensor-core layers).

A layer whose K is split over ksplit CTAs, with one work item a CTA, runs
its ksplit CTAs as one cluster: each CTA keeps its partial sums in its own
shared memory and CTA r adds every slice's partials for 1 / ksplit of the
columns through distributed shared memory, then applies the epilogue.  The
additions are the workspace reduction's, in its order, so the result must
equal NET_TC_XRED=0's (workspace + reduction launch) bit for bit, with one
launch fewer per split layer.  Cases force the N tile and split (64, 128,
256 columns; 2, 4, 8, 16 CTAs a cluster) on ragged maps, with and without the
fused 2x2/s2 pool, for both of the cluster epilogue's outputs: BF16 NHWC
(a layer followed by another) and FP32 NCHW (the last layer).
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
from paper_1811_03882_gb300 import synth

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (name, cin, layers [(k, cout, pool)], forced (bn, ksplit) of layer 0, batch, h, w)
CASES = [
    ("last_bn256_s2", 256, [(3, 256, synth.POOL_NONE)], (256, 2), 1, 12, 12),
    ("last_pool_bn128_s4", 256, [(3, 256, synth.POOL_2X2S2)], (128, 4), 2, 16, 16),
    ("last_1x1_bn128_s4", 1024, [(1, 125, synth.POOL_NONE)], (128, 4), 2, 13, 13),
    ("mid_bn64_s2", 128, [(3, 192, synth.POOL_NONE), (1, 10, synth.POOL_NONE)], (64, 2), 2, 20, 20),
    ("mid_pool_bn256_s8", 256, [(3, 256, synth.POOL_2X2S2), (1, 20, synth.POOL_NONE)], (256, 8), 2, 16, 16),
    ("mid_bn128_s8", 512, [(3, 128, synth.POOL_NONE), (1, 24, synth.POOL_NONE)], (128, 8), 1, 9, 11),
    # 16-CTA clusters (a non-portable size) and 8-column shares (one warpgroup reduces)
    ("last_bn256_s16", 512, [(3, 256, synth.POOL_NONE)], (256, 16), 1, 13, 13),
    ("mid_bn128_s16", 512, [(3, 128, synth.POOL_NONE), (1, 12, synth.POOL_NONE)], (128, 16), 1, 9, 11),
    ("mid_pool_bn64_s8", 256, [(3, 64, synth.POOL_2X2S2), (1, 8, synth.POOL_NONE)], (64, 8), 1, 16, 16),
]


def _spec(cin, layers):
    L = synth.Layer
    ls = [L(k, cout, True, synth.ACT_LEAKY, pool) for k, cout, pool in layers[:-1]]
    k, cout, pool = layers[-1]
    ls.append(L(k, cout, len(layers) == 1, synth.ACT_LEAKY if len(layers) == 1 else synth.ACT_LINEAR, pool))
    return synth.NetSpec("xred", cin, ls)


def _inputs(i, cin, layers, b, h, w):
    spec = _spec(cin, layers)
    s = synth.Stream(9100 + i)
    x = synth.make_frames(s, b, cin, h, w, -1, 1)
    blob = synth.pack_blob(spec, synth.make_params(s, spec))
    return spec, x, blob


CHILD = r'''
import sys, numpy as np
sys.path.insert(0, %r); sys.path.insert(0, %r)
import torch
from test_gpu_xred import CASES, _inputs
from helpers import make_net, run_device
out = {}
for i, (name, cin, layers, tiles, b, h, w) in enumerate(CASES):
    spec, x, blob = _inputs(i, cin, layers, b, h, w)
    with make_net(spec, prec="bf16", max_batch=b, max_side=max(h, w)) as net:
        net.load_weights(blob)
        net.set_layer_tiles(0, *tiles)
        assert net.plan_tiles(b, h, w)[0] == tuple(tiles), net.plan_tiles(b, h, w)
        y = run_device(net, x)
        l0 = net.launches()
        y2 = run_device(net, x)          # the captured graph's replay
        out[name] = y
        out[name + "_launches"] = np.int64(net.launches() - l0)
        assert np.array_equal(y, y2), name
np.savez(sys.argv[1], **out)
print("OK")
'''


def _run(tmp_path, tag, env_extra):
    path = os.path.join(str(tmp_path), tag + ".npz")
    code = CHILD % (ROOT, os.path.join(ROOT, "tests"))
    env = dict(os.environ, **env_extra)
    r = subprocess.run([sys.executable, "-c", code, path], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "OK" in r.stdout, r.stderr[-3000:]
    return np.load(path)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1811_03882_gb300 import build
    build.build()
    oracle.build()


def test_cluster_split_k_matches_workspace_reduction_and_oracle(tmp_path):
    on = _run(tmp_path, "xred", {})
    off = _run(tmp_path, "ws", {"NET_TC_XRED": "0"})
    for i, (name, cin, layers, tiles, b, h, w) in enumerate(CASES):
        spec, x, blob = _inputs(i, cin, layers, b, h, w)
        y = on[name]
        assert np.isfinite(y).all(), name
        # same additions in the same order as the workspace reduction
        np.testing.assert_array_equal(y, off[name], err_msg=name)
        # the reduction launch is gone
        assert int(on[name + "_launches"]) == int(off[name + "_launches"]) - 1, (
            name, int(on[name + "_launches"]), int(off[name + "_launches"]))
        precs = ["bf16"] * len(spec.layers)
        qa = oracle.forward_quant(spec.layers, spec.in_c, x, blob, precs, None)
        ex = oracle.forward(spec.layers, spec.in_c, x, blob)
        e_q = oracle.normwise_rel_err(y, qa)
        e_x = oracle.normwise_rel_err(y, ex)
        print("%s: vs quant-aware %.3e, vs exact %.3e" % (name, e_q, e_x))
        # one layer: FP32 against FP64 accumulation of the same BF16 operands;
        # two: a BF16-stored activation may round the other way now and then
        assert e_q <= (1e-4 if len(layers) == 1 else 4e-3), (name, e_q)
        assert e_x <= 2e-2, (name, e_x)
