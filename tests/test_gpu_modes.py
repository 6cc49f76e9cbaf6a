"""Launch-mode switches of the tensor-core conv, each in a child process (the
switches are read once per process): K-alternating MMA issuers off
(NET_TC_KALT=0), programmatic dependent launch off (NET_PDL=0), tap-merged
stages off (NET_TC_TAPM=0), the first layer as an im2col tile of 32
channels written by a pack kernel (NET_L0_PAIR=0) instead of two taps per
MMA over 8-channel pixels, and one CTA per SM everywhere (NET_TC_MB=1) or
two wherever the N tile allows (NET_TC_MB=2, which also runs long A + B
rings on half the shared memory and the 16-column epilogue), and CTA pairs
(NET_TC_PAIR=1: 2-CTA clusters, one M = 256 tile a pair, on the layers that
stream N tiles of 128 or 256 columns), the generic kernel for the
tap-pair first layer instead of its specialised variant (NET_TC_SPEC=0), and
split-K layers reduced through the workspace by a reduction launch instead
of inside their clusters (NET_TC_XRED=0), and every layer behind the
dependency wait on the whole previous kernel instead of the row-band
dataflow (NET_TC_FLOW=0), and the tap-pair first layer on 16 x 8 tiles
with three TMA boxes a stage instead of 8 x 16 tiles with one
(NET_L0_BOX1=0).
Every mode must give the oracle's answer within
the BF16 budget and agree with the default mode to BF16 rounding; the
19-conv network at 2 x 160 x 160 has layers with one and with several work
items per CTA, split-K layers and resident-weight layers."""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
from paper_1811_03882_gb300 import synth

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SIDE, BATCH = 160, 2

CHILD = r'''
import sys, json, numpy as np
sys.path.insert(0, %r); sys.path.insert(0, %r)
import torch
from paper_1811_03882_gb300 import synth
from helpers import make_net, run_device
spec = synth.net_19conv()
_, x, blob = synth.workload_net(spec, 71, %d, %d, %d)
with make_net(spec, prec="bf16", max_batch=%d, max_side=%d) as net:
    net.load_weights(blob)
    y = run_device(net, x)
    y2 = run_device(net, x)            # a second call replays the captured graph
    assert np.array_equal(y, y2)
np.save(sys.argv[1], y)
print("OK")
'''


def _run(tmp_path, name, env_extra):
    out = os.path.join(str(tmp_path), name + ".npy")
    code = CHILD % (ROOT, os.path.join(ROOT, "tests"), BATCH, SIDE, SIDE, BATCH, SIDE)
    env = dict(os.environ, **env_extra)
    r = subprocess.run([sys.executable, "-c", code, out], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "OK" in r.stdout, r.stderr[-2000:]
    return np.load(out)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1811_03882_gb300 import build
    build.build()
    oracle.build()


def test_launch_modes_match_oracle(tmp_path):
    spec = synth.net_19conv()
    _, x, blob = synth.workload_net(spec, 71, BATCH, SIDE, SIDE)
    ex = oracle.forward(spec.layers, 3, x, blob)
    ys = {}
    for name, env in (("default", {}), ("no_kalt", {"NET_TC_KALT": "0"}), ("no_pdl", {"NET_PDL": "0"}),
                      ("im2col", {"NET_L0_PAIR": "0"}), ("no_tapm", {"NET_TC_TAPM": "0"}),
                      ("mb1", {"NET_TC_MB": "1"}), ("mb2", {"NET_TC_MB": "2"}),
                      ("pair", {"NET_TC_PAIR": "1"}), ("pair_no_kalt", {"NET_TC_PAIR": "1", "NET_TC_KALT": "0"}),
                      ("no_spec", {"NET_TC_SPEC": "0"}), ("no_xred", {"NET_TC_XRED": "0"}),
                      ("no_flow", {"NET_TC_FLOW": "0"}), ("l0_three_boxes", {"NET_L0_BOX1": "0"})):
        y = _run(tmp_path, name, env)
        assert np.isfinite(y).all(), name
        e = oracle.normwise_rel_err(y, ex)
        agree, _, _ = oracle.argmax_agreement(y, ex, 2e-2)
        assert e <= 2e-2 and agree >= 0.99, (name, e, agree)
        ys[name] = y
    # programmatic launch and the row-band dataflow change only when kernels
    # start and what they wait for, never what they add
    np.testing.assert_array_equal(ys["no_pdl"], ys["default"])
    np.testing.assert_array_equal(ys["no_flow"], ys["default"])
    # the first-layer specialisation runs the generic kernel's operations
    np.testing.assert_array_equal(ys["no_spec"], ys["default"])
    # a CTA pair accumulates every row's products in the single-CTA order of
    # one MMA issuer: the same bits as that mode
    np.testing.assert_array_equal(ys["pair_no_kalt"], ys["no_kalt"])
    # the first layer's tap pairs sum the same products in another order
    # (without the cluster reduction the planner prices K splits differently,
    # so the splits and their summation order may change: tests/test_gpu_xred.py
    # checks bit-identity on fixed plans)
    for name in ("no_kalt", "no_tapm", "im2col", "mb1", "mb2", "pair", "no_xred", "l0_three_boxes"):
        assert oracle.normwise_rel_err(ys[name], ys["default"]) <= 2e-2, name
