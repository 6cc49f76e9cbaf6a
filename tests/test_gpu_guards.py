"""Canary guard regions (NET_GUARD=1, net_guard_check / net_guard_poke): a
child process runs every kind of pass the library has with a guard region
before and after each device buffer it allocates; afterwards no region may
have changed (no kernel wrote past either end of a buffer).  Then one byte
is written just past a live buffer on the host side and the check must
find exactly that buffer.  Regions are checked when a buffer is freed and,
for live buffers, when net_guard_check runs.  Every result is also compared with the same pass
without guards, which must be bit-identical."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import sys, numpy as np
sys.path.insert(0, %r); sys.path.insert(0, %r)
import torch
from paper_1811_03882_gb300 import synth, binding
from helpers import make_net, run_device
res = {}
# 19-conv BF16: tap-pair first layer, resident weights, split-K, K-alternating
spec = synth.net_19conv()
_, x, blob = synth.workload_net(spec, 71, 2, 160, 160)
with make_net(spec, prec="bf16", max_batch=2, max_side=160) as net:
    net.load_weights(blob)
    res["bf16"] = run_device(net, x)
    res["bf16_host"] = net.forward(x)
# the same network with an FP8 plan (calibrated activation scales)
with make_net(spec, prec="fp8", max_batch=2, max_side=160) as net:
    net.load_weights(blob)
    net.calibrate(torch.from_numpy(x[:1]).cuda(), 1, 160, 160)
    res["fp8"] = run_device(net, x)
# 9-conv FP32 (CUDA-core conv, split-K reduction, stride-1 pool), detection,
# nightmare gradient
spec9 = synth.net_9conv()
_, x9, blob9 = synth.workload_net(spec9, 72, 1, 128, 128)
with make_net(spec9, prec="fp32", max_batch=1, max_side=128) as net:
    net.load_weights(blob9)
    res["fp32"] = run_device(net, x9)
    net.set_region([(0.8, 1.2), (2.0, 3.1), (4.5, 2.2), (6.0, 7.5), (9.7, 5.0)], 20, 0.05, 0.45, 64)
    cnt, det = net.forward_detect(x9)
    res["det"] = np.concatenate([np.asarray(cnt, np.float64).ravel(), det.view(np.uint8).ravel().astype(np.float64)])
    d = torch.from_numpy(x9).cuda()
    g = torch.zeros_like(d)
    net.nightmare_grad(d, 1, 128, 128, 8, g)
    torch.cuda.synchronize()
    res["night"] = g.cpu().numpy()
# uneven batch (grouped launches) and the request queue
sides = [64, 96, 32, 128]
frames = [synth.frame_for(73, i, s) for i, s in enumerate(sides)]
with make_net(spec9, prec="bf16", max_side=128) as net:
    net.load_weights(blob9)
    d_in = [torch.from_numpy(f).cuda() for f in frames]
    outs = []
    for f in frames:
        c, ho, wo = net.output_shape(f.shape[2], f.shape[3])
        outs.append(torch.full((1, c, ho, wo), float("nan"), device="cuda"))
    net.forward_uneven(d_in, sides, outs)
    torch.cuda.synchronize()
    res["uneven"] = np.concatenate([o.cpu().numpy().ravel() for o in outs])
    ys = []
    for f in frames:
        rid = net.submit(f)
        c, ho, wo = net.output_shape(f.shape[2], f.shape[3])
        y = np.full((1, c, ho, wo), np.nan, np.float32)
        net.wait(rid, y, 20000)
        ys.append(y.ravel())
    res["serve"] = np.concatenate(ys)
# Jacobi
with binding.Jacobi(70, 2050) as J:
    out, k, ch = J.solve(synth.laplace_grid(74, 70, 2050, "random"), 0.0, 20)
    res["jacobi"] = out
np.savez(sys.argv[1], **res)
b, c = binding.guard_check()        # every buffer above was checked at its free
print("GUARDS", b, c)
with make_net(spec9, prec="bf16", max_side=64) as net:   # live buffers
    net.load_weights(blob9)
    run_device(net, x9[:, :, :64, :64].copy())
    b1, c1 = binding.guard_check()
    print("LIVE", b1 - b, c1 - c)
    if b1 > b:
        binding.guard_poke(0)
        b2, c2 = binding.guard_check()
        print("POKED", b2 - b1, c2 - c1)
b3, c3 = binding.guard_check()
print("FREED", b3, c3)
print("OK")
'''


def _run(tmp_path, name, guard):
    out = os.path.join(str(tmp_path), name + ".npz")
    env = dict(os.environ)
    env.pop("NET_GUARD", None)
    if guard:
        env["NET_GUARD"] = "1"
    r = subprocess.run([sys.executable, "-c", CHILD % (ROOT, os.path.join(ROOT, "tests")), out], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0 and "OK" in r.stdout, r.stdout[-2000:] + r.stderr[-3000:]
    lines = {l.split()[0]: [int(v) for v in l.split()[1:]] for l in r.stdout.splitlines()
             if l.startswith(("GUARDS", "LIVE", "POKED", "FREED"))}
    return np.load(out), lines


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1811_03882_gb300 import build
    build.build()


def test_no_pass_writes_past_a_buffer(tmp_path):
    ref, plain = _run(tmp_path, "plain", False)
    got, g = _run(tmp_path, "guarded", True)
    assert plain["GUARDS"] == [0, 0]                 # guards off: nothing checked
    buffers, corrupted = g["GUARDS"]
    print("guarded buffers %d (checked at their free), changed regions %d; live %s; after the poke %s; "
          "at the end %s" % (buffers, corrupted, g["LIVE"], g["POKED"], g["FREED"]))
    assert buffers >= 40 and corrupted == 0
    live = g["LIVE"][0]
    assert live >= 10 and g["LIVE"][1] == 0
    assert g["POKED"] == [0, 1]                      # the planted overrun is found while live
    assert g["FREED"][0] >= buffers + live and g["FREED"][1] == 1   # and once more at its free
    for k in ref.files:                              # guards change no result
        np.testing.assert_array_equal(got[k], ref[k], err_msg=k)
