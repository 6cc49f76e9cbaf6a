"""Row-band dataflow between the tensor-core layers of a pass: a layer whose
predecessor writes its own output starts on the tiles whose input rows are
complete instead of waiting for the whole previous kernel.  This changes
only when work starts, never what is added: every pass must be bit-identical
to the same pass with every layer behind the dependency wait
(NET_TC_FLOW=0, a child process, since the switch is read once).  Many
replays of the captured pass at full size give a race (a tile read before
its rows were written, a buffer overwritten while still being read) many
chances to show up as a changed bit."""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1811_03882_gb300 import synth

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
REPS = 30

CHILD = r'''
import sys, numpy as np
sys.path.insert(0, %r); sys.path.insert(0, %r)
import torch
from paper_1811_03882_gb300 import synth, binding
import oracle
from helpers import make_net
cases = [("19-conv", synth.net_19conv, 71, 8, 448, None),
         ("9-conv", synth.net_9conv, 72, 1, 416, None),
         ("9-conv-b4", synth.net_9conv, 73, 4, 320, None),
         ("19-conv-mix", synth.net_19conv, 74, 2, 224, ["bf16"] * 13 + ["fp8", "bf16", "fp8", "bf16", "bf16", "bf16"])]
out = {}
for name, mk, seed, batch, side, mix in cases:
    spec = mk()
    _, x, blob = synth.workload_net(spec, seed, batch, side, side)
    prec = "fp8" if mix else "bf16"
    with make_net(spec, prec=prec, max_batch=batch, max_side=side, layer_prec=mix) as net:
        net.load_weights(blob)
        if mix:
            xc = synth.make_frames(synth.Stream(synth.SEED_CALIB), 1, spec.in_c, 64, 64)
            net.set_act_scales(oracle.act_scales_from(spec.layers, spec.in_c, xc, blob))
        c, ho, wo = net.output_shape(side, side)
        d_in = torch.from_numpy(x).cuda()
        first = None
        for r in range(%d):
            d_out = torch.full((batch, c, ho, wo), float("nan"), device="cuda")
            net.forward_device(d_in, batch, side, side, d_out)
            torch.cuda.synchronize()
            y = d_out.cpu().numpy()
            if first is None:
                first = y
            elif not np.array_equal(y, first):
                print("MISMATCH", name, r, float(np.nanmax(np.abs(y - first))))
                sys.exit(3)
        out[name] = first
np.savez(sys.argv[1], **out)
print("OK")
'''


def _run(tmp_path, name, env_extra):
    path = os.path.join(str(tmp_path), name + ".npz")
    code = CHILD % (ROOT, os.path.join(ROOT, "tests"), REPS)
    env = dict(os.environ, **env_extra)
    r = subprocess.run([sys.executable, "-c", code, path], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0 and "OK" in r.stdout, (r.stdout[-2000:], r.stderr[-2000:])
    return dict(np.load(path))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1811_03882_gb300 import build
    build.build()
    import oracle
    oracle.build()


def test_dataflow_passes_bit_identical_to_whole_kernel_waits(tmp_path):
    flow = _run(tmp_path, "flow", {})
    wait = _run(tmp_path, "wait", {"NET_TC_FLOW": "0"})
    assert sorted(flow) == sorted(wait)
    for name in flow:
        assert np.isfinite(flow[name]).all(), name
        np.testing.assert_array_equal(flow[name], wait[name], err_msg=name)


def test_dataflow_passes_of_two_handles_on_two_streams():
    """Two handles, each on its own stream, issue passes without waiting for
    each other, so their kernels share the SMs.  A layer that polls another
    layer's counters only ever waits for kernels of its own stream that
    started before it, so the interleaving can delay a pass but not change
    it: every pass equals the same pass run alone."""
    import torch
    from paper_1811_03882_gb300 import binding
    spec = synth.net_19conv()
    batch, side = 4, 224
    _, x, blob = synth.workload_net(spec, 75, batch, side, side)
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    nets = [binding.Net(spec.layers, spec.in_c, prec="bf16", max_batch=batch, max_side=side,
                        stream=st.cuda_stream) for st in streams]
    try:
        for n in nets:
            n.load_weights(blob)
        c, ho, wo = nets[0].output_shape(side, side)
        d_in = torch.from_numpy(x).cuda()
        # alone (each handle's plan and captured pass are built here, with
        # nothing else running)
        ref = torch.empty((batch, c, ho, wo), device="cuda")
        for n in nets:
            n.forward_device(d_in, batch, side, side, ref)
            torch.cuda.synchronize()
        outs = [[torch.full((batch, c, ho, wo), float("nan"), device="cuda") for _ in range(8)] for _ in nets]
        torch.cuda.synchronize()
        for r in range(8):
            for k, n in enumerate(nets):
                n.forward_device(d_in, batch, side, side, outs[k][r])
        torch.cuda.synchronize()
        want = ref.cpu().numpy()
        for k in range(2):
            for r in range(8):
                np.testing.assert_array_equal(outs[k][r].cpu().numpy(), want, err_msg="handle %d pass %d" % (k, r))
    finally:
        for n in nets:
            n.close()

