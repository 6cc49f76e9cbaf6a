"""The nightmare pass on the GPU (net_nightmare_grad / net_nightmare_step)
against the FP64 oracle (oracle/nightmare.py).

The GPU runs forward and backward in FP32.  Its gradient matches the
oracle's to FP32 accumulation error, except where a max-pool window holds
two values closer than the forward pass's rounding: FP32 and FP64 can then
name different first maxima and route one gradient to a neighbouring
position.  On small maps no such window occurs and the whole gradient is
held to 1e-4; at 416 x 416 (millions of windows) each layer's backward step
is checked on the GPU's own activation and output gradient (both sides
then pick maxima from the same FP32 values) to 1e-5, and the whole
gradient to a looser bound."""
import numpy as np
import pytest

import oracle
from oracle import nightmare
from paper_1811_03882_gb300 import synth
from helpers import make_net

pytestmark = pytest.mark.gpu


def oracle_dims(spec, h, w):
    """Spatial size of every layer's input (and the final output)."""
    H, W = [h], [w]
    for l in spec.layers:
        s2 = l.pool == synth.POOL_2X2S2
        H.append(H[-1] // 2 if s2 else H[-1])
        W.append(W[-1] // 2 if s2 else W[-1])
    return None, H, W


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1811_03882_gb300 import build
    build.build()
    oracle.build()


def _gpu_grad(spec, x, blob, layer):
    import torch
    n, c, h, w = x.shape
    with make_net(spec, prec="fp32", max_batch=n, max_side=max(h, w)) as net:
        net.load_weights(blob)
        d_x = torch.from_numpy(x).cuda()
        d_g = torch.full_like(d_x, float("nan"))
        J = net.nightmare_grad(d_x, n, h, w, layer, d_g)
        torch.cuda.synchronize()
        return d_g.cpu().numpy(), J


def _compare(g, ref, J, Jref, nerr=1e-4, rms=2e-5, outliers=1e-3):
    assert np.isfinite(g).all()
    d = np.abs(g - ref)
    scale = np.abs(ref).max()
    far = float((d > 1e-3 * scale).mean())
    e_n = float(d.max() / scale)
    e_r = oracle.rms_rel_err(g, ref)
    print("grad: normwise %.3e rms %.3e, %.5f%% elements beyond 1e-3, J rel %.3e"
          % (e_n, e_r, 100 * far, float(np.abs(np.asarray(J) - Jref).max() / np.abs(Jref).max())))
    np.testing.assert_allclose(J, Jref, rtol=1e-5)
    assert e_r <= rms
    assert far <= outliers
    if far == 0.0:
        assert e_n <= nerr


def test_single_layer_grad():
    spec = synth.net_single_conv()
    s = synth.Stream(97)
    x = synth.make_frames(s, 2, 16, 32, 32, -1, 1)
    blob = synth.pack_blob(spec, synth.make_params(s, spec))
    g, J = _gpu_grad(spec, x, blob, 0)
    refs = [nightmare.input_grad(spec.layers, 16, x[f:f + 1], blob, 0) for f in range(2)]
    _compare(g, np.concatenate([r[0] for r in refs]), J, np.array([r[1] for r in refs]), nerr=1e-5)


@pytest.mark.parametrize("layer", [0, 2, 5, 8])
def test_9conv_grad(layer):
    spec = synth.net_9conv()
    _, x, blob = synth.workload_net(spec, 98, 2, 64, 96)
    g, J = _gpu_grad(spec, x, blob, layer)
    refs = [nightmare.input_grad(spec.layers, 3, x[f:f + 1], blob, layer) for f in range(2)]
    _compare(g, np.concatenate([r[0] for r in refs]), J, np.array([r[1] for r in refs]))


def test_9conv_416_full_size_local_and_step():
    """The 9-conv network at 416 x 416 (the single-frame workload), the
    gradient of its last layer's energy.  Per layer, the oracle's backward
    step applied to the GPU's own activation and output gradient (so both
    sides pick each window's maximum from the same FP32 values) must give
    the GPU's input gradient to 1e-5.  End to end, FP32 and FP64 name
    different maxima in a few of the millions of windows (values closer than
    the forward pass's rounding), so the whole gradient is held to a looser
    bound.  Then one ascent step, which moves the frame by
    rate * g / mean|g|."""
    import torch
    spec = synth.net_9conv()
    _, x, blob = synth.workload_net(spec, synth.SEED_9CONV, 1, 416, 416)
    layer = 8
    params = oracle.parse_blob(spec.layers, 3, blob)
    _, H, W = oracle_dims(spec, 416, 416)
    with make_net(spec, prec="fp32", max_batch=1, max_side=416) as net:
        net.load_weights(blob)
        d_x = torch.from_numpy(x).cuda()
        d_g = torch.full_like(d_x, float("nan"))
        acts = [torch.empty((1, l.cout, H[i], W[i]), device="cuda") for i, l in enumerate(spec.layers[:layer + 1])]
        gouts = [torch.empty((1, l.cout, H[i + 1], W[i + 1]), device="cuda")
                 for i, l in enumerate(spec.layers[:layer + 1])]
        net.nightmare_trace(d_x, 1, 416, 416, layer, d_g, acts, gouts)
        torch.cuda.synchronize()
        g = d_g.cpu().numpy()
        acts = [a.cpu().numpy().astype(np.float64) for a in acts]
        gouts = [t.cpu().numpy().astype(np.float64) for t in gouts]
    for l in range(layer, -1, -1):
        want = nightmare.layer_backward(spec.layers[l], params[l], acts[l], gouts[l])
        got = gouts[l - 1] if l > 0 else g
        e = oracle.normwise_rel_err(got, want)
        print("layer %d backward on the GPU's own inputs: normwise %.3e" % (l, e))
        assert e <= 1e-5, (l, e)
    ref, Jref = nightmare.input_grad(spec.layers, 3, x, blob, layer)
    far = float((np.abs(g - ref) > 1e-3 * np.abs(ref).max()).mean())
    print("end to end: rms %.3e, %.3f%% elements beyond 1e-3" % (oracle.rms_rel_err(g, ref), 100 * far))
    assert oracle.rms_rel_err(g, ref) <= 2e-2 and far <= 0.05
    with make_net(spec, prec="fp32", max_batch=1, max_side=416) as net:
        net.load_weights(blob)
        d_x = torch.from_numpy(x).cuda()
        J0 = net.nightmare_step(d_x, 1, 416, 416, layer, 0.01)
        x1 = d_x.cpu().numpy()
        J1 = net.nightmare_step(d_x, 1, 416, 416, layer, 0.01)
    np.testing.assert_allclose(J0, [Jref], rtol=1e-5)
    # the step itself, given the GPU's gradient (the same, deterministic pass)
    want = nightmare.ascent_step(x, g, 0.01)
    assert np.abs(x1 - want).max() <= 1e-5 * (1.0 + 0.01 * np.abs(g).max() / np.abs(g).mean())
    assert J1[0] > J0[0]        # an ascent step raises the layer's energy


def test_nightmare_argument_errors():
    import torch
    from paper_1811_03882_gb300 import binding
    spec = synth.net_9conv()
    blob = synth.weights_for(spec, 99)
    d = torch.zeros((1, 3, 32, 32), device="cuda")
    with make_net(spec, prec="bf16", max_side=32) as net:
        net.load_weights(blob)
        with pytest.raises(binding.NetError) as e:
            net.nightmare_grad(d, 1, 32, 32, 3, d)
        assert e.value.status == binding.NET_E_UNSUPPORTED
    with make_net(spec, prec="fp32", max_side=32) as net:
        net.load_weights(blob)
        with pytest.raises(binding.NetError) as e:
            net.nightmare_grad(d, 1, 32, 32, 9, d)
        assert e.value.status == binding.NET_E_INVAL
        with pytest.raises(binding.NetError) as e:
            net.nightmare_grad(d, 1, 30, 32, 3, d)       # odd size before a 2x2/s2 pool
        assert e.value.status == binding.NET_E_SHAPE
