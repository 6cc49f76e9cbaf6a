"""Shared test helpers: build a library handle for a synthetic network and
compare its output with the FP64 oracle."""
import numpy as np

from paper_1811_03882_gb300 import synth


def make_net(spec, prec="fp32", max_batch=1, max_side=416, layer_prec=None, budget=0):
    import torch
    from paper_1811_03882_gb300 import binding
    return binding.Net(spec.layers, spec.in_c, prec=prec, layer_prec=layer_prec,
                       max_batch=max_batch, max_side=max_side,
                       stream=torch.cuda.current_stream().cuda_stream, budget_bytes=budget)


def run_device(net, x):
    """x: host NCHW float32 -> device forward -> host array."""
    import torch
    n, _, h, w = x.shape
    c, ho, wo = net.output_shape(h, w)
    d_in = torch.from_numpy(x).cuda()
    d_out = torch.full((n, c, ho, wo), float("nan"), device="cuda")
    net.forward_device(d_in, n, h, w, d_out)
    torch.cuda.synchronize()
    return d_out.cpu().numpy()


def default_precs(spec, prec, layer_prec=None):
    """Per-layer operand format the library uses for a network at `prec`
    (or the per-layer list): a layer reading fewer than 16 channels keeps
    BF16 operands in an FP8 network."""
    out = []
    c = spec.in_c
    for i, l in enumerate(spec.layers):
        p = layer_prec[i] if layer_prec is not None else prec
        out.append("bf16" if (p == "fp8" and c < 16) else p)
        c = l.cout
    return out
