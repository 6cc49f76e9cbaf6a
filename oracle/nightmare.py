"""FP64 oracle of the "nightmare" pass: the gradient, with respect to the
input frames, of the energy of one layer's output.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper offloads Darknet's "nightmare" sample app (Sec. 5.1.1), which
changes an image by gradient ascent so that it excites a chosen layer more;
the paper prints none of its steps.  What follows is the plain definition:

* the objective of layer L is J = 1/2 * sum of the squares of its output
  (after its pool), so dJ/d(output of L) = that output;
* the gradient flows back through every layer l = L .. 0 in the reverse of
  the forward order:
    - 2x2/s2 max pool: each output's gradient goes to the first position of
      its window holding the window's maximum, scanning (0,0), (0,1), (1,0),
      (1,1); the other three get none;
    - 2x2/s1 "same" max pool (window (i..i+1, j..j+1) clipped at the bottom
      and right edges): each output's gradient goes to the first maximum of
      its own window, and a position sums what the windows it wins send it;
    - leaky rectifier: the gradient is multiplied by 1 where the
      pre-activation is positive and by 0.1 elsewhere;
    - batchnorm (running statistics): multiplied by gamma / sqrt(var + eps)
      per channel; the bias has no input gradient;
    - conv: the input gradient sum over (o, kh, kw) of dy[o, i-kh+p, j-kw+p]
      * w[o, c, kh, kw] (oracle.conv2d_bwd_data);
* one ascent step moves each frame by rate * g / mean(|g|) over that frame.
"""
from __future__ import annotations

import numpy as np

import oracle


def forward_saving(layers, in_c: int, x, blob, upto: int):
    """Exact FP64 forward pass through layer `upto`: per layer l a dict with
    its input 'a', pre-activation 'z' (after batchnorm / bias) and pre-pool
    activation 'h'; returns (per-layer list, output of layer upto)."""
    ps = oracle.parse_blob(layers, in_c, blob)
    a = oracle._f64(x)
    saved = []
    for l, p in zip(layers[:upto + 1], ps):
        y = oracle.conv2d(a, p["w"])
        if l.bn:
            z = oracle.batchnorm(y, p["gamma"], p["beta"], p["mean"], p["var"])
        else:
            z = oracle.add_bias(y, p["bias"])
        h = oracle.leaky(z) if l.act == oracle.ACT_LEAKY else z
        saved.append({"a": a, "z": z, "h": h, "p": p})
        a = oracle._pool(l, h)
    return saved, a


def maxpool2_s2_bwd(g, h):
    """Gradient through the 2x2/s2 max pool of h (N,C,H,W) given g (N,C,H/2,W/2)."""
    g, h = oracle._f64(g), oracle._f64(h)
    N, C, H, W = h.shape
    d = np.zeros_like(h)
    for n in range(N):
        for c in range(C):
            for i in range(H // 2):
                for j in range(W // 2):
                    best, bi, bj = None, 0, 0
                    for di in (0, 1):
                        for dj in (0, 1):
                            v = h[n, c, 2 * i + di, 2 * j + dj]
                            if best is None or v > best:
                                best, bi, bj = v, 2 * i + di, 2 * j + dj
                    d[n, c, bi, bj] += g[n, c, i, j]
    return d


def maxpool2_s1_same_bwd(g, h):
    """Gradient through the 2x2/s1 "same" max pool of h given g (same shape)."""
    g, h = oracle._f64(g), oracle._f64(h)
    N, C, H, W = h.shape
    d = np.zeros_like(h)
    for n in range(N):
        for c in range(C):
            for i in range(H):
                for j in range(W):
                    best, bi, bj = None, i, j
                    for di in (0, 1):
                        for dj in (0, 1):
                            if i + di < H and j + dj < W:
                                v = h[n, c, i + di, j + dj]
                                if best is None or v > best:
                                    best, bi, bj = v, i + di, j + dj
                    d[n, c, bi, bj] += g[n, c, i, j]
    return d


def leaky_bwd(g, z):
    return oracle._f64(g) * np.where(oracle._f64(z) > 0, 1.0, oracle.LEAKY_SLOPE)


def layer_backward(L, p, h, gout):
    """Gradient with respect to layer L's input from the gradient of its
    output, given its activation before the pool h (whose sign is the
    pre-activation's: the leaky rectifier keeps signs) and its parameters p
    (a dict of oracle.parse_blob)."""
    g = oracle._f64(gout)
    if L.pool == oracle.POOL_2X2S2:
        g = maxpool2_s2_bwd(g, h)
    elif L.pool == oracle.POOL_2X2S1_SAME:
        g = maxpool2_s1_same_bwd(g, h)
    if L.act == oracle.ACT_LEAKY:
        g = leaky_bwd(g, h)
    if L.bn:
        g = g * (p["gamma"] / np.sqrt(p["var"] + oracle.BN_EPS))[None, :, None, None]
    return oracle.conv2d_bwd_data(g, p["w"])


def input_grad(layers, in_c: int, x, blob, layer: int):
    """dJ/dx of J = 1/2 * sum(output of `layer`)^2, and J."""
    saved, out = forward_saving(layers, in_c, x, blob, layer)
    g = out.copy()
    for l in range(layer, -1, -1):
        g = layer_backward(layers[l], saved[l]["p"], saved[l]["h"], g)
    return g, 0.5 * float((out * out).sum())


def ascent_step(x, g, rate: float):
    """x + rate * g / mean(|g|), per frame."""
    x, g = oracle._f64(x), oracle._f64(g)
    m = np.abs(g).reshape(g.shape[0], -1).mean(axis=1)
    return x + rate * g / np.maximum(m, 1e-30)[:, None, None, None]
