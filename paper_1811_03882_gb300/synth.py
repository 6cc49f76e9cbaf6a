"""Seeded synthetic workloads: network descriptions, frames, weight blobs.

This module is the one piece that both the CUDA path (through tests and
``bench.py``) and the FP64 oracle consume.  It holds no arithmetic of the
forward pass itself: only random numbers, shapes and the weight-blob layout.

The paper offloads Darknet's image pipeline ("detection" and "nightmare"
sample apps, Sec. 5.1.1) but prints neither a network description, image
sizes, nor weights; Darknet's cfg files, trained weights and sample images
are not available.  The networks below are synthetic stand-ins shaped like
the Darknet models that pipeline runs (a 9-conv tiny detector and a 19-conv
classifier), with He-initialised weights and batchnorm statistics drawn from
fixed distributions.

Random numbers: SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), one counter-based stream per
seed.  Draw ``i`` (0-based) of seed ``s`` is ``mix(s + (i+1)*golden)`` with
golden = 0x9E3779B97F4A7C15.  Uniforms take the top 53 bits; normals use the
cosine branch of Box-Muller on two consecutive uniforms.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# activation / pool codes (mirrors include/net.h)
ACT_LINEAR, ACT_LEAKY = 0, 1
POOL_NONE, POOL_2X2S2, POOL_2X2S1_SAME = 0, 1, 2


def splitmix64(seed: int, start: int, n: int) -> np.ndarray:
    """Draws ``start .. start+n-1`` of the SplitMix64 stream for ``seed``."""
    with np.errstate(over="ignore"):
        idx = np.arange(start + 1, start + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


class Stream:
    """Sequential consumer of one seed's SplitMix64 stream."""

    def __init__(self, seed: int):
        self.seed = int(seed)
        self.pos = 0

    def bits(self, n: int) -> np.ndarray:
        out = splitmix64(self.seed, self.pos, n)
        self.pos += n
        return out

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        u = (self.bits(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u

    def normal(self, n: int, std: float = 1.0) -> np.ndarray:
        u = self.uniform(2 * n)
        u1, u2 = u[0::2], u[1::2]
        r = np.sqrt(-2.0 * np.log1p(-u1))  # 1-u1 in (0,1]
        return std * r * np.cos(2.0 * np.pi * u2)

    def choice(self, options: Sequence[int], n: int) -> np.ndarray:
        b = self.bits(n) % np.uint64(len(options))
        return np.asarray(options, dtype=np.int64)[b.astype(np.int64)]


@dataclass(frozen=True)
class Layer:
    k: int          # 1 or 3 (stride 1, pad k//2)
    cout: int
    bn: bool        # batchnorm (else a plain bias)
    act: int        # ACT_LINEAR or ACT_LEAKY (slope 0.1)
    pool: int       # POOL_NONE, POOL_2X2S2, POOL_2X2S1_SAME


@dataclass
class NetSpec:
    name: str
    in_c: int
    layers: List[Layer] = field(default_factory=list)

    def cins(self) -> List[int]:
        cs, c = [], self.in_c
        for l in self.layers:
            cs.append(c)
            c = l.cout
        return cs

    def out_hw(self, h: int, w: int) -> Tuple[int, int]:
        for l in self.layers:
            if l.pool == POOL_2X2S2:
                h, w = h // 2, w // 2
        return h, w

    def out_c(self) -> int:
        return self.layers[-1].cout

    def n_params(self) -> int:
        n = 0
        for l, c in zip(self.layers, self.cins()):
            n += l.cout * c * l.k * l.k + (4 if l.bn else 1) * l.cout
        return n

    def conv_flops(self, n: int, h: int, w: int) -> float:
        """Dense conv FLOPs: sum over layers of 2*N*H*W*Cout*Cin*k*k."""
        tot = 0.0
        for l, c in zip(self.layers, self.cins()):
            tot += 2.0 * n * h * w * l.cout * c * l.k * l.k
            if l.pool == POOL_2X2S2:
                h, w = h // 2, w // 2
        return tot


def leaky_bn(k, cout, pool=POOL_NONE):
    return Layer(k, cout, True, ACT_LEAKY, pool)


def net_single_conv() -> NetSpec:
    """One 3x3 conv 16->32 + BN + leaky 0.1 + 2x2/s2 max pool (32x32 input)."""
    return NetSpec("single-conv", 16, [leaky_bn(3, 32, POOL_2X2S2)])


def net_9conv() -> NetSpec:
    """Six 3x3 conv+BN+leaky+pool blocks (16..512; last pool 2x2/s1 same),
    two 3x3 1024 convs and a linear 1x1 conv to 125 channels."""
    ls = [leaky_bn(3, c, POOL_2X2S2) for c in (16, 32, 64, 128, 256)]
    ls.append(leaky_bn(3, 512, POOL_2X2S1_SAME))
    ls += [leaky_bn(3, 1024), leaky_bn(3, 1024)]
    ls.append(Layer(1, 125, False, ACT_LINEAR, POOL_NONE))
    return NetSpec("9-conv", 3, ls)


def net_19conv() -> NetSpec:
    """Alternating 3x3 / 1x1 convs, 32..1024 channels, 1x1 halving, five
    2x2/s2 pools, final linear 1x1 conv to 1000 channels."""
    P = POOL_2X2S2
    ls = [leaky_bn(3, 32, P), leaky_bn(3, 64, P),
          leaky_bn(3, 128), leaky_bn(1, 64), leaky_bn(3, 128, P),
          leaky_bn(3, 256), leaky_bn(1, 128), leaky_bn(3, 256, P),
          leaky_bn(3, 512), leaky_bn(1, 256), leaky_bn(3, 512), leaky_bn(1, 256),
          leaky_bn(3, 512, P),
          leaky_bn(3, 1024), leaky_bn(1, 512), leaky_bn(3, 1024), leaky_bn(1, 512),
          leaky_bn(3, 1024),
          Layer(1, 1000, False, ACT_LINEAR, POOL_NONE)]
    return NetSpec("19-conv", 3, ls)


NETS = {"single-conv": net_single_conv, "9-conv": net_9conv, "19-conv": net_19conv}


def make_frames(stream: Stream, n: int, c: int, h: int, w: int,
                lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """NCHW float32 frames, uniform in [lo, hi), drawn in row-major order."""
    return stream.uniform(n * c * h * w, lo, hi).astype(np.float32).reshape(n, c, h, w)


@dataclass
class LayerParams:
    w: np.ndarray                 # [cout, cin, k, k] float32
    gamma: np.ndarray = None      # [cout] float32 (bn)
    beta: np.ndarray = None
    mean: np.ndarray = None
    var: np.ndarray = None
    bias: np.ndarray = None       # [cout] float32 (no bn)


def make_params(stream: Stream, spec: NetSpec) -> List[LayerParams]:
    """He-init weights N(0, sqrt(2/fan_in)) (std), BN gamma U[0.5,1.5],
    beta U[-0.1,0.1], mean U[-0.1,0.1], var U[0.5,1.5]; linear layers get a
    bias U[-0.1,0.1].  Draw order per layer: W (o,c,kh,kw), then gamma, beta,
    mean, var (or bias)."""
    out = []
    for l, cin in zip(spec.layers, spec.cins()):
        fan_in = cin * l.k * l.k
        w = stream.normal(l.cout * fan_in, np.sqrt(2.0 / fan_in)).astype(np.float32)
        p = LayerParams(w.reshape(l.cout, cin, l.k, l.k))
        if l.bn:
            p.gamma = stream.uniform(l.cout, 0.5, 1.5).astype(np.float32)
            p.beta = stream.uniform(l.cout, -0.1, 0.1).astype(np.float32)
            p.mean = stream.uniform(l.cout, -0.1, 0.1).astype(np.float32)
            p.var = stream.uniform(l.cout, 0.5, 1.5).astype(np.float32)
        else:
            p.bias = stream.uniform(l.cout, -0.1, 0.1).astype(np.float32)
        out.append(p)
    return out


def pack_blob(spec: NetSpec, params: List[LayerParams]) -> np.ndarray:
    """Weight blob, float32, per layer in order: [beta, gamma, mean, var]
    (each cout) when bn else [bias] (cout); then W as [cout][cin][k][k]."""
    parts = []
    for l, p in zip(spec.layers, params):
        if l.bn:
            parts += [p.beta, p.gamma, p.mean, p.var]
        else:
            parts.append(p.bias)
        parts.append(p.w.reshape(-1))
    return np.ascontiguousarray(np.concatenate(parts).astype(np.float32))


def blob_floats(spec: NetSpec) -> int:
    return spec.n_params()


def unpack_blob(spec: NetSpec, blob: np.ndarray) -> List[LayerParams]:
    out, off = [], 0
    for l, cin in zip(spec.layers, spec.cins()):
        def take(n):
            nonlocal off
            a = blob[off:off + n]
            off += n
            return a
        if l.bn:
            beta, gamma, mean, var = take(l.cout), take(l.cout), take(l.cout), take(l.cout)
            w = take(l.cout * cin * l.k * l.k).reshape(l.cout, cin, l.k, l.k)
            out.append(LayerParams(w, gamma, beta, mean, var))
        else:
            bias = take(l.cout)
            w = take(l.cout * cin * l.k * l.k).reshape(l.cout, cin, l.k, l.k)
            out.append(LayerParams(w, bias=bias))
    assert off == blob.size, (off, blob.size)
    return out


# ---------------------------------------------------------------------------
# Workloads (seeds are fixed per workload so every consumer sees the same data)
# ---------------------------------------------------------------------------
SEED_SINGLE, SEED_9CONV, SEED_19CONV, SEED_UNEVEN, SEED_SERVE = 1, 2, 3, 4, 5
SEED_CALIB = 101


def workload_single():
    """1x16x32x32 U[-1,1] through one conv layer (seed 1)."""
    s = Stream(SEED_SINGLE)
    spec = net_single_conv()
    x = make_frames(s, 1, 16, 32, 32, -1.0, 1.0)
    params = make_params(s, spec)
    return spec, x, pack_blob(spec, params)


def workload_net(spec: NetSpec, seed: int, n: int, h: int, w: int):
    """Frames (n,3,h,w) U[0,1] then the weights, both from ``seed``."""
    s = Stream(seed)
    x = make_frames(s, n, spec.in_c, h, w)
    params = make_params(s, spec)
    return spec, x, pack_blob(spec, params)


def weights_for(spec: NetSpec, seed: int) -> np.ndarray:
    """Weights alone, from their own stream (seed) — used where frames come
    from elsewhere (uneven batches, serving, calibration)."""
    return pack_blob(spec, make_params(Stream(seed), spec))


def uneven_sides(n: int = 64, seed: int = SEED_UNEVEN, sides=(320, 416, 512, 608)) -> np.ndarray:
    return Stream(seed).choice(sides, n)


def frame_for(seed: int, index: int, side: int, c: int = 3) -> np.ndarray:
    """Frame ``index`` of a frame sequence: its own stream so that a frame
    does not depend on the sizes of the frames before it."""
    s = Stream((seed << 32) + index + 1)
    return make_frames(s, 1, c, side, side)


def laplace_grid(seed: int, ny: int, nx: int, interior: str = "zero") -> np.ndarray:
    """Initial grid of a Laplace problem (ny x nx float32, row-major): the
    boundary rows and columns uniform in [0, 1); the interior zero, or
    uniform in [0, 1) too ("random"), drawn after the boundary."""
    s = Stream(seed)
    g = np.zeros((ny, nx), np.float64)
    g[0, :] = s.uniform(nx)
    g[-1, :] = s.uniform(nx)
    g[1:-1, 0] = s.uniform(ny - 2)
    g[1:-1, -1] = s.uniform(ny - 2)
    if interior == "random":
        g[1:-1, 1:-1] = s.uniform((ny - 2) * (nx - 2)).reshape(ny - 2, nx - 2)
    return g.astype(np.float32)


def poisson_arrivals(rate_fps: float, duration_s: float, seed: int = SEED_SERVE,
                     sides=(320, 416, 608), cameras: int = 32):
    """Open-loop arrival schedule: ``cameras`` independent Poisson processes
    of rate rate_fps/cameras each.  Returns (t_seconds sorted, camera, side)."""
    s = Stream(seed)
    per = rate_fps / cameras
    ts, cams = [], []
    for cam in range(cameras):
        n_est = int(per * duration_s * 1.5 + 50)
        gaps = -np.log1p(-s.uniform(n_est)) / per
        t = np.cumsum(gaps)
        t = t[t < duration_s]
        ts.append(t)
        cams.append(np.full(t.size, cam))
    t = np.concatenate(ts)
    cam = np.concatenate(cams)
    order = np.argsort(t, kind="stable")
    t, cam = t[order], cam[order]
    side = s.choice(sides, t.size)
    return t, cam, side
