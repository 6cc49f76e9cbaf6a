"""FP64 CPU oracle for the device-resident CNN forward pass.

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only users.  The product library never
imports, links or runs anything here, and this package imports nothing from
the product: network layers arrive as plain objects with ``k, cout, bn, act,
pool`` attributes and the weights as the float32 blob that the library's
``net_load_weights`` also takes.

The arithmetic lives in ``oracle.c`` (plain nested loops in FP64, built with
gcc); this module composes the layers in the order conv -> batchnorm (or
bias) -> leaky 0.1 -> max pool, the order in which Darknet's convolutional
layer applies them.  The paper (Sec. 5.1.1) names Darknet's image-analysis
apps as the offloaded workload but prints no layer definitions, so each step
follows the textbook definition stated in ``oracle.c``.

Two forward passes are provided:

* ``forward``: exact FP64, batchnorm applied unfolded (so the library's
  fold is checked, not assumed).
* ``forward_quant``: FP64 arithmetic over operands rounded to the storage
  formats a reduced-precision path uses (BF16, or FP8 E4M3 with
  per-output-channel weight scales and a per-layer activation scale).  It
  separates rounding error from kernel bugs.

Parity pins for every function here are in tests/test_oracle_pins.py and,
for ``forward_quant`` and ``act_scales_from``, tests/test_oracle_quant_pins.py
(an independent float64 torch composition, matched to 1e-12 layer by layer).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_oracle.so")
_lock = threading.Lock()
_lib = None

BN_EPS = 1e-5          # batchnorm epsilon inside the square root
LEAKY_SLOPE = 0.1      # Darknet's leaky rectifier slope
FP8_MAX = 448.0        # largest finite E4M3 value

ACT_LINEAR, ACT_LEAKY = 0, 1
POOL_NONE, POOL_2X2S2, POOL_2X2S1_SAME = 0, 1, 2


def build(force: bool = False) -> str:
    """Compiles oracle.c with gcc (OpenMP) into oracle/_oracle.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99",
                               "-D_GNU_SOURCE", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            D = ctypes.POINTER(ctypes.c_double)
            i, l, d = ctypes.c_int, ctypes.c_long, ctypes.c_double
            L.oracle_conv2d.argtypes = [D, i, i, i, i, D, i, i, D]
            L.oracle_conv2d_bwd_data.argtypes = [D, i, i, i, i, D, i, i, D]
            L.oracle_batchnorm.argtypes = [D, i, i, l, D, D, D, D, d]
            L.oracle_bias.argtypes = [D, i, i, l, D]
            L.oracle_leaky.argtypes = [D, l, d]
            L.oracle_maxpool2_s2.argtypes = [D, i, i, i, i, D]
            L.oracle_maxpool2_s1_same.argtypes = [D, i, i, i, i, D]
            L.oracle_round_bf16.argtypes = [D, l]
            L.oracle_round_e4m3_sat.argtypes = [D, l]
            L.oracle_threads.restype = ctypes.c_int
            L.oracle_set_threads.argtypes = [i]
            _lib = L
    return _lib


def threads() -> int:
    return int(lib().oracle_threads())


def set_threads(n: int) -> None:
    """Threads of later oracle calls (OpenMP); timing use only."""
    lib().oracle_set_threads(int(n))


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


# ---------------------------------------------------------------- primitives
def conv2d(x, w) -> np.ndarray:
    """x: N,C,H,W; w: O,C,k,k (k odd) -> N,O,H,W; stride 1, zero pad (k-1)/2."""
    x, w = _f64(x), _f64(w)
    N, C, H, W = x.shape
    O, C2, k, k2 = w.shape
    assert C == C2 and k == k2 and k % 2 == 1
    y = np.empty((N, O, H, W), np.float64)
    if y.size:
        lib().oracle_conv2d(_p(x), N, C, H, W, _p(w), O, k, _p(y))
    return y


def conv2d_bwd_data(dy, w) -> np.ndarray:
    """Gradient of conv2d's input: dy: N,O,H,W; w: O,C,k,k -> N,C,H,W."""
    dy, w = _f64(dy), _f64(w)
    N, O, H, W = dy.shape
    O2, C, k, k2 = w.shape
    assert O == O2 and k == k2 and k % 2 == 1
    dx = np.empty((N, C, H, W), np.float64)
    if dx.size:
        lib().oracle_conv2d_bwd_data(_p(dy), N, O, H, W, _p(w), C, k, _p(dx))
    return dx


def batchnorm(y, gamma, beta, mean, var, eps: float = BN_EPS) -> np.ndarray:
    y = _f64(y).copy()
    N, O = y.shape[:2]
    hw = int(np.prod(y.shape[2:]))
    lib().oracle_batchnorm(_p(y), N, O, hw, _p(_f64(gamma)), _p(_f64(beta)),
                           _p(_f64(mean)), _p(_f64(var)), eps)
    return y


def add_bias(y, bias) -> np.ndarray:
    y = _f64(y).copy()
    N, O = y.shape[:2]
    lib().oracle_bias(_p(y), N, O, int(np.prod(y.shape[2:])), _p(_f64(bias)))
    return y


def leaky(y, slope: float = LEAKY_SLOPE) -> np.ndarray:
    y = _f64(y).copy()
    lib().oracle_leaky(_p(y), y.size, slope)
    return y


def maxpool2_s2(x) -> np.ndarray:
    x = _f64(x)
    N, C, H, W = x.shape
    assert H % 2 == 0 and W % 2 == 0
    y = np.empty((N, C, H // 2, W // 2), np.float64)
    lib().oracle_maxpool2_s2(_p(x), N, C, H, W, _p(y))
    return y


def maxpool2_s1_same(x) -> np.ndarray:
    x = _f64(x)
    N, C, H, W = x.shape
    y = np.empty_like(x)
    lib().oracle_maxpool2_s1_same(_p(x), N, C, H, W, _p(y))
    return y


def round_bf16(v) -> np.ndarray:
    v = _f64(v).copy()
    lib().oracle_round_bf16(_p(v), v.size)
    return v


def round_e4m3_sat(v) -> np.ndarray:
    v = _f64(v).copy()
    lib().oracle_round_e4m3_sat(_p(v), v.size)
    return v


# ------------------------------------------------------------- weight blob
def parse_blob(layers, in_c: int, blob):
    """Splits the float32 weight blob (per layer: [beta,gamma,mean,var] when
    bn else [bias], each cout long; then W as cout x cin x k x k)."""
    blob = np.asarray(blob, dtype=np.float32)
    out, off, cin = [], 0, in_c
    for l in layers:
        d = {}
        names = ("beta", "gamma", "mean", "var") if l.bn else ("bias",)
        for nm in names:
            d[nm] = blob[off:off + l.cout].astype(np.float64)
            off += l.cout
        nw = l.cout * cin * l.k * l.k
        d["w"] = blob[off:off + nw].astype(np.float64).reshape(l.cout, cin, l.k, l.k)
        off += nw
        out.append(d)
        cin = l.cout
    if off != blob.size:
        raise ValueError("weight blob has %d floats, layers need %d" % (blob.size, off))
    return out


def _pool(l, y):
    if l.pool == POOL_2X2S2:
        return maxpool2_s2(y)
    if l.pool == POOL_2X2S1_SAME:
        return maxpool2_s1_same(y)
    return y


# ------------------------------------------------------------ forward passes
def forward(layers, in_c: int, x, blob, keep_all: bool = False):
    """Exact FP64 forward pass.  Returns the final map (N, C_out, H', W'), or
    the list of every layer's output when keep_all."""
    ps = parse_blob(layers, in_c, blob)
    a = _f64(x)
    outs = []
    for l, p in zip(layers, ps):
        y = conv2d(a, p["w"])
        if l.bn:
            y = batchnorm(y, p["gamma"], p["beta"], p["mean"], p["var"])
        else:
            y = add_bias(y, p["bias"])
        if l.act == ACT_LEAKY:
            y = leaky(y)
        a = _pool(l, y)
        if keep_all:
            outs.append(a)
    return outs if keep_all else a


def fold(p):
    """Batchnorm fold in FP64: s = gamma/sqrt(var+eps), W' = s*W,
    b' = beta - mean*s; without batchnorm W' = W, b' = bias."""
    if "gamma" in p:
        s = p["gamma"] / np.sqrt(p["var"] + BN_EPS)
        return p["w"] * s[:, None, None, None], p["beta"] - p["mean"] * s
    return p["w"].copy(), p["bias"].copy()


def _store(v, prec: str, scale: float = 1.0):
    """Value of v after storing it in format `prec` (fp8 with `scale`)."""
    if prec == "fp32":
        return v.astype(np.float32).astype(np.float64)
    if prec == "bf16":
        return round_bf16(v)
    if prec == "fp8":
        return round_e4m3_sat(v / scale) * scale
    raise ValueError(prec)


def weight_scales_fp8(w_folded) -> np.ndarray:
    """Per-output-channel FP8 weight scale: max|W'_o| / 448."""
    amax = np.abs(w_folded).reshape(w_folded.shape[0], -1).max(axis=1)
    return np.maximum(amax, 1e-30) / FP8_MAX


def forward_quant(layers, in_c: int, x, blob, precs, act_scales=None,
                  keep_all: bool = False, out_store=None):
    """FP64 forward pass over operands rounded as a reduced-precision path
    stores them.  precs[l] in {'fp32','bf16','fp8'} is the operand format of
    layer l: its input activation and its folded weights are stored in it
    (FP8: activation / act_scales[l], weights / per-channel scale).  Bias is
    FP32; the epilogue (bias, leaky, pool) is exact; the final map is FP32,
    or, with out_store = (prec, scale), stored as a following layer of that
    format would read it (used to run one layer of a deeper network)."""
    ps = parse_blob(layers, in_c, blob)
    n = len(layers)
    a = _store(_f64(x), precs[0], act_scales[0] if precs[0] == "fp8" else 1.0)
    outs = []
    for li, (l, p) in enumerate(zip(layers, ps)):
        wf, bf = fold(p)
        if precs[li] == "fp8":
            sw = weight_scales_fp8(wf)
            wq = round_e4m3_sat(wf / sw[:, None, None, None]) * sw[:, None, None, None]
        else:
            wq = _store(wf, precs[li])
        y = conv2d(a, wq)
        y = add_bias(y, bf.astype(np.float32))
        if l.act == ACT_LEAKY:
            y = leaky(y)
        y = _pool(l, y)
        if li + 1 < n:
            nxt = precs[li + 1]
            a = _store(y, nxt, act_scales[li + 1] if nxt == "fp8" else 1.0)
        elif out_store is not None:
            a = _store(y, out_store[0], out_store[1])
        else:
            a = y.astype(np.float32).astype(np.float64)
        if keep_all:
            outs.append(a)
    return outs if keep_all else a


def act_scales_from(layers, in_c: int, x_calib, blob) -> np.ndarray:
    """Static per-layer FP8 activation scales: max|input of layer l| / 448
    over a calibration batch, from the exact FP64 forward pass."""
    outs = forward(layers, in_c, x_calib, blob, keep_all=True)
    ins = [_f64(x_calib)] + outs[:-1]
    return np.array([max(np.abs(t).max(), 1e-30) / FP8_MAX for t in ins])


# ----------------------------------------------------------------- metrics
def normwise_rel_err(y, r) -> float:
    """max_i |y_i - r_i| / max_i |r_i|."""
    y, r = _f64(y), _f64(r)
    den = np.abs(r).max()
    return float(np.abs(y - r).max() / (den if den > 0 else 1.0))


def rms_rel_err(y, r) -> float:
    """||y - r||_2 / ||r||_2."""
    y, r = _f64(y), _f64(r)
    den = np.sqrt((r * r).sum())
    return float(np.sqrt(((y - r) ** 2).sum()) / (den if den > 0 else 1.0))


def argmax_agreement(y, r, tie_tol: float):
    """Per spatial position, argmax over channels (axis 1).  Positions whose
    reference top-2 gap is below tie_tol * max|r| are near-ties and accepted
    either way.  Returns (agree_fraction, n_positions, n_ties)."""
    y, r = _f64(y), _f64(r)
    ay, ar = y.argmax(axis=1), r.argmax(axis=1)
    srt = np.sort(r, axis=1)
    gap = srt[:, -1] - srt[:, -2] if r.shape[1] > 1 else np.full(ar.shape, np.inf)
    tie = gap < tie_tol * np.abs(r).max()
    ok = (ay == ar) | tie
    return float(ok.mean()), int(ok.size), int(tie.sum())
