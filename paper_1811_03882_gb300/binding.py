"""ctypes binding of libnet.so (include/net.h): argument marshalling only.

Every step of the forward pass runs in the library's CUDA kernels; this
module only converts Python/NumPy/torch arguments into the C ABI's plain
pointers and sizes.  If libnet.so is missing the import of ``lib()`` raises:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnet.so")

NET_OK, NET_E_INVAL, NET_E_SHAPE, NET_E_WEIGHTS, NET_E_OOM, NET_E_BUDGET = 0, 1, 2, 3, 4, 5
NET_E_TIMEOUT, NET_E_CUDA, NET_E_DEVICE_WAIT, NET_E_STATE, NET_E_UNSUPPORTED = 6, 7, 8, 9, 10
NET_FP32, NET_BF16, NET_FP8 = 0, 1, 2
PREC = {"fp32": NET_FP32, "bf16": NET_BF16, "fp8": NET_FP8}

STATUS_NAMES = {0: "NET_OK", 1: "NET_E_INVAL", 2: "NET_E_SHAPE", 3: "NET_E_WEIGHTS", 4: "NET_E_OOM",
                5: "NET_E_BUDGET", 6: "NET_E_TIMEOUT", 7: "NET_E_CUDA", 8: "NET_E_DEVICE_WAIT",
                9: "NET_E_STATE", 10: "NET_E_UNSUPPORTED"}


class NetError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class net_layer(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("cout", ctypes.c_int), ("bn", ctypes.c_int),
                ("act", ctypes.c_int), ("pool", ctypes.c_int)]


class net_desc(ctypes.Structure):
    _fields_ = [("in_c", ctypes.c_int), ("n_layers", ctypes.c_int),
                ("layers", ctypes.POINTER(net_layer)), ("prec", ctypes.c_int),
                ("layer_prec", ctypes.POINTER(ctypes.c_int)), ("max_batch", ctypes.c_int),
                ("max_side", ctypes.c_int), ("hbm_budget_bytes", ctypes.c_size_t),
                ("cuda_stream", ctypes.c_void_p), ("device", ctypes.c_int)]


class net_ga_opts(ctypes.Structure):
    _fields_ = [("population", ctypes.c_int), ("generations", ctypes.c_int),
                ("crossover", ctypes.c_double), ("mutation", ctypes.c_double),
                ("max_err", ctypes.c_double), ("reps", ctypes.c_int), ("seed", ctypes.c_ulonglong)]


class net_ga_result(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double), ("err", ctypes.c_double),
                ("ms_all_bf16", ctypes.c_double), ("err_all_bf16", ctypes.c_double),
                ("ms_all_fp8", ctypes.c_double), ("err_all_fp8", ctypes.c_double),
                ("evaluations", ctypes.c_int), ("memo_hits", ctypes.c_int), ("fp8_layers", ctypes.c_int)]


class net_tile_result(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double), ("ms_analytic", ctypes.c_double),
                ("evaluations", ctypes.c_int), ("memo_hits", ctypes.c_int), ("changed_layers", ctypes.c_int)]


REGION_MAX_ANCHORS = 16


class net_region(ctypes.Structure):
    _fields_ = [("n_anchors", ctypes.c_int), ("n_classes", ctypes.c_int),
                ("anchors", ctypes.c_float * (2 * REGION_MAX_ANCHORS)), ("score_thresh", ctypes.c_float),
                ("nms_iou", ctypes.c_float), ("max_det", ctypes.c_int)]


# net_detection as a numpy record (32 bytes)
DETECTION = np.dtype([("x", np.float32), ("y", np.float32), ("w", np.float32), ("h", np.float32),
                      ("score", np.float32), ("cls", np.int32), ("id", np.int32), ("pad", np.int32)])

_lib = None
_lock = threading.Lock()

_SIGS = {
    "net_create": [ctypes.POINTER(net_desc), ctypes.POINTER(ctypes.c_void_p)],
    "net_load_weights": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t],
    "net_set_act_scales": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int],
    "net_calibrate": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                      ctypes.c_void_p],
    "net_output_shape": [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                         ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)],
    "net_forward": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                    ctypes.c_void_p, ctypes.c_size_t],
    "net_forward_async": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                          ctypes.c_void_p, ctypes.c_size_t],
    "net_forward_wait": [ctypes.c_void_p],
    "net_forward_device": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                           ctypes.c_void_p],
    "net_forward_trace": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                          ctypes.c_void_p],
    "net_forward_uneven": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                           ctypes.c_void_p],
    "net_submit": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                   ctypes.POINTER(ctypes.c_uint64)],
    "net_poll": [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_size_t,
                 ctypes.POINTER(ctypes.c_int)],
    "net_wait": [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int],
    "net_stats": [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                  ctypes.POINTER(ctypes.c_double)],
    "net_set_layer_prec": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int],
    "net_get_layer_prec": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int],
    "net_tune_precision": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                           ctypes.POINTER(net_ga_opts), ctypes.c_void_p, ctypes.POINTER(net_ga_result)],
    "net_set_layer_tiles": [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int],
    "net_set_layer_ctas": [ctypes.c_void_p, ctypes.c_int, ctypes.c_int],
    "net_tune_uneven": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                        ctypes.POINTER(net_ga_opts), ctypes.POINTER(net_tile_result)],
    "net_plan_grouped": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int],
    "net_plan_ctas": [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int],
    "net_plan_flow": [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int],
    "net_plan_tiles": [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                       ctypes.c_int],
    "net_tune_tiles": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                       ctypes.POINTER(net_ga_opts), ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(net_tile_result)],
    "net_stats_reset": [ctypes.c_void_p],
    "net_profile": [ctypes.c_void_p, ctypes.c_int],
    "net_layer_times": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int],
    "net_launches": [ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64)],
    "net_trace": [ctypes.c_void_p, ctypes.c_int],
    "net_trace_read": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t],
    "net_inject_device_fault": [ctypes.c_void_p, ctypes.c_int],
    "net_inject_flow_fault": [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int],
    "net_guard_check": [ctypes.c_void_p, ctypes.c_void_p],
    "net_guard_poke": [ctypes.c_uint64],
    "net_set_region": [ctypes.c_void_p, ctypes.POINTER(net_region)],
    "net_nightmare_grad": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                           ctypes.c_void_p, ctypes.c_void_p],
    "net_nightmare_trace": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
    "net_nightmare_step": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                           ctypes.c_float, ctypes.c_void_p],
    "net_jacobi_create": [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)],
    "net_jacobi_solve": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_float, ctypes.c_int, ctypes.c_void_p,
                         ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float)],
    "net_jacobi_solve_device": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_float, ctypes.c_int, ctypes.c_void_p,
                                ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float)],
    "net_jacobi_launches": [ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64)],
    "net_jacobi_free": [ctypes.c_void_p],
    "net_detect_device": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                          ctypes.c_void_p, ctypes.c_void_p],
    "net_forward_detect": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                           ctypes.c_void_p, ctypes.c_void_p],
    "net_conv2d_f32_noalloc": [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                               ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                               ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p],
    "net_free": [ctypes.c_void_p],
    "net_last_error": [],
    "net_version": [],
}


def lib():
    """Loads libnet.so (built by paper_1811_03882_gb300.build)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("libnet.so not built: run paper_1811_03882_gb300.build.build() "
                                   "(the CUDA library is the only implementation)")
            L = ctypes.CDLL(LIB_PATH)
            for name, args in _SIGS.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = ctypes.c_char_p if name in ("net_last_error", "net_version") else ctypes.c_int
            _lib = L
    return _lib


def guard_check():
    """(buffers checked, buffers with a changed guard region); (0, 0) unless
    NET_GUARD=1 (net_guard_check)."""
    b, c = ctypes.c_uint64(0), ctypes.c_uint64(0)
    check(lib().net_guard_check(ctypes.byref(b), ctypes.byref(c)))
    return int(b.value), int(c.value)


def guard_poke(index: int):
    """Test hook: one byte written past guarded buffer `index` (net_guard_poke)."""
    check(lib().net_guard_poke(int(index)))


def last_error() -> str:
    return lib().net_last_error().decode()


def check(status: int):
    if status != NET_OK:
        raise NetError(status, last_error())


def _ptr(a):
    """Address of a numpy array or torch tensor (host or device)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        return ctypes.c_void_p(a.ctypes.data)
    return ctypes.c_void_p(int(a))


class Jacobi:
    """Owning wrapper of a net_jacobi_t handle (Jacobi solver of the Laplace
    equation on an ny x nx float32 grid)."""

    def __init__(self, ny: int, nx: int, device: int = 0, stream=None):
        h = ctypes.c_void_p()
        check(lib().net_jacobi_create(ny, nx, device, stream, ctypes.byref(h)))
        self.h, self.ny, self.nx = h, ny, nx

    def solve(self, grid: np.ndarray, tol: float, iter_max: int, out: np.ndarray = None):
        """Host grid -> (host result, sweeps, last change)."""
        g = np.ascontiguousarray(grid, dtype=np.float32)
        out = np.empty_like(g) if out is None else out
        k, ch = ctypes.c_int(), ctypes.c_float()
        check(lib().net_jacobi_solve(self.h, _ptr(g), tol, iter_max, _ptr(out), ctypes.byref(k), ctypes.byref(ch)))
        return out, k.value, ch.value

    def solve_device(self, d_in, tol: float, iter_max: int, d_out):
        k, ch = ctypes.c_int(), ctypes.c_float()
        check(lib().net_jacobi_solve_device(self.h, _ptr(d_in), tol, iter_max, _ptr(d_out), ctypes.byref(k),
                                            ctypes.byref(ch)))
        return k.value, ch.value

    def launches(self) -> int:
        t = ctypes.c_uint64()
        check(lib().net_jacobi_launches(self.h, ctypes.byref(t)))
        return t.value

    def close(self):
        if getattr(self, "h", None):
            lib().net_jacobi_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Net:
    """Owning wrapper of a net_t handle."""

    def __init__(self, layers, in_c: int, prec="fp32", layer_prec=None, max_batch: int = 1,
                 max_side: int = 416, stream=None, budget_bytes: int = 0, device: int = 0):
        L = lib()
        self._layers = (net_layer * len(layers))(
            *[net_layer(l.k, l.cout, int(l.bn), l.act, l.pool) for l in layers])
        self.n_layers = len(layers)
        self.layers = list(layers)
        self.in_c = in_c
        lp = None
        if layer_prec is not None:
            self._lp = (ctypes.c_int * len(layers))(*[PREC.get(p, p) for p in layer_prec])
            lp = ctypes.cast(self._lp, ctypes.POINTER(ctypes.c_int))
        d = net_desc(in_c, len(layers), ctypes.cast(self._layers, ctypes.POINTER(net_layer)),
                     PREC.get(prec, prec), lp, max_batch, max_side, budget_bytes,
                     ctypes.c_void_p(stream) if stream else None, device)
        h = ctypes.c_void_p()
        check(L.net_create(ctypes.byref(d), ctypes.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().net_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def load_weights(self, blob: np.ndarray):
        blob = np.ascontiguousarray(blob, dtype=np.float32)
        check(lib().net_load_weights(self.h, _ptr(blob), blob.size))

    def set_act_scales(self, scales):
        s = np.ascontiguousarray(scales, dtype=np.float32)
        check(lib().net_set_act_scales(self.h, _ptr(s), s.size))

    def calibrate(self, d_frames, batch, h, w) -> np.ndarray:
        out = np.zeros(self.n_layers, np.float32)
        check(lib().net_calibrate(self.h, _ptr(d_frames), batch, h, w, _ptr(out)))
        return out

    def output_shape(self, h: int, w: int):
        c, ho, wo = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        check(lib().net_output_shape(self.h, h, w, ctypes.byref(c), ctypes.byref(ho), ctypes.byref(wo)))
        return c.value, ho.value, wo.value

    def forward(self, x: np.ndarray, out: np.ndarray = None) -> np.ndarray:
        """Host NCHW float32 in -> host NCHW float32 out (1 H2D + 1 D2H)."""
        n, _, h, w = x.shape
        c, ho, wo = self.output_shape(h, w)
        if out is None:
            out = np.empty((n, c, ho, wo), np.float32)
        check(lib().net_forward(self.h, _ptr(x), n, h, w, _ptr(out), out.size))
        return out

    def forward_async(self, x: np.ndarray, out: np.ndarray) -> None:
        """Enqueues net_forward's work and returns; x must stay unchanged and
        out unread until forward_wait() (pinned host arrays overlap best)."""
        n, _, h, w = x.shape
        check(lib().net_forward_async(self.h, _ptr(x), n, h, w, _ptr(out), out.size))

    def forward_wait(self) -> None:
        check(lib().net_forward_wait(self.h))

    def forward_device(self, d_in, batch, h, w, d_out):
        check(lib().net_forward_device(self.h, _ptr(d_in), batch, h, w, _ptr(d_out)))

    def forward_trace(self, d_in, batch, h, w, d_layer_outs):
        arr = (ctypes.c_void_p * len(d_layer_outs))(*[t.data_ptr() for t in d_layer_outs])
        check(lib().net_forward_trace(self.h, _ptr(d_in), batch, h, w, arr))

    def forward_uneven(self, d_ins, sides, d_outs):
        n = len(d_ins)
        a = (ctypes.c_void_p * n)(*[t.data_ptr() for t in d_ins])
        s = (ctypes.c_int * n)(*[int(v) for v in sides])
        o = (ctypes.c_void_p * n)(*[t.data_ptr() for t in d_outs])
        check(lib().net_forward_uneven(self.h, a, s, n, o))

    def submit(self, frame: np.ndarray) -> int:
        rid = ctypes.c_uint64()
        _, _, h, w = frame.shape
        check(lib().net_submit(self.h, _ptr(frame), h, w, ctypes.byref(rid)))
        return rid.value

    def poll(self, rid: int, out: np.ndarray) -> bool:
        done = ctypes.c_int()
        check(lib().net_poll(self.h, rid, _ptr(out), out.size, ctypes.byref(done)))
        return bool(done.value)

    def wait(self, rid: int, out: np.ndarray, timeout_ms: int = -1):
        check(lib().net_wait(self.h, rid, _ptr(out), out.size, timeout_ms))

    def set_layer_prec(self, precs):
        a = np.ascontiguousarray([PREC.get(p, p) for p in precs], dtype=np.int32)
        check(lib().net_set_layer_prec(self.h, _ptr(a), a.size))

    def layer_prec(self):
        a = np.zeros(self.n_layers, np.int32)
        check(lib().net_get_layer_prec(self.h, _ptr(a), a.size))
        names = {v: k for k, v in PREC.items()}
        return [names[int(v)] for v in a]

    def tune_precision(self, d_frames, batch, h, w, max_err, population=16, generations=12,
                       crossover=0.9, mutation=0.05, reps=3, seed=0):
        """Genetic FP8/BF16 plan search; returns (layer precisions, result dict)."""
        o = net_ga_opts(population, generations, crossover, mutation, max_err, reps, seed)
        r = net_ga_result()
        out = np.zeros(self.n_layers, np.int32)
        check(lib().net_tune_precision(self.h, _ptr(d_frames), batch, h, w, ctypes.byref(o), _ptr(out),
                                       ctypes.byref(r)))
        names = {v: k for k, v in PREC.items()}
        return [names[int(v)] for v in out], {f: getattr(r, f) for f, _ in net_ga_result._fields_}

    def set_layer_tiles(self, layer, bn=0, ksplit=0):
        """Overrides one tensor-core layer's N tile / split-K (0: analytic)."""
        check(lib().net_set_layer_tiles(self.h, layer, bn, ksplit))

    def tune_uneven(self, d_ins, sides, d_outs, max_err=1e-6, population=12, generations=8,
                    crossover=0.9, mutation=0.05, reps=3, seed=0):
        """Genetic search over the grouped launches of this uneven batch;
        returns (per-layer (bn, mb, nst) overrides, result dict)."""
        k = len(d_ins)
        a = (ctypes.c_void_p * k)(*[t.data_ptr() for t in d_ins])
        s = (ctypes.c_int * k)(*[int(v) for v in sides])
        o = (ctypes.c_void_p * k)(*[t.data_ptr() for t in d_outs])
        opts = net_ga_opts(population, generations, crossover, mutation, max_err, reps, seed)
        r = net_tile_result()
        check(lib().net_tune_uneven(self.h, a, s, k, o, ctypes.byref(opts), ctypes.byref(r)))
        return self.plan_grouped(), {f: getattr(r, f) for f, _ in net_tile_result._fields_}

    def plan_grouped(self):
        bn = np.zeros(self.n_layers, np.int32)
        mb = np.zeros(self.n_layers, np.int32)
        nst = np.zeros(self.n_layers, np.int32)
        check(lib().net_plan_grouped(self.h, _ptr(bn), _ptr(mb), _ptr(nst), self.n_layers))
        return [(int(a), int(b), int(c)) for a, b, c in zip(bn, mb, nst)]

    def set_layer_ctas(self, layer, mb=0):
        """Overrides one tensor-core layer's CTAs per SM (1, 2; 0: chosen)."""
        check(lib().net_set_layer_ctas(self.h, layer, mb))

    def plan_ctas(self, batch, h, w):
        """CTAs per SM of every layer's fixed-batch launch (0: CUDA cores)."""
        mb = np.zeros(self.n_layers, np.int32)
        check(lib().net_plan_ctas(self.h, batch, h, w, _ptr(mb), self.n_layers))
        return [int(v) for v in mb]

    def plan_flow(self, batch, h, w):
        """Per layer of the fixed-batch plan: 1 if it waits for the previous
        layer's row bands instead of the whole previous kernel."""
        dep = np.zeros(self.n_layers, np.int32)
        check(lib().net_plan_flow(self.h, batch, h, w, _ptr(dep), self.n_layers))
        return [int(v) for v in dep]

    def plan_tiles(self, batch, h, w):
        """[(bn, ksplit)] per layer of the fixed-batch plan ((0, 0): CUDA cores)."""
        bn = np.zeros(self.n_layers, np.int32)
        ks = np.zeros(self.n_layers, np.int32)
        check(lib().net_plan_tiles(self.h, batch, h, w, _ptr(bn), _ptr(ks), self.n_layers))
        return [(int(a), int(b)) for a, b in zip(bn, ks)]

    def tune_tiles(self, d_frames, batch, h, w, max_err=2e-2, population=12, generations=8,
                   crossover=0.9, mutation=0.05, reps=3, seed=0):
        """Genetic tile-plan search; returns ([(bn, ksplit)] per layer, result dict)."""
        o = net_ga_opts(population, generations, crossover, mutation, max_err, reps, seed)
        r = net_tile_result()
        bn = np.zeros(self.n_layers, np.int32)
        ks = np.zeros(self.n_layers, np.int32)
        check(lib().net_tune_tiles(self.h, _ptr(d_frames), batch, h, w, ctypes.byref(o), _ptr(bn), _ptr(ks),
                                   ctypes.byref(r)))
        return [(int(a), int(b)) for a, b in zip(bn, ks)], {f: getattr(r, f) for f, _ in net_tile_result._fields_}

    def stats_reset(self):
        check(lib().net_stats_reset(self.h))

    def profile(self, enable: bool = True):
        check(lib().net_profile(self.h, int(enable)))

    def layer_times(self) -> np.ndarray:
        ms = np.zeros(self.n_layers, np.float64)
        check(lib().net_layer_times(self.h, _ptr(ms), self.n_layers))
        return ms

    def set_region(self, anchors, n_classes: int, score_thresh: float, nms_iou: float, max_det: int):
        """Detection parameters (net_set_region); anchors: [(pw, ph)] in grid cells."""
        r = net_region()
        r.n_anchors = len(anchors)
        r.n_classes = n_classes
        for i, (pw, ph) in enumerate(anchors):
            r.anchors[2 * i] = pw
            r.anchors[2 * i + 1] = ph
        r.score_thresh = score_thresh
        r.nms_iou = nms_iou
        r.max_det = max_det
        check(lib().net_set_region(self.h, ctypes.byref(r)))
        self.max_det = max_det

    def detect_device(self, d_map, batch, gh, gw, d_counts, d_det):
        """Stream-ordered detection of a device map into device counts / rows
        (d_det: a uint8 tensor of batch * max_det * 32 bytes)."""
        check(lib().net_detect_device(self.h, _ptr(d_map), batch, gh, gw, _ptr(d_counts), _ptr(d_det)))

    def forward_detect(self, x: np.ndarray):
        """Host frames -> (counts[batch], detections[batch, max_det] as DETECTION records)."""
        x = np.ascontiguousarray(x, dtype=np.float32)
        n, _, h, w = x.shape
        counts = np.zeros(n, np.int32)
        det = np.zeros((n, self.max_det), DETECTION)
        check(lib().net_forward_detect(self.h, _ptr(x), n, h, w, _ptr(counts), _ptr(det)))
        return counts, det

    def nightmare_grad(self, d_in, batch, h, w, layer, d_grad):
        """dJ/d(frames) of J = 1/2 sum(output of `layer`)^2 into d_grad; returns J per frame."""
        obj = np.zeros(batch, np.float64)
        check(lib().net_nightmare_grad(self.h, _ptr(d_in), batch, h, w, layer, _ptr(d_grad), _ptr(obj)))
        return obj

    def nightmare_trace(self, d_in, batch, h, w, layer, d_grad, d_acts, d_gouts):
        """As nightmare_grad, also each layer's pre-pool activation and output gradient."""
        a = (ctypes.c_void_p * len(d_acts))(*[t.data_ptr() for t in d_acts])
        g = (ctypes.c_void_p * len(d_gouts))(*[t.data_ptr() for t in d_gouts])
        check(lib().net_nightmare_trace(self.h, _ptr(d_in), batch, h, w, layer, _ptr(d_grad), a, g))

    def nightmare_step(self, d_frames, batch, h, w, layer, rate):
        """One gradient-ascent step on the device frames in place; returns J before it."""
        obj = np.zeros(batch, np.float64)
        check(lib().net_nightmare_step(self.h, _ptr(d_frames), batch, h, w, layer, rate, _ptr(obj)))
        return obj

    def inject_device_fault(self, layer: int):
        """Test hook: the next fixed-batch pass faults layer `layer` (see net.h)."""
        check(lib().net_inject_device_fault(self.h, layer))

    def inject_flow_fault(self, layer: int, batch: int, h: int, w: int):
        """Test hook: the next batch x h x w pass makes layer `layer`'s band
        wait expire (see net.h)."""
        check(lib().net_inject_flow_fault(self.h, layer, batch, h, w))

    def launches(self) -> int:
        t = ctypes.c_uint64()
        check(lib().net_launches(self.h, ctypes.byref(t)))
        return t.value

    TRACE_CTAS, TRACE_EVENTS = 512, 10

    def trace(self, enable: bool = True):
        """Phase trace of the tensor-core launches on (clears it) or off (net_trace)."""
        check(lib().net_trace(self.h, int(enable)))

    def trace_read(self) -> np.ndarray:
        """[n_layers, 512, 10] uint64 globaltimer stamps of the last traced pass."""
        out = np.zeros((self.n_layers, self.TRACE_CTAS, self.TRACE_EVENTS), np.uint64)
        check(lib().net_trace_read(self.h, out.ctypes.data, out.size))
        return out

    def stats(self):
        f, p50, p99 = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        check(lib().net_stats(self.h, ctypes.byref(f), ctypes.byref(p50), ctypes.byref(p99)))
        return f.value, p50.value, p99.value


def conv2d_f32_noalloc(d_x, n, cin, h, w, d_weight, d_bias, cout, k, act, pool, d_y, stream=None):
    """net_conv2d_f32_noalloc: one FP32 conv layer using only the library's
    static scratch array (no device allocation)."""
    check(lib().net_conv2d_f32_noalloc(_ptr(d_x), n, cin, h, w, _ptr(d_weight), _ptr(d_bias), cout, k,
                                       act, pool, _ptr(d_y), ctypes.c_void_p(stream) if stream else None))
