"""Throughput benchmark of the device-resident CNN forward pass.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                [--workload NAME] [--no-cpu-baseline]

One step = one forward pass of the whole network over one batch of
synthetic frames that are already resident in device memory (value), and
the same through the host API (net_forward_async over two pinned buffer
pairs, then net_forward_wait), the H2D and D2H copies of every step inside
the timed region (e2e).  Under torchrun every
rank runs its own replica on its own GPU (frames are independent; no
collective on the data path) and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1811_03882_gb300 import synth  # noqa: E402

# name -> (network, frames, side, precision, weight/frame seed)
WORKLOADS = {
    # the single conv layer: 1 x 16 x 32 x 32, U[-1, 1] (latency-bound: report us per call)
    "single-conv-32-fp32": ("single-conv", 1, 32, "fp32", synth.SEED_SINGLE),
    "19conv-448-b8-bf16": ("19-conv", 8, 448, "bf16", synth.SEED_19CONV),
    "19conv-448-b8-fp8": ("19-conv", 8, 448, "fp8", synth.SEED_19CONV),
    "9conv-416-b1-fp32": ("9-conv", 1, 416, "fp32", synth.SEED_9CONV),
    "9conv-416-b1-bf16": ("9-conv", 1, 416, "bf16", synth.SEED_9CONV),
    # 64 frames, sides drawn from {320, 416, 512, 608}, one grouped launch per layer
    "uneven64-9conv-bf16": ("9-conv", 64, 0, "bf16", synth.SEED_UNEVEN),
}
# the configurations measured beside the default one in the same line
OTHER_CONFIGS = ("single-conv-32-fp32", "9conv-416-b1-fp32", "9conv-416-b1-bf16", "uneven64-9conv-bf16")
# open-loop serving streams: 32 cameras, Poisson arrivals, sides {320,416,608}
SERVE_RATES = (200.0, 1000.0, 4000.0)
DEFAULT = "19conv-448-b8-bf16"

# DRAM traffic per launch of the dominant kernel family (ncu
# dram__bytes_read.sum + dram__bytes_write.sum, averaged over the family's
# launches in one forward pass of the workload), with the first 16 hex digits
# of the SHA-256 of the conv kernel's source when it was captured: the figure
# is reported only while the source is unchanged, null otherwise.
TRAFFIC = {"19conv-448-b8-bf16": {"conv_tc_kernel": (208.4e6 / 19, "780366b9a898f6a2")}}
KERNEL_SRC = os.path.join(ROOT, "paper_1811_03882_gb300", "csrc", "k_conv_tc.cu")

L2_FLUSH_BYTES = 256 << 20   # > 129 MB L2


def kernel_sha16():
    import hashlib
    return hashlib.sha256(open(KERNEL_SRC, "rb").read()).hexdigest()[:16]


def cpu_model():
    """Host CPU model (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during timing."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        self.rows = []
        if self.p is None:
            return
        time.sleep(0.25)
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
            out, _ = self.p.communicate()
        for line in out.strip().splitlines():
            f = [t.strip() for t in line.split(",")]
            if len(f) >= 9:
                self.rows.append(f)

    def summary(self):
        if not getattr(self, "rows", None):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(torch, value: float, ws: int, device="cuda") -> float:
    """The slowest rank's time: replicas run independently, the job takes as
    long as its slowest replica."""
    if ws <= 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_frames_per_s(frames_per_rank: int, ws: int, slowest_s: float) -> float:
    """Whole-job throughput of ws replicas: all ranks' frames over the
    slowest rank's time."""
    return frames_per_rank * ws / slowest_s


def oracle_frames_per_s(spec, x1, blob, budget_s: float, threads: int = 0):
    """FP64 oracle timed on this host's cores over whole frames until
    budget_s of CPU work has passed (at least one frame); threads > 0 limits
    its OpenMP threads for this measurement."""
    import oracle
    oracle.build()
    full = oracle.threads()
    if threads:
        oracle.set_threads(threads)
    try:
        used = oracle.threads()
        n, t0 = 0, time.perf_counter()
        while True:
            oracle.forward(spec.layers, spec.in_c, x1, blob)
            n += 1
            el = time.perf_counter() - t0
            if el >= budget_s:
                break
    finally:
        oracle.set_threads(full)
    return n / el, n, el, used


def workload_config(wl, ws):
    """The line's config, shared by both arms: the workload and how this run
    lays it out (the reference arm times a bounded sample of the same
    workload, stated in its cpu_baseline.sample)."""
    netname, batch, side, prec, _ = WORKLOADS[wl]
    return {"workload": wl, "network": netname, "global_batch": batch * ws, "frames_per_step_per_gpu": batch,
            "side": side if side else "uneven {320,416,512,608}", "precision": prec,
            "parallelism": "replicas%d" % ws, "l2": "flushed between steps (256 MB write)"}


def run_reference(args, wl):
    """The oracle as the reference arm: each step is one frame of the
    workload through the FP64 CPU forward pass."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    netname, batch, side, prec, seed = WORKLOADS[wl]
    spec = synth.NETS[netname]()
    if side:
        if netname == "single-conv":
            _, x, blob = synth.workload_single()
        else:
            _, x, blob = synth.workload_net(spec, seed, 1, side, side)
        frames = [x] * args.steps
    else:
        blob = synth.weights_for(spec, seed)
        sides = synth.uneven_sides(batch, seed)
        frames = [synth.frame_for(seed, i % batch, int(sides[i % batch])) for i in range(args.steps)]
    import oracle
    oracle.build()
    oracle.forward(spec.layers, spec.in_c, frames[0], blob)   # warm-up (one frame)
    t0 = time.perf_counter()
    for f in frames:
        oracle.forward(spec.layers, spec.in_c, f, blob)
    el = time.perf_counter() - t0
    fps = args.steps / el
    line = {"impl": "reference", "metric": "frames/s", "value": fps, "unit": "frames/s",
            "n_gpus": 0, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": workload_config(wl, ws), "frames_per_step": 1,
            "cpu_baseline": {"value": fps, "unit": "frames/s", "cores": oracle.threads(),
                             "kind": "oracle", "cpu_model": cpu_model(),
                             "sample": "%d frames (side %s), one per step" % (args.steps, side or "uneven")},
            "e2e": {"value": fps, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_serving(args, torch, binding, dev):
    """Serving streams through the request queue (net_submit / net_wait):
    32 cameras with Poisson arrivals at each aggregate rate, frame sides
    drawn from {320, 416, 608}, the 19-conv network with a GA-tuned FP8/BF16
    plan, a 40 GB activation budget.  Latency = completion - submission,
    measured by the library; the submitters keep to the arrival schedule
    (their lag is reported) so the queue does not hide load."""
    import queue
    import threading
    spec = synth.net_19conv()
    blob = synth.weights_for(spec, synth.SEED_SERVE)
    sides = (320, 416, 608)
    pool = {s_: [synth.frame_for(synth.SEED_SERVE, i, s_) for i in range(4)] for s_ in sides}
    duration, warm = args.serve_seconds, 1.0
    out = {"rates": {}}

    def make(prec):
        net = binding.Net(spec.layers, 3, prec=prec, max_batch=1, max_side=608, budget_bytes=40 << 30, device=dev)
        net.load_weights(blob)
        return net

    # FP32 unbatched reference: each frame alone through the host API
    n32 = make("fp32")
    lat32 = []
    for s_ in sides:
        f = pool[s_][0]
        o = np.empty((1,) + n32.output_shape(s_, s_), np.float32)
        n32.forward(f, o)
        for _ in range(3):
            t0 = time.perf_counter()
            n32.forward(f, o)
            lat32.append((s_, 1e3 * (time.perf_counter() - t0)))
    n32.close()
    mean32 = {s_: float(np.mean([t for ss, t in lat32 if ss == s_])) for s_ in sides}
    out["fp32_unbatched_ms"] = mean32
    out["fp32_unbatched_max_fps"] = 1e3 / float(np.mean(list(mean32.values())))

    net = make("fp8")
    xc = synth.make_frames(synth.Stream(synth.SEED_CALIB), 1, 3, 416, 416)
    d_c = torch.from_numpy(xc).cuda()
    net.calibrate(d_c, 1, 416, 416)
    plan, ga = net.tune_precision(d_c, 1, 416, 416, max_err=0.05, population=12, generations=8, reps=2, seed=5)
    out["plan"] = plan
    out["ga"] = ga
    for rate in SERVE_RATES:
        t_arr, cam, side = synth.poisson_arrivals(rate, warm + duration, synth.SEED_SERVE)
        pending = queue.Queue()
        lag = []
        n_sub = 4
        t0 = time.perf_counter() + 0.05

        def submitter(k):
            for i in range(k, len(t_arr), n_sub):
                now = time.perf_counter() - t0
                if t_arr[i] > now:
                    time.sleep(t_arr[i] - now)
                f = pool[int(side[i])][i % 4]
                lag.append(time.perf_counter() - t0 - t_arr[i])
                pending.put((net.submit(f), int(side[i])))
            pending.put(None)

        done_ct = [0]

        def collector():
            ends = 0
            while ends < n_sub:
                it = pending.get()
                if it is None:
                    ends += 1
                    continue
                rid, s_ = it
                o = np.empty((1,) + net.output_shape(s_, s_), np.float32)
                net.wait(rid, o, 120000)
                done_ct[0] += 1

        def reset_after_warmup():
            time.sleep(max(0.0, t0 + warm - time.perf_counter()))
            net.stats_reset()

        ths = [threading.Thread(target=submitter, args=(k,)) for k in range(n_sub)]
        ths.append(threading.Thread(target=reset_after_warmup))
        col = threading.Thread(target=collector)
        col.start()
        for th in ths:
            th.start()
        for th in ths:
            th.join()
        col.join()
        fps, p50, p99 = net.stats()
        out["rates"][str(int(rate))] = {"offered_fps": rate, "frames": int(len(t_arr)), "measured_s": duration,
                                        "fps": fps,
                                        "p50_ms": p50, "p99_ms": p99,
                                        "submit_lag_p99_ms": 1e3 * float(np.percentile(lag, 99))}
    net.close()
    return out


JACOBI_SIDE, JACOBI_SWEEPS = 8192, 200


def run_jacobi(torch, binding, dev, cpu_budget_s=4.0):
    """Jacobi solver of the Laplace equation (paper Sec. 4's sample app) on an
    8192 x 8192 grid (each iterate 268 MB, above L2): JACOBI_SWEEPS sweeps
    (tol 0) timed with CUDA events on the solver's stream (device-resident),
    then end to end from host memory (one H2D, one D2H), and the FP64 oracle
    on the host over a bounded number of sweeps.  Sweeps run in fused pairs
    (one pass over the grid computes two): the roofline's algorithmic bytes
    are those of one pair, the grid read once and its interior written
    once (FP32), against the time of two sweeps."""
    from oracle import jacobi as ojac
    pk, pk_kind = peaks()
    ny = nx = JACOBI_SIDE
    u0 = synth.laplace_grid(24, ny, nx, "random")
    st = torch.cuda.Stream()
    d_in = torch.from_numpy(u0).cuda()
    d_out = torch.empty_like(d_in)
    J = binding.Jacobi(ny, nx, dev, st.cuda_stream)
    J.solve_device(d_in, 0.0, 32, d_out)     # warm-up: graphs captured
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    l0 = J.launches()
    e0.record(st)
    J.solve_device(d_in, 0.0, 0, d_out)      # the copies in and out alone
    e1.record(st)
    k, _ = J.solve_device(d_in, 0.0, JACOBI_SWEEPS, d_out)
    e2.record(st)
    torch.cuda.synchronize()
    launches = J.launches() - l0
    t_sweeps = (e1.elapsed_time(e2) - e0.elapsed_time(e1)) / 1e3
    per_sweep = t_sweeps / k
    alg = 4.0 * ny * nx + 4.0 * (ny - 2) * (nx - 2)   # one pass: a fused pair of sweeps
    gbs = alg / (2.0 * per_sweep) / 1e9
    h_in = torch.from_numpy(u0).pin_memory()     # pinned: the copies run at link speed
    h_out = torch.empty_like(h_in).pin_memory()
    t0 = time.perf_counter()
    _, k2, _ = J.solve(h_in.numpy(), 0.0, JACOBI_SWEEPS, h_out.numpy())
    e2e_s = time.perf_counter() - t0
    J.close()
    # oracle: FP64 sweeps of the same grid on the host, bounded sample
    n, t0, u = 0, time.perf_counter(), u0.astype(np.float64)
    while True:
        u, _ = ojac.sweep(u)
        n += 1
        el = time.perf_counter() - t0
        if el >= cpu_budget_s:
            break
    return {"grid": [ny, nx], "dtype": "f32", "sweeps": k, "ms_per_sweep": 1e3 * per_sweep,
            "sweeps_per_s": 1.0 / per_sweep, "gpu_launches": int(launches),
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
                         "frac": gbs / pk["hbm_gbs"], "traffic": None,
                         "kernel": "jacobi_sweep2_kernel (two sweeps a launch)",
                         "alg_bytes_per_launch": alg, "peak_source": "hbm copy, %s" % pk_kind},
            "e2e": {"sweeps_per_s": k2 / e2e_s, "h2d_bytes": int(u0.nbytes), "d2h_bytes": int(u0.nbytes),
                    "note": "%d sweeps with one H2D and one D2H of the grid" % k2},
            "cpu_baseline": {"sweeps_per_s": n / el, "kind": "oracle (numpy FP64)", "cores": 1,
                             "sample": "%d sweep(s) of the same grid, %.1f s" % (n, el)}}


def run_detect(torch, binding, dev, side=416, batch=8):
    """Detection post-processing after the 9-conv network (125 channels on a
    13 x 13 grid per 416 x 416 frame): the two device kernels timed with
    CUDA events on a batch's map, and frames -> detections end to end
    (net_forward_detect: one H2D of the frames, one D2H of the detections)."""
    spec = synth.net_9conv()
    _, x, blob = synth.workload_net(spec, synth.SEED_9CONV, batch, side, side)
    anchors = [(0.8, 1.2), (2.0, 3.1), (4.5, 2.2), (6.0, 7.5), (9.7, 5.0)]
    st = torch.cuda.Stream()
    net = binding.Net(spec.layers, 3, prec="bf16", max_batch=batch, max_side=side, stream=st.cuda_stream,
                      device=dev)
    net.load_weights(blob)
    net.set_region(anchors, 20, 0.04, 0.45, 256)
    d_x = torch.from_numpy(x).cuda()
    c, gh, gw = net.output_shape(side, side)
    d_map = torch.empty((batch, c, gh, gw), device="cuda")
    d_cnt = torch.zeros(batch, dtype=torch.int32, device="cuda")
    d_det = torch.zeros(batch * 256 * 32, dtype=torch.uint8, device="cuda")
    net.forward_device(d_x, batch, side, side, d_map)
    for _ in range(3):
        net.detect_device(d_map, batch, gh, gw, d_cnt, d_det)
    reps = 50
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record(st)
    for _ in range(reps):
        net.detect_device(d_map, batch, gh, gw, d_cnt, d_det)
    ev[1].record(st)
    torch.cuda.synchronize()
    det_ms = ev[0].elapsed_time(ev[1]) / reps
    for _ in range(3):
        net.forward_detect(x)
    t0 = time.perf_counter()
    for _ in range(reps):
        counts, _ = net.forward_detect(x)
    e2e = time.perf_counter() - t0
    net.close()
    return {"network": "9-conv", "batch": batch, "side": side, "grid": [gh, gw], "anchors": 5, "classes": 20,
            "score_thresh": 0.04, "nms_iou": 0.45, "detect_ms_per_batch": det_ms, "kernels": 2,
            "kept_per_frame": [int(v) for v in counts],
            "e2e_frames_per_s": batch * reps / e2e,
            "e2e_note": "frames -> detections through net_forward_detect (BF16 network + decode + NMS), "
                        "one H2D and one D2H per batch"}


def run_nightmare(torch, binding, dev, side=416, layer=8, reps=10, cpu_budget_s=4.0):
    """The nightmare pass (gradient ascent on the frame toward one layer's
    energy) on the 9-conv network, FP32 path, one 416 x 416 frame, through
    its last layer: ascent steps timed with CUDA events; algorithmic FLOPs
    per step = the forward convs through `layer` twice (forward and
    backward-data), against the FP32 ALU peak; the FP64 oracle's gradient
    timed on the host over a bounded sample."""
    from oracle import nightmare as onm
    pk, _ = peaks()
    spec = synth.net_9conv()
    _, x, blob = synth.workload_net(spec, synth.SEED_9CONV, 1, side, side)
    st = torch.cuda.Stream()
    net = binding.Net(spec.layers, 3, prec="fp32", max_batch=1, max_side=side, stream=st.cuda_stream, device=dev)
    net.load_weights(blob)
    d_x = torch.from_numpy(x).cuda()
    for _ in range(2):
        net.nightmare_step(d_x, 1, side, side, layer, 0.01)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    l0 = net.launches()
    ev[0].record(st)
    for _ in range(reps):
        J = net.nightmare_step(d_x, 1, side, side, layer, 0.01)
    ev[1].record(st)
    torch.cuda.synchronize()
    launches = (net.launches() - l0) // reps
    ms = ev[0].elapsed_time(ev[1]) / reps
    net.close()
    flops, h = 0.0, side
    for l, ci in list(zip(spec.layers, spec.cins()))[:layer + 1]:
        flops += 2.0 * 2.0 * h * h * l.cout * ci * l.k * l.k
        if l.pool == synth.POOL_2X2S2:
            h //= 2
    tf = flops / (ms / 1e3) / 1e12
    peak = 152 * 128 * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    n, t0 = 0, time.perf_counter()
    while True:
        onm.input_grad(spec.layers, 3, x, blob, layer)
        n += 1
        el = time.perf_counter() - t0
        if el >= cpu_budget_s:
            break
    return {"network": "9-conv", "side": side, "layer": layer, "dtype": "f32", "ms_per_step": ms,
            "steps_per_s": 1e3 / ms, "gpu_launches_per_step": int(launches), "objective_last": float(J[0]),
            "roofline": {"bound": "alu", "achieved": tf, "peak": peak, "unit": "TFLOP/s", "frac": tf / peak,
                         "traffic": None, "kernel": "conv_simt_kernel (forward + backward-data)",
                         "flops_per_step": flops, "peak_source": "152 SMs x 128 FP32 lanes x 2 x max SM clock"},
            "cpu_baseline": {"steps_per_s": n / el, "kind": "oracle (FP64 gradient)", "cores": onm.oracle.threads(),
                             "sample": "%d gradient(s), %.1f s" % (n, el)}}


class Workload:
    """Frames, weights and step functions of one bench workload."""

    def __init__(self, torch, binding, dev, wl, prec, stream):
        self.name = wl
        netname, batch, side, _, seed = WORKLOADS[wl]
        self.spec = spec = synth.NETS[netname]()
        self.batch, self.side, self.prec = batch, side, prec
        if netname == "single-conv":
            self.sides = [side]
            _, x, self.blob = synth.workload_single()
            self.frames = [x]
        elif side:
            self.sides = [side] * batch
            _, x, self.blob = synth.workload_net(spec, seed, batch, side, side)
            self.frames = [x]
        else:
            self.sides = [int(v) for v in synth.uneven_sides(batch, seed)]
            self.blob = synth.weights_for(spec, seed)
            self.frames = [synth.frame_for(seed, i, s) for i, s in enumerate(self.sides)]
        self.net = binding.Net(spec.layers, spec.in_c, prec=prec, max_batch=batch if side else 1,
                               max_side=max(self.sides), stream=stream.cuda_stream, device=dev)
        self.net.load_weights(self.blob)
        self.stream = stream
        self.d_in = [torch.from_numpy(f).cuda() for f in self.frames]
        self.d_out, self.h_in, self.h_out = [], [], []
        for f in self.frames:
            c, ho, wo = self.net.output_shape(f.shape[2], f.shape[3])
            self.d_out.append(torch.empty((f.shape[0], c, ho, wo), device="cuda"))
            self.h_in.append(torch.from_numpy(f).pin_memory())
            self.h_out.append(torch.empty((f.shape[0], c, ho, wo)).pin_memory())
        if side:
            # a second pinned pair: the async host API alternates between two
            self.h_in.append(self.h_in[0].clone().pin_memory())
            self.h_out.append(torch.empty_like(self.h_out[0]).pin_memory())
        else:
            # uneven batches, end to end: two device slots, so that one step's
            # uploads and downloads (own streams) overlap another step's pass
            self.slots = [(self.d_in, self.d_out)]
            self.slots.append(([torch.empty_like(t) for t in self.d_in], [torch.empty_like(t) for t in self.d_out]))
            self.h_out2 = [[torch.empty_like(o).pin_memory() for o in self.h_out] for _ in range(2)]
            self.s_up, self.s_down = torch.cuda.Stream(), torch.cuda.Stream()
            self.ev_up = [torch.cuda.Event() for _ in range(2)]
            self.ev_comp = [torch.cuda.Event() for _ in range(2)]
            self.ev_free = [None, None]   # slot's download done (its device buffers reusable)
        self.h2d = sum(int(f.nbytes) for f in self.frames)
        self.d2h = sum(int(o.numel() * 4) for o in self.d_out)
        cins = spec.cins()
        self.flops_l = np.zeros(len(spec.layers))
        for sd in self.sides:
            h = sd
            for i, (l, ci) in enumerate(zip(spec.layers, cins)):
                self.flops_l[i] += 2.0 * h * h * l.cout * ci * l.k * l.k
                if l.pool == synth.POOL_2X2S2:
                    h //= 2

    def step(self):
        if self.side:
            self.net.forward_device(self.d_in[0], self.batch, self.side, self.side, self.d_out[0])
        else:
            self.net.forward_uneven(self.d_in, self.sides, self.d_out)

    def step_e2e(self, i=0):
        if self.side:
            # the host API, stream-ordered: one H2D of the batch, the pass, one
            # D2H of the result per call; two pinned buffer pairs alternate so
            # one call's copies overlap the previous call's pass
            self.net.forward_async(self.h_in[i % 2].numpy(), self.h_out[i % 2].numpy())
        else:
            import torch
            k = i % 2
            d_in, d_out = self.slots[k]
            with torch.cuda.stream(self.s_up):
                if self.ev_free[k] is not None:
                    self.s_up.wait_event(self.ev_free[k])
                for a, b in zip(d_in, self.h_in):
                    a.copy_(b, non_blocking=True)
                self.ev_up[k].record(self.s_up)
            self.stream.wait_event(self.ev_up[k])
            self.net.forward_uneven(d_in, self.sides, d_out)
            self.ev_comp[k].record(self.stream)
            with torch.cuda.stream(self.s_down):
                self.s_down.wait_event(self.ev_comp[k])
                for a, b in zip(self.h_out2[k], d_out):
                    a.copy_(b, non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(self.s_down)
                self.ev_free[k] = ev

    def e2e_done(self):
        if self.side:
            self.net.forward_wait()
        else:
            import torch
            torch.cuda.synchronize()


def run_trace(torch, binding, wl, args):
    """Phase timeline of one fixed-batch pass (net_trace): per tensor-core
    layer, from the CTAs' globaltimer stamps, in microseconds from the first
    conv launch's start.  dep: first producer past the wait for the previous
    kernel; fill: from there to the first K step ready; mainloop: first K
    step to the last MMA issued; tail: last MMA issued to the epilogue's end
    (the MMAs still in the tensor pipe, then the last tile's epilogue);
    straggle: last CTA's end minus the median CTA's end; gap: this layer's
    dep minus the previous layer's last CTA end."""
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    W = Workload(torch, binding, 0, wl, WORKLOADS[wl][3], stream)
    if not W.side:
        raise SystemExit("trace: fixed-batch workloads only")
    flush = torch.empty(L2_FLUSH_BYTES // 4, device="cuda")
    for _ in range(args.warmup):
        W.step()
    W.net.trace(True)
    for _ in range(2):   # the first traced pass captures a new graph
        flush.zero_()
        W.step()
    buf = W.net.trace_read().astype(np.int64)
    ran = [l for l in range(buf.shape[0]) if buf[l, :, 0].any()]
    t0 = min(int(buf[l, buf[l, :, 0] > 0, 0].min()) for l in ran)
    layers, prev_end = [], None
    for l in ran:
        has9 = bool((buf[l, buf[l, :, 0] > 0, 9] > 0).all())   # (the tap-pair first layer leaves it out)
        B = (buf[l, buf[l, :, 0] > 0] - t0) / 1000.0
        ep_end = np.maximum(B[:, 6], B[:, 7])
        r = {"layer": l, "ctas": int(B.shape[0]), "start": float(B[:, 0].min()),
             "prologue": float(np.median(B[:, 1] - B[:, 0])), "dep": float(B[:, 2].min()),
             "fill": float(np.median(B[:, 3] - B[:, 2])), "mainloop": float(np.median(B[:, 4] - B[:, 3])),
             "tail": float(np.median(ep_end - B[:, 4])), "end": float(B[:, 8].max()),
             # the tail split at warp 2's last accumulator ready: the last MMAs
             # in the tensor pipe, then that tile's epilogue
             "mma_drain": float(np.median(B[:, 9] - B[:, 4])) if has9 else None,
             "last_epilogue": float(np.median(ep_end - B[:, 9])) if has9 else None,
             "straggle": float(B[:, 8].max() - np.median(B[:, 8]))}
        r["dep_to_end"] = r["end"] - r["dep"]
        r["gap"] = None if prev_end is None else r["dep"] - prev_end
        prev_end = r["end"]
        layers.append({k: (round(v, 2) if isinstance(v, float) else v) for k, v in r.items()})
    W.net.trace(False)
    tot = lambda k: round(sum(x[k] for x in layers if x[k] is not None), 2)
    return {"workload": wl, "unit": "us", "layers": layers,
            "sums": {k: tot(k) for k in ("fill", "mainloop", "tail", "straggle", "gap", "dep_to_end")},
            "span": round(layers[-1]["end"] - layers[0]["start"], 2)}


def measure(torch, W, args, flush, barrier, ws, with_clocks=False, dev=0):
    """Warm-up, K device-timed steps (L2 flushed between them, outside the
    events), a second pass with per-layer conv events, and the e2e pass."""
    for _ in range(args.warmup):
        W.step()
    barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    l0 = W.net.launches()
    barrier()
    clk = Clocks(dev) if with_clocks else None
    if clk:
        clk.__enter__()
    w0 = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(W.stream)
        W.step()
        ev[i][1].record(W.stream)
    barrier()
    wall = time.perf_counter() - w0
    if clk:
        clk.__exit__(None, None, None)
    launches = W.net.launches() - l0
    total_ms = max_over_ranks(torch, sum(a.elapsed_time(b) for a, b in ev), ws)
    W.net.profile(True)
    for _ in range(2):
        W.step()
    torch.cuda.synchronize()
    layer_ms = np.zeros(len(W.spec.layers))
    for i in range(args.steps):
        flush.zero_()
        W.step()
        layer_ms += W.net.layer_times()
    layer_ms /= args.steps
    W.net.profile(False)
    for i in range(2):
        W.step_e2e(i)
    W.e2e_done()
    barrier()
    t0 = time.perf_counter()
    for i in range(args.steps):
        W.step_e2e(i)
    W.e2e_done()
    barrier()
    e2e_s = max_over_ranks(torch, time.perf_counter() - t0, ws)
    frames_all = W.batch * args.steps * ws
    return {"value": job_frames_per_s(W.batch * args.steps, ws, total_ms / 1e3), "ms_per_step": total_ms / args.steps,
            "conv_tflops": float(W.flops_l.sum()) * args.steps * ws / (total_ms / 1e3) / 1e12,
            "layer_ms": layer_ms, "launches": launches, "wall": wall, "clocks": clk.summary() if clk else None,
            "e2e_fps": frames_all / e2e_s}


def per_layer(W, layer_ms, precs):
    """Each layer's achieved TFLOP/s and, against its algorithmic bytes
    (input activation + post-pool output activation + weights, each moved
    once, in the layer's storage type; the first layer reads the FP32
    frames), achieved GB/s and the fraction of the measured HBM peak."""
    pk, _ = peaks()
    esz = {"fp32": 4, "bf16": 2, "fp8": 1}
    cins = W.spec.cins()
    nl = len(W.spec.layers)
    out = []
    for i, (l, ci) in enumerate(zip(W.spec.layers, cins)):
        byt = 0.0
        for sd in W.sides:
            h = sd
            for j in range(i):
                if W.spec.layers[j].pool == synth.POOL_2X2S2:
                    h //= 2
            ho = h // 2 if l.pool == synth.POOL_2X2S2 else h
            ein = 4 if i == 0 else esz[precs[i]]
            eout = 4 if i + 1 == nl else esz[precs[i + 1]]
            byt += h * h * ci * ein + ho * ho * l.cout * eout
        byt += l.cout * ci * l.k * l.k * esz[precs[i]]
        t = float(layer_ms[i]) / 1e3
        out.append({"layer": i, "k": l.k, "cin": ci, "cout": l.cout, "ms": round(float(layer_ms[i]), 5),
                    "tflops": round(float(W.flops_l[i]) / t / 1e12, 2),
                    "alg_mb": round(byt / 1e6, 2), "gbs": round(byt / t / 1e9, 1),
                    "hbm_frac": round(byt / t / 1e9 / pk["hbm_gbs"], 3)})
    return out


def roofline(W, ms_per_step, precs):
    """The dominant kernel family (tensor-core conv, or the CUDA-core conv of
    the FP32 path): all its layers' algorithmic FLOPs per pass over the whole
    measured step time (which also holds the frame pack and any split-K
    reductions, so this is a lower bound on the conv kernels' own rate),
    against the measured burst peak (the timed region is tens of ms of
    sub-ms passes) of each layer's operand type."""
    pk, pk_kind = peaks()
    tc = [i for i, p in enumerate(precs) if p != "fp32"]
    sel = tc if tc else list(range(len(precs)))
    flops = float(sum(W.flops_l[i] for i in sel))
    achieved = flops / (ms_per_step / 1e3) / 1e12
    if not tc:
        peak = 152 * 128 * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        bound, kern = "alu", "conv_simt_kernel"
        pnote = "152 SMs x 128 FP32 lanes x 2 x %.0f MHz" % pk.get("sm_max_mhz", 2070.0)
    else:
        # FLOP-weighted: the time each layer's FLOPs take at its own type's peak
        bf = pk["bf16_tflops"]
        t_peak = sum(W.flops_l[i] / (bf * (2.0 if precs[i] == "fp8" else 1.0)) for i in sel)
        peak = flops / t_peak
        bound, kern = "tensor", "conv_tc_kernel"
        nfp8 = sum(1 for i in sel if precs[i] == "fp8")
        pnote = "bf16 burst, %s" % pk_kind + ("; fp8 layers at bf16 x 2 (nominal ratio), FLOP-weighted" if nfp8 else "")
    tr = TRAFFIC.get(W.name, {}).get(kern)
    traffic = tr[0] if tr and tr[1] == kernel_sha16() else None
    return {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": traffic, "kernel": "%s (%d launches per pass)" % (kern, len(sel)),
            "time_basis": "ms_per_step (whole pass, pack and split-K reductions included)",
            "flops_per_pass": flops, "peak_source": pnote, "kernel_src_sha16": kernel_sha16()}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT, choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true", help="skip the other-precision runs")
    ap.add_argument("--cpu-budget-s", type=float, default=12.0)
    ap.add_argument("--no-serve", action="store_true", help="leave the serving streams out of the line")
    ap.add_argument("--serve-seconds", type=float, default=3.0)
    ap.add_argument("--no-configs", action="store_true",
                    help="leave the other configurations (single conv, 9-conv b1 FP32/BF16, uneven 64) out")
    ap.add_argument("--no-extra", action="store_true",
                    help="leave the detection, nightmare and Jacobi measurements out of the line")
    ap.add_argument("--section", choices=["detect", "jacobi", "nightmare", "trace"],
                    help="run only this measurement and print its JSON (profiling entry point)")
    ap.add_argument("--no-tile-search", action="store_true",
                    help="keep the analytic tile plan (skip the genetic tile-plan search)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    wl = args.workload
    if args.impl == "reference":
        return run_reference(args, wl)

    import torch
    if args.section:
        from paper_1811_03882_gb300 import build, binding
        build.build()
        torch.cuda.set_device(0)
        if args.section == "trace":
            print(json.dumps({"section": "trace", **run_trace(torch, binding, wl, args)}), flush=True)
            return
        fn = {"detect": run_detect, "jacobi": run_jacobi, "nightmare": run_nightmare}[args.section]
        print(json.dumps({"section": args.section, **fn(torch, binding, 0)}), flush=True)
        return
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()

    from paper_1811_03882_gb300 import build, binding
    build.build()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    flush = torch.empty(L2_FLUSH_BYTES // 4, device="cuda")

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    netname, batch, side, prec, seed = WORKLOADS[wl]

    def setup(p, tune=False, wl=wl):
        _, batch, side, _, _ = WORKLOADS[wl]
        W = Workload(torch, binding, dev, wl, p, stream)
        info = {}
        if p == "fp8":
            cs = max(W.sides) if side else 416
            xc = synth.make_frames(synth.Stream(synth.SEED_CALIB), 1, 3, cs, cs)
            d_c = torch.from_numpy(xc).cuda()
            W.net.calibrate(d_c, 1, cs, cs)
            if tune:
                plan, ga = W.net.tune_precision(d_c, 1, cs, cs, max_err=0.05, population=12, generations=8,
                                                reps=2, seed=3)
                info = {"plan": plan, "ga": ga}
        if tune and not side and p != "fp32" and not args.no_tile_search:
            # uneven batch: the genetic search over its grouped launches (setup)
            plan, tr = W.net.tune_uneven(W.d_in, W.sides, W.d_out, population=12, generations=8, reps=3,
                                         seed=5)
            info["grouped_plan"] = plan
            info["tile_search"] = tr
        if tune and side and p != "fp32" and not args.no_tile_search:
            # the genetic tile-plan search on the workload's own batch shape
            # (setup, outside every timed region)
            tiles, tr = W.net.tune_tiles(W.d_in[0], batch, side, side, population=12, generations=8, reps=3,
                                         seed=5)
            info["tile_plan"] = tiles
            info["tile_search"] = tr
        if side and p != "fp32":
            info["cta_plan"] = W.net.plan_ctas(batch, side, side)
        return W, info

    W, info = setup(prec, tune=True)
    precs = W.net.layer_prec()
    m = measure(torch, W, args, flush, barrier, ws, with_clocks=True, dev=dev)
    roof = roofline(W, m["ms_per_step"], precs)
    line = {
        "metric": "frames/s", "value": m["value"], "unit": "frames/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": m["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "bf16": "bf16", "fp8": "e4m3"}[prec], "data": "synthetic",
        "config": workload_config(wl, ws),
        "layer_precision": precs,
        "conv_tflops": m["conv_tflops"],
        "roofline": roof,
        "layer_ms": [round(float(t), 5) for t in m["layer_ms"]],
        "layer_ms_basis": "CUDA events around each layer in a second pass; the events serialise "
                          "programmatic launch, so their sum exceeds ms_per_step",
        "layers": per_layer(W, m["layer_ms"], precs),
        "e2e": {"value": m["e2e_fps"], "unit": "frames/s", "h2d_bytes_per_step": W.h2d, "d2h_bytes_per_step": W.d2h},
        "gpu_launches": int(m["launches"]),
        "wall_s_timed": m["wall"],
        "clocks": m["clocks"],
    }
    if "plan" in info:
        line["precision_search"] = {"plan": info["plan"], "ga": info["ga"]}
    if "tile_plan" in info:
        # [N tile, split-K] per layer ([0, 0]: CUDA cores), from the genetic search
        line["tile_plan"] = info["tile_plan"]
        line["tile_search"] = info["tile_search"]
    if "grouped_plan" in info:
        # [N tile, CTAs per SM, stage cap] per layer of the grouped launches (0: analytic)
        line["grouped_plan"] = info["grouped_plan"]
        line["tile_search"] = info["tile_search"]
    if "cta_plan" in info:
        line["cta_plan"] = info["cta_plan"]   # CTAs per SM of each tensor-core layer
    W.net.close()
    if not args.no_compare and side:
        # the same workload on the other paths: FP32 (CUDA cores) and FP8 (GA-tuned plan) or BF16
        cmp = {}
        for p in ("fp32", "fp8" if prec != "fp8" else "bf16"):
            W2, info2 = setup(p, tune=(p == "fp8"))
            m2 = measure(torch, W2, args, flush, barrier, ws)
            cmp[p] = {"value": m2["value"], "ms_per_step": m2["ms_per_step"], "conv_tflops": m2["conv_tflops"],
                      "e2e": m2["e2e_fps"], "roofline_frac": roofline(W2, m2["ms_per_step"], W2.net.layer_prec())["frac"],
                      "layer_precision": W2.net.layer_prec()}
            if "plan" in info2:
                cmp[p]["precision_search"] = {"plan": info2["plan"], "ga": info2["ga"]}
            if "tile_plan" in info2:
                cmp[p]["tile_plan"] = info2["tile_plan"]
                cmp[p]["tile_search"] = info2["tile_search"]
            W2.net.close()
        line["compare"] = cmp
    if not args.no_configs and rank == 0:
        # the other configurations of the workload set, each on its own
        # network and batch shape (shorter runs: 20 timed steps)
        oc = {}
        sub = argparse.Namespace(**vars(args))
        sub.steps = min(args.steps, 20)
        for owl in OTHER_CONFIGS:
            if owl == wl:
                continue
            p = WORKLOADS[owl][3]
            W2, info2 = setup(p, tune=True, wl=owl)
            m2 = measure(torch, W2, sub, flush, barrier, 1)
            r2 = roofline(W2, m2["ms_per_step"], W2.net.layer_prec())
            oc[owl] = {"value": m2["value"], "unit": "calls/s" if WORKLOADS[owl][0] == "single-conv" else "frames/s",
                       "ms_per_step": m2["ms_per_step"], "frames_per_step": W2.batch,
                       "e2e": m2["e2e_fps"], "conv_tflops": m2["conv_tflops"],
                       "roofline": {"bound": r2["bound"], "achieved": r2["achieved"], "peak": r2["peak"],
                                    "unit": r2["unit"], "frac": r2["frac"]},
                       "gpu_launches_per_step": m2["launches"] / sub.steps, "steps": sub.steps,
                       "layer_precision": W2.net.layer_prec()}
            for k in ("tile_plan", "grouped_plan", "tile_search", "cta_plan"):
                if k in info2:
                    oc[owl][k] = info2[k]
            W2.net.close()
        line["other_configs"] = oc
    if not args.no_serve and rank == 0:
        line["serving"] = run_serving(args, torch, binding, dev)
    if not args.no_extra and rank == 0:
        line["detect"] = run_detect(torch, binding, dev)
        line["jacobi"] = run_jacobi(torch, binding, dev)
        line["nightmare"] = run_nightmare(torch, binding, dev)
    if rank == 0 and not args.no_cpu_baseline:
        f0 = W.frames[0][:1]
        fps, nfr, el, cores = oracle_frames_per_s(W.spec, f0, W.blob, args.cpu_budget_s)
        fps1, nfr1, el1, _ = oracle_frames_per_s(W.spec, f0, W.blob, 1.0, threads=1)
        line["cpu_baseline"] = {"value": fps, "unit": "frames/s", "cores": cores, "kind": "oracle",
                                "sample": "%d frame(s) of %dx%d, %.1f s" % (nfr, f0.shape[2], f0.shape[3], el),
                                "cpu_model": cpu_model(), "nproc": os.cpu_count(),
                                "single_thread": {"value": fps1, "unit": "frames/s",
                                                  "sample": "%d frame(s), %.1f s" % (nfr1, el1)}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
