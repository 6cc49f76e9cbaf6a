"""Throughput benchmark of the device-resident CNN forward pass.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                [--workload NAME] [--no-cpu-baseline]

One step = one forward pass of the whole network over one batch of
synthetic frames that are already resident in device memory (value), and
the same through the host API net_forward with pinned host buffers, the
H2D and D2H copies inside the timed region (e2e).  Under torchrun every
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
    "19conv-448-b8-bf16": ("19-conv", 8, 448, "bf16", synth.SEED_19CONV),
    "19conv-448-b8-fp8": ("19-conv", 8, 448, "fp8", synth.SEED_19CONV),
    "9conv-416-b1-fp32": ("9-conv", 1, 416, "fp32", synth.SEED_9CONV),
    "9conv-416-b1-bf16": ("9-conv", 1, 416, "bf16", synth.SEED_9CONV),
    # 64 frames, sides drawn from {320, 416, 512, 608}, one grouped launch per layer
    "uneven64-9conv-bf16": ("9-conv", 64, 0, "bf16", synth.SEED_UNEVEN),
}
DEFAULT = "9conv-416-b1-fp32"

# ncu DRAM traffic per launch of the dominant kernel (read + write bytes),
# from the capture summarised under profiles/; None until captured.
TRAFFIC = {}

L2_FLUSH_BYTES = 256 << 20   # > 129 MB L2


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


def oracle_frames_per_s(spec, x1, blob, budget_s: float):
    """FP64 oracle timed on this host's cores over whole frames until
    budget_s of CPU work has passed (at least one frame)."""
    import oracle
    oracle.build()
    n, t0 = 0, time.perf_counter()
    while True:
        oracle.forward(spec.layers, spec.in_c, x1, blob)
        n += 1
        el = time.perf_counter() - t0
        if el >= budget_s:
            break
    return n / el, n, el, oracle.threads()


def run_reference(args, wl):
    """The oracle as the reference arm: each step is one frame of the
    workload through the FP64 CPU forward pass."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    netname, batch, side, prec, seed = WORKLOADS[wl]
    spec = synth.NETS[netname]()
    if side:
        _, x, blob = synth.workload_net(spec, seed, 1, side, side)
        frames = [x] * args.steps
    else:
        blob = synth.weights_for(spec, seed)
        sides = synth.uneven_sides(batch, seed)
        frames = [synth.frame_for(seed, i % batch, int(sides[i % batch])) for i in range(args.steps)]
    import oracle
    oracle.build()
    oracle.forward(spec.layers, 3, frames[0], blob)   # warm-up (one frame)
    t0 = time.perf_counter()
    for f in frames:
        oracle.forward(spec.layers, 3, f, blob)
    el = time.perf_counter() - t0
    fps = args.steps / el
    line = {"impl": "reference", "metric": "frames/s", "value": fps, "unit": "frames/s",
            "n_gpus": 0, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": wl, "frames_per_step": 1, "side": side or "uneven", "network": netname},
            "cpu_baseline": {"value": fps, "unit": "frames/s", "cores": oracle.threads(),
                             "kind": "oracle", "sample": "%d frames (side %s)" % (args.steps, side or "uneven")},
            "e2e": {"value": fps, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT, choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget-s", type=float, default=12.0)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    wl = args.workload
    if args.impl == "reference":
        return run_reference(args, wl)

    import torch
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

    netname, batch, side, prec, seed = WORKLOADS[wl]
    spec = synth.NETS[netname]()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    if side:
        sides = [side] * batch
        _, x, blob = synth.workload_net(spec, seed, batch, side, side)
        frames = [x]
    else:
        # uneven batch: frame i has its own side and its own random stream
        sides = [int(v) for v in synth.uneven_sides(batch, seed)]
        blob = synth.weights_for(spec, seed)
        frames = [synth.frame_for(seed, i, s) for i, s in enumerate(sides)]
    net = binding.Net(spec.layers, 3, prec=prec, max_batch=batch if side else 1,
                      max_side=max(sides), stream=stream.cuda_stream, device=dev)
    net.load_weights(blob)
    if prec == "fp8":
        s = synth.Stream(synth.SEED_CALIB)
        cs = max(sides)
        xc = synth.make_frames(s, 2, 3, cs, cs)
        net.calibrate(torch.from_numpy(xc).cuda(), 2, cs, cs)
    d_in = [torch.from_numpy(f).cuda() for f in frames]
    d_out, h_in, h_out = [], [], []
    for f in frames:
        c, ho, wo = net.output_shape(f.shape[2], f.shape[3])
        d_out.append(torch.empty((f.shape[0], c, ho, wo), device="cuda"))
        h_in.append(torch.from_numpy(f).pin_memory())
        h_out.append(torch.empty((f.shape[0], c, ho, wo)).pin_memory())

    def step():
        if side:
            net.forward_device(d_in[0], batch, side, side, d_out[0])
        else:
            net.forward_uneven(d_in, sides, d_out)

    def step_e2e():
        if side:
            # the host API: one H2D of the batch, the pass, one D2H of the result
            net.forward(h_in[0].numpy(), h_out[0].numpy())
        else:
            for a, b in zip(d_in, h_in):
                a.copy_(b, non_blocking=True)
            net.forward_uneven(d_in, sides, d_out)
            for a, b in zip(h_out, d_out):
                a.copy_(b, non_blocking=True)
            stream.synchronize()

    flush = torch.empty(L2_FLUSH_BYTES // 4, device="cuda")

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    barrier()

    # ---- timed region: K steps, L2 flushed between steps (outside events)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    l0 = net.launches()
    barrier()
    with Clocks(dev) as clk:
        w0 = time.perf_counter()
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
        barrier()
        wall = time.perf_counter() - w0
    launches = net.launches() - l0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    if ws > 1:
        t = torch.tensor([total_ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    frames_all = batch * args.steps * ws
    value = frames_all / (total_ms / 1e3)

    # ---- per-layer conv-kernel times (second pass, events around each conv)
    net.profile(True)
    for _ in range(2):
        step()
    torch.cuda.synchronize()
    layer_ms = np.zeros(len(spec.layers))
    for i in range(args.steps):
        flush.zero_()
        step()
        layer_ms += net.layer_times()
    layer_ms /= args.steps
    net.profile(False)

    # ---- end to end through the host API (pinned host buffers)
    for _ in range(2):
        step_e2e()
    barrier()
    t0 = time.perf_counter()
    for i in range(args.steps):
        step_e2e()
    barrier()
    e2e_s = time.perf_counter() - t0
    if ws > 1:
        t = torch.tensor([e2e_s], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_s = float(t.item())
    h2d = sum(int(f.nbytes) for f in frames)
    d2h = sum(int(o.numel() * 4) for o in d_out)

    # ---- roofline of the dominant kernel (conv, by engine)
    pk, pk_kind = peaks()
    cins = spec.cins()
    flops_l = np.zeros(len(spec.layers))
    for sd, f in zip(sides, [1] * len(sides)):
        h = sd
        for i, (l, ci) in enumerate(zip(spec.layers, cins)):
            flops_l[i] += 2.0 * f * h * h * l.cout * ci * l.k * l.k
            if l.pool == synth.POOL_2X2S2:
                h //= 2
    engines = ["bf16" if (prec == "fp8" and ci < 16) else prec for ci in cins]
    dom = max(set(engines), key=lambda e: sum(t for t, en in zip(layer_ms, engines) if en == e))
    sel = [i for i, en in enumerate(engines) if en == dom]
    dom_flops = sum(flops_l[i] for i in sel)
    dom_ms = sum(layer_ms[i] for i in sel)
    achieved = dom_flops / (dom_ms / 1e3) / 1e12
    if dom == "fp32":
        peak = 152 * 128 * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        bound, pnote = "alu", "152 SMs x 128 FP32 lanes x 2 x %.0f MHz" % pk.get("sm_max_mhz", 2070.0)
    else:
        peak = pk.get("bf16_tflops_sustained", pk["bf16_tflops"]) * (2.0 if dom == "fp8" else 1.0)
        bound = "tensor"
        pnote = ("bf16 sustained of %s" % pk_kind) + (" x 2 (fp8/bf16 nominal ratio)" if dom == "fp8" else "")
    tr = TRAFFIC.get(wl)
    roof = {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": tr,
            "kernel": "conv_%s (%d layers)" % ("simt" if dom == "fp32" else "tc_" + dom, len(sel)),
            "peak_source": pnote, "launches_per_step": len(sel)}

    conv_flops = float(sum(flops_l))
    line = {
        "metric": "frames/s", "value": value, "unit": "frames/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "bf16": "bf16", "fp8": "e4m3"}[prec], "data": "synthetic",
        "config": {"workload": wl, "network": netname, "global_batch": batch * ws,
                   "frames_per_step_per_gpu": batch, "side": side if side else "uneven {320,416,512,608}",
                   "precision": prec,
                   "parallelism": "replicas%d" % ws, "l2": "flushed between steps (256 MB write)"},
        "conv_tflops": conv_flops * args.steps * ws / (total_ms / 1e3) / 1e12,
        "roofline": roof,
        "layer_ms": [round(float(t), 5) for t in layer_ms],
        "e2e": {"value": frames_all / e2e_s, "unit": "frames/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "wall_s_timed": wall,
        "clocks": clk.summary(),
    }
    if rank == 0 and not args.no_cpu_baseline:
        f0 = frames[0][:1]
        fps, nfr, el, cores = oracle_frames_per_s(spec, f0, blob, args.cpu_budget_s)
        line["cpu_baseline"] = {"value": fps, "unit": "frames/s", "cores": cores, "kind": "oracle",
                                "sample": "%d frame(s) of %dx%d, %.1f s" % (nfr, f0.shape[2], f0.shape[3], el)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    net.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
