"""Benchmark of the lens-transport hot path on GB300.

Workload (the one the headline metric is quoted on): the seeded 6-element
double-Gauss-like 11-surface lens, 4,194,304 entrance rays (uniform disk of
radius 1.2 a_1, +-10 deg, lambda uniform 380-780 nm).  One step = one pass
of the per-batch hot path over that batch: the FP32 map query of the
transmission-path map (lattice 32^4 x 8, fitted from 16,777,216 traced rays;
valid/occluded mask + multilinear table + exact-tracer fallback near mask
boundaries) and, beside it, the brute-force FP32 trace of the same rays.
`value` is map-query rays/s; the trace's rays/s is reported next to it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 runs under torchrun: every rank runs an independent replica on its own
GPU over its own batch (rays are independent; no collective on the data
path), timed between barriers, max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "rays/s map query vs FP32 trace at ≤1e-4 mm error; % roofline; p99 batch latency"
WORKLOAD = ("11-surface seeded double-Gauss-like lens (6 elements, stop after surface 6), "
            "4,194,304 rays (disk r=1.2*a1, +-10 deg, lambda U[380,780] nm), transmission path; "
            "map 32^4x8 fitted from 16,777,216 traced rays, FP32 query with tracer fallback")

# ncu DRAM traffic per ray of each kernel (dram__bytes_read.sum + dram__bytes_write.sum
# of one launch / rays in it), keyed by kernel, with the hash of the sources it was
# measured on.  A kernel whose sources changed since reports traffic = null.
NCU_TRAFFIC = {}


def src_hash(files):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


TRACE_SRCS = ["paper_2605_04017_gb300/csrc/trace.cu", "paper_2605_04017_gb300/csrc/tracer.cuh",
              "paper_2605_04017_gb300/csrc/lt_internal.h"]


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": d["hbm_gbs"], "src": "measured", "sm_max_mhz": d.get("sm_max_mhz", 2070.0)}
    return {"hbm_gbs": 6800.0, "src": "fallback", "sm_max_mhz": 2070.0}


# FP32 non-tensor peak: 152 SMs x 128 FP32 lanes x 2 flop per FMA x max SM clock.
def fp32_peak_tflops(sm_mhz):
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


class ClockSampler:
    """nvidia-smi sampling during the timed region (200 ms period)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_accept(p):
    import oracle
    try:
        e, b = oracle.Lens(p).paraxial(587.6)
        return e > 0 and b > 0
    except ValueError:
        return False


def lib_accept(p):
    from paper_2605_04017_gb300 import lt
    try:
        lt.Lens(p)
        return True
    except lt.LTError:
        return False


def timed_steps(step, steps, warmup, flush, stream):
    """Per-step CUDA-event times (ms) on `stream`, L2 flushed before every step."""
    import torch
    for _ in range(warmup):
        flush()
        step()
    torch.cuda.synchronize()
    times = []
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    for a, b in evs:
        flush()
        a.record(stream)
        step()
        b.record(stream)
    torch.cuda.synchronize()
    for a, b in evs:
        times.append(a.elapsed_time(b))
    return times


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2605_04017_gb300 import batch, lt, workloads as w

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()

    presc = w.eleven_surface_lens(lib_accept)
    lens = lt.Lens(presc)
    n = w.ELEVEN_N
    rays = w.entrance_rays(n, w.SEED_BASE + 2 + 7919 * rank, w.eleven_rho(presc))
    d = batch.DeviceRays(rays)
    o = batch.DeviceOut(n)
    flush_buf = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    def flush():
        flush_buf.fill_(rank + 1)

    def trace_step():
        lt.trace(lens, d.inp, d.lam, 0, o.out, n, stream)

    # warm-up + timed trace arm
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    t_trace = timed_steps(trace_step, args.steps, args.warmup, flush, stream)
    clocks = sampler.stop()
    if world > 1:
        dist.barrier()

    ms_trace = statistics.mean(t_trace)
    total_ms = sum(t_trace)
    tt = torch.tensor([total_ms], device="cuda")
    if world > 1:
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    total_ms = float(tt.item())
    value = world * n * args.steps / (total_ms * 1e-3)

    # end-to-end through the host-buffer entry point (pinned host memory)
    h = batch.HostRays(rays)
    for _ in range(2):
        lt.trace_host(lens, h.inp[:5], h.inp[5], 0, h.out + [h.flags], n)
    e2e_steps = max(3, args.steps // 4)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        lt.trace_host(lens, h.inp[:5], h.inp[5], 0, h.out + [h.flags], n)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e_rays_s = n / e2e_s

    peaks = load_peaks()
    bytes_per_ray = 6 * 4 + 6 * 4 + 1
    achieved_gbs = n * bytes_per_ray / (ms_trace * 1e-3) / 1e9
    th = src_hash(TRACE_SRCS)
    tr = NCU_TRAFFIC.get("trace_kernel")
    traffic = tr["bytes_per_ray"] * n if tr and tr["hash"] == th else None
    roofline = {"kernel": "trace_kernel", "bound": "hbm", "achieved": round(achieved_gbs, 1),
                "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": round(achieved_gbs / peaks["hbm_gbs"], 4), "traffic": traffic,
                "peak_src": peaks["src"],
                "algorithmic_bytes_per_ray": bytes_per_ray}

    line = {
        "metric": METRIC, "value": round(value, 1), "unit": "rays/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_trace, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "rays_per_gpu": n, "l2": "flushed (256 MB write) before every step",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "trace": {"rays_per_s": round(value, 1), "ms": round(ms_trace, 4)},
        "roofline": roofline,
        "e2e": {"value": round(e2e_rays_s, 1), "unit": "rays/s",
                "h2d_bytes_per_step": n * 24, "d2h_bytes_per_step": n * 25},
        "gpu_launches": args.steps,
        "clocks": clocks,
    }
    if rank == 0 and not args.skip_cpu:
        line["cpu_baseline"] = cpu_baseline(presc, rays)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def cpu_baseline(presc, rays, budget_s=12.0):
    """The FP64 oracle, as it stands, single-threaded on a bounded sample."""
    import oracle
    ol = oracle.Lens(presc)
    m = 1 << 16
    sample = rays.subset(slice(0, m))
    t0 = time.perf_counter()
    reps = 0
    while True:
        ol.trace(sample)
        reps += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": round(reps * m / dt, 1), "unit": "rays/s", "cores": 1, "kind": "oracle",
            "sample": f"{m} rays of the same workload traced {reps} times (transmission path)"}


def run_reference(args):
    """The oracle arm: the FP64 CPU oracle as it stands, on host cores, same
    workload, metric and unit; each step a bounded sample."""
    import numpy as np
    from paper_2605_04017_gb300 import workloads as w

    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    presc = w.eleven_surface_lens(oracle_accept)
    rays = w.eleven_rays(presc, 1 << 15)
    ol = oracle.Lens(presc)
    for _ in range(args.warmup):
        ol.trace(rays)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ol.trace(rays)
    dt = time.perf_counter() - t0
    value = args.steps * len(rays) / dt
    line = {"metric": METRIC, "value": round(value, 1), "unit": "rays/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "rays_per_step": len(rays)}, "impl": "reference",
            "cpu_baseline": {"value": round(value, 1), "unit": "rays/s", "cores": 1,
                             "kind": "oracle",
                             "sample": f"{len(rays)} rays of the same workload per step"},
            "e2e": {"value": round(value, 1), "unit": "rays/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--skip-cpu", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
