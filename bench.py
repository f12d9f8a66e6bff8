"""Benchmark of the lens-transport hot path on GB300.

Workload (the one the headline metric is quoted on): the seeded 6-element
double-Gauss-like 11-surface lens, 4,194,304 entrance rays (uniform disk of
radius 1.2 a_1, +-10 deg, lambda uniform 380-780 nm), transmission path.
Set-up (untimed, reported): the polynomial-patch map -- degree-4 patch
polynomials over the symmetry-reduced input (r, rotated slopes, 1/lambda^2)
fitted to traced rays of the unclipped lens, a 128 x 128 x 64 x 8 validity
mask, every cell certified at 1e-4 mm against its corners and 16,777,216
traced fit rays.  One step = the FP32 map query of the whole batch: mask
lookup, patch polynomial on VALID cells, the exact tracer on BOUNDARY cells.
`value` is map-query rays/s; the brute-force FP32 trace of the same rays is
timed the same way ("trace"), and so is the 32^4 x 8 multilinear table map
with its 16-bit node table ("table_map", which misses the 1e-4 mm bound).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 runs under torchrun: each rank is an independent replica on its own GPU
with its own batch (rays are independent; there is no collective on the data
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
            "polynomial-patch map (degree 4, 4x4x2x1 patches over (r, p, q, w=1/lambda^2), "
            "128x128x64x8 mask cells) certified at 1e-4 mm against 16,777,216 traced rays; "
            "FP32 query with tracer fallback")
RES = [32, 32, 32, 32, 8]          # the multilinear table map reported beside it
SMAX = math.tan(math.radians(10.0)) * math.sqrt(2.0)   # slope bound of the +-10 deg rays
POLY = {"degree": 4, "patches": [4, 4, 2, 1], "cells": [32, 32, 32, 8], "samples": 6,
        "max_residual_mm": 1e-4}

# FP32 operations of one ray-surface interaction of the tracer (intersection,
# aperture test, normal, Snell/mirror, Fresnel, renormalisation), counting an
# FMA as 2; the output plane and stop tests are folded into the same unit.
FLOPS_PER_INTERACTION = 89

# Sources a kernel's code comes from: the file that holds it and the headers
# it includes.
_CSRC = "paper_2605_04017_gb300/csrc/"
_HDRS = [_CSRC + f for f in ("lt_internal.h", "map_internal.h", "rays.cuh", "tracer.cuh", "profile.h")] + \
    ["include/lt.h"]
POLY_SRCS = [_CSRC + "poly.cu"] + _HDRS
MAP_SRCS = [_CSRC + "map.cu"] + _HDRS

# ncu DRAM traffic per ray of each kernel (dram__bytes_read.sum +
# dram__bytes_write.sum of one launch / rays in it) with the hash of the
# kernel's sources it was measured on; stale hashes report traffic = null.
NCU_TRAFFIC = {
    # ncu --metrics gpu__time_duration.sum,dram__bytes_read.sum,dram__bytes_write.sum,
    # one launch of each kernel of the polynomial-patch query of the headline's
    # 4,194,304 rays: 102,805,760 + 7,710,464 bytes (sort) and 46,535,680 +
    # 53,677,824 bytes (evaluation and the queue's trace)
    "poly_sort_kernel": {"bytes_per_ray": 110516224 / 4194304, "srcs": POLY_SRCS, "hash": "a98669c5dc0a7af3"},
    "poly_eval_kernel": {"bytes_per_ray": 100213504 / 4194304, "srcs": POLY_SRCS, "hash": "a98669c5dc0a7af3"},
    # the same metrics, one launch of the 16-bit table's classify-and-gather
    # kernel on the same rays: 134,202,368 + 88,067,584 bytes
    "map_query_kernel": {"bytes_per_ray": 222269952 / 4194304, "srcs": MAP_SRCS, "hash": "27a803adcc21d91c"},
}


def src_hash(files):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": float(d["hbm_gbs"]), "src": "measured",
                "sm_max_mhz": float(d.get("sm_max_mhz", 2070.0))}
    return {"hbm_gbs": 6800.0, "src": "fallback", "sm_max_mhz": 2070.0}


def fp32_peak_tflops(sm_mhz):
    """Non-tensor FP32 peak: 152 SMs x 128 FP32 lanes x 2 flop (FMA) x SM clock."""
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons (200 ms period)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,utilization.gpu")

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
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, util, reasons = [], [], [], set()
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
            try:
                util.append(float(parts[9]))
            except (IndexError, ValueError):
                pass
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm),
                "gpu_util_pct_mean": round(statistics.mean(util), 1) if util else None}


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


def build_poly(lt, lens, rho, fit=None, cfg=POLY, path_id=0):
    """The polynomial-patch map of the workload's box (r <= rho, |slopes| <= SMAX)."""
    return lt.Map.build_poly(lens, path_id, rho, SMAX, cfg["degree"], cfg["patches"], cfg["cells"],
                             cfg["samples"], fit=fit, max_residual_mm=cfg["max_residual_mm"])


def map_error(qout, qflags, tout, tflags, lt):
    """A map query's answers against the FP32 trace of the same rays: over the
    rays the map interpolated, the largest per-component and Euclidean exit
    position errors (mm), their p99 and RMS, the direction and throughput
    errors, and the validity agreement over all rays."""
    import numpy as np
    interp = ((qflags & lt.FLAG_VALID) != 0) & ((qflags & lt.FLAG_TRACED) == 0)
    tv = (tflags & lt.FLAG_VALID) != 0
    both = interp & tv
    mism = ((qflags & lt.FLAG_VALID) != 0) != tv
    rep = {"rays_interpolated": int(interp.sum()), "interpolated_but_trace_invalid": int((interp & ~tv).sum()),
           "validity_mismatches": int(mism.sum()),
           "validity_mismatches_near_edge": int((mism & ((tflags & lt.FLAG_NEAR_EDGE) != 0)).sum()),
           "valid_agreement": round(float(1.0 - mism.mean()), 8)}
    if both.any():
        d = qout[both].astype(np.float64) - tout[both]
        comp = np.abs(d[:, :2]).max(axis=1)
        eu = np.hypot(d[:, 0], d[:, 1])
        rep.update(pos_max_mm=float(comp.max()), pos_p99_mm=float(np.percentile(comp, 99)),
                   pos_euclid_max_mm=float(eu.max()), pos_rms_mm=float(np.sqrt((eu ** 2).mean())),
                   dir_max=float(np.abs(d[:, 2:5]).max()), I_max=float(np.abs(d[:, 5]).max()))
    return rep


def map_box(rho):
    sm = math.tan(math.radians(10.0))
    return [-rho, -rho, -sm, -sm, 380.0], [rho, rho, sm, sm, 780.0]


def timed_steps(step, steps, warmup, flush, stream, on_timed_start=None):
    """Per-step device times (ms) from CUDA events on `stream`; L2 flushed
    (256 MB write) before every step, outside the events."""
    import torch
    for _ in range(warmup):
        flush()
        step()
    torch.cuda.synchronize()
    if on_timed_start:
        on_timed_start()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    for a, b in evs:
        flush()
        a.record(stream)
        step()
        b.record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def combine_ranks(step_ms, world, n, steps, dist=None, device="cpu"):
    """Whole-job numbers of the replicas: for each timed arm (a list of per-step
    ms), the maximum over ranks of its summed time, and the aggregate rays/s
    world * n * steps / that time (every rank processed n rays per step)."""
    import torch
    tt = torch.tensor([sum(x) for x in step_ms], device=device, dtype=torch.float64)
    if world > 1:
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    totals = [float(v) for v in tt.cpu()]
    return totals, [world * n * steps / (t * 1e-3) for t in totals]


def kernel_roofline(name, prof, peaks, steps, units_bytes=None, flops_per_work=None):
    """Roofline of one kernel over the timed steps: `units_bytes` (or the
    counted work x flops_per_work) of one step over the kernel's summed
    CUDA-event time per step (a step may launch it several times)."""
    launches, ms, work = prof[name]
    step_s = ms / steps * 1e-3
    base = {"kernel": name, "launches_per_step": round(launches / steps, 2),
            "kernel_ms_per_step": round(ms / steps, 5)}
    if units_bytes is not None:
        ach = units_bytes / step_s / 1e9
        return {**base, "bound": "hbm", "achieved": round(ach, 1),
                "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": round(ach / peaks["hbm_gbs"], 4),
                "peak_src": peaks["src"] + " (hbm_gbs, burst copy)",
                "algorithmic_bytes_per_step": int(units_bytes)}
    flops = work / steps * flops_per_work
    ach = flops / step_s / 1e12
    peak = fp32_peak_tflops(peaks["sm_max_mhz"])
    return {**base, "bound": "alu", "achieved": round(ach, 2), "peak": round(peak, 1),
            "unit": "TFLOP/s", "frac": round(ach / peak, 4),
            "peak_src": "derived: 152 SMs x 128 FP32 lanes x 2 x %.0f MHz" % peaks["sm_max_mhz"],
            "interactions_per_step": int(work / steps), "flops_per_interaction": flops_per_work}


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
    rho = w.eleven_rho(presc)
    n = args.rays or w.ELEVEN_N
    # each rank draws its own batch (weak scaling); rank 0 uses the standard seed
    rays = w.entrance_rays(n, w.SEED_BASE + 2 + 7919 * rank, rho)
    fit = batch.DeviceRays(w.eleven_fit_rays(presc))
    lo, hi = map_box(rho)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pmap = build_poly(lt, lens, rho, fit)
    pbuild_s = time.perf_counter() - t0
    pstats, ppoly = pmap.stats(), pmap.poly_stats()
    t0 = time.perf_counter()
    gmap = lt.Map.build(lens, 0, RES, lo, hi, fit=fit, node_format=lt.NODE_S16)
    build_s = time.perf_counter() - t0
    mstats = gmap.stats()
    del fit
    torch.cuda.empty_cache()

    d = batch.DeviceRays(rays)
    o = batch.DeviceOut(n)
    flush_buf = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    def flush():
        flush_buf.fill_(rank + 1)

    def query_step():
        pmap.query(d.inp, d.lam, o.out, n, lt.QUERY_TABLE, stream)

    def table_step():
        gmap.query(d.inp, d.lam, o.out, n, lt.QUERY_TABLE, stream)

    def trace_step():
        lt.trace(lens, d.inp, d.lam, 0, o.out, n, stream)

    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    # the steps are timed twice: once as they run (the headline numbers), and
    # once with the library's per-kernel CUDA events on (their records add
    # about 3 us per kernel boundary) for the kernels' durations and work
    reset = lambda: lt.profile_read(reset=True)  # noqa: E731
    lt.profile_enable(False)
    t_query = timed_steps(query_step, args.steps, args.warmup, flush, stream)
    t_trace = timed_steps(trace_step, args.steps, args.warmup, flush, stream)
    t_table = timed_steps(table_step, args.steps, args.warmup, flush, stream)
    lt.profile_enable(True)
    tp_query = timed_steps(query_step, args.steps, args.warmup, flush, stream, reset)
    pq = lt.profile_read(reset=True)
    qflags = o.flags.cpu().numpy()
    qout = torch.stack(o.f, 1).cpu().numpy()
    tp_table = timed_steps(table_step, args.steps, args.warmup, flush, stream, reset)
    pm = lt.profile_read(reset=True)
    mflags = o.flags.cpu().numpy()
    mout = torch.stack(o.f, 1).cpu().numpy()
    tp_trace = timed_steps(trace_step, args.steps, args.warmup, flush, stream, reset)
    pt = lt.profile_read(reset=True)
    lt.profile_enable(False)
    clocks = sampler.stop()
    tout = torch.stack(o.f, 1).cpu().numpy()
    tflags = o.flags.cpu().numpy()
    if world > 1:
        dist.barrier()

    # max over ranks of the summed step time
    (q_total_ms, t_total_ms, m_total_ms), (value, trace_value, table_value) = combine_ranks(
        [t_query, t_trace, t_table], world, n, args.steps, dist if world > 1 else None, "cuda")

    traced = (qflags & lt.FLAG_TRACED) != 0
    n_fb = int(traced.sum())
    interp = (~traced) & ((qflags & lt.FLAG_VALID) != 0)
    n_interp = int(interp.sum())
    m_fb = int(((mflags & lt.FLAG_TRACED) != 0).sum())
    peaks = load_peaks()
    # algorithmic bytes of one launch of each of the polynomial map's kernels:
    # the sort kernel reads every ray's 24 B and the class table once, and
    # writes a 28 B queue entry per ray it hands to the tracer and a 32 B
    # record per ray the polynomial answers; the evaluation kernel reads
    # those records, the coefficient table once and the queue entries, and
    # writes every ray's 25 B row
    coef_bytes = ppoly["patches"] * ((ppoly["terms"] + 3) // 4) * 80
    s_bytes = n * 24 + (pstats["n_cells"] + 15) // 16 * 4 + n_fb * 28 + n_interp * 32
    e_bytes = n_interp * 32 + coef_bytes + n * 25 + n_fb * 28
    # the table map's classify-and-gather kernel: 24 B in, 25 B out per answered
    # ray, 4 B per queued ray, the 16-bit node table (6 values of 2 B per node)
    # and classes once
    table_bytes = mstats["n_nodes"] * 12 + (mstats["n_cells"] + 15) // 16 * 4
    m_bytes = n * 24 + (n - m_fb) * 25 + m_fb * 4 + table_bytes
    kernels = {
        "poly_sort_kernel": kernel_roofline("poly_sort_kernel", pq, peaks, args.steps, units_bytes=s_bytes),
        # the evaluation kernel also traces the step's queued rays (its work
        # counter counts their interactions)
        "poly_eval_kernel": kernel_roofline("poly_eval_kernel", pq, peaks, args.steps, units_bytes=e_bytes),
        "trace_kernel": kernel_roofline("trace_kernel", pt, peaks, args.steps,
                                        flops_per_work=FLOPS_PER_INTERACTION),
        "map_query_kernel": kernel_roofline("map_query_kernel", pm, peaks, args.steps, units_bytes=m_bytes),
    }
    kernels["poly_eval_kernel"]["traced_rays_per_step"] = n_fb
    kernels["poly_eval_kernel"]["traced_interactions_per_step"] = int(pq["poly_eval_kernel"][2] / args.steps)
    # the roofline reported is that of the step's longer kernel
    dom = max(("poly_sort_kernel", "poly_eval_kernel"), key=lambda k: kernels[k]["kernel_ms_per_step"])
    # the ncu DRAM bytes of one launch of each kernel, where a capture of the
    # current kernel sources exists
    for name, kr in kernels.items():
        tr = NCU_TRAFFIC.get(name)
        kr["traffic"] = round(tr["bytes_per_ray"] * n) if tr and tr["hash"] == src_hash(tr["srcs"]) else None
    roof = dict(kernels[dom])

    # end to end through the host-buffer entry point (pinned host memory)
    h = batch.HostRays(rays)
    for _ in range(2):
        pmap.query_host(h.inp[:5], h.inp[5], h.out + [h.flags], n)
    e2e_steps = max(3, args.steps // 4)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        pmap.query_host(h.inp[:5], h.inp[5], h.out + [h.flags], n)
    e2e_s = (time.perf_counter() - t0) / e2e_steps

    launches = sum(v[0] for v in pq.values())
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": "rays/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(statistics.mean(t_query), 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "rays_per_gpu": n, "poly_map": POLY,
                   "l2": "flushed (256 MB write) before every step",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "p99_batch_ms": round(float(np.percentile(t_query, 99)), 4),
        "trace": {"rays_per_s": round(trace_value, 1), "ms_per_step": round(statistics.mean(t_trace), 4),
                  "p99_batch_ms": round(float(np.percentile(t_trace, 99)), 4),
                  "ms_per_step_profiled": round(statistics.mean(tp_trace), 4)},
        "ms_per_step_profiled": round(statistics.mean(tp_query), 4),
        "map_over_trace": round(value / trace_value, 3),
        "query_mix": {"mask_only": round(1 - (n_fb + n_interp) / n, 4),
                      "interpolated": round(n_interp / n, 4), "traced": round(n_fb / n, 4)},
        "map": {"build_s": round(pbuild_s, 3), "cells_valid": pstats["cells_valid"],
                "cells_boundary": pstats["cells_boundary"], "cells_invalid": pstats["cells_invalid"],
                "patches": ppoly["patches"], "patches_fit": ppoly["patches_fit"], "terms": ppoly["terms"],
                "fit_rays_residual_max_mm": pstats["fit_residual_max_mm"],
                "corner_residual_max_mm": ppoly["corner_residual_max_mm"],
                "table_bytes": pstats["table_bytes"],
                "err_vs_fp32_trace": map_error(qout, qflags, tout, tflags, lt)},
        "table_map": {"res": RES, "node_format": "s16", "table_bytes": mstats["table_bytes"],
                      "rays_per_s": round(table_value, 1),
                      "ms_per_step": round(statistics.mean(t_table), 4),
                      "ms_per_step_profiled": round(statistics.mean(tp_table), 4),
                      "map_over_trace": round(table_value / trace_value, 3), "build_s": round(build_s, 3),
                      "traced": round(m_fb / n, 4),
                      "err_vs_fp32_trace": map_error(mout, mflags, tout, tflags, lt),
                      "note": "multilinear interpolation of traced nodes (16-bit node table); outside the "
                              "1e-4 mm bound"},
        "roofline": roof,
        "kernels": kernels,
        "e2e": {"value": round(n / e2e_s, 1), "unit": "rays/s",
                "h2d_bytes_per_step": n * 24, "d2h_bytes_per_step": n * 25},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    if world == 1 and not args.skip_extra:
        extra = {}
        for key, fn in (("singlet_65k", bench_singlet), ("precision_16M", bench_precision),
                        ("flares_56x1M", bench_flares), ("mcmc_ghost", bench_mcmc)):
            extra[key] = fn(args, stream, flush, peaks)
            torch.cuda.empty_cache()
        extra["serving"] = bench_serving(args, peaks, seconds=args.serve_seconds)
        line["configs"] = extra
    if world == 1 and not args.skip_cpu:
        # the oracle baseline is taken at N = 1 only (the replicas' GPUs are not held for it)
        line["cpu_baseline"] = cpu_baseline(presc, rays)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


# ----------------------------------------------------------------------------- other configs

MLP_REG_SIZES = [4, 32, 32, 32, 32, 32, 6]
MLP_CLS_SIZES = [4, 32, 32, 1]
MLP_MACS = sum(a * b for a, b in zip(MLP_REG_SIZES[:-1], MLP_REG_SIZES[1:])) + \
    sum(a * b for a, b in zip(MLP_CLS_SIZES[:-1], MLP_CLS_SIZES[1:]))      # 4,416 + 1,184


def xavier_flat(sizes, rng):
    import numpy as np
    from paper_2605_04017_gb300 import workloads as w
    parts = []
    for a, b in zip(sizes[:-1], sizes[1:]):
        parts += [w.xavier_uniform(a, b, rng).reshape(-1), np.zeros(b)]
    return np.concatenate(parts).astype(np.float32)


def pos_err(a_out, a_flags, b_out, b_flags, FLAG_VALID, FLAG_GRAZING=0x40):
    """Exit-position distance (mm) over rays valid in both (grazing excluded)."""
    import numpy as np
    both = ((a_flags & FLAG_VALID) != 0) & ((b_flags & FLAG_VALID) != 0) & ((b_flags & FLAG_GRAZING) == 0)
    e = np.hypot(a_out[both, 0].astype(np.float64) - b_out[both, 0], a_out[both, 1].astype(np.float64) - b_out[both, 1])
    agree = float((((a_flags & FLAG_VALID) != 0) == ((b_flags & FLAG_VALID) != 0)).mean())
    if not e.size:
        return {"rms_mm": 0.0, "p99_mm": 0.0, "valid_agreement": agree}
    return {"rms_mm": float(np.sqrt((e ** 2).mean())), "p99_mm": float(np.percentile(e, 99)),
            "valid_agreement": round(agree, 6)}


def time_kernel(step, name, args, flush, stream, n, lt):
    """rays/s, mean and p99 step ms of the steps as they run, and the
    profiler's record of a second timed run with the library's per-kernel
    events on (their records add a few microseconds per launch, so the
    headline figures come from the first run)."""
    import numpy as np
    lt.profile_enable(False)
    t = timed_steps(step, args.steps, args.warmup, flush, stream)
    lt.profile_enable(True)
    lt.profile_read(reset=True)
    tp = timed_steps(step, args.steps, args.warmup, flush, stream, lambda: lt.profile_read(reset=True))
    prof = lt.profile_read(reset=True)
    lt.profile_enable(False)
    return {"rays_per_s": round(n * len(t) / (sum(t) * 1e-3), 1), "ms_per_step": round(statistics.mean(t), 4),
            "p99_batch_ms": round(float(np.percentile(t, 99)), 4),
            "ms_per_step_profiled": round(statistics.mean(tp), 4)}, prof


def bench_singlet(args, stream, flush, peaks):
    """The 2-surface singlet, 65,536 rays; its 32^4 x 8 map fitted on the same rays."""
    import torch
    from paper_2605_04017_gb300 import batch, lt, workloads as w
    presc = w.singlet_lens()
    lens = lt.Lens(presc)
    rays = w.singlet_rays()
    n = len(rays)
    d = batch.DeviceRays(rays)
    lo, hi = map_box(w.SINGLET_RHO)
    gmap = lt.Map.build(lens, 0, RES, lo, hi, fit=d)
    gmap16 = lt.Map.build(lens, 0, RES, lo, hi, fit=d, node_format=lt.NODE_S16)
    oq, ot = batch.DeviceOut(n), batch.DeviceOut(n)
    q16, pq16 = time_kernel(lambda: gmap16.query(d.inp, d.lam, oq.out, n, lt.QUERY_TABLE, stream), "q16", args,
                            flush, stream, n, lt)
    torch.cuda.synchronize()
    q16o, q16f = oq.numpy()
    q, pq = time_kernel(lambda: gmap.query(d.inp, d.lam, oq.out, n, lt.QUERY_TABLE, stream), "q", args, flush,
                        stream, n, lt)
    t, pt = time_kernel(lambda: lt.trace(lens, d.inp, d.lam, 0, ot.out, n, stream), "t", args, flush, stream, n,
                        lt)
    torch.cuda.synchronize()
    qo, qf = oq.numpy()
    to, tf = ot.numpy()
    # the one-kernel query's algorithmic bytes: 24 B in and 25 B out per ray,
    # and per interpolated ray the 32 corners' 24-byte node values it gathers
    n_interp = int((((qf & lt.FLAG_VALID) != 0) & ((qf & lt.FLAG_TRACED) == 0)).sum())
    q["kernel"] = kernel_roofline("map_query_fused_kernel", pq, peaks, args.steps,
                                  units_bytes=n * 49 + n_interp * 32 * 24)
    q["kernel"]["note"] = "algorithmic bytes: 49 B per ray + 768 B of corner gathers per interpolated ray"
    t["kernel"] = kernel_roofline("trace_kernel", pt, peaks, args.steps, flops_per_work=FLOPS_PER_INTERACTION)
    n16 = int((((q16f & lt.FLAG_VALID) != 0) & ((q16f & lt.FLAG_TRACED) == 0)).sum())
    q16["kernel"] = kernel_roofline("map_query_fused_kernel", pq16, peaks, args.steps,
                                    units_bytes=n * 49 + n16 * 32 * 12)
    q16["kernel"]["note"] = "algorithmic bytes: 49 B per ray + 384 B of 16-bit corner gathers per interpolated ray"
    q16["map_err_vs_fp32_trace"] = pos_err(q16o, q16f, to, tf, lt.FLAG_VALID)
    return {"workload": "2-surface singlet (R +-50 mm, t 5 mm, a 10 mm), 65,536 rays, map 32^4x8 fitted on them",
            "query": q, "query_s16": q16, "trace": t,
            "map_err_vs_fp32_trace": pos_err(qo, qf, to, tf, lt.FLAG_VALID)}


def bench_precision(args, stream, flush, peaks):
    """Config-1 lens, 16,777,216 rays: the learned map (classifier + regressor)
    in FP32, BF16 and FP16 (tensor cores), the FP32 table map and the FP32
    tracer on the same batch."""
    import numpy as np
    import torch
    from paper_2605_04017_gb300 import batch, lt, workloads as w
    presc = w.singlet_lens()
    lens = lt.Lens(presc)
    rho = w.SINGLET_RHO
    rng = np.random.Generator(np.random.PCG64(w.SEED_BASE + 3))
    fit = batch.DeviceRays(w.entrance_rays(1 << 21, w.SEED_BASE + 3 + 1000, rho))
    lt.profile_enable(True)
    lt.profile_read(reset=True)
    t0 = time.perf_counter()
    if args.untrained:
        # random Xavier networks (profiling: no training launches before the query)
        m = lt.Mlp.create(lens, lt.mlp_frame(0, rho, 0.2421), xavier_flat(MLP_REG_SIZES, rng),
                          xavier_flat(MLP_CLS_SIZES, rng), np.zeros(6), np.ones(6))
    else:
        m = lt.Mlp.train(lens, lt.mlp_frame(0, rho, 0.2421), fit, xavier_flat(MLP_REG_SIZES, rng),
                         xavier_flat(MLP_CLS_SIZES, rng), reg_steps=6000, reg_batch=8192, cls_steps=4000,
                         cls_batch=8192, lr=1e-3, lr_decay=0.95, decay_every=500, seed=5)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    ptrain = lt.profile_read(reset=True)
    lt.profile_enable(False)
    train_kernels = {}
    if not args.untrained:
        fp32 = fp32_peak_tflops(peaks["sm_max_mhz"])
        macs = {"mlp_train_reg_kernel": MLP_MACS - 1184, "mlp_train_cls_kernel": 1184}
        for k, nm in (("mlp_train_reg_kernel", 6000), ("mlp_train_cls_kernel", 4000)):
            if k in ptrain:
                launches, ms, _ = ptrain[k]
                # forward + backward of a batch: 3 x 2 flop per MAC per ray
                fl = 6.0 * macs[k] * 8192 * launches
                train_kernels[k] = {"launches": launches, "avg_launch_ms": round(ms / launches, 5),
                                    "bound": "alu", "achieved": round(fl / (ms * 1e-3) / 1e12, 2),
                                    "peak": round(fp32, 1), "unit": "TFLOP/s",
                                    "frac": round(fl / (ms * 1e-3) / 1e12 / fp32, 4),
                                    "note": "6 flop per MAC per ray (forward + both backward products), "
                                            "batch 8192"}
        if "mlp_adam_kernel" in ptrain:
            launches, ms, _ = ptrain["mlp_adam_kernel"]
            # per parameter: P read + written (8 B), the moments read + written
            # (FP64: 32 B) and one gradient partial per training block read (4 B
            # x 64 blocks of 128 rays)
            by = (6000 * 4582 + 4000 * 1249) * (8 + 32 + 4 * 64)   # reg 4,582 and cls 1,249 parameters
            ach = by / (ms * 1e-3) / 1e9
            train_kernels["mlp_adam_kernel"] = {
                "launches": launches, "avg_launch_ms": round(ms / launches, 5), "bound": "hbm",
                "achieved": round(ach, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": round(ach / peaks["hbm_gbs"], 4),
                "note": "per parameter and step: 8 B of parameter, 32 B of FP64 moments, 4 B x 64 "
                        "gradient partials"}
    lo, hi = map_box(rho)
    gmap = lt.Map.build(lens, 0, RES, lo, hi, fit=fit)
    gmap16 = lt.Map.build(lens, 0, RES, lo, hi, fit=fit, node_format=lt.NODE_S16)
    del fit
    rays = w.precision_rays(args.precision_rays or w.PRECISION_N)
    n = len(rays)
    d = batch.DeviceRays(rays)
    del rays
    o = batch.DeviceOut(n)
    res, outs = {}, {}
    runs = [("mlp_f32", lambda: m.query(d.inp, d.lam, o.out, n, lt.MLP_F32, stream), "mlp_query_f32_kernel"),
            ("mlp_bf16", lambda: m.query(d.inp, d.lam, o.out, n, lt.MLP_BF16, stream), "mlp_query_bf16_kernel"),
            ("mlp_f16", lambda: m.query(d.inp, d.lam, o.out, n, lt.MLP_F16, stream), "mlp_query_f16_kernel"),
            ("table_f32", lambda: gmap.query(d.inp, d.lam, o.out, n, lt.QUERY_TABLE, stream), None),
            ("table_s16", lambda: gmap16.query(d.inp, d.lam, o.out, n, lt.QUERY_TABLE, stream), None),
            ("trace_f32", lambda: lt.trace(lens, d.inp, d.lam, 0, o.out, n, stream), None)]
    bf16_peak = None
    if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        bf16_peak = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"])
    for key, step, kname in runs:
        r, prof = time_kernel(step, key, args, flush, stream, n, lt)
        torch.cuda.synchronize()
        outs[key] = o.numpy()
        if kname and kname in prof:
            launches, ms, _ = prof[kname]
            avg_s = ms / launches * 1e-3
            tflops = 2.0 * MLP_MACS * n / avg_s / 1e12
            r["kernel"] = {"name": kname, "mlp_tflops": round(tflops, 2), "avg_launch_ms": round(ms / launches, 4),
                           "hbm_gbs": round(49.0 * n / avg_s / 1e9, 1)}
            if key != "mlp_f32" and bf16_peak:
                peak = bf16_peak
                r["kernel"]["tensor_frac"] = round(tflops / peak, 4)
                r["kernel"]["tensor_peak"] = "%.1f TFLOP/s of measured (bf16 burst; fp16 taken equal)" % peak
            r["kernel"]["hbm_frac"] = round(49.0 * n / avg_s / 1e9 / peaks["hbm_gbs"], 4)
        if key in ("table_f32", "table_s16") and "map_query_kernel" in prof:
            # as the headline's table map: 24 B in, 25 B out per answered ray, 4 B
            # per queued ray, the node table (6 values per node: FP32 or 16-bit)
            # and classes once
            qf = outs[key][1]
            m_fb = int(((qf & lt.FLAG_TRACED) != 0).sum())
            ms_ = gmap.stats()
            vb = 24 if key == "table_f32" else 12
            r["kernel"] = kernel_roofline("map_query_kernel", prof, peaks, args.steps,
                                          units_bytes=n * 24 + (n - m_fb) * 25 + m_fb * 4 + ms_["n_nodes"] * vb +
                                          (ms_["n_cells"] + 15) // 16 * 4)
        if key == "trace_f32" and "trace_kernel" in prof:
            r["kernel"] = kernel_roofline("trace_kernel", prof, peaks, args.steps,
                                          flops_per_work=FLOPS_PER_INTERACTION)
        res[key] = r
    to, tf = outs["trace_f32"]
    errs = {k: pos_err(outs[k][0], outs[k][1], to, tf, lt.FLAG_VALID) for k in outs if k != "trace_f32"}
    f32o, f32f = outs["mlp_f32"]
    for k in ("mlp_bf16", "mlp_f16"):
        errs[k]["vs_mlp_f32"] = pos_err(outs[k][0], outs[k][1], f32o, f32f, lt.FLAG_VALID)
    st = m.stats()
    return {"workload": "singlet, 16,777,216 rays (seed +3); learned map = classifier 4-32-32-1 + "
                        "regressor 4-(32x5)-6, trained on the GPU from 2,097,152 traced rays",
            "train": {"s": round(train_s, 2), "kernels": train_kernels,
                      "reg_loss": st["reg_loss"], "cls_loss": st["cls_loss"],
                      "steps": "reg 6000 + cls 4000, batch 8192, Adam lr 1e-3 x0.95/500"},
            "rays_per_s": res, "pos_err_vs_fp32_trace": errs}


def bench_flares(args, stream, flush, peaks):
    """The 11-surface lens, main path + all 55 two-bounce ghosts, 1,048,576 rays
    each with wavelengths redrawn per path, one lt_trace_paths launch."""
    import numpy as np
    import torch
    from paper_2605_04017_gb300 import batch, lt, workloads as w
    presc = w.eleven_surface_lens(lib_accept)
    lens = lt.Lens(presc)
    P = lens.n_paths
    rays = w.flare_rays(presc, args.flare_rays or w.FLARE_N_PER_PATH)
    n = len(rays)
    d = batch.DeviceRays(rays)
    lam = torch.from_numpy(np.concatenate([w.flare_wavelengths(p, n) for p in range(P)])).cuda()
    po = batch.PathsOut(P, n)
    ids = list(range(P))
    r, prof = time_kernel(lambda: lt.trace_paths(lens, d.inp, lam, n, ids, po, n, stream), "paths", args, flush,
                          stream, n * P, lt)
    counts = po.counts()
    launches, ms, work = prof["trace_paths_kernel"]
    avg_s = ms / launches * 1e-3
    useful = work / launches * FLOPS_PER_INTERACTION / avg_s / 1e12
    peak = fp32_peak_tflops(peaks["sm_max_mhz"])
    del po
    torch.cuda.empty_cache()
    # forward light tracing of the same rays onto a 24 mm, 512 x 512 sensor
    # (Eq. 8; per-sample average): the same trace with the deposits fused in
    W = 512
    img = torch.zeros((1, W, W), dtype=torch.float32, device="cuda")
    rs, prof_s = time_kernel(lambda: lt.splat_paths(lens, d.inp, lam, n, ids, n, W, W, 24.0 / W, img,
                                                    weight=1.0 / n, stream=stream),
                             "splat", args, flush, stream, n * P, lt)
    sl, sms, swork = prof_s["splat_paths_kernel"]
    del img
    bf16 = None if args.no_flare_map else bench_flares_bf16_map(args, stream, flush, lens, presc, d, lam, n, P)
    return {"workload": "11-surface lens, 56 paths (main + 55 ghosts) x 1,048,576 rays, lambda per path",
            "rays_per_s": r["rays_per_s"], "ms_per_step": r["ms_per_step"], "p99_batch_ms": r["p99_batch_ms"],
            "valid_rays_per_launch": int(counts.sum()),
            "valid_rays_per_s": round(int(counts.sum()) / avg_s, 1),
            "roofline": {"kernel": "trace_paths_kernel", "bound": "alu", "achieved": round(useful, 2),
                         "peak": round(peak, 1), "unit": "TFLOP/s", "frac": round(useful / peak, 4),
                         "interactions_per_launch": int(work / launches),
                         "note": "useful FP32 flop: interactions actually executed x 89"},
            "splat": {"workload": "the same 56 x 1,048,576 rays traced and splatted onto a 24 mm 512 x 512 "
                                  "sensor (tent filter, G = exit d_z, weight 1/n)",
                      "rays_per_s": rs["rays_per_s"], "ms_per_step": rs["ms_per_step"],
                      "p99_batch_ms": rs["p99_batch_ms"],
                      "useful_tflops": round(swork / sl * FLOPS_PER_INTERACTION / (sms / sl * 1e-3) / 1e12, 2)},
            "bf16_map": bf16}


def bench_flares_bf16_map(args, stream, flush, lens, presc, d, lam, n, P, m_err=65536):
    """The BF16 map variant of the flare workload: one learned map per path
    (classifier + regressor trained on the GPU, short schedule), all 56
    queried in BF16 on tensor cores over the same rays and wavelengths as the
    trace.  Two training sets per path, the same schedule: 262,144 uniform
    draws of the input box, and 131,072 uniform draws followed by the
    valid-region sampler's 2,048 chains x 64 states (Sec. 5.1, data
    collection), whose maps are the ones timed.  Error of both against the
    FP32 tracer on the first m_err rays of every path."""
    import numpy as np
    import torch
    from paper_2605_04017_gb300 import batch, lt, workloads as w
    rho = w.eleven_rho(presc)
    lo, hi = map_box(rho)
    uni = batch.DeviceRays(w.entrance_rays(1 << 18, w.SEED_BASE + 4 + 1001, rho))
    half = batch.DeviceRays(w.entrance_rays(1 << 17, w.SEED_BASE + 4 + 1002, rho))
    kw = dict(reg_steps=1500, reg_batch=8192, cls_steps=1500, cls_batch=8192, lr=1e-3, lr_decay=0.95,
              decay_every=500)

    def train_all(sampler):
        rng = np.random.Generator(np.random.PCG64(w.SEED_BASE + 4 + 1000))
        maps, t_mcmc = [], 0.0
        t0 = time.perf_counter()
        for p in range(P):
            fit = uni
            if sampler:
                t1 = time.perf_counter()
                fit = lt.valid_region_fit(lens, p, lo, hi, half, chains=2048, steps=64, seed=w.SEED_BASE + 4 + 2000 + p)
                t_mcmc += time.perf_counter() - t1
            maps.append(lt.Mlp.train(lens, lt.mlp_frame(p, rho, 0.2421), fit, xavier_flat(MLP_REG_SIZES, rng),
                                     xavier_flat(MLP_CLS_SIZES, rng), seed=100 + p, **kw))
        torch.cuda.synchronize()
        return maps, time.perf_counter() - t0, t_mcmc

    maps_u, train_u, _ = train_all(False)
    maps, train_s, mcmc_s = train_all(True)
    del uni, half
    o = batch.DeviceOut(n)

    def step():
        for p in range(P):
            maps[p].query(d.inp, lam[p * n:(p + 1) * n], o.out, n, lt.MLP_BF16, stream)

    r, _ = time_kernel(step, "flares_bf16", args, flush, stream, n * P, lt)
    # error against the FP32 tracer, path by path, on the first m_err rays
    m = min(m_err, n)
    sub = [t[:m] for t in d.inp]
    tq, qq = batch.DeviceOut(m), batch.DeviceOut(m)

    def errors(ms):
        agree, iou, rms, p99, nboth = [], [], [], [], 0
        for p in range(P):
            lp = lam[p * n:p * n + m]
            lt.trace(lens, sub, lp, p, tq.out, m, stream)
            ms[p].query(sub, lp, qq.out, m, lt.MLP_BF16, stream)
            torch.cuda.synchronize()
            to, tf = tq.numpy()
            qo, qf = qq.numpy()
            tv, qv = (tf & lt.FLAG_VALID) != 0, (qf & lt.FLAG_VALID) != 0
            agree.append(float((tv == qv).mean()))
            iou.append(float((tv & qv).sum() / max(1, (tv | qv).sum())))
            both = tv & qv
            if both.sum() >= 10:
                e = np.hypot(qo[both, 0] - to[both, 0], qo[both, 1] - to[both, 1])
                rms.append(float(np.sqrt((e ** 2).mean())))
                p99.append(float(np.percentile(e, 99)))
                nboth += int(both.sum())
        return {"rays_per_path": m, "valid_agreement_mean": round(float(np.mean(agree)), 5),
                "valid_agreement_min": round(float(np.min(agree)), 5),
                "valid_iou_mean": round(float(np.mean(iou)), 5), "valid_iou_min": round(float(np.min(iou)), 5),
                "pos_rms_mm_median_over_paths": round(float(np.median(rms)), 5) if rms else None,
                "pos_rms_mm_main_path": round(rms[0], 5) if rms else None,
                "pos_p99_mm_median_over_paths": round(float(np.median(p99)), 5) if p99 else None,
                "pos_p99_mm_max_over_paths": round(float(np.max(p99)), 5) if p99 else None,
                "paths_compared": len(rms), "rays_valid_in_both": nboth}

    return {"workload": "one learned map per path (classifier 4-32-32-1 + regressor 4-(32x5)-6, "
                        "1,500 + 1,500 Adam steps of 8,192, lr 1e-3 x 0.95 per 500 steps), trained on 131,072 "
                        "uniform rays + 2,048 x 64 valid-region samples of the path; 56 BF16 tensor-core queries "
                        "of 1,048,576 rays each",
            "train_s": round(train_s, 2), "sampler_s": round(mcmc_s, 2), "rays_per_s": r["rays_per_s"],
            "ms_per_step": r["ms_per_step"], "p99_batch_ms": r["p99_batch_ms"],
            "err_vs_fp32_trace": errors(maps),
            "uniform_training": {"workload": "the same maps trained on 262,144 uniform rays of the box instead",
                                 "train_s": round(train_u, 2), "err_vs_fp32_trace": errors(maps_u)}}


def bench_mcmc(args, stream, flush, peaks):
    """The valid-region sampler (Sec. 5.1) on a ghost path of the 11-surface
    lens: 65,536 chains x 64 steps, against uniform draws of the same box."""
    import numpy as np
    import torch
    from paper_2605_04017_gb300 import batch, lt, workloads as w
    presc = w.eleven_surface_lens(lib_accept)
    lens = lt.Lens(presc)
    rho = w.eleven_rho(presc)
    lo, hi = map_box(rho)
    pid, chains, steps = 20, 65536, 64
    box = [(a, b) for a, b in zip(lo, hi)]
    res = {}

    def step():
        res["out"] = lt.mcmc_sample(lens, pid, lo, hi, 20260510, chains, steps, 0.03, 0.05, 64, stream)

    r, prof = time_kernel(step, "mcmc", args, flush, stream, chains * steps, lt)
    f, flags, acc = res["out"]
    started = float((flags[:chains] != 0).float().mean())
    a = acc.cpu().numpy()
    launches, ms, work = prof["mcmc_kernel"]
    # uniform draws of the same box through the tracer: the valid fraction they would give
    u = np.random.default_rng(20260511)
    n = 1 << 22
    cols = [u.uniform(b[0], b[1], n) for b in box]
    s = np.sqrt(cols[2] ** 2 + cols[3] ** 2 + 1.0)
    rays = w.Rays(*(np.asarray(c, np.float32) for c in (cols[0], cols[1], cols[2] / s, cols[3] / s, 1.0 / s, cols[4])))
    d = batch.DeviceRays(rays)
    o = batch.DeviceOut(n)
    lt.trace(lens, d.inp, d.lam, pid, o.out, n, stream)
    torch.cuda.synchronize()
    uniform_valid = float(((o.flags & 1) != 0).float().mean())
    useful = work / launches * FLOPS_PER_INTERACTION / (ms / launches * 1e-3) / 1e12
    return {"workload": "11-surface lens, ghost path 20, 65,536 chains x 64 steps (small 0.03, p_large 0.05, "
                        "64 start draws)",
            "samples_per_s": r["rays_per_s"], "ms_per_step": r["ms_per_step"], "p99_batch_ms": r["p99_batch_ms"],
            "chains_started": round(started, 4),
            "acceptance": round(float(a[a > 0].mean()) / steps, 4) if (a > 0).any() else 0.0,
            "valid_fraction_of_uniform_draws": round(uniform_valid, 5),
            "useful_tflops": round(useful, 2),
            "roofline": kernel_roofline("mcmc_kernel", prof, peaks, args.steps,
                                        flops_per_work=FLOPS_PER_INTERACTION)}


def bench_serving(args, peaks, seconds=10.0, warm=1.0, rate=2000.0):
    """8 seeded lenses (S ~ U{4..22}); Poisson arrivals; sizes log-uniform on
    [1,024, 4,194,304]; lens uniform; main path (its resident table map) with
    probability 0.5, else a uniform ghost (traced).  Latency = submission ->
    completion on the host clock, requests submitted after the warm-up."""
    import queue
    import numpy as np
    import torch
    from paper_2605_04017_gb300 import batch, lt, workloads as w
    pres = w.serving_lenses(lib_accept, 8)
    lenses = [lt.Lens(p) for p in pres]
    NMAX = 1 << 22
    inputs, maps = [], []
    for k, p in enumerate(pres):
        rho = 1.2 * p.surfaces[0].aperture_r
        lo, hi = map_box(rho)
        fit = batch.DeviceRays(w.entrance_rays(1 << 21, w.SEED_BASE + 5 + 7 * k, rho))
        maps.append(lt.Map.build(lenses[k], 0, RES, lo, hi, fit=fit, node_format=lt.NODE_S16))
        del fit
        inputs.append(batch.DeviceRays(w.entrance_rays(NMAX, w.SEED_BASE + 5 + 7 * k + 1, rho)))
    # each resident map's error against the FP32 tracer on the first 65,536
    # rays of its lens's requests (interpolated rays; traced ones are exact)
    m_err = 1 << 16
    eq, et = batch.DeviceOut(m_err), batch.DeviceOut(m_err)
    map_err = []
    for k in range(len(pres)):
        sub = [t[:m_err] for t in inputs[k].inp]
        lam = inputs[k].lam[:m_err]
        maps[k].query(sub, lam, eq.out, m_err)
        lt.trace(lenses[k], sub, lam, 0, et.out, m_err)
        torch.cuda.synchronize()
        qo, qf = eq.numpy()
        to, tf = et.numpy()
        interp = (qf & lt.FLAG_TRACED) == 0
        e = pos_err(qo[interp], qf[interp], to[interp], tf[interp], lt.FLAG_VALID)
        map_err.append({"surfaces": pres[k].n_surfaces, "rms_mm": round(e["rms_mm"], 6),
                        "p99_mm": round(e["p99_mm"], 6), "valid_agreement": e["valid_agreement"],
                        "traced_fraction": round(float((~interp).mean()), 4)})
    del eq, et
    SLOTS = 48
    slots = [batch.DeviceOut(NMAX) for _ in range(SLOTS)]
    torch.cuda.synchronize()

    def run(rate, window_us, seed):
        """One serving run: Poisson arrivals at `rate` for `warm` + `seconds`."""
        free = queue.Queue()
        for i in range(SLOTS):
            free.put(i)
        rng = np.random.Generator(np.random.PCG64(w.SEED_BASE + 5 + seed))
        total = seconds + warm
        n_req = int(rate * total * 1.2) + 16
        t_arr = np.cumsum(rng.exponential(1.0 / rate, n_req))
        n_req = int(np.searchsorted(t_arr, total))
        t_arr = t_arr[:n_req]
        sizes = np.exp(rng.uniform(np.log(1024), np.log(NMAX), n_req)).astype(np.int64)
        which = rng.integers(0, len(pres), n_req)
        main = rng.uniform(size=n_req) < 0.5
        ghost = [int(rng.integers(1, lenses[k].n_paths)) for k in which]
        srv = lt.Server(n_streams=4, batch_window_us=window_us)
        tickets = queue.Queue()
        stalls = [0]

        def submitter():
            t0 = time.perf_counter()
            for i in range(n_req):
                while True:
                    dt = t0 + t_arr[i] - time.perf_counter()
                    if dt <= 0:
                        break
                    time.sleep(dt if dt > 2e-4 else 0)
                try:
                    slot = free.get_nowait()
                except queue.Empty:
                    stalls[0] += 1
                    slot = free.get()
                k, nn = int(which[i]), int(sizes[i])
                d, o = inputs[k], slots[slot]
                if main[i]:
                    t = srv.submit_query(maps[k], d.inp, d.lam, o.out, nn)
                else:
                    t = srv.submit_trace(lenses[k], d.inp, d.lam, ghost[i], o.out, nn)
                tickets.put((i, t, slot))
            tickets.put(None)

        lat, rays_done, fused_lat = [], 0, 0
        th = threading.Thread(target=submitter)
        sampler = ClockSampler(torch.cuda.current_device())
        sampler.start()
        wall0 = time.perf_counter()
        th.start()
        fails = 0
        while True:
            item = tickets.get()
            if item is None:
                break
            i, t, slot = item
            st, info = srv.poll(t, 60_000_000)
            free.put(slot)
            if st != lt.OK:
                fails += 1
                continue
            if t_arr[i] >= warm:
                lat.append(info["latency_us"])
                rays_done += int(sizes[i])
                fused_lat += int(info["fused"] > 1)
        wall = time.perf_counter() - wall0
        th.join()
        smi = sampler.stop()
        stats = srv.stats()
        srv.close()
        lat = np.array(lat)
        return {"offered_req_per_s": rate, "batch_window_us": window_us,
                "requests": int(len(lat)), "failed": fails,
                "achieved_req_per_s": round(n_req / wall, 1),
                "p50_latency_ms": round(float(np.percentile(lat, 50)) / 1e3, 4) if lat.size else None,
                "p99_latency_ms": round(float(np.percentile(lat, 99)) / 1e3, 4) if lat.size else None,
                "rays_per_s": round(rays_done / seconds, 1),
                "gpu_util_pct_mean": smi.get("gpu_util_pct_mean"),
                "fused_launches": int(stats["fused_launches"]), "fused_requests": int(stats["fused_requests"]),
                "fused_fraction": round(int(stats["fused_requests"]) / max(1, int(stats["completed"])), 4),
                "launches": int(stats["launches"]), "client_slot_stalls": stalls[0]}

    base = run(rate, 0, 0)
    loaded = run(args.serve_high_rate, 0, 1)
    windowed = run(args.serve_high_rate, 200, 2)
    return {"workload": "8 seeded lenses (S 4..22), Poisson arrivals, sizes log-uniform [1024, 4194304], "
                        "main path via resident 32^4x8 16-bit table map else a uniform ghost traced; "
                        "%g s after %g s warm-up "
                        "per run" % (seconds, warm),
            **base,
            "high_load": loaded,
            "high_load_batch_window": windowed,
            "map_err_vs_fp32_trace": map_err}


SWEEP_POLY = [
    # (degree, patches, cells per patch, max_residual_mm): the headline first
    (4, [4, 4, 2, 1], [32, 32, 32, 8], 1e-4),
    (4, [4, 4, 2, 1], [32, 32, 32, 8], 0.0),
    (4, [4, 4, 2, 1], [16, 16, 16, 4], 1e-4),
    (4, [4, 4, 2, 1], [64, 64, 64, 8], 1e-4),
    (4, [4, 4, 1, 1], [32, 32, 64, 8], 1e-4),
    (4, [2, 2, 2, 1], [64, 64, 32, 8], 1e-4),
    (4, [2, 2, 1, 1], [64, 64, 64, 8], 1e-4),
    (3, [4, 4, 2, 1], [32, 32, 32, 8], 1e-4),
    (5, [4, 4, 2, 1], [32, 32, 32, 8], 1e-4),
    (3, [8, 8, 4, 2], [16, 16, 16, 4], 1e-4),
    (2, [16, 16, 8, 2], [8, 8, 8, 4], 1e-4),
    (2, [16, 16, 8, 2], [8, 8, 8, 4], 0.0),
    (2, [4, 4, 2, 1], [32, 32, 32, 8], 1e-4),
    (2, [4, 4, 2, 1], [32, 32, 32, 8], 0.0),
]
SWEEP_TABLE = [  # (lattice, max_residual_mm, node format: 0 FP32, 1 16-bit)
    ([16, 16, 16, 16, 8], 0.0, 0), ([24, 24, 24, 24, 8], 0.0, 0), ([32, 32, 32, 32, 8], 0.0, 0),
    ([40, 40, 40, 40, 8], 0.0, 0), ([32, 32, 32, 32, 8], 1e-4, 0),
    ([32, 32, 32, 32, 8], 0.0, 1), ([40, 40, 40, 40, 8], 0.0, 1)]


def bench_sweep(args, stream, flush, peaks):
    """Accuracy against speed on the headline workload (11-surface lens, the
    same 4,194,304 rays): the polynomial-patch map over degree, patch grid,
    mask resolution and certification limit, and the multilinear table map
    over lattice resolution, each fitted from the same 16,777,216 traced rays;
    rays/s of the query, its error against the FP32 trace of the same rays
    and the share of rays it traces, beside the FP32 trace itself."""
    import torch
    from paper_2605_04017_gb300 import batch, lt, workloads as w
    presc = w.eleven_surface_lens(lib_accept)
    lens = lt.Lens(presc)
    rho = w.eleven_rho(presc)
    n = args.rays or w.ELEVEN_N
    d = batch.DeviceRays(w.entrance_rays(n, w.SEED_BASE + 2, rho))
    fit = batch.DeviceRays(w.eleven_fit_rays(presc))
    o, ot = batch.DeviceOut(n), batch.DeviceOut(n)
    steps = max(3, args.steps // 2)

    def timed(step):
        t = timed_steps(step, steps, args.warmup, flush, stream)
        return {"rays_per_s": round(n * len(t) / (sum(t) * 1e-3), 1), "ms_per_step": round(statistics.mean(t), 4)}

    tr = timed(lambda: lt.trace(lens, d.inp, d.lam, 0, ot.out, n, stream))
    torch.cuda.synchronize()
    tout = torch.stack(ot.f, 1).cpu().numpy()
    tflags = ot.flags.cpu().numpy()

    def measured(m, build_s, extra):
        r = timed(lambda: m.query(d.inp, d.lam, o.out, n, lt.QUERY_TABLE, stream))
        torch.cuda.synchronize()
        qflags = o.flags.cpu().numpy()
        qout = torch.stack(o.f, 1).cpu().numpy()
        traced = float(((qflags & lt.FLAG_TRACED) != 0).mean())
        e = map_error(qout, qflags, tout, tflags, lt)
        keep = ("pos_max_mm", "pos_p99_mm", "pos_rms_mm", "dir_max", "I_max", "valid_agreement",
                "validity_mismatches", "validity_mismatches_near_edge")
        row = dict(extra)
        row.update(r)
        row.update({"map_over_trace": round(r["rays_per_s"] / tr["rays_per_s"], 3), "build_s": round(build_s, 4),
                    "traced": round(traced, 4), "answered_by_map": round(e["rays_interpolated"] / n, 4)})
        row.update({k: e[k] for k in keep if k in e})
        return row

    rows = []
    lo, hi = map_box(rho)
    for deg, pt, cells, tol in SWEEP_POLY:
        cfg = {"degree": deg, "patches": pt, "cells": cells, "samples": deg + 2, "max_residual_mm": tol}
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m = build_poly(lt, lens, rho, fit, cfg)
        torch.cuda.synchronize()
        bs = time.perf_counter() - t0
        ps = m.poly_stats()
        rows.append(measured(m, bs, {"map": "poly", "degree": deg, "patches": pt,
                                     "mask_cells": [a * b for a, b in zip(pt, cells)], "max_residual_mm": tol,
                                     "table_bytes": m.stats()["table_bytes"], "patches_fit": ps["patches_fit"]}))
        del m
        torch.cuda.empty_cache()
    for res, tol, fmt in SWEEP_TABLE:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m = lt.Map.build(lens, 0, res, lo, hi, fit=fit, max_residual_mm=tol, node_format=fmt)
        torch.cuda.synchronize()
        bs = time.perf_counter() - t0
        rows.append(measured(m, bs, {"map": "table", "res": res, "max_residual_mm": tol,
                                     "node_format": "s16" if fmt else "f32",
                                     "table_bytes": m.stats()["table_bytes"]}))
        del m
        torch.cuda.empty_cache()
    return {"workload": "11-surface lens, %d rays, transmission path; maps fitted from 16,777,216 traced rays; "
                        "%d timed steps each, L2 flushed before every step" % (n, steps),
            "trace": tr, "maps": rows}


def run_only(args):
    """One of the other workloads alone (1 GPU): prints {"workload_key": ..., ...}."""
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    stream = torch.cuda.current_stream()
    flush_buf = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    peaks = load_peaks()

    def flush():
        flush_buf.fill_(1)

    fns = {"singlet": bench_singlet, "precision": bench_precision, "flares": bench_flares, "mcmc": bench_mcmc,
           "sweep": bench_sweep}
    if args.only == "serving":
        out = bench_serving(args, peaks, seconds=args.serve_seconds)
    else:
        out = fns[args.only](args, stream, flush, peaks)
    print(json.dumps({"only": args.only, **out}), flush=True)


def oracle_poly_map(presc, rays):
    """The oracle's polynomial-patch map of the headline configuration with the
    classes of the cells `rays` fall in (classify_cells: their corners traced
    afresh plus the fit rays inside them), built single-threaded beforehand and
    not timed."""
    import numpy as np
    from oracle import poly
    from paper_2605_04017_gb300 import workloads as w
    t0 = time.perf_counter()
    om = poly.PolyMap(presc, (0, 0), w.eleven_rho(presc), SMAX, 380.0, 780.0, POLY["degree"], POLY["patches"],
                      POLY["cells"], POLY["samples"], tol=POLY["max_residual_mm"],
                      fit_rays=w.eleven_fit_rays(presc), build_mask=False)
    inside, cells = om.locate(rays)
    cid = np.ravel_multi_index(tuple(cells.T), tuple(om.grid.C))
    uc, inv = np.unique(cid[inside], return_inverse=True)
    ucls, _ = om.classify_cells(np.stack(np.unravel_index(uc, tuple(om.grid.C)), 1))
    classes = np.full(len(rays), 2, np.uint8)
    classes[np.nonzero(inside)[0]] = ucls[inv]
    return om, classes, time.perf_counter() - t0


def oracle_query_threads(om, rays, classes, cores):
    """The oracle's query of `rays` (given their cells' classes) split into
    `cores` equal parts run on as many threads (numpy and the C tracer release
    the GIL); returns the wall time."""
    import concurrent.futures
    n = len(rays)
    cuts = [(n * k // cores, n * (k + 1) // cores) for k in range(cores)]
    parts = [(rays.subset(slice(a, b)), classes[a:b]) for a, b in cuts]
    with concurrent.futures.ThreadPoolExecutor(cores) as ex:
        t0 = time.perf_counter()
        list(ex.map(lambda pc: om.query(pc[0], classes=pc[1]), parts))
        return time.perf_counter() - t0


CPU_SAMPLE = 1 << 18


def cpu_baseline(presc, rays):
    """The FP64 oracle's query of the polynomial-patch map, as it stands, on a
    bounded sample of the batch (its first 262,144 rays), on one host core: the
    oracle is a plain single-threaded numpy program, and threads over it only
    contend for the interpreter (measured slower than one)."""
    sample = rays.subset(slice(0, min(len(rays), CPU_SAMPLE)))
    om, classes, build = oracle_poly_map(presc, sample)
    m = len(sample)
    om.query(sample, classes=classes)
    t0 = time.perf_counter()
    om.query(sample, classes=classes)
    dt = time.perf_counter() - t0
    return {"value": round(m / dt, 1), "unit": "rays/s", "cores": 1, "kind": "oracle",
            "sample": f"the first {m} rays of the batch through the oracle's own polynomial-patch map "
                      f"(fitted, and the sample's cells classified, single-threaded in {build:.1f} s, "
                      f"untimed), one thread; host has {os.cpu_count()} cores"}


def run_reference(args):
    """The oracle arm: the FP64 CPU oracle's query of the polynomial-patch map,
    as it stands, on one host core (threads over the numpy oracle only contend
    for the interpreter), same workload, metric and unit; each step 262,144 rays
    of the batch."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2605_04017_gb300 import workloads as w
    presc = w.eleven_surface_lens(oracle_accept)
    rays = w.eleven_rays(presc, CPU_SAMPLE)
    om, classes, build = oracle_poly_map(presc, rays)
    cores = 1
    for _ in range(args.warmup):
        om.query(rays, classes=classes)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        om.query(rays, classes=classes)
    dt = time.perf_counter() - t0
    value = args.steps * len(rays) / dt
    line = {"metric": METRIC, "value": round(value, 1), "unit": "rays/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "rays_per_step": len(rays)}, "impl": "reference",
            "cpu_baseline": {"value": round(value, 1), "unit": "rays/s", "cores": cores,
                             "kind": "oracle",
                             "sample": f"{len(rays)} rays of the same workload per step on one "
                                       f"thread; map fitted and the sample's cells classified "
                                       f"single-threaded in {build:.1f} s, untimed"},
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
    ap.add_argument("--skip-extra", action="store_true", help="headline workload only")
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--serve-high-rate", type=float, default=16000.0,
                    help="offered request rate of the serving workload's loaded runs")
    ap.add_argument("--only", choices=["singlet", "precision", "flares", "mcmc", "serving", "sweep"],
                    help="run one of the other workloads alone and print its object")
    ap.add_argument("--rays", type=int, default=0, help="headline batch size (default 4,194,304)")
    ap.add_argument("--precision-rays", type=int, default=0)
    ap.add_argument("--flare-rays", type=int, default=0, help="rays per flare path")
    ap.add_argument("--no-flare-map", action="store_true",
                    help="leave out the flare workload's BF16 learned-map variant (56 trainings)")
    ap.add_argument("--untrained", action="store_true",
                    help="precision workload with random networks (no training launches)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        run_reference(args)
    elif args.only:
        run_only(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
