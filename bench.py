"""Benchmark: ray-segments per second of the coupled trace + ionisation step.

Workload (the Strömgren convergence configuration): 128^3 uniform grid, box
6.6 kpc, n_H = 1e-3 cm^-3, one 13.6 eV source of 5e48 photons/s at the
corner, sigma = 6.3e-18 cm^2, HEALPix level 1, Phi_c = 5.1, f_term = 1e-10;
state = the seeded-free synthetic snapshot with the I-front at the analytic
500 Myr radius (synth.stromgren_snapshot).  One step = one rt_trace plus one
rt_chem_update (dt = 0.5 Myr, 10 backward-Euler substeps), starting every time
from that snapshot, so every step does identical work.

Output: one JSON line (rank 0).  ``value`` = segments/s with inputs resident
in HBM (device-timed with CUDA events on the library's stream, L2 flushed
between steps); ``e2e`` = the same through the C ABI with pinned host
buffers, host->device state upload and device->host k_ph/x_HI readback inside
the timed region.  Beside it: the Strömgren convergence run (1000 coupled steps
from the neutral medium in each precision, R_IF against the closed-form R_s)
and, in the leg that times the oracle, each GPU path's k_ph and x_HI after the
benchmark step against the oracle's.  ``--impl reference`` times the FP64 CPU
oracle on the same step instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ray-segments/sec FP32-mixed vs FP64 at ≤1e-3 k_ph rel err; p50/p99 solve latency"
UNIT = "ray-segments/s"
WORKLOAD = ("stromgren-128^3: Test-1 medium (6.6 kpc, n_H=1e-3, corner source 5e48 ph/s, 13.6 eV), "
            "I-front at the 500 Myr radius; step = rt_trace (level 1, Phi_c 5.1, f_term 1e-10) + "
            "rt_chem_update (0.5 Myr, 10 substeps)")
WORKLOAD_CLUMPY = ("clumpy-256^3: log-normal medium (P(k) ~ k^-3, sigma_ln 1, mean n_H 1e-2), 1000 sources "
                   "of 1e48-1e50 ph/s at random cell centres, x_HI = 1; step = rt_trace (level 1, Phi_c 5.1, "
                   "f_term 1e-10) + rt_chem_update (0.5 Myr, 10 substeps)")
DT_S = 0.5 * 3.15576e13
# the trace kernel's sources: a profile summary's DRAM traffic holds only for these exact files
TRACE_SOURCES = ("trace.cu", "rt_internal.cuh", "f2.cuh", "healpix.cuh")


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self) -> dict:
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                smax.append(float(p[1]))
            except ValueError:
                continue
            for nm, v in zip(names, p[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm)}


def barrier():
    """Barrier across ranks (no-op without an initialised process group)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def reduce_over_ranks(total_s: float, segments: int):
    """Replicas: the slowest rank's timed seconds and the work of all ranks."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return total_s, segments
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([total_s], dtype=torch.float64, device=dev)
    n = torch.tensor([segments], dtype=torch.int64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t.item()), int(n.item())


def _kernel_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in TRACE_SOURCES:
        with open(os.path.join(ROOT, "paper_1012_2865_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def _profiled_traffic(precision: str, workload: str):
    """DRAM bytes per trace launch from the committed ncu summary of this
    workload, or None when there is none or the kernel changed since."""
    path = os.path.join(ROOT, "profiles", f"trace_kernel_{precision}_{workload}.md")
    try:
        fields = {}
        with open(path) as f:
            for line in f:
                if ":" in line and line.startswith("- "):
                    k, v = line[2:].split(":", 1)
                    fields[k.strip()] = v.strip().strip("`")
        if fields.get("kernel_source_sha256") != _kernel_source_hash():
            return None
        return float(fields["dram_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        return None


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0}, "fallback"


def queue_capacity_for(b, level0=1):
    """Queue records that a repeat of trace `b` can need: every child other
    than child 0 of every split (how many of them a free lane of the splitting
    warp takes instead of the queue depends on scheduling), with a margin."""
    kids = sum(int(c) for c in np.asarray(b["counts"])[level0 + 1:])
    return max(1 << 20, kids // 4 * 3 * 9 // 8 + 1024)


# bytes of one queue record (written once, read once) per precision, for
# traces without a finite speed of light (FP32-mixed records of FSL traces,
# which carry the package's age, take 48)
REC_BYTES = {"fp64": 48, "fp32_mixed": 32}


def red_peak(native, device: int, precision: str, cells: int):
    """Reductions per second the probe measures (rt_probe_red): into a 64 MB
    array, which stays in L2 -- the roof of the deposits -- and, as context,
    into an array of the workload's rate-array size (scattered addresses; the
    deposits of a ray are spatially coherent, so they can exceed that one)."""
    dt = native.RT_DTYPE_F64 if precision == "fp64" else native.RT_DTYPE_F32
    esz = 8 if precision == "fp64" else 4
    roof_words = (64 << 20) // esz
    size_words = min(1 << 30, 1 << int(np.ceil(np.log2(max(cells, 1024)))))
    return native.rt_probe_red(device, dt, roof_words), roof_words, native.rt_probe_red(device, dt, size_words), \
        size_words


def trace_roofline(precision, segments, pushed, kernel_ms, gamma, red, peaks, peak_kind, traffic):
    """Roofline figures of one trace launch.

    HBM: algorithmic bytes per launch -- per segment the n_HI read (FP64, or
    the FP32 pair: 8 bytes) and the k_ph reduction (8 / 4 bytes), plus the
    Gamma reduction where photons carry energy above the threshold; per queue
    record one write and one read -- over the kernel's event-timed duration,
    against the measured copy bandwidth.
    L2 reductions: one k_ph reduction per segment (and one Gamma reduction
    where photons heat) over the same duration, against the L2-resident
    reduction rate the probe measured in this run (`red`, from red_peak; the
    per-package residual deposits and the queue's atomics, a few per cent,
    are left out, so the fraction is a lower bound)."""
    red_b = 8 if precision == "fp64" else 4
    nred = 2 if gamma else 1
    alg = segments * (8 + red_b * nred) + pushed * 2 * REC_BYTES[precision]
    s = kernel_ms / 1e3
    achieved = alg / s / 1e9
    hbm = peaks.get("hbm_gbs", 6800.0)
    out = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
           "traffic": traffic, "peak_kind": peak_kind, "algorithmic_bytes": alg, "kernel": "trace_kernel",
           "kernel_ms": kernel_ms}
    if red:
        roof, roof_words, at_size, size_words = red
        reds = segments * nred
        out["l2_red"] = {"reds_per_launch": reds, "achieved": reds / s / 1e9, "peak": roof / 1e9,
                         "unit": "G RED/s", "frac": reds / s / roof,
                         "peak_kind": f"measured in this run (rt_probe_red, {'f64' if red_b == 8 else 'f32'}, "
                                      f"{roof_words} words = 64 MB, L2-resident, scattered addresses)",
                         "scattered_rate_at_array_size": {"words": size_words, "G_per_s": at_size / 1e9}}
    return out


def run_native(args, rank, world, local):
    import torch
    from paper_1012_2865_gb300 import build, native, synth

    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    ctx = native.rt_ctx_create(local)
    g = synth.clumpy() if args.workload == "clumpy" else synth.stromgren_snapshot(args.grid)
    params = dict(synth.DEFAULT_PARAMS)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 512 MB > L2

    x0 = torch.tensor(g["x_HI"], dtype=torch.float64, device=dev)
    z0 = torch.tensor(g["x_HII"], dtype=torch.float64, device=dev)

    def measure(precision, **extra):
        grid = native.Grid(ctx, g, precision, stream=stream.cuda_stream)
        b = grid.trace(**params, **extra)  # sizes the queue
        cap = queue_capacity_for(b, params["level0"])
        qp = dict(params, queue_capacity=cap, **extra)
        seg_per_step = b["segments"]
        pushed = b["queue_pushed"]
        for _ in range(max(3, args.warmup)):
            native.rt_set_state(grid.h, x0, z0)
            grid.trace(sync=False, **qp)
            grid.chem(DT_S, 10, synth.ALPHA_B)
        torch.cuda.synchronize()
        step_ms, kern_ms = [], []
        segs = 0
        launches = 0
        torch.cuda.synchronize()
        barrier()
        with ClockSampler(local) as clk:
            for _ in range(args.steps):
                native.rt_set_state(grid.h, x0, z0)  # restore the snapshot (untimed)
                flush.zero_()                         # evict L2 between steps (untimed)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                l0 = native.rt_kernel_launches()
                e0.record(stream)
                grid.trace(sync=False, **qp)
                grid.chem(DT_S, 10, synth.ALPHA_B)
                e1.record(stream)
                launches += native.rt_kernel_launches() - l0
                e1.synchronize()
                bb = native.rt_get_budget(grid.h)
                step_ms.append(e0.elapsed_time(e1))
                kern_ms.append(bb["kernel_ms"])
                segs += bb["segments"]
                assert bb["segments"] == seg_per_step, (bb["status"], bb["segments"], seg_per_step)
        torch.cuda.synchronize()
        barrier()
        final = grid.rates()  # one step from the snapshot: k_ph of the trace, x_HI after the update
        grid.close()
        return dict(step_ms=step_ms, kern_ms=kern_ms, segments=segs, seg_per_step=seg_per_step,
                    pushed=pushed, launches=launches, clocks=clk.summary(), final=final)

    def e2e(precision):
        """The step through the C ABI from host memory, pipelined as a caller
        that streams states in and rates out would run it: each step uploads
        its state from pinned host memory (rt_set_state_async, on the
        library's upload stream, while the previous step's kernels run),
        traces, updates, and reads k_ph (the path's precision) and x_HI (FP64)
        back into pinned host buffers (rt_get_rates_async); before enqueueing
        the read-back the host waits for the previous step's copies
        (rt_wait_rates), so one step's results are on the host while the next
        runs.  The timed region ends when the last step's results are on the
        host."""
        grid = native.Grid(ctx, g, precision, stream=stream.cuda_stream)
        b = grid.trace(**params)
        qp = dict(params, queue_capacity=queue_capacity_for(b, params["level0"]))
        n = grid.ncell
        hx = torch.tensor(g["x_HI"], dtype=torch.float64).pin_memory()
        hz = torch.tensor(g["x_HII"], dtype=torch.float64).pin_memory()
        kdt = native.RT_DTYPE_F64 if precision == "fp64" else native.RT_DTYPE_F32
        kt = torch.float64 if precision == "fp64" else torch.float32
        hk = [torch.empty(n, dtype=kt).pin_memory() for _ in range(2)]
        hxo = [torch.empty(n, dtype=torch.float64).pin_memory() for _ in range(2)]
        lib = native.lib()
        warm = max(3, args.warmup)
        t0 = None
        for i in range(warm + args.steps):
            if i == warm:
                native.rt_synchronize(grid.h)
                t0 = time.perf_counter()
            native.check(lib.rt_set_state_async(grid.h, None, hx.data_ptr(), hz.data_ptr(), native.RT_MEM_HOST))
            grid.trace(sync=False, **qp)
            grid.chem(DT_S, 10, synth.ALPHA_B)
            native.check(lib.rt_wait_rates(grid.h))
            native.check(lib.rt_get_rates_async(grid.h, hk[i % 2].data_ptr(), None, None, kdt, native.RT_MEM_HOST))
            native.check(lib.rt_get_rates_async(grid.h, None, None, hxo[i % 2].data_ptr(), native.RT_DTYPE_F64,
                                                native.RT_MEM_HOST))
        native.rt_synchronize(grid.h)
        dt = time.perf_counter() - t0
        last = native.rt_get_budget(grid.h)
        assert last["segments"] == b["segments"], (last["segments"], b["segments"])
        # the last step's read-back is the one-step result of the snapshot
        ref = grid.rates(dtype=kdt)
        assert np.array_equal(hk[(warm + args.steps - 1) % 2].numpy(), np.asarray(ref["kph"]))
        grid.close()
        return dict(value=b["segments"] * args.steps / dt, h2d=2 * n * 8, d2h=n * (hk[0].element_size() + 8),
                    ms_per_step=1e3 * dt / args.steps)

    res = {}
    for prec in args.precisions:
        res[prec] = measure(prec)
    head = args.precisions[0]
    r = res[head]
    total_s = sum(r["step_ms"]) / 1e3
    kern_s = sum(r["kern_ms"]) / 1e3
    # the slowest rank's time, the work of all ranks
    total_s, all_segments = reduce_over_ranks(total_s, r["segments"])
    value = all_segments / total_s
    ee = e2e(head) if not args.no_e2e else dict(value=None, h2d=0, d2h=0)
    peaks, peak_kind = _peaks()
    wtag = "clumpy256" if args.workload == "clumpy" else f"stromgren{args.grid}"
    traffic = _profiled_traffic(head, wtag)
    red = red_peak(native, local, head, int(np.prod(g["dims"])))
    gamma = bool(np.any(np.asarray(g["e_ph_eV"]) > 13.6))
    if args.workload == "clumpy":
        wl = WORKLOAD_CLUMPY
    else:
        wl = WORKLOAD if args.grid == 128 else WORKLOAD.replace("128^3", f"{args.grid}^3")
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": 1e3 * total_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if head == "fp64" else "f32", "data": "synthetic",
        "config": {"workload": wl,
                   "precision": head, "segments_per_step": r["seg_per_step"],
                   "queue_records_per_step": r["pushed"], "l2": "flushed (512 MB write) between steps",
                   "parallelism": f"replicas x{world}"},
        "roofline": trace_roofline(head, r["seg_per_step"], r["pushed"], 1e3 * kern_s / args.steps, gamma,
                                   red, peaks, peak_kind, traffic),
        "e2e": {"value": ee["value"], "unit": UNIT, "h2d_bytes_per_step": ee["h2d"],
                "d2h_bytes_per_step": ee["d2h"], "ms_per_step": ee.get("ms_per_step"),
                "how": "C ABI, pinned host buffers, rt_set_state_async / rt_get_rates_async pipelined "
                       "one step deep"},
        "gpu_launches": int(r["launches"]),
        "clocks": r["clocks"],
    }
    for prec in args.precisions[1:]:
        q = res[prec]
        out[f"{prec}_path"] = {"value": q["segments"] * world / (sum(q["step_ms"]) / 1e3),
                               "ms_per_step": sum(q["step_ms"]) / args.steps,
                               "kernel_ms": sum(q["kern_ms"]) / args.steps}
    # the same step with the covering-factor correction of Sec. 2.3 (optional)
    if not args.no_fc:
        q = measure(head, fc=True)
        out["fc_path"] = {"value": q["segments"] / (sum(q["step_ms"]) / 1e3),
                          "ms_per_step": sum(q["step_ms"]) / args.steps,
                          "kernel_ms": sum(q["kern_ms"]) / args.steps, "precision": head}
    # the adaptive RT timestep of Sec. 3.4 on the same state (one synchronous call)
    if not args.no_timestep:
        grid = native.Grid(ctx, g, head, stream=stream.cuda_stream)
        grid.trace(**params)
        t = []
        for i in range(8):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            dt_p = native.rt_timestep(grid.h, eps_ion=0.05, dt_max=DT_S)
            t.append(time.perf_counter() - t0)
        grid.close()
        cells = int(np.prod(g["dims"]))
        ms = 1e3 * float(np.median(t[3:]))
        # per cell: n_H, x_HI (FP64), k_ph read, the per-cell value written and read back
        out["timestep"] = {"ms": ms, "dt_s": dt_p, "cells": cells,
                           "gb_s": cells * (8 + 8 + (8 if head == "fp64" else 4) + 4 + 4) / (ms / 1e3) / 1e9}
    # the clumpy multi-source configuration: 256^3, 1000 sources, one trace per step
    if not args.no_clumpy and args.workload != "clumpy":
        out["clumpy256"] = clumpy_leg(args, ctx, stream, flush, head, peaks, peak_kind, local)
    # photon types (Sec. 3.2): the clumpy configuration with H I, He I and He II sources
    if not args.no_types:
        out["photon_types"] = photon_types(args, ctx, stream, flush, head)
    # finite speed of light: the Application 5 pulse (Sec. 9)
    if not args.no_fsl:
        out["finite_light"] = finite_light(args, ctx, stream, flush, head)
    # the batched and serving configurations are measured on one GPU
    if not args.no_batched and world == 1:
        out["batched"] = batched(args, ctx, stream, dev, world)
    if not args.no_serving and world == 1:
        out["serving"] = serving(args, ctx)
    # the Strömgren convergence run: 500 Myr of coupled steps from the neutral medium
    if not args.no_convergence:
        out["stromgren_500myr"] = stromgren_500myr(ctx, stream, args.precisions)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        bench_step = args.workload == "stromgren" and args.grid == 128
        out["cpu_baseline"], ref = cpu_baseline(args.cpu_seconds)
        if bench_step:
            out["precision_error"] = precision_error(g, ref, {p: res[p]["final"] for p in args.precisions})
    return out


def run_partition(args, rank, world, local):
    """One large grid shared by the ranks by sources (the clumpy 256^3
    configuration, 1000 sources): each rank holds the whole medium, traces its
    contiguous share of the sources, the ranks sum k_ph, Gamma (FP32) and the
    photon budget with one all-reduce per trace (NCCL), and every rank runs
    the same update.  The timed step includes the exchange; the state is
    restored (untimed) before each step.  Total work is fixed as ranks are
    added (strong scaling)."""
    import torch
    from paper_1012_2865_gb300 import build, native, shard, synth
    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ctx = native.rt_ctx_create(local)
    g = synth.clumpy()
    prec = args.precisions[0]
    sg = shard.ShardGrid(ctx, g, prec, rank, world)
    x0 = torch.tensor(g["x_HI"], dtype=torch.float64, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    params = dict(synth.DEFAULT_PARAMS)
    sg.step(DT_S, 10, synth.ALPHA_B, **params)  # sizes the queue
    for _ in range(max(3, args.warmup)):
        native.rt_set_state(sg.grid.h, x0)
        sg.step(DT_S, 10, synth.ALPHA_B, **params)
    total_s, segs = 0.0, 0
    torch.cuda.synchronize()
    barrier()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            native.rt_set_state(sg.grid.h, x0)
            flush.zero_()
            torch.cuda.synchronize()
            barrier()
            t0 = time.perf_counter()
            b = sg.step(DT_S, 10, synth.ALPHA_B, **params)
            torch.cuda.synchronize()
            total_s += time.perf_counter() - t0
            segs += b["segments"]
    barrier()
    # the slowest rank's time; every rank already holds the whole trace's segments
    t_max, _ = reduce_over_ranks(total_s, 0)
    sg.close()
    return {"metric": METRIC, "value": segs / t_max, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f64" if prec == "fp64" else "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD_CLUMPY, "precision": prec, "segments_per_step": segs // args.steps,
                       "parallelism": f"sources partitioned over {world} ranks; one all-reduce of k_ph, Gamma and "
                                      "the photon budget per trace",
                       "l2": "flushed (512 MB write) between steps"},
            "e2e": {"value": None, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0,
                    "note": "device-resident mode; see the default run for the end-to-end figure"},
            "clocks": clk.summary(), "gpu_launches": None}


def stromgren_500myr(ctx, stream, precisions) -> dict:
    """Test 1 at 128^3 evolved over 500 Myr (1000 steps of trace + update, dt 0.5 Myr)
    in each precision: the volume-equivalent I-front radius against the closed form
    R_s = (3 Ndot / (4 pi alpha_B n_H^2))^(1/3) (Eq. Rstr; the analytic r_s(500 Myr)
    is 0.9944 R_s), the two precisions against each other, and the device time of
    the whole evolution."""
    import torch
    from paper_1012_2865_gb300 import native, synth
    N = 128
    g = synth.stromgren(N)
    V = (g["box_len_cm"] / N) ** 3
    rs = (3 * g["ndot"][0] / (4 * np.pi * synth.ALPHA_B * 1e-3 ** 2)) ** (1 / 3)
    out, state = {"workload": "stromgren-128^3 from neutral, 1000 steps of 0.5 Myr",
                  "R_s_cm": rs, "r_s_500myr_over_R_s": (1.0 - np.exp(-500 * synth.MYR_S * synth.ALPHA_B * 1e-3)) ** (1 / 3)}, {}
    for prec in precisions:
        grid = native.Grid(ctx, g, prec, stream=stream.cuda_stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(1000):
            grid.trace(sync=False, queue_capacity=1 << 22, **synth.DEFAULT_PARAMS)
            grid.chem(DT_S, 10, synth.ALPHA_B)
        e1.record(stream)
        e1.synchronize()
        b = native.rt_get_budget(grid.h)
        z = grid.x_HII()
        r_if = (6 * float(np.sum(z)) * V / np.pi) ** (1 / 3)
        state[prec] = grid.rates()
        out[prec] = {"R_IF_over_R_s": r_if / rs, "evolve_s": e0.elapsed_time(e1) / 1e3,
                     "status": b["status"], "last_step_segments": b["segments"]}
        grid.close()
    if "fp32_mixed" in state and "fp64" in state:
        a, c = state["fp32_mixed"], state["fp64"]
        pos = c["x_HI"] > 0
        rx = np.abs(a["x_HI"][pos] - c["x_HI"][pos]) / c["x_HI"][pos]
        out["fp32_mixed_vs_fp64"] = {
            "R_IF_rel": out["fp32_mixed"]["R_IF_over_R_s"] / out["fp64"]["R_IF_over_R_s"] - 1.0,
            "x_HI_max_rel": float(rx.max()), "x_HI_median_rel": float(np.median(rx))}
    return out


def precision_error(g, ref, final) -> dict:
    """Each GPU path's k_ph and x_HI after one benchmark step against the FP64 oracle's
    step from the same snapshot: k_ph in the cells receiving more than 1e-8 of the
    emitted photons (photon path length k_ph dx^2 / sigma), x_HI in every cell.
    Gamma is zero on this workload (13.6 eV photons)."""
    dx = g["box_len_cm"] / g["dims"][0]
    kph_o, x_o, emitted = ref
    m = kph_o * dx * dx / float(np.max(g["sigma_cm2"])) > 1e-8 * emitted
    out = {"vs": "FP64 C oracle, the same step from the same snapshot", "cells_compared_kph": int(m.sum())}
    for prec, r in final.items():
        rk = np.abs(r["kph"][m] - kph_o[m]) / kph_o[m]
        pos = x_o > 0
        rx = np.abs(r["x_HI"][pos] - x_o[pos]) / x_o[pos]
        out[prec] = {"kph_max_rel": float(rk.max()), "kph_median_rel": float(np.median(rk)),
                     "x_HI_max_rel": float(rx.max()), "x_HI_median_rel": float(np.median(rx))}
    return out


def clumpy_leg(args, ctx, stream, flush, precision, peaks, peak_kind, local) -> dict:
    """The clumpy multi-source configuration (256^3 log-normal medium, 1000
    sources, Ndot log-uniform in [1e48, 1e50], 13.6-29.6 eV; HEALPix level 1,
    Phi_c 5.1, f_term 1e-10, FP32-mixed, FP32 rate grids): one rt_trace per
    timed step, L2 flushed between steps, with the trace kernel's HBM and L2
    reduction rooflines."""
    import torch
    from paper_1012_2865_gb300 import native, synth
    g = synth.clumpy()
    grid = native.Grid(ctx, g, precision, stream=stream.cuda_stream)
    params = dict(synth.DEFAULT_PARAMS)
    b = grid.trace(**params)  # sizes the queue
    qp = dict(params, queue_capacity=queue_capacity_for(b, params["level0"]))
    for _ in range(max(3, args.warmup)):
        grid.trace(sync=False, **qp)
    torch.cuda.synchronize()
    steps = max(3, args.steps // 2)
    step_ms, kern_ms, launches = [], [], 0
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        l0 = native.rt_kernel_launches()
        e0.record(stream)
        grid.trace(sync=False, **qp)
        e1.record(stream)
        e1.synchronize()
        launches += native.rt_kernel_launches() - l0
        bb = native.rt_get_budget(grid.h)
        assert bb["segments"] == b["segments"]
        step_ms.append(e0.elapsed_time(e1))
        kern_ms.append(bb["kernel_ms"])
    grid.close()
    red = red_peak(native, local, precision, int(np.prod(g["dims"])))
    t = sum(step_ms) / 1e3
    km = sum(kern_ms) / steps
    return {"workload": WORKLOAD_CLUMPY.replace(" + rt_chem_update (0.5 Myr, 10 substeps)", ""),
            "value": b["segments"] * steps / t, "unit": UNIT, "ms_per_step": 1e3 * t / steps,
            "segments_per_step": b["segments"], "queue_records_per_step": b["queue_pushed"],
            "precision": precision, "gpu_launches": int(launches), "l2": "flushed (512 MB write) between steps",
            "roofline": trace_roofline(precision, b["segments"], b["queue_pushed"], km, True, red, peaks,
                                       peak_kind, _profiled_traffic(precision, "clumpy256"))}


def photon_types(args, ctx, stream, flush, precision) -> dict:
    """Photon types (Sec. 3.2) on a clumpy 128^3 medium: 30 sources cycling
    through H I, He I and He II ionising photons, each absorbed by its own
    species (helium at 0.079 n_H, 90 % He I, so He II photons cross most of
    the box); each timed step traces and updates from the neutral initial
    state (restored untimed)."""
    import torch
    from paper_1012_2865_gb300 import native, synth

    g = synth.typed_clumpy()
    grid = native.Grid(ctx, g, precision, stream=stream.cuda_stream)
    grid.set_absorbers(g["n_he"][0], g["n_he"][1])
    grid.set_source_types(g["types"])
    params = dict(synth.DEFAULT_PARAMS)
    b = grid.trace(**params)  # sizes the queue
    qp = dict(params, queue_capacity=queue_capacity_for(b, params["level0"]))
    x0 = torch.tensor(g["x_HI"], dtype=torch.float64, device=stream.device)
    for _ in range(max(3, args.warmup)):
        native.rt_set_state(grid.h, x0)
        grid.trace(sync=False, **qp)
        grid.chem(DT_S, 10, synth.ALPHA_B)
    torch.cuda.synchronize()
    step_ms, kern_ms, segs, launches = [], [], 0, 0
    for _ in range(args.steps):
        native.rt_set_state(grid.h, x0)
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        l0 = native.rt_kernel_launches()
        e0.record(stream)
        grid.trace(sync=False, **qp)
        grid.chem(DT_S, 10, synth.ALPHA_B)
        e1.record(stream)
        e1.synchronize()
        launches += native.rt_kernel_launches() - l0
        bb = native.rt_get_budget(grid.h)
        step_ms.append(e0.elapsed_time(e1))
        kern_ms.append(bb["kernel_ms"])
        segs += bb["segments"]
    grid.close()
    t = sum(step_ms) / 1e3
    return {"value": segs / t, "unit": UNIT, "ms_per_step": 1e3 * t / args.steps,
            "kernel_ms": sum(kern_ms) / args.steps, "segments_per_step": segs // args.steps,
            "precision": precision, "gpu_launches": int(launches),
            "workload": "typed-clumpy-128^3: clumpy medium, 30 sources cycling H I / He I / He II ionising "
                        "(E_i..E_i+16 eV, threshold cross sections), n_He = 0.079 n_H (90 % He I); "
                        "step = rt_trace + rt_chem_update from the neutral state",
            "l2": "flushed (512 MB write) between steps"}


def finite_light(args, ctx, stream, flush, precision) -> dict:
    """Application 5 (Sec. 9, Eq. "test12") with a finite speed of light
    (Sec. 2.1, Step 3j): a 1 Mpc box of 128^3 cells, optically thin, a corner
    source whose rate pulses with period 0.5 Myr, radiative-transfer timestep
    50 kyr (light crosses 1.96 cells per step).  After 6 Myr of steps
    (untimed; light has crossed the box diagonal, so packages of every age
    are in flight) each timed step sets the source's rate, traces (continuing
    every package in flight and halting them again c dt_P further on) and
    updates the chemistry."""
    import torch
    from paper_1012_2865_gb300 import native, synth

    g = synth.pulse(128)
    dt, light = g["dt_s"], g["light_cm"]
    grid = native.Grid(ctx, g, precision, stream=stream.cuda_stream)
    params = dict(synth.DEFAULT_PARAMS, light_cm=light)
    fill = int(round(6.0 * synth.MYR_S / dt))
    for n in range(fill):
        grid.set_source_rates([float(synth.pulse_rate(n * dt))])
        grid.trace(**params)  # synchronous: sizes the queue and the stores of packages in flight
        grid.chem(dt, 10, synth.ALPHA_B)
    torch.cuda.synchronize()
    step_ms, kern_ms, segs, moved, pushed = [], [], 0, 0, 0
    launches = 0
    for k in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        l0 = native.rt_kernel_launches()
        e0.record(stream)
        grid.set_source_rates([float(synth.pulse_rate((fill + k) * dt))])
        grid.trace(sync=False, **params)
        grid.chem(dt, 10, synth.ALPHA_B)
        e1.record(stream)
        e1.synchronize()
        launches += native.rt_kernel_launches() - l0
        bb = native.rt_get_budget(grid.h)
        step_ms.append(e0.elapsed_time(e1))
        kern_ms.append(bb["kernel_ms"])
        segs += bb["segments"]
        moved += bb["n_resumed"] + bb["n_halted"]
        pushed += bb["queue_pushed"]
    grid.close()
    t = sum(step_ms) / 1e3
    kt = sum(kern_ms) / 1e3
    # algorithmic bytes: per segment the n_HI pair read and the k_ph and Gamma
    # reductions; 48 bytes per package continued or halted; 96 per queue record
    red = 8 if precision == "fp64" else 4
    alg = segs * (8 + 2 * red) + moved * 48 + pushed * 96
    return {"value": segs / t, "unit": UNIT, "ms_per_step": 1e3 * t / args.steps,
            "kernel_ms": 1e3 * kt / args.steps, "segments_per_step": segs // args.steps,
            "in_flight_per_step": moved // (2 * args.steps), "queue_records_per_step": pushed // args.steps,
            "algorithmic_bytes_per_step": alg // args.steps, "precision": precision,
            "trace_gb_s": alg / kt / 1e9, "gpu_launches": int(launches),
            "workload": "application5-pulse-128^3: 1 Mpc box, n_H 1e-4, x_HI 1e-5, corner source "
                        "L(t) of Eq. test12 (1e55 ph/s, t0 0.5 Myr, A 4), dt_P 50 kyr, timed after 6 Myr",
            "l2": "flushed (512 MB write) between steps"}


def batched(args, ctx, stream, dev, world, n_grids=64, tune=True, warm=None):
    """Batched configuration: 64 grids (sides 32-192, 1-256 sources) per launch,
    autotuned, one coupled step captured as a CUDA graph.  (n_grids, tune and
    warm shrink it for a profiler capture: the first n_grids grids of the same
    draw, 8 segments per queue visit and 2 blocks per SM, `warm` warm-up steps.)"""
    import torch
    from paper_1012_2865_gb300 import native, synth
    gs = synth.batch(64)[:n_grids]
    b = native.Batch(ctx, stream.cuda_stream)
    grids = [native.Grid(ctx, g, "fp32_mixed") for g in gs]
    slots = [b.add(gr) for gr in grids]
    # every timed step is the first coupled step from the initial conditions:
    # the neutral state is restored from device copies (untimed) before each
    # step, so that all steps do the same work (traces grow by ~1.4x per step
    # as the media ionise)
    x0 = [torch.tensor(g["x_HI"], dtype=torch.float64, device=dev) for g in gs]

    def restore():
        for gr, x in zip(grids, x0):
            native.rt_set_state(gr.h, x)
        torch.cuda.synchronize()

    if tune:
        p = native.rt_batch_autotune(b.h, native.trace_params(**synth.DEFAULT_PARAMS))
    else:
        p = native.trace_params(**dict(synth.DEFAULT_PARAMS, segs_per_iter=8, blocks_per_sm=2))
    tuned = dict(synth.DEFAULT_PARAMS, segs_per_iter=p.segs_per_iter, blocks_per_sm=p.blocks_per_sm)
    for _ in range(max(3, args.warmup) if warm is None else warm):
        restore()
        b.step(1, DT_S, 10, synth.ALPHA_B, **tuned)  # the first call captures the graph
    torch.cuda.synchronize()
    steps = max(3, args.steps // 2)
    ms, segs, launches, kms, pushed = 0.0, 0, 0, 0.0, 0
    for _ in range(steps):  # one graph replay per timed step, exact segments per step
        restore()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        l0 = native.rt_kernel_launches()
        e0.record(stream)
        b.step(1, DT_S, 10, synth.ALPHA_B, **tuned)
        e1.record(stream)
        e1.synchronize()
        launches += native.rt_kernel_launches() - l0
        ms += e0.elapsed_time(e1)
        buds = [b.budget(s) for s in slots]
        segs += sum(bb["segments"] for bb in buds)
        pushed += buds[0]["queue_pushed"]
    # the trace launch's own duration for the roofline (a graph replay does not
    # time its events): the same trace enqueued without the graph, after the
    # timed steps
    tms = []
    for _ in range(3):
        restore()
        b.trace(sync=True, **tuned)
        tms.append(b.budget(slots[0])["kernel_ms"])
    kms = float(np.median(tms)) * steps
    cells = sum(int(np.prod(g["dims"])) for g in gs)
    b.close()
    for gr in grids:
        gr.close()
    peaks, peak_kind = _peaks()
    red = red_peak(native, dev.index or 0, "fp32_mixed", cells)
    return {"workload": f"{n_grids} grids, sides from {{32,48,64,96,128,192}}, 1-256 sources, log-normal medium, "
                        "neutral; one CUDA-graph step = zero + emit + trace + update (0.5 Myr), the neutral "
                        "state restored (untimed) before each step",
            "value": segs * world / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps,
            "segments_per_step": segs // steps, "cells": cells, "gpu_launches": int(launches),
            "queue_records_per_step": pushed // steps, "trace_ms": kms / steps,
            "autotuned": {"segs_per_iter": p.segs_per_iter, "blocks_per_sm": p.blocks_per_sm},
            "l2": "inputs larger than L2 (no flush)",
            "roofline": trace_roofline("fp32_mixed", segs // steps, pushed // steps, kms / steps, True, red,
                                       peaks, peak_kind, _profiled_traffic("fp32_mixed", f"batch{n_grids}"))}


def serving(args, ctx):
    """The serving configuration as stated: a Poisson stream at 200 requests/s
    for its args.serve_seconds of arrivals (grids 64^3-256^3 log-uniform in
    cells, 1-500 sources, 1-20 coupled steps of 0.5 Myr from neutral), served
    live by FP32-mixed continuous batching and stopped at the end of the
    arrivals.  The offered load exceeds one GB300 many times over, so the
    report says what happens to the stream in that time: requests completed
    (p50/p99 latency over them), still queued, in progress, rejected or
    failed, and the service capacity -- completions per second with the queue
    never empty, the highest arrival rate the server sustains.  Then the first
    args.serve_fp64_requests requests of the same stream are served live, one
    at a time, on the plain FP64 path (the reference server), beside their
    latencies in the batched run."""
    from paper_1012_2865_gb300 import serve, synth
    specs = synth.request_stream(rate_hz=200.0, duration_s=args.serve_seconds)
    pool = serve.MediumPool()
    reqs = [pool.request(sp, i, lazy=True) for i, sp in enumerate(specs)]
    srv = serve.Server(ctx, "fp32_mixed", max_slots=64)
    rep = srv.run(reqs, time_limit_s=args.serve_seconds)
    srv.close()
    first = [pool.request(sp, i) for i, sp in enumerate(specs[:args.serve_fp64_requests])]
    ref = serve.serve_one_at_a_time(ctx, first, "fp64", time_limit_s=args.serve_fp64_budget_s)
    mixed_lat = {r.rid: r.latency for r in srv.done}
    same = [mixed_lat[i] for i in ref["rids"] if i in mixed_lat]
    return {"workload": f"Poisson stream at 200 req/s, {args.serve_seconds:.0f} s of arrivals ({len(specs)} "
                        "requests), 64^3-256^3 log-uniform cells, 1-500 sources, 1-20 coupled steps of 0.5 Myr "
                        "from neutral; served live, stopped at the end of the arrivals",
            "value": rep["segments_per_s"], "unit": UNIT, "p50_ms": rep["p50_ms"], "p99_ms": rep["p99_ms"],
            "latency_over": "completed requests", "arrived": len(specs) - rep["not_arrived"],
            "completed": rep["completed"], "queued": rep["queued"], "in_progress": rep["in_progress"],
            "failed": rep["failed"], "rejected": rep["rejected"],
            "requests_per_s": rep["requests_per_s"],
            "capacity_req_per_s": rep["requests_per_s"],
            "capacity_note": "highest arrival rate the server sustains: completions per second while the "
                             "queue was never empty",
            "wall_s": rep["wall_s"], "segments": rep["segments"], "batch_steps": rep["steps"],
            "fp64_one_at_a_time": {"requests": ref["completed"], "how": "live, arrival order, one grid at a time",
                                   "p50_ms": ref["p50_ms"], "p99_ms": ref["p99_ms"],
                                   "service_s_total": float(np.sum(ref["service_s"])),
                                   "fp32_mixed_batched_same_requests_p50_ms":
                                       float(np.percentile(same, 50) * 1e3) if same else None,
                                   "fp32_mixed_batched_same_requests_p99_ms":
                                       float(np.percentile(same, 99) * 1e3) if same else None}}


def oracle_step(g, x, z):
    """One step of the oracle: (segments, k_ph, x_HI after the update, emitted)."""
    import oracle
    from paper_1012_2865_gb300 import synth
    o = oracle.trace(g["dims"], g["box_len_cm"], g["n_H"], x, g["pos_cm"], g["ndot"], g["e_ph_eV"],
                     g["sigma_cm2"], **synth.DEFAULT_PARAMS)
    x1, _ = oracle.chem(g["n_H"], x, z, o["kph"], DT_S, 10, synth.ALPHA_B)
    return o["segments"], o["kph"], x1, o["budget"][0]


def host_threads() -> int:
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def oracle_step_threads(g, x, z, threads: int):
    """One step of the oracle shared by `threads` host threads: each takes root
    packages one at a time from a shared counter and traces them
    (oracle.trace_roots) into its own k_ph (thread-private), the partial fields
    are summed at the end, and the update runs on equal cell ranges.  Returns
    (segments, k_ph, x_HI after the update, emitted)."""
    from concurrent.futures import ThreadPoolExecutor
    import oracle
    from paper_1012_2865_gb300 import synth
    p = synth.DEFAULT_PARAMS
    nroots = len(g["ndot"]) * 12 * 4 ** p["level0"]
    lock = threading.Lock()
    nxt = [0]

    def work(_):
        acc, segs, emitted = None, 0, 0.0
        while True:
            with lock:
                r = nxt[0]
                nxt[0] += 1
            if r >= nroots:
                return acc, segs, emitted
            o = oracle.trace_roots(g["dims"], g["box_len_cm"], g["n_H"], x, g["pos_cm"], g["ndot"], g["e_ph_eV"],
                                   g["sigma_cm2"], r, 1, **p)
            if acc is None:
                acc = o["kph"]
            else:
                np.add(acc, o["kph"], out=acc)
            segs += o["segments"]
            emitted += float(o["budget"][0])

    with ThreadPoolExecutor(threads) as ex:
        parts = list(ex.map(work, range(threads)))
        kph = np.zeros(int(np.prod(g["dims"])))
        for acc, _, _ in parts:
            if acc is not None:
                kph += acc
        n = kph.size
        cuts = [n * i // threads for i in range(threads + 1)]
        upd = list(ex.map(lambda i: oracle.chem(g["n_H"][cuts[i]:cuts[i + 1]], x[cuts[i]:cuts[i + 1]],
                                                z[cuts[i]:cuts[i + 1]], kph[cuts[i]:cuts[i + 1]], DT_S, 10,
                                                synth.ALPHA_B)[0], range(threads)))
    return sum(q[1] for q in parts), kph, np.concatenate(upd), sum(q[2] for q in parts)


def cpu_baseline(seconds: float):
    """The oracle timed on the benchmark step on the machine's host cores: shared by
    one thread per core over the root packages (thread-private k_ph, summed),
    and, beside it, on one thread.  Also returns the first step's (k_ph, x_HI,
    emitted) for the precision report."""
    from paper_1012_2865_gb300 import synth
    g = synth.stromgren_snapshot(128)
    threads = host_threads()

    def timed(step, budget):
        segs, n, first = 0, 0, None
        t0 = time.perf_counter()
        while True:
            s, kph, x1, em = step()
            segs += s
            first = first or (kph, x1, em)
            n += 1
            if time.perf_counter() - t0 >= budget:
                return segs / (time.perf_counter() - t0), n, time.perf_counter() - t0, first

    v1, n1, t1, ref = timed(lambda: oracle_step(g, g["x_HI"], g["x_HII"]), seconds / 2)
    vt, nt, tt, _ = timed(lambda: oracle_step_threads(g, g["x_HI"], g["x_HII"], threads), seconds / 2)
    return ({"value": vt, "unit": UNIT, "cores": threads, "kind": "oracle",
             "sample": f"{nt} full steps of the bench workload, FP64 C oracle shared by {threads} host threads "
                       f"over the root packages (thread-private k_ph, summed), {tt:.1f} s",
             "single_thread": {"value": v1, "cores": 1, "sample": f"{n1} full steps, {t1:.1f} s"}}, ref)


def run_reference(args, rank, world):
    """The reference arm: the FP64 oracle on the benchmark step, shared by one
    thread per host core over the root packages."""
    if rank != 0:
        return None
    from paper_1012_2865_gb300 import synth
    import oracle
    oracle.build()
    g = synth.stromgren_snapshot(128)
    threads = host_threads()
    for _ in range(args.warmup):
        oracle_step_threads(g, g["x_HI"], g["x_HII"], threads)
    segs = 0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        segs += oracle_step_threads(g, g["x_HI"], g["x_HII"], threads)[0]
    dt = time.perf_counter() - t0
    v = segs / dt
    return {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference", "config": {"workload": WORKLOAD, "precision": "fp64 oracle"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{args.steps} full steps of the bench workload, shared by {threads} host "
                                       "threads over the root packages"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--precisions", default="fp32_mixed,fp64")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-fc", action="store_true", help="skip the covering-factor (Sec. 2.3) leg")
    ap.add_argument("--no-timestep", action="store_true", help="skip the adaptive-timestep (Sec. 3.4) leg")
    ap.add_argument("--no-fsl", action="store_true", help="skip the finite-speed-of-light (Application 5) leg")
    ap.add_argument("--no-types", action="store_true", help="skip the photon-types (Sec. 3.2) leg")
    ap.add_argument("--no-clumpy", action="store_true", help="skip the clumpy 256^3, 1000-source leg")
    ap.add_argument("--profile-batched", type=int, default=0, metavar="N",
                    help="run only the batched leg on its first N grids (fixed tuning, one warm-up step), "
                         "for a profiler capture")
    ap.add_argument("--partition", default="replicas", choices=["replicas", "sources"],
                    help="replicas: one independent problem per rank (default); sources: the clumpy 256^3 grid "
                         "shared by the ranks by sources, one all-reduce per trace")
    ap.add_argument("--no-convergence", action="store_true",
                    help="skip the 500 Myr Strömgren evolution in each precision")
    ap.add_argument("--serve-seconds", type=float, default=60.0, help="arrival window of the serving stream")
    ap.add_argument("--serve-fp64-requests", type=int, default=8,
                    help="first requests of the stream served one at a time on the FP64 path")
    ap.add_argument("--serve-fp64-budget-s", type=float, default=40.0)
    ap.add_argument("--grid", type=int, default=128, help="cells per side (128 = the benchmark workload)")
    ap.add_argument("--workload", default="stromgren", choices=["stromgren", "clumpy"],
                    help="stromgren: the benchmark workload; clumpy: the 256^3 multi-source case (profiling)")
    args = ap.parse_args()
    args.precisions = [p.strip() for p in args.precisions.split(",") if p.strip()]
    rank, world, local = _dist()
    if args.profile_batched:
        # a profiler's capture of the batched trace on a smaller batch: the
        # trace launches are the sizing trace, one warm-up replay, then the
        # timed replays
        import torch
        from paper_1012_2865_gb300 import build, native
        build.build()
        torch.cuda.set_device(local)
        ctx = native.rt_ctx_create(local)
        stream = torch.cuda.current_stream()
        print(json.dumps(batched(args, ctx, stream, torch.device("cuda", local), 1, n_grids=args.profile_batched,
                                 tune=False, warm=1)), flush=True)
        return
    if args.impl == "reference":
        out = run_reference(args, rank, world)
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
        dist.barrier()
    out = run_partition(args, rank, world, local) if args.partition == "sources" else \
        run_native(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
