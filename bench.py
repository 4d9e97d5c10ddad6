#!/usr/bin/env python3
"""Throughput of the 2D/3D type 1 + type 2 NUFFT hot path on GB300.

One step = the whole hot path over one batch of synthetic points: for a type 1
plan and a type 2 plan on the same M points, setpts (bin-sort) then execute
(spread -> cuFFT -> deconvolve, and precorrect -> cuFFT -> interpolate).
value = nonuniform points transformed per second over both plans
        (2 * M * ntransf per step), inputs resident in HBM, L2 flushed between steps;
        the two plans run on two streams (their kernels may overlap); the one-stream
        form is reported as "serial".
e2e   = the same through the public API with host buffers: pinned host->device
        copies of x, y(, z), c, f and device->host copies of both results inside
        the timed region (two streams; "serial" inside it is the one-stream form).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                       [--impl reference]
Under torchrun (N > 1) every rank runs an independent replica on its own GPU
(the transform has no exchange step); value sums the ranks' points over the
slowest rank's time.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2102_08463_gb300 import workloads as wl  # noqa: E402

UNIT = "points/s"


def metric_for(W):
    """The headline metric's name for a workload (its tolerance and precision)."""
    return "NU points/sec (spread/interp and full exec) at eps=%g %s" % (
        W["eps"], "fp32" if W["prec"] == 0 else "fp64")

WORKLOADS = {
    "2d-1024-rand-eps1e-5": dict(dim=2, N=(1024, 1024), M=4194304, eps=1e-5, prec=0, kind="rand"),
    "2d-1024-rand-eps1e-2": dict(dim=2, N=(1024, 1024), M=4194304, eps=1e-2, prec=0, kind="rand"),
    "2d-1024-rand-eps1e-9": dict(dim=2, N=(1024, 1024), M=4194304, eps=1e-9, prec=1, kind="rand"),
    "2d-1024-rand-eps1e-12": dict(dim=2, N=(1024, 1024), M=4194304, eps=1e-12, prec=1, kind="rand"),
    "3d-128-rand-eps1e-2": dict(dim=3, N=(128, 128, 128), M=16777216, eps=1e-2, prec=0, kind="rand"),
    "3d-128-rand-eps1e-6": dict(dim=3, N=(128, 128, 128), M=16777216, eps=1e-6, prec=0, kind="rand"),
    "3d-128-gauss-eps1e-2": dict(dim=3, N=(128, 128, 128), M=16777216, eps=1e-2, prec=0, kind="gauss"),
    "3d-128-gauss-eps1e-6": dict(dim=3, N=(128, 128, 128), M=16777216, eps=1e-6, prec=0, kind="gauss"),
    "2d-64-rand-eps1e-5": dict(dim=2, N=(64, 64), M=4096, eps=1e-5, prec=0, kind="rand"),
    # reduced 3D case for kernel captures: the same kernels and tiles at a quarter of the points
    "3d-128-rand-eps1e-6-m4m": dict(dim=3, N=(128, 128, 128), M=4194304, eps=1e-6, prec=0, kind="rand"),
}
DEFAULT_WORKLOAD = "2d-1024-rand-eps1e-5"
SEED = wl.BASE_SEED + 1

# Roofline denominators.  HBM: the measured copy bandwidth of this GPU pool
# (MEASURED_PEAKS.json), else 6800 GB/s.  FP32 ALU: the device's SM count (queried)
# x 128 FP32 lanes x 2 flop x the maximum SM clock (MEASURED_PEAKS.json, else
# 2070 MHz).  FP64 ALU: the FMA rate measured on the device by the library's
# nufft_fma_peak kernel (the FP64 unit count per SM is not published for this GPU).
FP32_LANES_PER_SM = 128

# DRAM traffic per launch from ncu captures (dram__bytes_read.sum +
# dram__bytes_write.sum), keyed by kernel and workload, with the hash of the
# kernel sources at capture time; a stale hash reports null.
TRAFFIC = {
    # dram__bytes_read.sum + dram__bytes_write.sum of one launch (ncu --metrics ... -k
    # regex:"spread_sweep2|interp_warp2" -c 2 on the bench command of
    # profiles/launches_2d-1024-rand-eps1e-5.md; the 3D rows on --workload 3d-128-rand-eps1e-6
    # with -k regex:"spread_sweep3|interp_planes3"; see profiles/traffic_2d-1024_3d-128.md)
    "spread:2d-1024-rand-eps1e-5:e4182cc8d343359e": 140114944 + 19632128,
    "interp:2d-1024-rand-eps1e-5:e4182cc8d343359e": 126882560 + 25981440,
    "spread:3d-128-rand-eps1e-6:e4182cc8d343359e": 1798426368 + 229019136,
    "interp:3d-128-rand-eps1e-6:e4182cc8d343359e": 1070203904 + 506863872,
}


def _src_hash():
    """Hash of the sources that define the spreading / interpolation kernels and
    their launch parameters (tiles, defaults)."""
    h = hashlib.sha256()
    for f in ("spread_interp.cuh", "nufft_internal.cuh", "plan.cu"):
        with open(os.path.join(ROOT, "paper_2102_08463_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _peaks():
    hbm, src = 6800.0, "fallback"
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            with open(p) as fh:
                hbm = float(json.load(fh)["hbm_gbs"])
            src = "measured"
        except Exception:
            pass
    return hbm, src


def _sm_max_mhz():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            return float(json.load(fh)["sm_max_mhz"]), "measured"
    except Exception:
        return 2070.0, "fallback"


def alu_peaks(dev):
    """FP32 (derived) and FP32 / FP64 (measured FMA kernel) peaks in TFLOP/s."""
    import torch
    from paper_2102_08463_gb300 import binding
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz, mhz_src = _sm_max_mhz()
    return {"sm_count": sms, "sm_max_mhz": mhz, "sm_max_mhz_source": mhz_src,
            "fp32_derived_tflops": round(sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12, 2),
            "fp32_measured_tflops": round(binding.fma_peak(0), 2),
            "fp64_measured_tflops": round(binding.fma_peak(1), 3)}


def roofline_of(W, w, kernel_ms, peaks):
    """Roofline of one spread / interp launch: the slower of algorithmic bytes at
    the measured HBM bandwidth and algorithmic flops at the ALU peak."""
    hbm, hbm_src = _peaks()
    byts, flops = algorithmic_cost(W, w, "spread")
    if W["prec"] == 0:
        fp_peak, fp_src = peaks["fp32_derived_tflops"], "derived: %d SMs x 128 FP32 lanes x 2 x %g MHz" % (
            peaks["sm_count"], peaks["sm_max_mhz"])
    else:
        fp_peak, fp_src = peaks["fp64_measured_tflops"], "measured: nufft_fma_peak FP64 kernel"
    t = kernel_ms / 1e3
    if byts / (hbm * 1e9) >= flops / (fp_peak * 1e12):
        ach = byts / t / 1e9
        r = {"bound": "hbm", "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s",
             "frac": round(ach / hbm, 4), "peak_source": hbm_src}
    else:
        ach = flops / t / 1e12
        r = {"bound": "alu", "achieved": round(ach, 3), "peak": fp_peak, "unit": "TFLOP/s",
             "frac": round(ach / fp_peak, 4), "peak_source": fp_src}
    r["algorithmic_bytes"] = byts
    r["algorithmic_flops"] = flops
    r["kernel_ms"] = round(kernel_ms, 5)
    return r


def algorithmic_cost(W, w, kernel):
    """Bytes and flops per launch of one spread / interp kernel (ntransf = 1).

    bytes = M (d s + 2 s) + n_tot 2 s: coordinates and strengths once, the fine
    grid written (spread) or read (interp) once.  flops = M (8 d w + (d + 3) w^d):
    d w kernel evaluations of 8 operations, then per window cell (d - 1) weight
    products and a complex-by-real accumulate (4).
    """
    d = W["dim"]
    s = 4 if W["prec"] == 0 else 8
    nf = 1
    for v in W["nf"]:
        nf *= v
    M = W["M"]
    byts = M * (d * s + 2 * s) + nf * 2 * s
    flops = M * (8 * d * w + (d + 3) * w ** d)
    return byts, flops


# ---------------------------------------------------------------------------
# nvidia-smi clock sampler
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], 0.0, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = max(smax, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def make_inputs(W, seed):
    dt = np.float32 if W["prec"] == 0 else np.float64
    ct = np.complex64 if W["prec"] == 0 else np.complex128
    pts = wl.points(W["kind"], W["dim"], W["M"], seed, dt, n=W.get("nf"))
    c = wl.strengths(W["M"], seed + 1, ct)
    f = wl.modes(W["N"], seed + 2, ct)
    return pts, c, f


def max_over_ranks(values, device="cpu"):
    """Element-wise maximum over the ranks of a list of floats (the list itself
    without an initialised process group or at world size 1)."""
    import torch
    import torch.distributed as dist
    vals = [float(v) for v in values]
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return vals
    t = torch.tensor(vals, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def choose_form(ms_by_form, device="cpu"):
    """The step schedule with the smallest slowest-rank time; every rank gets
    the same answer (ties go to the first listed)."""
    order = list(ms_by_form)
    worst = max_over_ranks([ms_by_form[k] for k in order], device)
    return order[min(range(len(order)), key=lambda i: worst[i])]


def replica_value(units_per_rank, world, ms_per_step):
    """Whole-job throughput of `world` replicas: the units all ranks processed
    over the slowest rank's time per step."""
    return units_per_rank * world / (ms_per_step / 1e3)


def run_gpu(args, W, rank, world, local_rank):
    import torch
    from paper_2102_08463_gb300 import binding

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    method1 = args.method1
    method2 = args.method2
    p1 = binding.Plan(1, W["N"], W["eps"], prec=W["prec"], method=method1, stream=stream)
    p2 = binding.Plan(2, W["N"], W["eps"], prec=W["prec"], method=method2, stream=stream)
    W["nf"] = p1.params["nf"][: W["dim"]]
    w = p1.params["w"]
    pts, c, f = make_inputs(W, SEED + 17 * rank)
    rd = p1.real_dtype
    cd = p1.complex_dtype
    dpts = [torch.from_numpy(p).to(dev) for p in pts]
    dc = torch.from_numpy(c).to(dev)
    df = torch.from_numpy(f).to(dev)
    fout = torch.empty(tuple(reversed(W["N"])), dtype=cd, device=dev)
    cout = torch.empty(W["M"], dtype=cd, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def serial_step():
        p1.setpts(*dpts)
        p1.execute(c=dc, f=fout)
        p2.setpts(*dpts)
        p2.execute(f=df, c=cout)

    # The two plans are independent, so the step has three schedules, all doing
    # the same work: one stream (serial_step); two streams, type 1 plan on t1
    # and type 2 plan on t2, started together (overlap_step); and two streams
    # with the type 2 plan's sort started after the type 1 plan's sort, so that
    # each sort overlaps the other plan's spreading / FFT / interpolation
    # instead of the other sort (staggered_step).  An untimed selection pass
    # picks the fastest; the timed region runs it, and the others are timed
    # after it and reported beside it.
    t1, t2 = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    r1 = binding.Plan(1, W["N"], W["eps"], prec=W["prec"], method=method1, stream=t1)
    r2 = binding.Plan(2, W["N"], W["eps"], prec=W["prec"], method=method2, stream=t2)
    rout = torch.empty_like(fout)
    rcout = torch.empty_like(cout)

    def two_stream_step(stagger):
        start = torch.cuda.Event()
        start.record(stream)
        t1.wait_event(start)
        t2.wait_event(start)
        r1.setpts(*dpts)
        if stagger:
            sorted1 = torch.cuda.Event()
            sorted1.record(t1)
            t2.wait_event(sorted1)
        r1.execute(c=dc, f=rout)
        r2.setpts(*dpts)
        r2.execute(f=df, c=rcout)
        stream.wait_stream(t1)
        stream.wait_stream(t2)

    forms = {
        "one stream": serial_step,
        "two streams": lambda: two_stream_step(False),
        "two streams, sorts staggered": lambda: two_stream_step(True),
    }

    def time_form(fn, n):
        ee = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(n)]
        for i in range(n):
            flush.zero_()
            ee[i][0].record(stream)
            fn()
            ee[i][1].record(stream)
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in ee]

    for _ in range(args.warmup):
        for fn in forms.values():
            fn()
    torch.cuda.synchronize()
    form = choose_form({k: sorted(time_form(fn, 5))[2] for k, fn in forms.items()}, dev)
    step = forms[form]

    # ---- timed region: K steps, L2 flushed before each, CUDA events on the stream ----
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    sampler = ClockSampler(local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    launches0 = binding.get_launch_count()
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    launches = binding.get_launch_count() - launches0
    clocks = sampler.stop()
    ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(ms)
    # the same K steps in the other schedules
    form_ms = {form: total_ms / args.steps}
    for k, fn in forms.items():
        if k != form:
            form_ms[k] = sum(time_form(fn, args.steps)) / args.steps
    form_ms = dict(zip(form_ms, max_over_ranks(list(form_ms.values()), dev)))
    r1.close()
    r2.close()
    total_ms = max_over_ranks([total_ms], dev)[0]
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    ms_per_step = total_ms / args.steps
    units = 2 * W["M"] * world
    value = replica_value(2 * W["M"], world, ms_per_step)

    # ---- stage breakdown and the kernels' own durations (outside the timed region) ----
    def timed(fn, reps=args.stage_reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        tot = 0.0
        for _ in range(reps):
            flush.zero_()
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            tot += a.elapsed_time(b)
        return tot / reps

    h1, h2 = p1.handle, p2.handle
    dcp = binding._dptr(dc)
    dfp = binding._dptr(df)
    fop = binding._dptr(fout)
    cop = binding._dptr(cout)
    stages = {
        "setpts_ms": timed(lambda: p1.setpts(*dpts)),
        "spread_ms": timed(lambda: binding.spread_add(h1, dcp)),
        "spread_with_clear_ms": timed(lambda: binding.spread(h1, dcp)),
        "fft_ms": timed(lambda: binding.fft(h1)),
        "deconvolve_ms": timed(lambda: binding.deconvolve(h1, fop)),
        "precorrect_ms": timed(lambda: binding.precorrect(h2, dfp)),
        "interp_ms": timed(lambda: binding.interp(h2, cop)),
        "exec_type1_ms": timed(lambda: binding.execute(h1, dcp, fop)),
        "exec_type2_ms": timed(lambda: binding.execute(h2, cop, dfp)),
    }
    # restore correct outputs for the accuracy check
    serial_step()
    torch.cuda.synchronize()

    # ---- roofline of the dominant kernel ----
    peaks = alu_peaks(dev)
    roof = {name: roofline_of(W, w, stages[key], peaks)
            for name, key in (("spread", "spread_ms"), ("interp", "interp_ms"))}
    dom = "spread" if stages["spread_ms"] >= stages["interp_ms"] else "interp"
    roofline = dict(roof[dom])
    roofline["kernel"] = dom
    tkey = "%s:%s:%s" % (dom, args.workload, _src_hash())
    roofline["traffic"] = TRAFFIC.get(tkey)

    # ---- end to end through the public API with host buffers ----
    hpts = [torch.from_numpy(p).pin_memory() for p in pts]
    hc = torch.from_numpy(c).pin_memory()
    hf = torch.from_numpy(f).pin_memory()
    hfo = torch.empty(fout.shape, dtype=cd).pin_memory()
    hco = torch.empty(cout.shape, dtype=cd).pin_memory()
    h2d = sum(t.numel() * t.element_size() for t in hpts) + hc.numel() * hc.element_size() \
        + hf.numel() * hf.element_size()
    d2h = hfo.numel() * hfo.element_size() + hco.numel() * hco.element_size()

    def e2e_serial_step():
        for hsrc, ddst in zip(hpts, dpts):
            ddst.copy_(hsrc, non_blocking=True)
        dc.copy_(hc, non_blocking=True)
        df.copy_(hf, non_blocking=True)
        serial_step()
        hfo.copy_(fout, non_blocking=True)
        hco.copy_(cout, non_blocking=True)

    # Overlapped form (host buffers in, host results out): the type 1 plan on
    # stream s1, the type 2 plan on stream s2, the strengths and modes copied on
    # s3.  The points go first (s1: x, y in); both sorts start as soon as they
    # have arrived while s3 copies f and then c; each plan's execute waits only
    # for the array it reads; each result is copied out on its plan's stream.
    s1, s2, s3 = (torch.cuda.Stream(device=dev) for _ in range(3))
    q1 = binding.Plan(1, W["N"], W["eps"], prec=W["prec"], method=method1, stream=s1)
    q2 = binding.Plan(2, W["N"], W["eps"], prec=W["prec"], method=method2, stream=s2)
    ep = [torch.from_numpy(p).to(dev) for p in pts]
    ec = torch.empty_like(dc)
    ef = torch.empty_like(df)
    efo = torch.empty_like(fout)
    eco = torch.empty_like(cout)

    def e2e_step():
        start = torch.cuda.Event()
        start.record(stream)
        for q in (s1, s2, s3):
            q.wait_event(start)
        with torch.cuda.stream(s1):
            for hsrc, ddst in zip(hpts, ep):
                ddst.copy_(hsrc, non_blocking=True)
            have_pts = torch.cuda.Event()
            have_pts.record(s1)
        s3.wait_event(have_pts)
        with torch.cuda.stream(s3):
            ef.copy_(hf, non_blocking=True)
            have_f = torch.cuda.Event()
            have_f.record(s3)
            ec.copy_(hc, non_blocking=True)
            have_c = torch.cuda.Event()
            have_c.record(s3)
        s2.wait_event(have_pts)
        q1.setpts(*ep)
        q2.setpts(*ep)
        s1.wait_event(have_c)
        s2.wait_event(have_f)
        with torch.cuda.stream(s1):
            q1.execute(c=ec, f=efo)
            hfo.copy_(efo, non_blocking=True)
        with torch.cuda.stream(s2):
            q2.execute(f=ef, c=eco)
            hco.copy_(eco, non_blocking=True)
        stream.wait_stream(s1)
        stream.wait_stream(s2)

    def time_e2e(fn):
        for _ in range(max(1, args.warmup // 2)):
            fn()
        torch.cuda.synchronize()
        ee = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        for i in range(args.steps):
            flush.zero_()
            ee[i][0].record(stream)
            fn()
            ee[i][1].record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in ee) / args.steps

    e2e_serial_ms = time_e2e(e2e_serial_step)
    e2e_ms = time_e2e(e2e_step)
    # the overlapped form's host results against the one-stream step's (same inputs)
    serial_step()
    torch.cuda.synchronize()

    def _rd(a, b):
        a = a.to(torch.complex128)
        b = b.cpu().to(torch.complex128)
        return float(torch.linalg.vector_norm(a - b) / max(float(torch.linalg.vector_norm(b)), 1e-300))

    e2e_diff = {"type1": _rd(hfo, fout), "type2": _rd(hco, cout)}
    q1.close()
    q2.close()
    e2e_ms = max_over_ranks([e2e_ms], dev)[0]


    out = {
        "metric": metric_for(W),
        "value": round(value, 1),
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_per_step, 5),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32" if W["prec"] == 0 else "f64",
        "data": "synthetic (seeded SplitMix64: %s points, N(0,1) strengths and modes)" % W["kind"],
        "step_form": form,
        "step_forms": {k: {"value": round(units / (v / 1e3), 1), "ms_per_step": round(v, 5)}
                       for k, v in form_ms.items()},
        "config": {"workload": "%s: %dD type 1 + type 2, N=%s, fine grid %s, M=%d, eps=%g, %s"
                               % (args.workload, W["dim"], "x".join(map(str, W["N"])),
                                  "x".join(map(str, W["nf"])), W["M"], W["eps"],
                                  "complex64" if W["prec"] == 0 else "complex128"),
                   "methods": {"type1": p1.params["method"], "type2": p2.params["method"]},
                   "kernel_width": w, "ntransf": 1,
                   "l2": "flushed before every step (256 MiB write)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": roofline,
        "roofline_kernels": roof,
        "alu_peaks": peaks,
        "stages_ms": {k: round(v, 5) for k, v in stages.items()},
        "pts_per_s": {
            "spread": round(W["M"] / (stages["spread_ms"] / 1e3), 1),
            "interp": round(W["M"] / (stages["interp_ms"] / 1e3), 1),
            "exec_type1": round(W["M"] / (stages["exec_type1_ms"] / 1e3), 1),
            "exec_type2": round(W["M"] / (stages["exec_type2_ms"] / 1e3), 1),
        },
        "e2e": {"value": round(units / (e2e_ms / 1e3), 1), "unit": UNIT,
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "ms_per_step": round(e2e_ms, 5),
                "form": "two plans on two streams; points copied first, strengths and modes on a "
                        "third stream while the sorts run",
                "rel_diff_vs_device_step": e2e_diff,
                "serial": {"value": round(units / (e2e_serial_ms / 1e3), 1),
                           "ms_per_step": round(e2e_serial_ms, 5)}},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    # outputs of the last step, for the sampled check in the CPU oracle leg
    out["_outputs"] = (pts, c, f, hfo.numpy(), hco.numpy())
    p1.close()
    p2.close()
    return out


CONFIG_ROWS = ("3d-128-rand-eps1e-6", "2d-1024-rand-eps1e-9", "2d-64-rand-eps1e-5")


def measure_config(name, reps=5, nsamp=32):
    """One more workload measured beside the headline: setpts, spread, interp and
    both executes (median of `reps`, L2 flushed before each), the roofline of
    spreading and interpolation, and the relative l2 error of both types against
    the exact sums on `nsamp` sampled modes / targets."""
    import torch
    from paper_2102_08463_gb300 import binding

    W = dict(WORKLOADS[name])
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    p1 = binding.Plan(1, W["N"], W["eps"], prec=W["prec"], stream=stream)
    p2 = binding.Plan(2, W["N"], W["eps"], prec=W["prec"], stream=stream)
    W["nf"] = p1.params["nf"][: W["dim"]]
    w = p1.params["w"]
    pts, c, f = make_inputs(W, SEED + 29)
    dpts = [torch.from_numpy(p).to(dev) for p in pts]
    dc = torch.from_numpy(c).to(dev)
    df = torch.from_numpy(f).to(dev)
    fout = torch.empty(tuple(reversed(W["N"])), dtype=p1.complex_dtype, device=dev)
    cout = torch.empty(W["M"], dtype=p1.complex_dtype, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    p1.setpts(*dpts)
    p2.setpts(*dpts)

    def med(fn):
        ts = []
        for _ in range(reps + 1):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        ts = sorted(ts[1:])
        return ts[len(ts) // 2]

    h1, h2 = p1.handle, p2.handle
    st = {"setpts_ms": med(lambda: p1.setpts(*dpts)),
          "spread_ms": med(lambda: binding.spread_add(h1, binding._dptr(dc))),
          "interp_ms": med(lambda: binding.interp(h2, binding._dptr(cout))),
          "exec_type1_ms": med(lambda: binding.execute(h1, binding._dptr(dc), binding._dptr(fout))),
          "exec_type2_ms": med(lambda: binding.execute(h2, binding._dptr(cout), binding._dptr(df)))}
    peaks = alu_peaks(dev)
    p1.execute(c=dc, f=fout)
    p2.execute(f=df, c=cout)
    torch.cuda.synchronize()
    acc = sampled_accuracy(W, pts, c, f, fout.cpu().numpy(), cout.cpu().numpy(), nsamp=nsamp)
    p1.close()
    p2.close()
    M = W["M"]
    return {
        "workload": "%dD type 1 + type 2, N=%s, fine grid %s, M=%d, eps=%g, %s, %s points"
                    % (W["dim"], "x".join(map(str, W["N"])), "x".join(map(str, W["nf"])), M,
                       W["eps"], "complex64" if W["prec"] == 0 else "complex128", W["kind"]),
        "kernel_width": w,
        "stages_ms": {k: round(v, 5) for k, v in st.items()},
        "pts_per_s": {"spread": round(M / (st["spread_ms"] / 1e3), 1),
                      "interp": round(M / (st["interp_ms"] / 1e3), 1),
                      "exec_type1": round(M / (st["exec_type1_ms"] / 1e3), 1),
                      "exec_type2": round(M / (st["exec_type2_ms"] / 1e3), 1)},
        "roofline": {"spread": roofline_of(W, w, st["spread_ms"], peaks),
                     "interp": roofline_of(W, w, st["interp_ms"], peaks)},
        "rel_l2_vs_exact": acc,
    }


def sampled_accuracy(W, pts, c, f, f_gpu, c_gpu, nsamp=48):
    """Relative l2 error of the GPU outputs on sampled modes / targets (exact sums)."""
    import oracle
    p64 = [p.astype(np.float64) for p in pts]
    Ntot = int(np.prod(W["N"]))
    kidx = wl.sample_indices(Ntot, nsamp, SEED + 5)
    jidx = wl.sample_indices(W["M"], nsamp, SEED + 6)
    f_ref = oracle.direct_type1(p64, c.astype(np.complex128), W["N"], +1, modes=kidx)
    c_ref = oracle.direct_type2(p64, f.astype(np.complex128), +1, targets=jidx)
    return {"type1": oracle.rel_l2(f_gpu.ravel()[kidx], f_ref),
            "type2": oracle.rel_l2(c_gpu.ravel()[jidx], c_ref),
            "samples": nsamp, "reference": "FP64 exact sums (oracle O1)"}


# ---------------------------------------------------------------------------
# CPU oracle arm
# ---------------------------------------------------------------------------
def oracle_step(W, pts, c, f):
    import oracle
    p64 = [p.astype(np.float64) for p in pts]
    oracle.nufft_type1(p64, c.astype(np.complex128), W["N"], eps=W["eps"])
    oracle.nufft_type2(p64, f.astype(np.complex128), eps=W["eps"])


def cpu_sample(W, budget_s):
    """Pick a point count for one oracle step of about budget_s seconds."""
    import oracle
    if "nf" not in W:
        P = oracle.Params(W["N"], W["eps"])
        W["nf"] = P.n
    m0 = min(W["M"], 65536)
    Ws = dict(W, M=m0)
    pts, c, f = make_inputs(Ws, SEED)
    t0 = time.perf_counter()
    oracle_step(Ws, pts, c, f)
    t_small = time.perf_counter() - t0
    Ws = dict(W, M=min(W["M"], 4 * m0))
    pts, c, f = make_inputs(Ws, SEED)
    t0 = time.perf_counter()
    oracle_step(Ws, pts, c, f)
    t_big = time.perf_counter() - t0
    per_pt = max((t_big - t_small) / max(Ws["M"] - m0, 1), 1e-9)
    fixed = max(t_small - per_pt * m0, 0.0)
    m = int(max(m0, min(W["M"], (budget_s - fixed) / per_pt)))
    return m


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the platform)."""
    try:
        r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10)
        for ln in r.stdout.splitlines():
            if ln.strip().lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for ln in fh:
                if ln.lower().startswith(("model name", "cpu model")):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def run_cpu_baseline(W, budget_s=15.0, steps=1, gpu_outputs=None):
    """The oracle timed on the host cores; with the GPU arm's outputs, also the
    relative l2 error of those outputs on sampled modes / targets against the
    oracle's exact sums."""
    import oracle
    oracle.set_num_threads(os.cpu_count() or 1)
    cores = oracle.num_threads()
    m = cpu_sample(W, budget_s / max(steps, 1))
    Ws = dict(W, M=m)
    pts, c, f = make_inputs(Ws, SEED)
    t0 = time.perf_counter()
    for _ in range(steps):
        oracle_step(Ws, pts, c, f)
    dt = (time.perf_counter() - t0) / steps
    # the same step on one thread, on a quarter of the sample
    m1 = max(1, m // 4)
    W1 = dict(W, M=m1)
    pts1, c1, f1 = make_inputs(W1, SEED)
    oracle.set_num_threads(1)
    t0 = time.perf_counter()
    oracle_step(W1, pts1, c1, f1)
    dt1 = time.perf_counter() - t0
    oracle.set_num_threads(cores)
    out = {"value": round(2 * m / dt, 1), "unit": UNIT, "cores": cores, "kind": "oracle",
           "cpu_model": cpu_model(),
           "sample": "one type 1 + type 2 FP64 oracle pipeline step (C spread/interp with "
                     "OpenMP, numpy FFT) on %d of the %d points, full %s fine grid, eps=%g"
                     % (m, W["M"], "x".join(map(str, W["nf"])), W["eps"]),
           "s_per_step": round(dt, 3),
           "one_thread": {"value": round(2 * m1 / dt1, 1), "unit": UNIT, "points": m1,
                          "s_per_step": round(dt1, 3)}}
    if gpu_outputs is not None:
        out["gpu_rel_l2_sampled"] = sampled_accuracy(W, *gpu_outputs)
    return out


def run_reference(args, W, rank):
    if rank != 0:
        return None
    import oracle
    oracle.build()
    oracle.set_num_threads(os.cpu_count() or 1)
    cores = oracle.num_threads()
    per_step_budget = max(0.5, 150.0 / max(args.steps + args.warmup, 1))
    m = cpu_sample(W, per_step_budget)
    Ws = dict(W, M=m)
    pts, c, f = make_inputs(Ws, SEED)
    for _ in range(args.warmup):
        oracle_step(Ws, pts, c, f)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_step(Ws, pts, c, f)
    dt = (time.perf_counter() - t0) / args.steps
    value = 2 * m / dt
    return {
        "impl": "reference",
        "metric": metric_for(W), "value": round(value, 1), "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dt * 1e3, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded SplitMix64), bounded sample of the workload",
        "config": {"workload": "%s: %dD type 1 + type 2, N=%s, M=%d (sample %d), eps=%g"
                               % (args.workload, W["dim"], "x".join(map(str, W["N"])), W["M"],
                                  m, W["eps"])},
        "cpu_baseline": {"value": round(value, 1), "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "%d of %d points per step, full fine grid" % (m, W["M"])},
        "e2e": {"value": round(value, 1), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


# ---------------------------------------------------------------------------
# Many-plan workload: 256 independent plans of uneven N and M plus one
# ntransf = 32 plan, one-by-one with the heuristic tiles versus autotuned tiles
# in one captured batched launch.
# ---------------------------------------------------------------------------
def batch_specs(seed=SEED + 40):
    """256 plans: half 2D / half 3D, half type 1 / half type 2; square / cube N
    log-uniform in [32, 512] (2D) or [16, 128] (3D); M log-uniform in [1e4, 2e6];
    plus one 2D N = 512^2, M = 1e6, ntransf = 32 plan.  eps = 1e-5, single precision."""
    u = wl.uniform01(seed, 4 * 256, stream=50).reshape(256, 4)
    specs = []
    for i in range(256):
        dim = 2 if i % 2 == 0 else 3
        tp = 1 if (i // 2) % 2 == 0 else 2
        lo, hi = (32, 512) if dim == 2 else (16, 128)
        n1 = int(round(math.exp(math.log(lo) + u[i, 0] * (math.log(hi) - math.log(lo)))))
        M = int(round(math.exp(math.log(1e4) + u[i, 1] * (math.log(2e6) - math.log(1e4)))))
        specs.append(dict(type=tp, N=(n1,) * dim, M=M, ntransf=1))
    specs.append(dict(type=1, N=(512, 512), M=1000000, ntransf=32))
    return specs


def run_batch_bench(args):
    import torch
    from paper_2102_08463_gb300 import binding

    stream = torch.cuda.Stream()
    specs = batch_specs()
    eps = 1e-5
    torch.cuda.set_device(0)
    with torch.cuda.stream(stream):
        data = []
        for i, sp in enumerate(specs):
            dim = len(sp["N"])
            pts = [torch.from_numpy(a).cuda() for a in wl.points("rand", dim, sp["M"], SEED + 1000 + i,
                                                                 np.float32)]
            if sp["type"] == 1:
                c = torch.from_numpy(wl.strengths(sp["M"], SEED + 3000 + i, np.complex64,
                                                  ntransf=sp["ntransf"])).cuda()
                shp = tuple(reversed(sp["N"]))
                f = torch.zeros(((sp["ntransf"],) + shp) if sp["ntransf"] > 1 else shp,
                                dtype=torch.complex64, device="cuda")
            else:
                f = torch.from_numpy(wl.modes(sp["N"], SEED + 5000 + i, np.complex64)).cuda()
                c = torch.zeros(sp["M"], dtype=torch.complex64, device="cuda")
            data.append((pts, c, f))
        total_pts = sum(sp["M"] * sp["ntransf"] for sp in specs)

        def make_plans(opts_for):
            plans = []
            for sp, (pts, c, f) in zip(specs, data):
                kw = opts_for(sp)
                p = binding.Plan(sp["type"], sp["N"], eps, prec=0, ntransf=sp["ntransf"],
                                 stream=stream, **kw)
                p.setpts(*pts)
                plans.append(p)
            return plans

        def time_it(fn, steps):
            for _ in range(args.warmup):
                fn()
            stream.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(steps):
                fn()
            b.record(stream)
            b.synchronize()
            return a.elapsed_time(b) / steps

        # heuristic tiles, one plan after another
        heur = make_plans(lambda sp: {})

        def one_by_one(plans):
            def run():
                for p, (pts, c, f) in zip(plans, data):
                    p.execute(c=c, f=f)
            return run
        ms_heur = time_it(one_by_one(heur), args.steps)
        for p in heur:
            p.close()

        # autotune one representative per (type, dim) class and the ntransf plan
        tuned = {}
        t0 = time.perf_counter()
        for key in sorted({(sp["type"], len(sp["N"]), sp["ntransf"]) for sp in specs}):
            idx = [i for i, sp in enumerate(specs)
                   if (sp["type"], len(sp["N"]), sp["ntransf"]) == key]
            idx.sort(key=lambda i: specs[i]["M"] * max(specs[i]["N"]))
            i = idx[len(idx) // 2]
            sp = specs[i]
            pts, c, f = data[i]
            best, best_ms, _ = binding.autotune(sp["type"], sp["N"], eps, sp["M"], pts[0], pts[1],
                                                pts[2] if len(pts) == 3 else None, c.clone(),
                                                f.clone(), ntransf=sp["ntransf"], prec=0, reps=2,
                                                stream=stream)
            tuned[key] = dict(method=best.method, bins=tuple(best.bin)[: len(sp["N"])],
                              msub=best.msub, threads=best.threads)
        tune_s = time.perf_counter() - t0
        plans = make_plans(lambda sp: tuned[(sp["type"], len(sp["N"]), sp["ntransf"])])
        ms_tuned = time_it(one_by_one(plans), args.steps)
        for p in plans:
            p.close()
        # The batch keeps the library's default tiles: the autotuner times one plan
        # alone, where the unsorted GM method can win because that plan's fine grid
        # sits in L2; in a grouped launch many plans' grids are live at once and
        # the sorted SM forms win (measured per class with every method).
        binding.tune_cache_clear()      # automatic tiles would otherwise adopt the cache
        plans = make_plans(lambda sp: {})
        batch = binding.Batch(plans, stream=stream)
        cs = [d[1] for d in data]
        fs = [d[2] for d in data]
        ms_batch = time_it(lambda: batch.execute(cs, fs), args.steps)
        launches0 = binding.get_launch_count()
        batch.capture(cs, fs)
        graph_launches = binding.get_launch_count() - launches0
        ms_graph = time_it(batch.launch, args.steps)
        batch.close()
        for p in plans:
            p.close()
    value = total_pts / (ms_graph / 1e3)
    return {
        "metric": "aggregate NU points/sec, 256 uneven plans + ntransf=32 plan, batched",
        "batch_tiles": "library defaults (heuristic); the one-by-one autotuned arm uses tuned_tiles",
        "value": round(value, 1), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_graph, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded SplitMix64 uniform points, N(0,1) strengths / modes)",
        "config": {"workload": "batch-256: 128 2D (N in [32,512]^2) + 128 3D (N in [16,128]^3) "
                               "plans, half type 1 / half type 2, M log-uniform in [1e4, 2e6], "
                               "+ 2D 512^2 M=1e6 ntransf=32; eps=1e-5 complex64; execute only "
                               "(points set once)",
                   "tuned_tiles": {"%d-%dd-nt%d" % k: v for k, v in tuned.items()},
                   "autotune_seconds": round(tune_s, 2)},
        "arms_ms_per_step": {"one_by_one_heuristic": round(ms_heur, 4),
                             "one_by_one_autotuned": round(ms_tuned, 4),
                             "batched_execute": round(ms_batch, 4),
                             "batched_graph": round(ms_graph, 4)},
        "speedup_vs_one_by_one_heuristic": round(ms_heur / ms_graph, 3),
        "total_points_per_step": int(total_pts),
        "gpu_launches": int(graph_launches) * args.steps,
    }


def run_picker_bench(args):
    """Held-out problems of the picker's distribution (seeds past the training
    data's, in the evaluation split): every candidate tiling timed, then the
    total execute time of the learned picker's choice against the heuristic
    tiles and the fastest candidate."""
    import torch
    from paper_2102_08463_gb300 import binding, picker

    torch.cuda.set_device(0)
    weights = picker.DEFAULT_WEIGHTS
    p = binding.Picker(path=weights)
    probs = picker.sample_problems(args.picker_problems, first_seed=100000, heldout=True)
    t0 = time.perf_counter()
    rows = picker.collect(probs, reps=3)
    collect_s = time.perf_counter() - t0
    tot, per = picker.evaluate(p, rows)
    p.close()
    return {
        "metric": "held-out total execute time with the learned tile picker",
        "value": round(tot["picker"], 4), "unit": "ms", "n_gpus": 1, "steps": 1,
        "warmup": args.warmup, "ms_per_step": round(tot["picker"], 4),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64",
        "data": "synthetic (seeded SplitMix64 points: uniform, wrapped Gaussian, 8-Gaussian "
                "mixture)",
        "config": {"workload": "picker-holdout: %d problems, 2D/3D, type 1/2, N_i in [32,1024], "
                               "M in [1e4,3e7], eps in [1e-12,1e-2] (work-bounded), every "
                               "candidate tiling at sigma 2 and (where it reaches eps) 1.25 "
                               "timed (median of 3 executes)" % tot["problems"],
                   "weights": os.path.relpath(weights, ROOT)},
        "heuristic_ms": round(tot["heuristic"], 4), "best_ms": round(tot["best"], 4),
        "regret_vs_best": round(tot["regret"], 4),
        "picked_sigma125": tot["picked_sigma125"],
        "speedup_vs_heuristic": round(tot["speedup_vs_heuristic"], 4),
        "collect_seconds": round(collect_s, 1),
        "per_problem": per,
    }


def run_method_sweep(args):
    """The paper's method comparison on this GPU: spreading and interpolation time
    per point for each method (GM, GM-sort, SM), by fine-grid size, for uniform and
    box-clustered points at densities 0.1, 1 and 10; 2D single precision at
    eps = 1e-5.  Sizes with more than 2^24 points are left out; each time is the
    median of 5 launches (L2 flushed before each)."""
    import torch
    from paper_2102_08463_gb300 import binding

    torch.cuda.set_device(0)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")

    def timed(fn, reps=5):
        ts = []
        for _ in range(reps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            b.synchronize()
            ts.append(a.elapsed_time(b))
        ts.sort()
        return ts[len(ts) // 2]

    rows = []
    launches0 = binding.get_launch_count()
    for n in (256, 512, 1024, 2048, 4096):
        for rho in (0.1, 1.0, 10.0):
            M = int(round(rho * n * n))
            if M > (1 << 24):
                continue
            for kind in ("rand", "cluster"):
                N = (n // 2, n // 2)
                pts = [torch.from_numpy(a).cuda()
                       for a in wl.points(kind, 2, M, SEED + 77, np.float32, n=(n, n))]
                c = torch.from_numpy(wl.strengths(M, SEED + 78, np.complex64)).cuda()
                co = torch.empty_like(c)
                row = {"n": n, "rho": rho, "M": M, "dist": kind}
                for method in ("gm", "gmsort", "sm"):
                    p1 = binding.Plan(1, N, 1e-5, prec=0, method=method)
                    p1.setpts(*pts)
                    t_s = timed(lambda: binding.spread_add(p1.handle, binding._dptr(c)))
                    t_set = timed(lambda: p1.setpts(*pts))
                    p1.close()
                    p2 = binding.Plan(2, N, 1e-5, prec=0, method=method)
                    p2.setpts(*pts)
                    t_i = timed(lambda: binding.interp(p2.handle, binding._dptr(co)))
                    p2.close()
                    row[method] = {"spread_ns_per_pt": round(t_s * 1e6 / M, 4),
                                   "interp_ns_per_pt": round(t_i * 1e6 / M, 4),
                                   "setpts_ns_per_pt": round(t_set * 1e6 / M, 4)}
                rows.append(row)
                del pts, c, co
    launches = binding.get_launch_count() - launches0
    sm = [r["sm"]["spread_ns_per_pt"] for r in rows if r["rho"] == 1.0 and r["dist"] == "rand"]
    return {
        "metric": "2D spread / interp ns per point by method (GM, GM-sort, SM) vs fine grid",
        "value": round(min(sm), 4) if sm else None, "unit": "ns/pt (SM spread, rho=1 rand, best n)",
        "n_gpus": 1, "steps": 5, "warmup": 0, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded SplitMix64: uniform on [-pi,pi)^2 and the box [0, 8h]^2)",
        "config": {"workload": "method-sweep: 2D eps=1e-5 complex64, fine grid n^2 for n in "
                               "256..4096, density M/n^2 in {0.1, 1, 10} (M <= 2^24)"},
        "gpu_launches": int(launches),
        "table": rows,
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD,
                    choices=sorted(WORKLOADS) + ["batch-256", "picker-holdout", "method-sweep"])
    ap.add_argument("--picker-problems", type=int, default=24)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--method1", default="auto")
    ap.add_argument("--method2", default="auto")
    ap.add_argument("--stage-reps", type=int, default=10)
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-accuracy", action="store_true", help="skip the sampled accuracy check")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the extra workloads measured beside the headline")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.workload == "batch-256":
        print(json.dumps(run_batch_bench(args)), flush=True)
        return
    if args.workload == "picker-holdout":
        print(json.dumps(run_picker_bench(args)), flush=True)
        return
    if args.workload == "method-sweep":
        print(json.dumps(run_method_sweep(args)), flush=True)
        return
    W = dict(WORKLOADS[args.workload])

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        out = run_reference(args, W, rank)
        if out is not None:
            print(json.dumps(out), flush=True)
        return

    import torch
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    out = run_gpu(args, W, rank, world, local_rank)
    outputs = out.pop("_outputs")
    if rank == 0 and world == 1 and not args.no_cpu:
        out["cpu_baseline"] = run_cpu_baseline(
            W, gpu_outputs=None if args.no_accuracy else outputs)
    if rank == 0 and world == 1 and not args.no_configs:
        # the other spec rows, measured in the same run (outside the timed region)
        out["configs"] = {name: measure_config(name) for name in CONFIG_ROWS
                          if name != args.workload}
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
