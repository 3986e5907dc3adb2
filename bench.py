"""Benchmark: cell-updates/s of the per-cell uniform-patch RHD update on GB300.

Default workload: 3-D periodic 128^3 RHD, FP64 (lognormal density with a |k|^-4
Gaussian random field, sigma_ln rho = 1, T_gas = 1, T_r ~ U(0.5, 2),
kappa_P = kappa_R = 1, a_r = 1, c = 100, chat = 10 max c_s, CFL 0.3,
N_sub,max = 10).  A "step" is one full update: hydro RK2 stage pair plus every
radiation substep (RK2 pair + exchange); one cell-update is one cell advanced
by one such step (the paper's Mzones/s unit, Sec. 4).

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                [--workload rhd128|hydro128|...] [--precision fp64|fp32]
Prints ONE JSON line (rank 0).  Under torchrun each rank runs an independent
replica of the workload on its own GPU (weak scaling, no data-path collective).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
# ALU peaks from the unit counts and the maximum SM clock (152 SMs, 2.07 GHz):
# FP64 2 FMA/clk/SM -> 1.26 TFLOP/s; FP32 128 FMA/clk/SM -> 80.6 TFLOP/s.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12

# Algorithmic flops per interior cell of one launch (add, sub, mul, div, sqrt),
# counted on the oracle's formulas by oracle/count_flops.cpp on a seeded
# workload: con2prim 13, PPM 21.3 per call, HLLC 119.6 per face, radiation
# face work 283.4 (closures, HLL, optical depth), f = F/(c E_r) 6, exchange
# 256.4 (4.2 Newton iterations); divergence 2 per variable and direction,
# RK combine 2 (stage 1) or 5 (stage 2) per variable.
ALGO_FLOPS = {
    "hydro1": 13 + 3 * (5 * 21.3 + 119.6) + 30 + 10 + 10,
    "hydro2": 13 + 3 * (5 * 21.3 + 119.6) + 30 + 10 + 25,
    "rad1": 6 + 3 * (4 * 21.1 + 283.4) + 24 + 8 + 8,
    "rad2": 6 + 3 * (4 * 21.1 + 283.4) + 24 + 8 + 20,
    "exchange": 256.4,
}

# kernels launched per step (captured in one CUDA graph; substeps beyond N_sub
# are predicated off but still launched)
def launches_per_step(hydro_only: bool, nsub_max: int) -> int:
    n = 2 + 2 + 2  # max-speed + timestep, 2 ghost fills, 2 hydro stages
    if not hydro_only:
        n += 1 + nsub_max * 5  # rho ghost fill; per substep: 2 fills, 2 rad stages, exchange
    return n


def workload(name: str):
    from paper_2110_01792_gb300 import inputs as I
    if name == "rhd128":
        return I.rhd_lognormal(128, steps=20)
    if name == "rhd256":
        return I.rhd_lognormal(256, steps=20)
    if name == "hydro128":
        return I.hydro_waves(128)
    if name == "hydro256":
        return I.hydro_waves(256)
    if name == "hydro32":
        return I.hydro_waves(32)
    if name == "rhd512":
        return I.rhd_lognormal(512, sigma=1.5, kappa_mode=1, steps=10)
    if name == "patches":
        return I.rhd_lognormal(layout=I.patch_tiling(), steps=10)
    raise SystemExit(f"unknown workload {name}")


def describe(name: str, prob, precision: str) -> dict:
    lay = prob.layout
    d = {"workload": f"{name} ({'RHD' if prob.R is not None else 'hydro'}, "
                     f"{'x'.join(str(v) for v in lay.dom_n)} periodic, {lay.nbox} patch"
                     f"{'es' if lay.nbox > 1 else ''}, {precision})",
         "cells": lay.ncells, "ghost": lay.ng, "patches": lay.nbox,
         "precision": precision}
    return d


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": FALLBACK_HBM_GBS}, "fallback"


def algorithmic_bytes_per_cell(kernel: str, elem: int) -> float:
    """Minimum HBM traffic per interior cell of one launch (values x elem size):
    hydro stage 1 reads 5, writes 5; stage 2 reads 10, writes 5; radiation
    stage 1 reads 4 + rho, writes 4; stage 2 reads 8 + rho, writes 4;
    exchange reads 9, writes 8."""
    vals = {"hydro1": 10, "hydro2": 15, "rad1": 9, "rad2": 13, "exchange": 17}[kernel]
    return vals * elem


def cpu_baseline(precision: str, budget_s: float = 12.0):
    """The oracle as it stands, single-threaded on the host, on a bounded sample
    of the same workload: one RHD update of a 32^3 periodic box drawn with the
    same generators and parameters (same N_sub,max, CFL, chat rule)."""
    import numpy as np
    import oracle as O
    from paper_2110_01792_gb300 import inputs as I
    prob = I.rhd_lognormal(32)
    g = O.Grid(prob.layout.lo, prob.layout.n, prob.layout.off, prob.layout.dom_n, prob.layout.ng)
    p = O.make_params(**prob.params)
    U = [a.copy() for a in prob.U]
    R = [a.copy() for a in prob.R]
    steps, t0 = 0, time.perf_counter()
    while True:
        rc, ts, _ = O.step(g, p, U, R)
        steps += 1
        el = time.perf_counter() - t0
        if el > budget_s or steps >= 12:
            break
    cells = prob.layout.ncells
    return {"value": cells * steps / el, "unit": "cell-updates/s", "cores": 1, "kind": "oracle",
            "sample": f"{steps} full RHD update(s) of a 32^3 periodic box of the same generator "
                      f"(N_sub={ts[1]}), FP64, {el:.1f} s"}


def run_reference(args):
    """--impl reference: the FP64 oracle on the host cores, each step one
    bounded sample (one RHD update of a 32^3 box of the same workload)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O
    from paper_2110_01792_gb300 import inputs as I
    prob = I.rhd_lognormal(32) if args.workload.startswith("rhd") else I.hydro_waves(32)
    g = O.Grid(prob.layout.lo, prob.layout.n, prob.layout.off, prob.layout.dom_n, prob.layout.ng)
    p = O.make_params(**prob.params)
    U = [a.copy() for a in prob.U]
    R = [a.copy() for a in prob.R] if prob.R is not None else None
    for _ in range(args.warmup):
        O.step(g, p, U, R)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.step(g, p, U, R)
    el = time.perf_counter() - t0
    v = prob.layout.ncells * args.steps / el
    sample = (f"each step one full update of a 32^3 periodic box of the {args.workload} generator, "
              f"FP64 oracle, single thread")
    line = {"impl": "reference", "metric": "cell-updates/s", "value": v, "unit": "cell-updates/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload + " (32^3 sample per step)", "precision": "fp64"},
            "cpu_baseline": {"value": v, "unit": "cell-updates/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "cell-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def time_kernel(torch, fn, reps, stream):
    """Average device duration of one launch of fn() (CUDA events on `stream`)."""
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    fn()
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(reps):
        fn()
    ev1.record(stream)
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1) / 1e3 / reps


def run_variants(args, steps=5, warmup=3):
    """Cell-updates/s of the other precision / physics combinations on the same
    GPU (device time over `steps` full updates after `warmup`)."""
    import torch
    from paper_2110_01792_gb300 import qk
    out = {}
    for name, prec in (("rhd128", "fp32"), ("hydro128", "fp64"), ("hydro128", "fp32"),
                       ("rhd128", "fp64")):
        if name == args.workload and prec == args.precision:
            continue
        prob = workload(name)
        p = qk.FP64 if prec == "fp64" else qk.FP32_MIXED
        tdt = torch.float64 if p == qk.FP64 else torch.float32
        ctx = qk.Context(prob.layout, prob.params, p)
        U = [torch.from_numpy(a).cuda().to(tdt) for a in prob.U]
        R = None if prob.R is None else [torch.from_numpy(a).cuda().to(tdt) for a in prob.R]
        for _ in range(warmup):
            ctx.step(U, R)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            ctx.step(U, R)
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        st = ctx.status()
        ctx.close()
        out[f"{name}_{prec}"] = {"value": prob.layout.ncells * steps / t, "unit": "cell-updates/s",
                                 "ms_per_step": 1e3 * t / steps, "steps": steps,
                                 "status_ok": st[0] == qk.OK}
    return out


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import __graft_entry__
    from paper_2110_01792_gb300 import qk

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    __graft_entry__.build()
    prec = qk.FP64 if args.precision == "fp64" else qk.FP32_MIXED
    tdt = torch.float64 if prec == qk.FP64 else torch.float32
    elem = 8 if prec == qk.FP64 else 4
    prob = workload(args.workload)
    lay = prob.layout
    ctx = qk.Context(lay, prob.params, prec)
    hydro_only = prob.R is None
    dev = torch.device("cuda", local)
    U = [torch.from_numpy(a).to(dev, tdt) for a in prob.U]
    R = None if hydro_only else [torch.from_numpy(a).to(dev, tdt) for a in prob.R]
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(args.warmup):
        ctx.step(U, R)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        ctx.step(U, R)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    t_dev = ev0.elapsed_time(ev1) / 1e3
    clk = clocks.stop()
    rc, flags, bad, maxit = ctx.status()
    if rc != qk.OK:
        raise SystemExit(f"exchange status {rc} flags {flags} first bad cell {bad}")
    tt = torch.tensor([t_dev], device=dev, dtype=torch.float64)
    if world > 1:
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    t_max = float(tt.item())
    cells = lay.ncells
    value = cells * args.steps * world / t_max

    # ---- end to end through the public API with host buffers ----
    hostU = [torch.from_numpy(a).to(tdt).pin_memory() for a in prob.U]
    hostR = None if hydro_only else [torch.from_numpy(a).to(tdt).pin_memory() for a in prob.R]
    outU = [torch.empty_like(h).pin_memory() for h in hostU]
    outR = None if hydro_only else [torch.empty_like(h).pin_memory() for h in hostR]
    fields_h = hostU + (hostR or [])
    fields_o = outU + (outR or [])
    dfields = U + (R or [])
    h2d = sum(h.numel() * h.element_size() for h in fields_h)
    d2h = h2d

    def e2e_step():
        for d, h in zip(dfields, fields_h):
            d.copy_(h, non_blocking=True)
        ctx.step(U, R)
        for o, d in zip(fields_o, dfields):
            o.copy_(d, non_blocking=True)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    t_e2e = e0.elapsed_time(e1) / 1e3
    te = torch.tensor([t_e2e], device=dev, dtype=torch.float64)
    if world > 1:
        dist.all_reduce(te, op=dist.ReduceOp.MAX)
    e2e_value = cells * args.steps * world / float(te.item())

    # ---- dominant kernel, timed alone through its entry point ----
    pk, pk_kind = peaks()
    reps = 20
    if hydro_only:
        U1 = [torch.empty_like(a) for a in U]
        ctx.fill_ghosts(U)
        dt = ctx.timestep(U)[0]
        kname = "hydro1"
        t_k = time_kernel(torch, lambda: ctx.hydro_stage(1, U, None, U1, dt), reps, stream)
    else:
        R1 = [torch.empty_like(a) for a in R]
        ctx.fill_ghosts(R + [U[0]])
        dtr = ctx.timestep(U)[2]
        kname = "rad1"
        t_k = time_kernel(torch, lambda: ctx.rad_stage(1, R, None, R1, U[0], dtr), reps, stream)
    bytes_launch = algorithmic_bytes_per_cell(kname, elem) * cells
    flops_launch = ALGO_FLOPS[kname] * cells
    hbm_ach = bytes_launch / t_k / 1e9
    hbm_peak = pk.get("hbm_gbs", FALLBACK_HBM_GBS)
    alu_peak = FP64_PEAK_TFLOPS if prec == qk.FP64 else FP32_PEAK_TFLOPS
    alu_ach = flops_launch / t_k / 1e12
    kern = {"hydro1": "hydro_stage_kernel<%s,1>", "rad1": "rad_stage_kernel<%s,1>"}[kname] % (
        "double" if prec == qk.FP64 else "float")
    hbm = {"bound": "hbm", "achieved": hbm_ach, "peak": hbm_peak, "unit": "GB/s",
           "frac": hbm_ach / hbm_peak, "peak_source": f"{pk_kind} (MEASURED_PEAKS.json hbm_gbs)"}
    alu = {"bound": "alu", "achieved": alu_ach, "peak": alu_peak, "unit": "TFLOP/s",
           "frac": alu_ach / alu_peak,
           "peak_source": ("FP64" if prec == qk.FP64 else "FP32") +
                          " unit counts x 2.07 GHz (no measured FP64/FP32 peak in MEASURED_PEAKS.json)"}
    main_, other = (alu, hbm) if alu["frac"] >= hbm["frac"] else (hbm, alu)
    roofline = dict(main_, kernel=kern, traffic=None, launch_s=t_k,
                    algorithmic_bytes_per_launch=bytes_launch,
                    algorithmic_flops_per_launch=flops_launch, other=other)

    ctx.close()
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    cpu = None if args.no_cpu_baseline or world > 1 else cpu_baseline(args.precision)
    variants = None if args.no_variants or world > 1 else run_variants(args)
    nl = launches_per_step(hydro_only, int(prob.params.get("nsub_max", 10)))
    line = {
        "metric": "cell-updates/s", "value": value, "unit": "cell-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if prec == qk.FP64 else "f32+f64", "data": "synthetic",
        "config": dict(describe(args.workload, prob, args.precision),
                       l2="inputs larger than L2 (state %.0f MB > 129 MB), no flush" %
                          (h2d / 1e6), parallelism=f"{world} independent replica(s)"),
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "cell-updates/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": nl * args.steps,
        "clocks": clk,
        "variants": variants,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rhd128")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
