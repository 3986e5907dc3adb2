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
# radiation stage 2 with the exchange in its epilogue (what qk_step launches)
ALGO_FLOPS["rad2x"] = ALGO_FLOPS["rad2"] + ALGO_FLOPS["exchange"]

# kernels launched per step (captured in one CUDA graph; substeps beyond N_sub
# are predicated off but still launched)
def launches_per_step(hydro_only: bool, nsub_max: int, fused: bool = True) -> int:
    n = 2 + 2 + 2  # max-speed + timestep, 2 ghost fills, 2 hydro stages
    if not hydro_only:
        # rho ghost fill; per substep: 2 fills, 2 rad stages (+ the exchange
        # unless it runs in the epilogue of stage 2)
        n += 1 + nsub_max * (4 if fused else 5)
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
    exchange reads 9, writes 8; stage 2 with the exchange fused reads 8 + rho
    + m, E (12 + 1), writes 4 + m, E (8)."""
    vals = {"hydro1": 10, "hydro2": 15, "rad1": 9, "rad2": 13, "exchange": 17,
            # fused: the exchange's E_r, F come from the stage, rho is read once
            "rad2x": 21}[kernel]
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


def measure_alu_peak(torch, qk, fp64: bool, stream) -> float:
    """FMA throughput of this GPU in TFLOP/s from the library's probe
    (qk_fma_probe: 8 independent FMA chains per thread, 64 warps per SM),
    best of three launches timed with CUDA events on `stream`."""
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    sink = torch.empty(8 * 256 * nsm, dtype=torch.float64 if fp64 else torch.float32,
                       device="cuda")
    iters = 2000 if fp64 else 100000      # ~10 ms per launch
    h = stream.cuda_stream
    qk.fma_probe(fp64, iters, sink, h)
    best = 0.0
    for _ in range(3):
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        fl = qk.fma_probe(fp64, iters, sink, h)
        ev1.record(stream)
        torch.cuda.synchronize()
        best = max(best, fl / (ev0.elapsed_time(ev1) / 1e3) / 1e12)
    return best


def l2_note(state_bytes: float) -> str:
    """How the timed steps avoid an L2-resident state: a step reads the whole
    state and writes the stage-1 copy of it (the context's scratch, as large
    again) before writing the state back, so its working set is twice the
    state; with that above the 129 MB L2 no flush is added."""
    ws = 2.0 * state_bytes
    if ws > 129e6:
        return ("working set larger than L2 (state %.0f MB + its stage-1 copy %.0f MB > 129 MB),"
                " no flush" % (state_bytes / 1e6, state_bytes / 1e6))
    return ("working set %.0f MB below the 129 MB L2: timings of this workload include L2 reuse"
            % (ws / 1e6))


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


# dram__bytes_read.sum + dram__bytes_write.sum per launch from one ncu capture
# (profiles/ncu_*_128.md), valid only while the kernel's sources hash to the
# value recorded at capture time.
NCU_TRAFFIC = {
    ("rhd128", "rad_stage_ex_kernel<double>"): (342.76e6, "rad", "8d7d55bb2947"),
    ("rhd128", "rad_stage_kernel<double,1>"): (135.02e6, "rad", "8d7d55bb2947"),
    ("rhd128", "hydro_stage_kernel<double,1>"): (150.91e6, "hydro", "89f91359c44a"),
    ("rhd128", "rad_column_kernel<float,2,EX>"): (164.92e6, "radcol", "715cee76a212"),
    ("rhd128", "rad_column_kernel<float,1>"): (54.69e6, "radcol", "715cee76a212"),
    ("rhd128", "hydro_column_kernel<float,1>"): (58.73e6, "hydrocol", "f2e0909c7b7a"),
}


def _src_hash(kind: str) -> str:
    import hashlib
    cs = os.path.join(ROOT, "paper_2110_01792_gb300", "csrc")
    files = {"rad": ["qk_rad.cu", "qk_rad.cuh", "qk_exchange.cuh"], "hydro": ["qk_hydro.cu"],
             "radcol": ["qk_column_rad.cu", "qk_column_rad.cuh", "qk_rad.cuh",
                        "qk_exchange.cuh"],
             "hydrocol": ["qk_column.cu"],
             "cell": ["qk_cell.cu", "qk_exchange.cuh"]}[kind]
    h = hashlib.sha1()
    for f in files + ["qk_device.cuh", "qk_internal.cuh"]:
        with open(os.path.join(cs, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def ncu_traffic(workload: str, kernel: str):
    ent = NCU_TRAFFIC.get((workload, kernel))
    if ent is None or _src_hash(ent[1]) != ent[2]:
        return None
    return ent[0]


def run_kernel_only(args):
    """Launch one stage kernel three times on the workload through the C ABI
    (a small, self-contained case for ncu --set full)."""
    import torch
    import __graft_entry__
    from paper_2110_01792_gb300 import qk
    __graft_entry__.build()
    prec = qk.FP64 if args.precision == "fp64" else qk.FP32_MIXED
    tdt = torch.float64 if prec == qk.FP64 else torch.float32
    prob = workload(args.workload)
    ctx = qk.Context(prob.layout, prob.params, prec)
    U = [torch.from_numpy(a).cuda().to(tdt) for a in prob.U]
    R = None if prob.R is None else [torch.from_numpy(a).cuda().to(tdt) for a in prob.R]
    if args.tile_shape == "auto":
        tuned = None if args.no_autotune else ctx.autotune(U, R)
    else:
        # pinned launch configuration (deterministic captures)
        cfg = (256, "columns") if args.tile_shape == "columns" else (args.threads, "strided")
        tuned = {k: cfg for k in ("hydro1", "hydro2", "rad1", "rad2")}
        ctx.set_launch_config(tuned)
    ctx.fill_ghosts(U + (R or []))
    dt, _, dtr, _ = ctx.timestep(U)
    for _ in range(3):
        if args.kernel_only == "hydro1":
            ctx.hydro_stage(1, U, None, [torch.empty_like(a) for a in U], dt)
        elif args.kernel_only == "rad1":
            ctx.rad_stage(1, R, None, [torch.empty_like(a) for a in R], U[0], dtr)
        elif args.kernel_only == "rad2x":
            R1 = [a.clone() for a in R]
            ctx.rad_stage2_exchange(R, R1, [torch.empty_like(a) for a in R], U, dtr)
        else:
            ctx.exchange(U, R, dtr)
    torch.cuda.synchronize()
    ctx.close()
    print(json.dumps({"kernel_only": args.kernel_only, "workload": args.workload,
                      "precision": args.precision, "launch_config": tuned, "ok": True}))


def run_variants(args, steps=5, warmup=3):
    """Cell-updates/s of the other precision / physics / size combinations and
    of the ~1700-patch set (batched persistent launches vs one launch per patch)
    on the same GPU (device time over `steps` full updates after `warmup`)."""
    import torch
    from paper_2110_01792_gb300 import qk
    out = {}
    specs = [("rhd128", "fp32", False, steps, warmup), ("hydro128", "fp64", False, steps, warmup),
             ("hydro128", "fp32", False, steps, warmup), ("rhd128", "fp64", False, steps, warmup),
             ("rhd256", "fp32", False, steps, warmup), ("hydro256", "fp32", False, steps, warmup),
             ("patches", "fp32", False, 3, 2), ("patches", "fp32", True, 3, 2),
             ("patches", "fp64", False, 2, 1)]
    for name, prec, per_patch, st_, wu in specs:
        if name == args.workload and prec == args.precision and not per_patch:
            continue
        prob = workload(name)
        p = qk.FP64 if prec == "fp64" else qk.FP32_MIXED
        tdt = torch.float64 if p == qk.FP64 else torch.float32
        ctx = qk.Context(prob.layout, prob.params, p)
        ctx.set_launch_mode(per_patch)
        U = [torch.from_numpy(a).cuda().to(tdt) for a in prob.U]
        R = None if prob.R is None else [torch.from_numpy(a).cuda().to(tdt) for a in prob.R]
        del prob.U, prob.R
        tuned = None if args.no_autotune else ctx.autotune(U, R)
        for _ in range(wu):
            ctx.step(U, R)
        torch.cuda.synchronize()
        i0 = ctx.step_info()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(st_):
            ctx.step(U, R)
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        i1 = ctx.step_info()
        stt = ctx.status()
        ctx.close()
        key = f"{name}_{prec}" + ("_per_patch_launches" if per_patch else "")
        out[key] = {"value": prob.layout.ncells * st_ / t, "unit": "cell-updates/s",
                    "ms_per_step": 1e3 * t / st_, "steps": st_,
                    "nsub_mean": (i1[4] - i0[4]) / max(1.0, i1[5] - i0[5]),
                    "patches": prob.layout.nbox, "status_ok": stt[0] == qk.OK,
                    "launch_config": tuned}
        del U, R
        torch.cuda.empty_cache()
    return out


def run_precision_report(steps_hydro=10, steps_rhd=20):
    """Per-field error and conservation drift of the reduced-precision forms at
    256^3: the hydro and RHD workloads advanced from the same initial state in
    FP64, FP32-mixed and compensated FP32 (hi + lo per conserved field).  The
    error of each field is the relative L1 distance to the FP64 result (the
    FP64 path matches the oracle to 1e-10 per cell; the oracle itself would
    take hours at this size).  Drift: max over the steps of |total(t) -
    total(0)|, relative to |total(0)| for sum rho and sum (E + (c/chat) E_r),
    and to the L1 norm of the final momenta (sum |m| + |F|/(c chat)) for each
    component of sum (m + F/(c chat)), a total near zero.  Also the
    cell-updates/s of each form."""
    import numpy as np
    import torch
    from paper_2110_01792_gb300 import qk

    def interior(lay, a):
        g = lay.ng
        out = []
        for b in range(lay.nbox):
            n = lay.n[b]
            blk = a[lay.off[b]:lay.off[b] + int(np.prod(n + 2 * g))].reshape(
                n[2] + 2 * g, n[1] + 2 * g, n[0] + 2 * g)
            out.append(blk[g:g + n[2], g:g + n[1], g:g + n[0]].ravel())
        return np.concatenate(out)

    report = {}
    for name, steps in (("hydro256", steps_hydro), ("rhd256", steps_rhd)):
        prob = workload(name)
        lay = prob.layout
        cr = prob.params["c"] / prob.params["chat"] if prob.R is not None else 0.0
        icc = 1.0 / (prob.params["c"] * prob.params["chat"]) if prob.R is not None else 0.0
        results, entry, sums_by = {}, {}, {}
        for form in ("fp64", "fp32", "fp32_compensated"):
            prec = qk.FP64 if form == "fp64" else qk.FP32_MIXED
            tdt = torch.float64 if prec == qk.FP64 else torch.float32
            ctx = qk.Context(lay, prob.params, prec)
            U = [torch.from_numpy(a).cuda().to(tdt) for a in prob.U]
            R = None if prob.R is None else [torch.from_numpy(a).cuda().to(tdt) for a in prob.R]
            lo = None
            if form == "fp32_compensated":
                lo = ([torch.from_numpy(a - a.astype(np.float32)).float().cuda() for a in prob.U],
                      None if R is None else
                      [torch.from_numpy(a - a.astype(np.float32)).float().cuda() for a in prob.R])
            sums = [ctx.conserved_sums(U, R, lo=lo)]
            times = []
            for _ in range(steps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                ctx.step(U, R, lo=lo)
                e1.record()
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1) / 1e3)
                sums.append(ctx.conserved_sums(U, R, lo=lo))
            ok = ctx.status()[0] == qk.OK
            ctx.close()
            fields = [u.double().cpu().numpy() for u in U + (R or [])]
            if lo is not None:
                fields = [a + b.double().cpu().numpy() for a, b in zip(fields, lo[0] + (lo[1] or []))]
            results[form] = [interior(lay, a) for a in fields]
            del U, R, lo, fields
            torch.cuda.empty_cache()
            sums_by[form] = np.array(sums)
            entry[form] = {
                # the first step captures the step graph: timed from the second
                "cell_updates_per_s": lay.ncells * (steps - 1) / sum(times[1:])
                if steps > 1 else None,
                "status_ok": ok}
        # drift scales: |total(0)| for rho and E + (c/chat) E_r; for the
        # momentum totals (near zero) the L1 norm sum |m| + |F|/(c chat) of
        # the final FP64 state, times the cell volume as in the sums
        ref = results["fp64"]
        vol = 1.0 / lay.ncells
        mom = [vol * (np.abs(ref[1 + a]).sum() +
                      (icc * np.abs(ref[6 + a]).sum() if prob.R is not None else 0.0))
               for a in range(3)]
        for form, S in sums_by.items():
            d = np.abs(S - S[0]).max(axis=0)
            entry[form]["drift"] = {
                "rho": float(d[0] / abs(S[0, 0])),
                "E_total": float(d[9] / abs(S[0, 9])),
                "momentum": float(max(d[10 + a] / mom[a] for a in range(3)))}
        names = ["rho", "m_x", "m_y", "m_z", "E", "E_r", "F_x", "F_y", "F_z"]
        for form in ("fp32", "fp32_compensated"):
            entry[form]["rel_l1_vs_fp64"] = {
                names[q]: float(np.abs(results[form][q] - ref[q]).sum() / np.abs(ref[q]).sum())
                for q in range(len(ref))}
        entry["steps"] = steps
        entry["cells"] = lay.ncells
        report[name] = entry
        del results, ref
    return report


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
    ctx.set_fused_exchange(not args.no_fused_exchange)
    hydro_only = prob.R is None
    dev = torch.device("cuda", local)
    U = [torch.from_numpy(a).to(dev, tdt) for a in prob.U]
    R = None if hydro_only else [torch.from_numpy(a).to(dev, tdt) for a in prob.R]
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()

    tuned = None if args.no_autotune else ctx.autotune(U, R)
    for _ in range(args.warmup):
        ctx.step(U, R)
    torch.cuda.synchronize()
    # the state the timed steps start from, replayed by the end-to-end run so
    # that both time the same steps (N_sub changes as the state evolves)
    host = [d.cpu().pin_memory() for d in U + (R or [])]
    info_start = ctx.step_info()
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

    info_end = ctx.step_info()
    nsub_mean = (info_end[4] - info_start[4]) / max(1.0, info_end[5] - info_start[5])

    # ---- end to end through the public API with a host-resident state ----
    # the state lives in pinned host memory (from the start of the timed
    # steps); every step is one qk_step_host call, which copies it to the
    # device, runs the update and copies it back (in place)
    h2d = sum(h.numel() * h.element_size() for h in host)
    d2h = h2d
    hU, hR = host[:5], (host[5:] if R is not None else None)

    def e2e_step():
        ctx.step_host(hU, hR, stream=stream.cuda_stream)

    snap = [h.clone() for h in host]
    e2e_step()  # allocates the context's device copy of the state
    for h, h0 in zip(host, snap):
        h.copy_(h0)  # back to the start of the timed steps
    del snap
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

    # ---- dominant kernel: each kernel of the step timed alone through its
    # entry point (CUDA events on the launching stream), weighted by its
    # launches per update; the largest share is reported against the peak of
    # the unit its arithmetic runs on (FP64 for the FP64 path; FP32 for the
    # FP32-mixed kernels), from the unit counts and clocks and, beside it,
    # from the FMA throughput measured by the library's probe ----
    pk, pk_kind = peaks()
    reps = 10
    fused = not args.no_fused_exchange
    times = {}
    U1 = [torch.empty_like(a) for a in U]
    U2 = [torch.empty_like(a) for a in U]
    ctx.fill_ghosts(U)
    dt, _, dtr, _ = ctx.timestep(U)
    times["hydro1"] = (time_kernel(torch, lambda: ctx.hydro_stage(1, U, None, U1, dt), reps,
                                   stream), 1.0)
    ctx.fill_ghosts(U1)
    times["hydro2"] = (time_kernel(torch, lambda: ctx.hydro_stage(2, U, U1, U2, dt), reps,
                                   stream), 1.0)
    del U1, U2
    if not hydro_only:
        R1 = [torch.empty_like(a) for a in R]
        R2 = [torch.empty_like(a) for a in R]
        ctx.fill_ghosts(R + [U[0]])
        times["rad1"] = (time_kernel(torch, lambda: ctx.rad_stage(1, R, None, R1, U[0], dtr),
                                     reps, stream), nsub_mean)
        ctx.fill_ghosts(R1)
        Uc = [a.clone() for a in U]
        if fused:
            times["rad2x"] = (time_kernel(
                torch, lambda: ctx.rad_stage2_exchange(R, R1, R2, Uc, dtr), reps, stream),
                nsub_mean)
        else:
            times["rad2"] = (time_kernel(torch, lambda: ctx.rad_stage(2, R, R1, R2, U[0], dtr),
                                         reps, stream), nsub_mean)
            times["exchange"] = (time_kernel(torch, lambda: ctx.exchange(Uc, R2, dtr), reps,
                                             stream), nsub_mean)
        ctx.status(reset=True)
        del R1, R2, Uc
    kname = max(times, key=lambda k: times[k][0] * times[k][1])
    tot_k = sum(v[0] * v[1] for v in times.values())
    t_k = times[kname][0]
    tname = "double" if prec == qk.FP64 else "float"
    stage_of = {"hydro1": "hydro1", "hydro2": "hydro2", "rad1": "rad1", "rad2": "rad2",
                "rad2x": "rad2"}
    cols = bool(tuned) and kname in stage_of and tuned[stage_of[kname]][1] == "columns"
    if cols:
        kern = {"hydro1": f"hydro_column_kernel<{tname},1>",
                "hydro2": f"hydro_column_kernel<{tname},2>",
                "rad1": f"rad_column_kernel<{tname},1>", "rad2": f"rad_column_kernel<{tname},2>",
                "rad2x": f"rad_column_kernel<{tname},2,EX>"}[kname]
    else:
        kern = {"hydro1": f"hydro_stage_kernel<{tname},1>",
                "hydro2": f"hydro_stage_kernel<{tname},2>",
                "rad1": f"rad_stage_kernel<{tname},1>", "rad2": f"rad_stage_kernel<{tname},2>",
                "rad2x": f"rad_stage_ex_kernel<{tname}>",
                "exchange": "exchange_kernel<double>" if prec == qk.FP64
                            else "exchange_kernel_mixed"}[kname]
    bytes_launch = algorithmic_bytes_per_cell(kname, elem) * cells
    flops_launch = ALGO_FLOPS[kname] * cells
    hbm_ach = bytes_launch / t_k / 1e9
    hbm_peak = pk.get("hbm_gbs", FALLBACK_HBM_GBS)
    fp64_unit = prec == qk.FP64
    alu_peak = FP64_PEAK_TFLOPS if fp64_unit else FP32_PEAK_TFLOPS
    alu_ach = flops_launch / t_k / 1e12
    hbm = {"bound": "hbm", "achieved": hbm_ach, "peak": hbm_peak, "unit": "GB/s",
           "frac": hbm_ach / hbm_peak, "peak_source": f"{pk_kind} (MEASURED_PEAKS.json hbm_gbs)"}
    alu_meas = measure_alu_peak(torch, qk, fp64_unit, stream)
    alu = {"bound": "alu", "achieved": alu_ach, "peak": alu_peak, "unit": "TFLOP/s",
           "frac": alu_ach / alu_peak,
           "peak_source": ("FP64" if fp64_unit else "FP32") +
                          " unit counts x 2.07 GHz (no measured FP64/FP32 peak in MEASURED_PEAKS.json)",
           "measured_peak": alu_meas, "frac_of_measured": alu_ach / alu_meas,
           "measured_peak_source": "qk_fma_probe in this run (independent FMA chains, "
                                   "64 warps per SM, best of 3)"}
    main_, other = (alu, hbm) if alu["frac"] >= hbm["frac"] else (hbm, alu)
    roofline = dict(main_, kernel=kern, traffic=ncu_traffic(args.workload, kern),
                    launch_s=t_k, algorithmic_bytes_per_launch=bytes_launch,
                    algorithmic_flops_per_launch=flops_launch, other=other,
                    kernel_s_per_update={k: v[0] * v[1] for k, v in times.items()},
                    kernel_shares={k: v[0] * v[1] / tot_k for k, v in times.items()})

    ctx.close()
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    cpu = None if args.no_cpu_baseline or world > 1 else cpu_baseline(args.precision)
    variants = None if args.no_variants or world > 1 else run_variants(args)
    precision = None if args.no_variants or world > 1 else run_precision_report()
    nl = launches_per_step(hydro_only, int(prob.params.get("nsub_max", 10)),
                           not args.no_fused_exchange)
    line = {
        "metric": "cell-updates/s", "value": value, "unit": "cell-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if prec == qk.FP64 else "f32+f64", "data": "synthetic",
        "config": dict(describe(args.workload, prob, args.precision),
                       l2=l2_note(h2d), parallelism=f"{world} independent replica(s)",
                       launch_config=tuned or "default (256 threads, strided tiles)"),
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "cell-updates/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": nl * args.steps,
        "nsub_mean": nsub_mean,
        "clocks": clk,
        "variants": variants,
        "precision_report": precision,
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
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-fused-exchange", action="store_true",
                    help="run the exchange as its own launch after radiation stage 2")
    ap.add_argument("--tile-shape", choices=["auto", "tiles", "columns"], default="auto",
                    help="with --kernel-only: autotune, or pin 8^3 tiles / 16x16 columns")
    ap.add_argument("--threads", type=int, default=256, choices=[128, 256, 512],
                    help="with --kernel-only --tile-shape tiles: threads per 8^3 tile CTA")
    ap.add_argument("--kernel-only", choices=["hydro1", "rad1", "rad2x", "exchange"], default=None,
                    help="launch one stage kernel 3 times and exit (for ncu captures)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.kernel_only:
        run_kernel_only(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
