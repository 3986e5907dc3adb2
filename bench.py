"""Benchmark: cell-updates/s of the per-cell uniform-patch RHD update on GB300.

Default workload: 3-D periodic 128^3 RHD, FP64 (lognormal density with a |k|^-4
Gaussian random field, sigma_ln rho = 1, T_gas = 1, T_r ~ U(0.5, 2),
kappa_P = kappa_R = 1, a_r = 1, c = 100, chat = 10 max c_s, CFL 0.3,
N_sub,max = 10).  A "step" is one full update: hydro RK2 stage pair plus every
radiation substep (RK2 pair + exchange); one cell-update is one cell advanced
by one such step (the paper's Mzones/s unit, Sec. 4).

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                [--workload rhd128|hydro128|...] [--precision fp64|fp32]
                [--mode sharded|replicas]
Prints ONE JSON line (rank 0).  With N = 1 it times the workload through
qk_step (one CUDA graph per update), then the other precision / size / patch
variants, the 512^3 case and the reduced-precision error report, each in a
compact entry at the end of the line.  Under torchrun (N > 1) the default is
the sharded run: the periodic domain (128 N) x 128 x 128 with one 128^3 patch
per rank (weak scaling), ghost cells moved between ranks over NCCL with the
transfers overlapped with the interior tiles; --mode replicas instead runs N
independent copies of the single-GPU workload.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
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
L2_BYTES = 129e6
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

# values moved per cell-update (face fluxes on chip, Delta t fused, stage 2 in
# place): hydro stage 1 reads 5 and writes 5, stage 2 reads 10 and writes 5;
# a radiation substep with the exchange fused into stage 2 moves 9 + 21
HYDRO_VALUES = 25
SUBSTEP_VALUES = 30


def values_per_update(hydro_only: bool, nsub: float) -> float:
    return HYDRO_VALUES + (0.0 if hydro_only else SUBSTEP_VALUES * nsub)


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
    if name == "rhd32":
        return I.rhd_lognormal(32, steps=20)
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


def hbm_peak() -> float:
    return peaks()[0].get("hbm_gbs", FALLBACK_HBM_GBS)


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


def host_cpu() -> dict:
    """Host core count and CPU model (reported beside the oracle timings)."""
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    model = platform.processor() or platform.machine()
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().startswith("Model name:"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"cores": int(cores or 1), "model": model}


def _oracle_step_timed(O, g, p, U, R, threads):
    O.set_threads(threads)
    try:
        t0 = time.perf_counter()
        rc, ts, _ = O.step(g, p, U, R)
        el = time.perf_counter() - t0
    finally:
        O.set_threads(1)
    if rc != 0:
        raise SystemExit(f"oracle step failed: status {rc}")
    return el, ts


def cpu_baseline(name: str, single_core: bool = True) -> dict:
    """The oracle as it stands on the host cores, on the bench workload itself:
    one full update of its initial state on every host core (z-planes over
    OpenMP threads, bit-identical to one thread) and, beside it, the same
    update on one core."""
    import oracle as O
    prob = workload(name)
    lay = prob.layout
    g = O.Grid(lay.lo, lay.n, lay.off, lay.dom_n, lay.ng)
    p = O.make_params(**prob.params)
    host = host_cpu()
    U = [a.copy() for a in prob.U]
    R = [a.copy() for a in prob.R] if prob.R is not None else None
    el, ts = _oracle_step_timed(O, g, p, U, R, host["cores"])
    out = {"value": lay.ncells / el, "unit": "cell-updates/s", "cores": host["cores"],
           "kind": "oracle", "cpu": host["model"],
           "sample": f"one full update of the {name} initial state ({lay.ncells} cells, "
                     f"N_sub={int(ts[1])}), FP64 oracle on {host['cores']} threads, {el:.1f} s"}
    if single_core:
        U = [a.copy() for a in prob.U]
        R = [a.copy() for a in prob.R] if prob.R is not None else None
        el1, _ = _oracle_step_timed(O, g, p, U, R, 1)
        out["single_core"] = {"value": lay.ncells / el1, "s": round(el1, 2)}
    return out


def run_reference(args):
    """--impl reference: the FP64 oracle on all host cores, each step one full
    update of the same workload as the GPU arm (z-planes over OpenMP threads,
    bit-identical to one thread)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O
    name = args.workload
    prob = workload(name)
    lay = prob.layout
    g = O.Grid(lay.lo, lay.n, lay.off, lay.dom_n, lay.ng)
    p = O.make_params(**prob.params)
    host = host_cpu()
    U = [a.copy() for a in prob.U]
    R = [a.copy() for a in prob.R] if prob.R is not None else None
    O.set_threads(host["cores"])
    try:
        for _ in range(args.warmup):
            O.step(g, p, U, R)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            rc, _, _ = O.step(g, p, U, R)
            if rc != 0:
                raise SystemExit(f"oracle step failed: status {rc}")
        el = time.perf_counter() - t0
    finally:
        O.set_threads(1)
    v = lay.ncells * args.steps / el
    sample = (f"each step one full update of the {name} workload ({lay.ncells} cells), "
              f"FP64 oracle on {host['cores']} host threads")
    line = {"impl": "reference", "metric": "cell-updates/s", "value": v, "unit": "cell-updates/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": describe(name, prob, "fp64"),
            "cpu_baseline": {"value": v, "unit": "cell-updates/s", "cores": host["cores"],
                             "kind": "oracle", "cpu": host["model"], "sample": sample},
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


def working_set(state_bytes: float) -> float:
    """A step reads the whole state and writes the stage-1 copy of it (the
    context's scratch, as large again) before writing the state back."""
    return 2.0 * state_bytes


def l2_note(state_bytes: float) -> str:
    """How the timed steps avoid an L2-resident state: with the working set
    above the 129 MB L2 no flush is added."""
    ws = working_set(state_bytes)
    if ws > L2_BYTES:
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
# (profiles/ncu_*.md), valid only while the kernel's code (comments and
# whitespace removed) hashes to the value recorded at capture time.
NCU_TRAFFIC = {
    ("rhd128", "rad_stage_ex_kernel<double>"): (343.05e6, "rad", "5e02440890a4"),
    ("rhd128", "rad_stage_kernel<double,1>"): (135.91e6, "rad", "5e02440890a4"),
    ("rhd128", "hydro_stage_kernel<double,1>"): (150.50e6, "hydro", "08c0e4e62ed0"),
    ("hydro256", "hydro_column_kernel<float,1>"): (843.54e6, "hydrocol", "a98b6816d223"),
    ("rhd128", "rad_column_kernel<float,2,EX>"): (170.06e6, "radcol", "8bc1abbe78e3"),
    ("rhd128", "rad_column_kernel<float,1>"): (56.11e6, "radcol", "8bc1abbe78e3"),
}


def _strip_code(text: str) -> str:
    """C/C++/CUDA source without its comments and whitespace: what the
    compiler sees of it (the sources quote no comment markers in strings)."""
    import re
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return "".join(text.split())


def _src_hash(kind: str, read=None) -> str:
    """sha1 prefix of a kernel's code (its sources plus qk_device.cuh and
    qk_internal.cuh, comments and whitespace removed); read(name) returns a
    source's text (default: the working tree)."""
    import hashlib
    cs = os.path.join(ROOT, "paper_2110_01792_gb300", "csrc")
    if read is None:
        def read(name):
            with open(os.path.join(cs, name), encoding="utf-8") as fh:
                return fh.read()
    files = {"rad": ["qk_rad.cu", "qk_rad.cuh", "qk_exchange.cuh"], "hydro": ["qk_hydro.cu"],
             "radcol": ["qk_column_rad.cu", "qk_column_rad.cuh", "qk_rad.cuh",
                        "qk_exchange.cuh", "qk_pair.cuh"],
             "hydrocol": ["qk_column.cu", "qk_pair.cuh"],
             "cell": ["qk_cell.cu", "qk_exchange.cuh"]}[kind]
    h = hashlib.sha1()
    for f in files + ["qk_device.cuh", "qk_internal.cuh"]:
        h.update(_strip_code(read(f)).encode())
    return h.hexdigest()[:12]


def ncu_traffic(workload_name: str, kernel: str):
    ent = NCU_TRAFFIC.get((workload_name, kernel))
    if ent is None or _src_hash(ent[1]) != ent[2]:
        return None
    return ent[0]


def _to_device(torch, arrays, dtype, dev="cuda"):
    return [torch.from_numpy(a).to(dev, dtype) for a in arrays]


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
    U = _to_device(torch, prob.U, tdt)
    R = None if prob.R is None else _to_device(torch, prob.R, tdt)
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


def _r(x, n=4):
    """Round to n significant digits (compact JSON)."""
    if x is None:
        return None
    if x == 0 or x != x:
        return x
    from math import floor, log10
    return round(x, -int(floor(log10(abs(x)))) + n - 1)


def stage_kernel_times(torch, ctx, U, R, stream, reps=10, fused=True):
    """Each stage kernel of the update timed alone through its entry point
    (CUDA events on the launching stream): {kernel: seconds per launch}."""
    times = {}
    U1 = [torch.empty_like(a) for a in U]
    U2 = [torch.empty_like(a) for a in U]
    ctx.fill_ghosts(U)
    if ctx.nranks > 1:
        dt, _, dtr, _ = ctx.set_timestep(ctx.signal_speed(U))
    else:
        dt, _, dtr, _ = ctx.timestep(U)
    times["hydro1"] = time_kernel(torch, lambda: ctx.hydro_stage(1, U, None, U1, dt), reps, stream)
    ctx.fill_ghosts(U1)
    times["hydro2"] = time_kernel(torch, lambda: ctx.hydro_stage(2, U, U1, U2, dt), reps, stream)
    del U1, U2
    if R is not None:
        R1 = [torch.empty_like(a) for a in R]
        R2 = [torch.empty_like(a) for a in R]
        ctx.fill_ghosts(R + [U[0]])
        times["rad1"] = time_kernel(torch, lambda: ctx.rad_stage(1, R, None, R1, U[0], dtr),
                                    reps, stream)
        ctx.fill_ghosts(R1)
        Uc = [a.clone() for a in U]
        if fused:
            times["rad2x"] = time_kernel(
                torch, lambda: ctx.rad_stage2_exchange(R, R1, R2, Uc, dtr), reps, stream)
        else:
            times["rad2"] = time_kernel(torch, lambda: ctx.rad_stage(2, R, R1, R2, U[0], dtr),
                                        reps, stream)
            times["exchange"] = time_kernel(torch, lambda: ctx.exchange(Uc, R2, dtr), reps,
                                            stream)
        ctx.status(reset=True)
        del R1, R2, Uc
    return times


def kernel_name(kname: str, fp64: bool, tuned) -> str:
    tname = "double" if fp64 else "float"
    stage_of = {"hydro1": "hydro1", "hydro2": "hydro2", "rad1": "rad1", "rad2": "rad2",
                "rad2x": "rad2"}
    cols = bool(tuned) and kname in stage_of and tuned[stage_of[kname]][1].startswith("columns")
    if cols:
        return {"hydro1": f"hydro_column_kernel<{tname},1>",
                "hydro2": f"hydro_column_kernel<{tname},2>",
                "rad1": f"rad_column_kernel<{tname},1>", "rad2": f"rad_column_kernel<{tname},2>",
                "rad2x": f"rad_column_kernel<{tname},2,EX>"}[kname]
    return {"hydro1": f"hydro_stage_kernel<{tname},1>",
            "hydro2": f"hydro_stage_kernel<{tname},2>",
            "rad1": f"rad_stage_kernel<{tname},1>", "rad2": f"rad_stage_kernel<{tname},2>",
            "rad2x": f"rad_stage_ex_kernel<{tname}>",
            "exchange": "exchange_kernel<double>" if fp64 else "exchange_kernel_mixed"}[kname]


def dominant_roofline(torch, qk, ctx, U, R, prec, tuned, nsub_mean, cells, wname, stream,
                      fused=True):
    """The dominant kernel of the update (largest share of the device time:
    each stage kernel timed alone, weighted by its launches per update),
    reported against the peak of the unit its arithmetic runs on (FP64 for
    the FP64 path; FP32 for the FP32-mixed kernels), from the unit counts and
    clocks and, beside it, from the FMA throughput measured by the library's
    probe; the HBM fraction of the same kernel beside it."""
    times = stage_kernel_times(torch, ctx, U, R, stream, fused=fused)
    weight = {"hydro1": 1.0, "hydro2": 1.0}
    weight.update({k: nsub_mean for k in ("rad1", "rad2", "rad2x", "exchange")})
    share = {k: times[k] * weight[k] for k in times}
    tot_k = sum(share.values())
    kname = max(share, key=share.get)
    t_k = times[kname]
    fp64 = prec == qk.FP64
    elem = 8 if fp64 else 4
    kern = kernel_name(kname, fp64, tuned)
    bytes_launch = algorithmic_bytes_per_cell(kname, elem) * cells
    flops_launch = ALGO_FLOPS[kname] * cells
    pk, pk_kind = peaks()
    hbm_ach = bytes_launch / t_k / 1e9
    hpk = pk.get("hbm_gbs", FALLBACK_HBM_GBS)
    hbm = {"bound": "hbm", "achieved": hbm_ach, "peak": hpk, "unit": "GB/s",
           "frac": hbm_ach / hpk, "peak_source": f"{pk_kind} (MEASURED_PEAKS.json hbm_gbs)"}
    alu_peak = FP64_PEAK_TFLOPS if fp64 else FP32_PEAK_TFLOPS
    alu_ach = flops_launch / t_k / 1e12
    alu_meas = measure_alu_peak(torch, qk, fp64, stream)
    alu = {"bound": "alu", "achieved": alu_ach, "peak": alu_peak, "unit": "TFLOP/s",
           "frac": alu_ach / alu_peak,
           "peak_source": ("FP64" if fp64 else "FP32") +
                          " unit counts x 2.07 GHz (no measured FP64/FP32 peak in "
                          "MEASURED_PEAKS.json)",
           "measured_peak": alu_meas, "frac_of_measured": alu_ach / alu_meas,
           "measured_peak_source": "qk_fma_probe in this run (independent FMA chains, "
                                   "64 warps per SM, best of 3)"}
    main_, other = (alu, hbm) if alu["frac"] >= hbm["frac"] else (hbm, alu)
    return dict(main_, kernel=kern, traffic=ncu_traffic(wname, kern), launch_s=t_k,
                algorithmic_bytes_per_launch=bytes_launch,
                algorithmic_flops_per_launch=flops_launch, other=other,
                kernel_shares={k: _r(v / tot_k, 3) for k, v in share.items()})


def run_variant(torch, qk, name, prec_name, steps, warmup, autotune=True, per_patch=False,
                stage_hbm=False):
    """Cell-updates/s of one workload in one precision through qk_step (device
    time over `steps` full updates after `warmup`), compact: v (cell-updates/s),
    ms (per step), hbm (algorithmic bytes per update x v / measured HBM peak),
    gbs (that algorithmic rate in GB/s), l2 (1: working set below the L2),
    nsub (mean substeps), cfg (tuned shape per stage kernel: c columns, C
    columns of 288 threads, t tiles); with stage_hbm the HBM fraction of each
    hydro stage kernel alone."""
    prob = workload(name)
    p = qk.FP64 if prec_name == "fp64" else qk.FP32_MIXED
    tdt = torch.float64 if p == qk.FP64 else torch.float32
    elem = 8 if p == qk.FP64 else 4
    lay = prob.layout
    ctx = qk.Context(lay, prob.params, p)
    ctx.set_launch_mode(per_patch)
    U = _to_device(torch, prob.U, tdt)
    R = None if prob.R is None else _to_device(torch, prob.R, tdt)
    hydro_only = prob.R is None
    del prob.U, prob.R
    tuned = ctx.autotune(U, R) if autotune else None
    for _ in range(warmup):
        ctx.step(U, R)
    torch.cuda.synchronize()
    i0 = ctx.step_info()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        ctx.step(U, R)
    e1.record()
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    i1 = ctx.step_info()
    ok = ctx.status()[0] == qk.OK
    nsub = (i1[4] - i0[4]) / max(1.0, i1[5] - i0[5])
    v = lay.ncells * steps / t
    bpu = values_per_update(hydro_only, nsub) * elem
    state = sum(a.numel() * a.element_size() for a in U + (R or []))
    out = {"v": _r(v), "ms": _r(1e3 * t / steps), "hbm": _r(v * bpu / 1e9 / hbm_peak(), 3),
           "gbs": _r(v * bpu / 1e9, 3), "l2": int(working_set(state) <= L2_BYTES)}
    if not hydro_only:
        out["nsub"] = _r(nsub, 3)
    if lay.nbox > 1:
        out["patches"] = lay.nbox
    if tuned:
        out["cfg"] = "".join(("C" if tuned[k][0] > 256 else "c")
                             if tuned[k][1].startswith("columns") else "t"
                             for k in ("hydro1", "hydro2", "rad1", "rad2"))
    if not ok:
        out["status"] = "exchange error"
    if stage_hbm:
        st = stage_kernel_times(torch, ctx, U, R, torch.cuda.current_stream())
        cells = lay.ncells
        out["stage_hbm"] = [
            _r(algorithmic_bytes_per_cell(k, elem) * cells / st[k] / 1e9 / hbm_peak(), 3)
            for k in ("hydro1", "hydro2")]
    ctx.close()
    del U, R
    torch.cuda.empty_cache()
    return out


VARIANTS = [
    # (key, workload, precision, steps, warmup, per_patch, stage_hbm)
    ("rhd128_fp64", "rhd128", "fp64", 5, 3, False, False),
    ("rhd128_fp32", "rhd128", "fp32", 10, 3, False, False),
    ("hydro128_fp64", "hydro128", "fp64", 10, 3, False, False),
    ("hydro128_fp32", "hydro128", "fp32", 10, 3, False, False),
    ("hydro256_fp64", "hydro256", "fp64", 5, 3, False, True),
    ("hydro256_fp32", "hydro256", "fp32", 10, 3, False, True),
    ("rhd256_fp32", "rhd256", "fp32", 5, 3, False, False),
    ("patches_fp32", "patches", "fp32", 3, 2, False, False),
    ("patches_fp32_per_patch", "patches", "fp32", 2, 1, True, False),
    ("patches_fp64", "patches", "fp64", 2, 1, False, False),
    # the largest single-grid case: 512^3, sigma_ln rho = 1.5, kappa = kappa0 rho
    ("rhd512_fp64", "rhd512", "fp64", 3, 2, False, False),
    ("rhd512_fp32", "rhd512", "fp32", 5, 2, False, False),
]


def run_variants(args):
    import torch
    from paper_2110_01792_gb300 import qk
    out = {}
    for key, name, prec, st, wu, pp, sh in VARIANTS:
        if name == args.workload and prec == args.precision and not pp:
            continue
        out[key] = run_variant(torch, qk, name, prec, st, wu, autotune=not args.no_autotune,
                               per_patch=pp, stage_hbm=sh)
    return out


def run_precision_report(autotune=True, steps_hydro=10, steps_rhd=20):
    """Per-field error and conservation drift of the reduced-precision forms at
    256^3: the hydro and RHD workloads advanced from the same initial state in
    FP64, FP32-mixed and compensated FP32 (hi + lo per conserved field, lo as
    FP32 or in 16 bits), each with its tuned launch configuration.  The error of each field is the
    relative L1 distance to the GPU's FP64 result (the FP64 path is pinned to
    the oracle to 1e-10 per cell on grids up to 40^3; the oracle itself would
    take hours here).  Drift: max over the steps of |total(t) - total(0)|,
    relative to |total(0)| for sum rho and sum (E + (c/chat) E_r), and to the
    L1 norm of the final momenta (sum |m| + |F|/(c chat)) for each component
    of sum (m + F/(c chat)), a total near zero.  Compact: per form v
    (cell-updates/s), l1 {rho, E, E_r, max over all fields}, drift [rho,
    E_total, momentum]."""
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
        icc = 1.0 / (prob.params["c"] * prob.params["chat"]) if prob.R is not None else 0.0
        results, entry, sums_by = {}, {}, {}

        def lo_parts(arrays, fmt):
            out = []
            for a in arrays:
                hi = a.astype(np.float32)
                res = a - hi.astype(np.float64)
                out.append(torch.from_numpy(qk.lo16_encode(hi, res)).cuda() if fmt == "i16"
                           else torch.from_numpy(res).float().cuda())
            return out

        for form in ("fp64", "fp32", "fp32c", "fp32c16"):
            prec = qk.FP64 if form == "fp64" else qk.FP32_MIXED
            tdt = torch.float64 if prec == qk.FP64 else torch.float32
            ctx = qk.Context(lay, prob.params, prec)
            U = _to_device(torch, prob.U, tdt)
            R = None if prob.R is None else _to_device(torch, prob.R, tdt)
            lo = None
            if form in ("fp32c", "fp32c16"):
                fmt = "i16" if form == "fp32c16" else "f32"
                if fmt == "i16":
                    ctx.set_lo_format(qk.LO_I16)
                lo = (lo_parts(prob.U, fmt), None if R is None else lo_parts(prob.R, fmt))
            if autotune:
                # tuned on a scratch copy so that every form starts from the same state
                Ut = [a.clone() for a in U]
                Rt = None if R is None else [a.clone() for a in R]
                ctx.autotune(Ut, Rt)
                del Ut, Rt
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
                los = lo[0] + (lo[1] or [])
                if form == "fp32c16":
                    fields = [a + qk.lo16_decode(a.astype(np.float32), b.cpu().numpy())
                              for a, b in zip(fields, los)]
                else:
                    fields = [a + b.double().cpu().numpy() for a, b in zip(fields, los)]
            results[form] = [interior(lay, a) for a in fields]
            del U, R, lo, fields
            torch.cuda.empty_cache()
            sums_by[form] = np.array(sums)
            # the first step captures the step graph: timed from the second
            entry[form] = {"v": _r(lay.ncells * (steps - 1) / sum(times[1:])),
                           "bytes_per_value": {"fp64": 8, "fp32": 4, "fp32c": 8,
                                               "fp32c16": 6}[form]}
            if not ok:
                entry[form]["status"] = "exchange error"
        ref = results["fp64"]
        vol = 1.0 / lay.ncells
        mom = [vol * (np.abs(ref[1 + a]).sum() +
                      (icc * np.abs(ref[6 + a]).sum() if prob.R is not None else 0.0))
               for a in range(3)]
        for form, S in sums_by.items():
            d = np.abs(S - S[0]).max(axis=0)
            entry[form]["drift"] = [_r(float(d[0] / abs(S[0, 0])), 2),
                                    _r(float(d[9] / abs(S[0, 9])), 2),
                                    _r(float(max(d[10 + a] / mom[a] for a in range(3))), 2)]
        for form in ("fp32", "fp32c", "fp32c16"):
            l1 = [float(np.abs(results[form][q] - ref[q]).sum() / np.abs(ref[q]).sum())
                  for q in range(len(ref))]
            e = {"rho": _r(l1[0], 2), "E": _r(l1[4], 2), "max": _r(max(l1), 2)}
            if prob.R is not None:
                e["E_r"] = _r(l1[5], 2)
            entry[form]["l1"] = e
        report[name] = entry
        del results, ref
    return report


SUMMARY_KEY = ("v M cell-updates/s; hbm: algorithmic bytes x v / measured HBM peak; hydro256 "
               "+ each hydro stage's; rhd512 + GB/s; prec: [v, B/value, L1 rho, E, (E_r), "
               "max, drift rho, E+(c/chat)E_r, m+F/(c chat)]")


def summary(value, step_hbm, variants, precision, headline) -> dict:
    """The compact record printed last on the line: the headline workload's
    rate (under its own name, e.g. rhd128_fp64), every variant's rate and HBM
    fraction, the 512^3 rates with GB/s, and the precision forms (errors
    against the GPU's FP64 result)."""
    M = lambda v: _r(v / 1e6)
    out = {"key": SUMMARY_KEY, headline: [M(value), step_hbm]}
    for k, d in (variants or {}).items():
        row = [M(d["v"]), d["hbm"]]
        if "stage_hbm" in d:
            row += d["stage_hbm"]
        if k.startswith("rhd512"):
            row.append(d["gbs"])
        if d.get("l2"):
            row.append("in L2")
        out[k] = row
    for name, ent in (precision or {}).items():
        rows = {}
        for form, e in ent.items():
            l1 = e.get("l1")
            row = [M(e["v"]), e["bytes_per_value"]]
            if l1:
                row += [l1["rho"], l1["E"]] + ([l1["E_r"]] if "E_r" in l1 else []) + [l1["max"]]
            rows[form] = row + e["drift"]
        out["prec_" + name.replace("256", "")] = rows
    return out


def _e2e_host_steps(torch, ctx, host, R_present, steps, stream):
    """Device-timed steps through qk_step_host (state in pinned host memory,
    copied in and out by every call); returns seconds."""
    hU, hR = host[:5], (host[5:] if R_present else None)
    snap = [h.clone() for h in host]
    ctx.step_host(hU, hR, stream=stream.cuda_stream)  # allocates the device copy
    for h, h0 in zip(host, snap):
        h.copy_(h0)  # back to the start of the timed steps
    del snap
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        ctx.step_host(hU, hR, stream=stream.cuda_stream)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3


def run_ours(args):
    """N = 1 (or N independent replicas under torchrun with --mode replicas)."""
    import torch
    import torch.distributed as dist

    import __graft_entry__
    from paper_2110_01792_gb300 import qk

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    __graft_entry__.build()
    prec = qk.FP64 if args.precision == "fp64" else qk.FP32_MIXED
    tdt = torch.float64 if prec == qk.FP64 else torch.float32
    prob = workload(args.workload)
    lay = prob.layout
    ctx = qk.Context(lay, prob.params, prec)
    ctx.set_fused_exchange(not args.no_fused_exchange)
    hydro_only = prob.R is None
    dev = torch.device("cuda", local)
    U = _to_device(torch, prob.U, tdt, dev)
    R = None if hydro_only else _to_device(torch, prob.R, tdt, dev)
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
    h2d = sum(h.numel() * h.element_size() for h in host)
    d2h = h2d
    barrier()
    t_e2e = _e2e_host_steps(torch, ctx, host, R is not None, args.steps, stream)
    te = torch.tensor([t_e2e], device=dev, dtype=torch.float64)
    if world > 1:
        dist.all_reduce(te, op=dist.ReduceOp.MAX)
    e2e_value = cells * args.steps * world / float(te.item())

    roofline = dominant_roofline(torch, qk, ctx, U, R, prec, tuned, nsub_mean, cells,
                                 args.workload, stream, fused=not args.no_fused_exchange)
    ctx.close()
    del U, R
    torch.cuda.empty_cache()
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    single = world == 1
    cpu = cpu_baseline(args.workload, not args.no_cpu_single_core) \
        if single and not args.no_cpu_baseline else None
    variants = run_variants(args) if single and not args.no_variants else None
    precision = run_precision_report(not args.no_autotune) \
        if single and not args.no_variants else None
    nl = launches_per_step(hydro_only, int(prob.params.get("nsub_max", 10)),
                           not args.no_fused_exchange)
    elem = 8 if prec == qk.FP64 else 4
    bpu = values_per_update(hydro_only, nsub_mean) * elem
    step_hbm = _r(value / world * bpu / 1e9 / hbm_peak(), 3)
    line = {
        "metric": "cell-updates/s", "value": value, "unit": "cell-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if prec == qk.FP64 else "f32+f64", "data": "synthetic",
        "config": dict(describe(args.workload, prob, args.precision),
                       l2=l2_note(h2d), parallelism=f"{world} independent replica(s)",
                       launch_config=tuned or "default (256 threads, strided tiles)",
                       step_hbm_frac=step_hbm),
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "cell-updates/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": nl * args.steps,
        "nsub_mean": nsub_mean,
        "clocks": clk,
        "precision_report": precision,
        "variants": variants,
        # printed last: the part of the line a tail of the output keeps
        "summary": (summary(value, step_hbm, variants, precision,
                            f"{args.workload}_{args.precision}") if single else None),
    }
    print(json.dumps(line, separators=(",", ":")), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_sharded(args):
    """N ranks (one per GPU) advance the periodic domain (128 N) x 128 x 128,
    one 128^3 patch per rank (the RHD workload's generator per patch, same
    cell size for every N: weak scaling).  Every ghost fill moves the x faces
    between neighbouring ranks: qk_halo_pack, NCCL isend / irecv from a
    separate stream, qk_halo_unpack, with each stage run on its interior tiles
    while the transfer is in flight (shard.RankStepper, overlap on); the
    timestep takes an all-reduce (MAX) of the signal speed."""
    import numpy as np
    import torch
    import torch.distributed as dist

    import __graft_entry__
    from paper_2110_01792_gb300 import inputs as I
    from paper_2110_01792_gb300 import qk
    from paper_2110_01792_gb300 import shard as S

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    __graft_entry__.build()
    prec = qk.FP64 if args.precision == "fp64" else qk.FP32_MIXED
    tdt = torch.float64 if prec == qk.FP64 else torch.float32
    n = 128
    lay = I.make_layout([[n * r, 0, 0] for r in range(world)], [[n, n, n]] * world,
                        (n * world, n, n), 4)
    prob = I.rhd_lognormal(layout=lay, seed=2110)
    prm = dict(prob.params, dx=1.0 / n)
    owner = np.arange(world, dtype=np.int32)
    rlay = S.rank_layout(lay, owner, rank)
    ctx = qk.Context(rlay, prm, prec, owner=owner, rank=rank)
    dev = torch.device("cuda", local)

    def mine(arrays):
        out = []
        for a in arrays:
            r = np.zeros(rlay.field_len)
            rlay.full(r, rank)[...] = lay.full(a, rank)
            out.append(torch.from_numpy(r).to(dev, tdt))
        return out

    U, R = mine(prob.U), mine(prob.R)
    del prob
    st = S.RankStepper(ctx, U, R, overlap=world > 1)
    comm = torch.cuda.Stream() if world > 1 else None

    def one_step():
        if world > 1:
            return S.run_distributed(st, comm)
        return S.run_local([st])[0]

    def barrier():
        if world > 1:
            dist.barrier()

    # one update fills every ghost cell (the remote ones included) before the
    # autotuner times the stage kernels on this state
    one_step()
    tuned = None if args.no_autotune else ctx.autotune(U, R)
    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    host = [d.cpu().pin_memory() for d in U + R]
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    nsubs = []
    ev0.record(stream)
    for _ in range(args.steps):
        nsubs.append(one_step()[1])
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    t_dev = ev0.elapsed_time(ev1) / 1e3
    clk = clocks.stop()
    rc, flags, bad, _ = ctx.status()
    if rc != qk.OK:
        raise SystemExit(f"exchange status {rc} flags {flags} first bad cell {bad}")
    tt = torch.tensor([t_dev], device=dev, dtype=torch.float64)
    if world > 1:
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    t_max = float(tt.item())
    cells = lay.ncells
    value = cells * args.steps / t_max
    nsub_mean = float(np.mean(nsubs))

    # end to end: the rank's state in pinned host memory, copied to the device
    # and back around every step
    h2d = sum(h.numel() * h.element_size() for h in host)
    dU = U + R
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        for d, h in zip(dU, host):
            d.copy_(h, non_blocking=True)
        one_step()
        for d, h in zip(dU, host):
            h.copy_(d, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    te = torch.tensor([e0.elapsed_time(e1) / 1e3], device=dev, dtype=torch.float64)
    if world > 1:
        dist.all_reduce(te, op=dist.ReduceOp.MAX)
    e2e_value = cells * args.steps / float(te.item())

    # a rank's patch is the 128^3 RHD box: the kernel traffic of that workload applies
    roofline = dominant_roofline(torch, qk, ctx, U, R, prec, tuned, nsub_mean, n ** 3,
                                 "rhd128", stream)
    peers = len(st.peers)
    # launches per step: signal speed + timestep; per ghost fill the local fill,
    # one pack and one unpack per peer with cells, and the stage (two parts
    # when overlapped); fills: 2 hydro, rho, 2 per substep
    per_fill = 1 + 2 * peers + (2 if st.overlap else 1)
    launches = sum(2 + 2 * per_fill + (1 + 2 * peers) + 2 * ns * per_fill for ns in nsubs)
    ctx.close()
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    line = {
        "metric": "cell-updates/s", "value": value, "unit": "cell-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if prec == qk.FP64 else "f32+f64", "data": "synthetic",
        "config": {"workload": f"sharded RHD ({n * world}x{n}x{n} periodic, one {n}^3 patch "
                               f"per rank, {args.precision})",
                   "cells": cells, "ghost": 4, "patches": world, "precision": args.precision,
                   "l2": l2_note(h2d),
                   "parallelism": (f"{world} ranks, patches sharded, NCCL halo exchange overlapped"
                                   if world > 1 else "1 rank (sharded path, no halo)"),
                   "launch_config": tuned or "default"},
        "roofline": roofline,
        "cpu_baseline": None,
        "e2e": {"value": e2e_value, "unit": "cell-updates/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": h2d},
        "gpu_launches": launches,
        "nsub_mean": nsub_mean,
        "clocks": clk,
    }
    print(json.dumps(line, separators=(",", ":")), flush=True)
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
    ap.add_argument("--mode", default=None, choices=["sharded", "replicas"],
                    help="N > 1: sharded weak-scaling run (default) or independent replicas")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-cpu-single-core", action="store_true",
                    help="skip the single-core oracle timing beside the all-cores one")
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
    world = int(os.environ.get("WORLD_SIZE", "1"))
    mode = args.mode or ("sharded" if world > 1 else "replicas")
    if args.kernel_only:
        run_kernel_only(args)
    elif args.impl == "reference":
        run_reference(args)
    elif mode == "sharded":
        run_sharded(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
