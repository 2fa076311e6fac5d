"""Benchmark of the RT step (injection + transport + thermochemistry +
photon budget) on GB300 through the rtgb C-ABI.

Metric: cell-group RT updates per second = cells x groups x steps / time.
Default workload: the 128^3, 3-group, H+He, evolving-temperature HLL
cosmological box with 16 sources (synthetic seeded log-normal density),
200 steps from its initial state, FP64.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-group RT updates/s (transport+thermochem)"
UNIT = "cell-group updates/s"

# Denominators.  HBM: the measured copy bandwidth of this GB300 pool
# (MEASURED_PEAKS.json when present).  FP64 and FP32: cuBLAS DGEMM and SGEMM
# (TF32 off) measured in the same run (measure_fp_peaks), the library's own
# best FMA throughput on this part.
# Algorithmic work per unit: the op-counting build of the oracle
# (oracle/make_counts.py writes tests/golden/op_counts.json): FP64 flops per
# thermochemistry attempt and per transport cell-group, as the oracle states
# the method.  Transport bytes: N, F read and written once per cell-group.
# the library's default routing: attempts of the first pass, and of the
# first lane-per-cell drain stage
PASS1_ATTEMPTS = 6
DRAIN1_BUDGET = 128
# DRAM bytes (read + write) per launch, from the ncu captures of the current
# kernels summarised in profiles/ (128^3 x 3 groups, HLL)
TRAFFIC = {"transport": 399187712 + 192541696,
           # the two drains and thermo_hard of one step (the phase's three kernels)
           "thermo_drain": 830720 + 77568 + 594688 + 5888}


def _op_counts():
    d = json.load(open(os.path.join(ROOT, "tests", "golden", "op_counts.json")))
    return d["thermo_per_attempt"], d["transport_per_cell_group"]


def measure_fp_peaks():
    """FP64 and FP32 FMA throughput of this GPU: cuBLAS DGEMM (4096^3) and
    SGEMM with TF32 off (8192^3) through torch.matmul, best of 5 (CUDA
    events), in GFLOP/s."""
    import torch
    out = {}
    tf32 = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        for name, dtype, n in (("fp64", torch.float64, 4096), ("fp32", torch.float32, 8192)):
            a = torch.randn(n, n, dtype=dtype, device="cuda")
            b = torch.randn(n, n, dtype=dtype, device="cuda")
            c = torch.matmul(a, b)
            best = None
            for _ in range(5):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(a, b, out=c)
                e1.record()
                e1.synchronize()
                t = e0.elapsed_time(e1) / 1e3
                best = t if best is None else min(best, t)
            out[name + "_gflops"] = 2.0 * n ** 3 / best / 1e9
            del a, b, c
    finally:
        torch.backends.cuda.matmul.allow_tf32 = tf32
    out["how"] = "cuBLAS DGEMM 4096^3 and SGEMM 8192^3 (TF32 off) via torch.matmul, best of 5"
    return out


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        self.f.flush()
        rows = []
        try:
            for line in open(self.f.name):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        finally:
            os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x, ws, device):
    """The largest x over the ranks of the default process group (x itself
    on one rank): the job's time is its slowest rank's."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_units(units_per_rank, ws):
    """Cell-group updates of the whole job: every rank runs its own replica
    of the workload (weak scaling, no exchange between ranks)."""
    return units_per_rank * ws


def workload(name):
    from paper_1304_7126_gb300 import workloads as W
    return {"cosmo128": W.cosmo128, "stromgren32": W.stromgren32, "cosmo256": W.cosmo256}[name]()


def run_reference(args):
    """The FP64 CPU oracle on this host's cores, on the GPU arm's workload and
    metric: after min(W, 1) untimed warm-up step, K RT steps of the full
    workload from its initial state (stopping early, with the steps done
    reported, if they take more than four minutes)."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    from oracle import oracle as O
    w = workload(args.workload)
    cores = os.cpu_count() or 1
    p = O.Problem(w.shape, w.dx, w.G, w.cr, w.sigN, w.sigE, w.egy, X=w.X,
                  isothermal=w.isothermal, otsa=w.otsa, flux=w.flux, bc=w.bc, nthreads=cores)
    dt = O.courant_dt(w.cfl, w.dx, w.cr)
    s = w.state()
    for _ in range(min(args.warmup, 1)):
        p.step(s, dt, w.src_ijk, w.src_L)
    s = w.state()
    t0 = time.perf_counter()
    n = 0
    while n < args.steps:
        st, _, _, _ = p.step(s, dt, w.src_ijk, w.src_L)
        assert st == 0
        n += 1
        if time.perf_counter() - t0 > 240.0:
            break
    t = time.perf_counter() - t0
    val = w.ncells * w.G * n / t
    sample = "RT steps 1-%d of the full %s workload from its initial state (%d requested)" % (n, w.name, args.steps)
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / n,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _config(w),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                             "cpu": cpu_info()["cpu"]},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _config(w):
    nz, ny, nx = w.shape
    return {"workload": "%s: %dx%dx%d cells, %d groups, %s, %s, X=%.2f, %d sources, c_r=c/%g, %d steps"
            % (w.name, nx, ny, nz, w.G, "HLL" if w.flux == 1 else "GLF",
               "isothermal" if w.isothermal else "evolving T", w.X, len(w.src_ijk),
               round(2.99792458e10 / w.cr), w.steps),
            "cells": w.ncells, "groups": w.G, "precision": "fp64",
            "l2": "inputs larger than L2 (state %.0f MB)" % ((5 + 8 * w.G) * w.ncells * 8 / 1e6)}


# kernels each profiled phase of one RT step launches (the thermochemistry
# drain phase: two lane-per-cell drains and the warp-per-cell kernel)
KERNELS_PER_PHASE = {"inject": 1, "transport": 1, "thermo_pass1": 1, "thermo_drain": 3, "reduce": 1, "finalize": 1}


def oracle_rate(w, nthreads, max_steps, seconds=30.0, boxes=None):
    """The oracle on this host: RT steps of workload w from its initial state
    (at least one, at most max_steps, stopping once `seconds` have passed),
    its cells spread over nthreads cores (OpenMP over cells, the oracle's only
    parallelism).  boxes: a list of workloads run one step each instead
    (batched boxes; stops likewise).  Returns (cell-group updates/s, steps)."""
    from oracle import oracle as O
    t0 = time.perf_counter()
    units, n = 0, 0
    for wb in (boxes if boxes is not None else [w]):
        p = O.Problem(wb.shape, wb.dx, wb.G, wb.cr, wb.sigN, wb.sigE, wb.egy, X=wb.X, isothermal=wb.isothermal,
                      otsa=wb.otsa, flux=wb.flux, bc=wb.bc, nthreads=nthreads,
                      inflow=(wb.extra or {}).get("inflow"))
        dt = O.courant_dt(wb.cfl, wb.dx, wb.cr)
        s = wb.state()
        k = 0
        while True:
            st, _, _, _ = p.step(s, dt, wb.src_ijk, wb.src_L)
            assert st == 0
            k += 1
            units += wb.ncells * wb.G
            if k >= (1 if boxes is not None else max_steps) or time.perf_counter() - t0 > seconds:
                break
        n += k
        if time.perf_counter() - t0 > seconds:
            break
    return units / (time.perf_counter() - t0), n


def cpu_info():
    """Core count and CPU model (lscpu's model name, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu part")):
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return {"cores": os.cpu_count() or 1, "cpu": model}


def cpu_baseline(w, steps, seconds=40.0):
    """The oracle on this host's cores over the same window as the GPU arm:
    RT steps of the same workload from its initial state (all K, unless that
    takes more than `seconds`), cells spread over all cores; then its first
    step on a single thread."""
    cores = os.cpu_count() or 1
    v, n = oracle_rate(w, cores, steps, seconds)
    out = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": "RT steps 1-%d of the same %s workload from its initial state (the GPU arm times steps 1-%d)"
                     % (n, w.name, steps), "cpu": cpu_info()["cpu"]}
    if cores > 1:
        v1, n1 = oracle_rate(w, 1, 1, 0.0)
        out["single_thread"] = {"value": v1, "unit": UNIT, "cores": 1,
                                "sample": "first RT step of the same workload, one thread"}
    return out


def variant_cpu_baseline(w, all_steps, one_steps, boxes=None, seconds=15.0):
    """Single-thread and all-core oracle timings of a variant's workload
    (bounded samples, as cpu_baseline)."""
    cores = os.cpu_count() or 1
    v, n = oracle_rate(w, cores, all_steps, seconds, boxes=boxes)
    out = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": ("%d boxes, one RT step each" % n) if boxes is not None else
           "RT steps 1-%d from the initial state" % n}
    if cores > 1:
        v1, n1 = oracle_rate(w, 1, one_steps, seconds, boxes=boxes)
        out["single_thread"] = {"value": v1, "unit": UNIT, "cores": 1,
                                "sample": ("%d boxes, one RT step each" % n1) if boxes is not None else
                                "RT steps 1-%d from the initial state" % n1}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cosmo128")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-mixed", action="store_true", help="skip timing the RT_MIXED variants")
    ap.add_argument("--no-batched", action="store_true", help="skip timing the batched-boxes variant")
    ap.add_argument("--batched-boxes", type=int, default=512)
    ap.add_argument("--no-c3", action="store_true", help="skip the 256^3 precision comparison")
    ap.add_argument("--smooth", action="store_true",
                    help="also time smoothed RT (Sec. 3.4); off by default: on this workload cells whose net "
                         "outflow rate and absorption empty them within a step sub-cycle without end under the "
                         "10%% rule with its 1e-30 floor")
    ap.add_argument("--no-adjoint", action="store_true", help="skip timing the adjoint")
    ap.add_argument("--no-shadow", action="store_true", help="skip the dense-cloud shadow workload")
    ap.add_argument("--no-stromgren", action="store_true", help="skip the 32^3 Stromgren-sphere workload")
    ap.add_argument("--adjoint-steps", type=int, default=200)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1304_7126_gb300 import rt as R

    w = workload(args.workload)
    hbm_peak, peak_kind = _peaks()
    sim = R.RT.from_workload(w)
    stream = torch.cuda.Stream()
    sim.set_stream(stream.cuda_stream)
    dt = sim.courant_dt()
    init = w.state()
    dev_init = {k: torch.from_numpy(v).cuda() for k, v in init.items()}
    torch.cuda.synchronize()

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    # warm-up (also captures the CUDA graph of a pair of steps)
    sim.run(dt, max(args.warmup, 3))
    sim.sync()
    sim.set_state(dev_init)
    sim.sync()

    # ---- timed region: K steps from the initial state, device-resident ----
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    with Clocks(local) as clk:
        ev0.record(stream)
        sim.run(dt, args.steps)
        ev1.record(stream)
        ev1.synchronize()
    barrier()
    sim.sync()
    t = max_over_ranks(ev0.elapsed_time(ev1) / 1e3, ws, "cuda")
    units = job_units(w.ncells * w.G * args.steps, ws)
    value = units / t
    clocks = clk.summary()

    # ---- per-kernel breakdown: same K steps, eager launches with events ----
    sim.set_state(dev_init)
    sim.set_profiling(True)
    attempts = 0
    att_max = 0
    queued = 0
    queued_att = 0
    long_cells = 0
    pass1_att = []
    sub = torch.empty(w.ncells, dtype=torch.int32, device="cuda")
    for _ in range(args.steps):
        sim.step(dt)
        sim.L.rt_get_subcycles(sim.h, sub.data_ptr(), 1)
        attempts += int(sub.sum().item())
        att_max = max(att_max, int(sub.max().item()))
        q = sub > PASS1_ATTEMPTS
        queued += int(q.sum().item())
        queued_att += int((sub[q] - PASS1_ATTEMPTS).sum().item())
        long_cells += int((sub > PASS1_ATTEMPTS + DRAIN1_BUDGET).sum().item())
        pass1_att.append(int(torch.clamp(sub, max=PASS1_ATTEMPTS).sum().item()))
    prof = sim.profile()
    sim.set_profiling(False)
    phases = {k: {"ms_total": round(v[0], 4), "launches": v[1],
                  "ms_per_launch": round(v[0] / v[1], 5) if v[1] else None} for k, v in prof.items()}
    dominant = max(prof, key=lambda k: prof[k][0])
    ms_launch = prof[dominant][0] / max(prof[dominant][1], 1)
    cg = w.ncells * w.G
    th_ops, tr_ops = _op_counts()
    fp_peaks = measure_fp_peaks()
    fp64_peak = fp_peaks["fp64_gflops"]
    # FP64 transport: HBM-bound by its bytes (64 B per cell-group), FP64-bound
    # by its flops (the oracle's count per cell-group); both fractions
    tr_ms = prof["transport"][0] / max(prof["transport"][1], 1)
    tr_bytes = 64.0 * cg
    tr_fpc = tr_ops["hll" if w.flux == R.RT_HLL else "glf"]["flop"]
    tr_flop = tr_fpc * cg
    tr_gbs = tr_bytes / (tr_ms / 1e3) / 1e9
    tr_gfl = tr_flop / (tr_ms / 1e3) / 1e9
    roof_ms = 1e3 * max(tr_bytes / (hbm_peak * 1e9), tr_flop / (fp64_peak * 1e9))
    transport_roof = {
        "kernel": "transport_kernel<double>", "ms_per_launch": tr_ms,
        "bound": "fp64" if tr_flop / fp64_peak > tr_bytes / hbm_peak else "hbm",
        "roof_ms_per_launch": roof_ms, "frac_of_roof": roof_ms / tr_ms,
        "hbm": {"achieved": tr_gbs, "peak": hbm_peak, "unit": "GB/s", "frac": tr_gbs / hbm_peak,
                "algorithmic_bytes_per_launch": tr_bytes, "peak_kind": peak_kind,
                "traffic": TRAFFIC.get("transport") if w.name == "cosmo128_s7" else None},
        "fp64": {"achieved": tr_gfl, "peak": fp64_peak, "unit": "GFLOP/s", "frac": tr_gfl / fp64_peak,
                 "flop_per_cell_group": tr_fpc, "algorithmic_flop_per_launch": tr_flop,
                 "peak_kind": "measured (cuBLAS DGEMM)"}}
    if dominant == "transport":
        roof = {"bound": "hbm", "achieved": tr_gbs, "peak": hbm_peak, "unit": "GB/s", "frac": tr_gbs / hbm_peak,
                "traffic": TRAFFIC.get("transport") if w.name == "cosmo128_s7" else None, "kernel": "transport",
                "peak_kind": peak_kind,
                "algorithmic_bytes_per_launch": tr_bytes}
    else:
        # thermochemistry: FP64-ALU work = algorithmic flops per attempt x
        # the attempts the phase made (first pass: up to PASS1_ATTEMPTS per
        # cell; queue drains: the rest)
        if dominant == "thermo_pass1":
            att_per_launch = (attempts - queued_att) / args.steps
        else:
            att_per_launch = queued_att / args.steps
        fpa = th_ops["flop"]
        ach = fpa * att_per_launch / (ms_launch / 1e3) / 1e9
        roof = {"bound": "alu", "achieved": ach, "peak": fp64_peak, "unit": "GFLOP/s",
                "frac": ach / fp64_peak,
                "traffic": TRAFFIC.get(dominant) if w.name == "cosmo128_s7" else None,
                "kernel": dominant + " (two lane-per-cell drains + warp-per-cell thermo_hard)"
                if dominant == "thermo_drain" else dominant,
                "peak_kind": "measured (cuBLAS DGEMM, FP64)",
                "flop_per_attempt": fpa, "transcendental_calls_per_attempt":
                    th_ops["exp"] + th_ops["log"] + th_ops["pow"],
                "attempts_per_launch": att_per_launch,
                "ms_per_launch": ms_launch}

    # ---- end to end: host buffers through the C-ABI, copies in the timed region ----
    e2e = None
    if not args.no_e2e:
        pin = {k: torch.from_numpy(v).pin_memory() for k, v in init.items()}
        host = {k: v.numpy() for k, v in pin.items()}
        outp = {k: torch.empty_like(v).pin_memory() for k, v in pin.items()}
        outh = {k: v.numpy() for k, v in outp.items()}
        sim.set_state(dev_init)
        sim.sync()
        h2d = sum(v.nbytes for v in host.values())
        d2h = sum(v.nbytes for v in outh.values())
        barrier()
        t0 = time.perf_counter()
        cur_in, cur_out = host, outh
        for _ in range(args.steps):
            sim.set_state(cur_in)           # H2D of the step's input state
            sim.step(dt)
            sim.get_state(cur_out)          # D2H of the step's result
            cur_in, cur_out = cur_out, cur_in
        barrier()
        te = max_over_ranks(time.perf_counter() - t0, ws, "cuda")
        e2e = {"value": units / te, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "how": "per step: rt_set_state from pinned host buffers, rt_step, rt_get_state to pinned host"}

    # ---- variants on the same workload: RT_MIXED, RT_MIXED32 and smoothed RT (Sec. 3.4) ----
    variants = {}
    vlist = [] if args.no_mixed else [("mixed", R.RT_MIXED, 0), ("mixed32", R.RT_MIXED32, 0)]
    if args.smooth:
        vlist += [("smoothed", R.RT_FP64, 1), ("smoothed_mixed32", R.RT_MIXED32, 1)]
    for vname, vprec, vsmooth in vlist:
        simm = R.RT.from_workload(w, precision=vprec, smooth=vsmooth)
        simm.set_stream(stream.cuda_stream)
        simm.run(dt, max(args.warmup, 3))
        simm.sync()
        simm.set_state(dev_init)
        simm.sync()
        barrier()
        ev0.record(stream)
        simm.run(dt, args.steps)
        ev1.record(stream)
        ev1.synchronize()
        simm.sync()
        tm = max_over_ranks(ev0.elapsed_time(ev1) / 1e3, ws, "cuda")
        simm.set_state(dev_init)
        simm.set_profiling(True)
        for _ in range(args.steps):
            simm.step(dt)
        pm = simm.profile()
        simm.set_profiling(False)
        subm = simm.subcycles()
        tr_ms = pm["transport"][0] / max(pm["transport"][1], 1)
        alg32 = 32.0 * cg
        ach32 = alg32 / (tr_ms / 1e3) / 1e9
        variants[vname] = {
            "value": units / tm, "ms_per_step": 1e3 * tm / args.steps, "speedup_vs_fp64": t / tm,
            "smoothed_rt": bool(vsmooth), "last_step_attempts": {"total": int(subm.sum()), "max": int(subm.max())},
            "phases_ms_per_launch": {k: round(v[0] / v[1], 5) if v[1] else None for k, v in pm.items()},
            "transport_roofline": {"bound": "hbm", "achieved": ach32, "peak": hbm_peak, "unit": "GB/s",
                                   "frac": ach32 / hbm_peak, "algorithmic_bytes_per_launch": alg32}}
        simm.close()

    # ---- batched uneven boxes (512 boxes of 16..64 cells a side, 1 or 3
    # groups, FP32 transport + FP64 thermochemistry), one graph per step pair ----
    if not args.no_batched:
        from paper_1304_7126_gb300 import workloads as W
        boxes = W.batched(args.batched_boxes)
        kb = min(args.steps, 100)
        cgb = sum(wb.ncells * wb.G for wb in boxes)
        bres = {}
        for bname, bprec in (("mixed", R.RT_MIXED), ("fp64", R.RT_FP64)):
            bt = R.RTBatch.from_workloads(boxes, precision=bprec)
            bt.set_stream(stream.cuda_stream)
            dtb = bt.courant_dt()
            bt.autotune(1)
            bt.run(dtb, max(args.warmup, 3))
            bt.sync()
            for i, wb in enumerate(boxes):
                bt.set_box_state(i, wb.state())
            bt.sync()
            barrier()
            ev0.record(stream)
            bt.run(dtb, kb)
            ev1.record(stream)
            ev1.synchronize()
            bt.sync()
            tb = max_over_ranks(ev0.elapsed_time(ev1) / 1e3, ws, "cuda")
            bres[bname] = {"value": job_units(cgb * kb, ws) / tb, "ms_per_step": 1e3 * tb / kb}
            bt.close()
        # the plain FP64 path, one single-box handle per box, on the first 16
        # boxes (one after another, kb steps each)
        t_single, cg_single = 0.0, 0
        for wb in boxes[:16]:
            sb = R.RT.from_workload(wb)
            sb.set_stream(stream.cuda_stream)
            dts = sb.courant_dt()
            sb.step(dts)
            sb.set_state(wb.state())
            sb.sync()
            ev0.record(stream)
            sb.run(dts, kb)
            ev1.record(stream)
            ev1.synchronize()
            sb.sync()
            t_single += ev0.elapsed_time(ev1) / 1e3
            cg_single += wb.ncells * wb.G * kb
            sb.close()
        variants["batched%d" % len(boxes)] = {
            "value": bres["mixed"]["value"], "ms_per_step": bres["mixed"]["ms_per_step"], "steps": kb,
            "cell_groups": cgb, "cells": sum(wb.ncells for wb in boxes),
            "precision": "mixed (FP32 transport, FP64 thermochemistry)",
            "fp64_same_boxes": dict(bres["fp64"], precision="FP64 batch, same boxes and steps"),
            "speedup_vs_fp64": bres["mixed"]["value"] / bres["fp64"]["value"],
            "single_box_fp64_first16": {"value": cg_single / t_single, "boxes": 16,
                                        "how": "one FP64 single-box handle per box, boxes run one after another"},
            "workload": "%d boxes, side in {16,24,32,48,64}, 1 or 3 groups, HLL, c_r=c/100" % len(boxes)}
        del boxes

    # ---- the 32^3 Stromgren sphere (isothermal, one group, GLF, FP64), 500 steps ----
    if not args.no_stromgren:
        from paper_1304_7126_gb300 import workloads as W
        w1 = W.stromgren32(32)
        k1 = 500
        s1 = R.RT.from_workload(w1)
        s1.set_stream(stream.cuda_stream)
        dt1 = s1.courant_dt()
        s1.run(dt1, 3)
        s1.set_state(w1.state())
        s1.sync()
        barrier()
        ev0.record(stream)
        s1.run(dt1, k1)
        ev1.record(stream)
        ev1.synchronize()
        s1.sync()
        t1 = max_over_ranks(ev0.elapsed_time(ev1) / 1e3, ws, "cuda")
        variants["stromgren32"] = {
            "value": job_units(w1.ncells * w1.G * k1, ws) / t1, "ms_per_step": 1e3 * t1 / k1, "steps": k1,
            "workload": "32^3 Stromgren sphere, box 6.6 kpc, n_H 1e-3, T 1e4 K fixed, 1 group, corner source, "
                        "GLF, c_r = c/100, FP64"}
        s1.close()

    # ---- 256^3 (seed 11, 64 sources): FP64, RT_MIXED and RT_MIXED32 from the
    # same state, per-field error of the reduced-precision states against FP64 ----
    if not args.no_c3:
        from paper_1304_7126_gb300 import workloads as W
        w3 = W.cosmo256()
        k3 = min(args.steps, w3.steps)
        init3 = {k: torch.from_numpy(v).cuda() for k, v in w3.state().items()}
        cg3 = w3.ncells * w3.G
        res, fin = {}, {}
        for name, prec in (("fp64", R.RT_FP64), ("mixed", R.RT_MIXED), ("mixed32", R.RT_MIXED32)):
            s3 = R.RT.from_workload(w3, precision=prec)
            s3.set_stream(stream.cuda_stream)
            dt3 = s3.courant_dt()
            s3.run(dt3, 3)
            s3.set_state(init3)
            s3.sync()
            barrier()
            ev0.record(stream)
            s3.run(dt3, k3)
            ev1.record(stream)
            ev1.synchronize()
            s3.sync()
            t3 = max_over_ranks(ev0.elapsed_time(ev1) / 1e3, ws, "cuda")
            fin[name] = s3.get_state(device=True)
            res[name] = {"value": job_units(cg3 * k3, ws) / t3, "ms_per_step": 1e3 * t3 / k3}
            s3.close()
        ref = fin["fp64"]
        nmax = float(ref["N"].abs().max())
        for name in ("mixed", "mixed32"):
            g = fin[name]
            res[name]["speedup_vs_fp64"] = res["fp64"]["ms_per_step"] / res[name]["ms_per_step"]
            res[name]["error_vs_fp64_gpu"] = {
                "xHII_abs": float((g["xHII"] - ref["xHII"]).abs().max()),
                "xHeII_abs": float((g["xHeII"] - ref["xHeII"]).abs().max()),
                "xHeIII_abs": float((g["xHeIII"] - ref["xHeIII"]).abs().max()),
                "T_rel": float(((g["T"] - ref["T"]).abs() / ref["T"]).max()),
                "N_rel": float(((g["N"] - ref["N"]).abs() / ref["N"].abs().clamp_min(1e-6 * nmax)).max())}
        variants["cosmo256"] = {"steps": k3, "cell_groups": cg3,
                                "workload": "256^3, 3 groups, seed 11, 64 sources of 1e52/s, HLL, c_r=c/10",
                                "tolerance": {"x_abs": 1e-4, "T_rel": 1e-3, "N_rel": 1e-4}, **res}
        del fin, ref, init3

    # ---- the dense-cloud shadow workload (Sec. 6 test 3 on a uniform 128^3
    # grid): a constant flux entering through x = 0, HLL, FP64 ----
    if not args.no_shadow:
        from paper_1304_7126_gb300 import workloads as W
        w6 = W.shadow(128)
        k6 = min(args.steps, 200)
        s6 = R.RT.from_workload(w6)
        s6.set_stream(stream.cuda_stream)
        dt6 = s6.courant_dt()
        s6.run(dt6, 3)
        init6 = {k: torch.from_numpy(v).cuda() for k, v in w6.state().items()}
        s6.set_state(init6)
        s6.sync()
        barrier()
        ev0.record(stream)
        s6.run(dt6, k6)
        ev1.record(stream)
        ev1.synchronize()
        s6.sync()
        t6 = max_over_ranks(ev0.elapsed_time(ev1) / 1e3, ws, "cuda")
        sub6 = s6.subcycles()
        variants["shadow128"] = {
            "value": job_units(w6.ncells * w6.G * k6, ws) / t6, "ms_per_step": 1e3 * t6 / k6, "steps": k6,
            "last_step_attempts": {"total": int(sub6.sum()), "max": int(sub6.max())},
            "workload": "128^3, box 6.6 kpc, cloud r = 0.8 kpc (n_H 4e-2, 40 K) in n_H 2e-4, 8000 K, H only, "
                        "3 groups, 1e6 photons/cm^2/s entering through x = 0, HLL, c_r = c/10, FP64"}
        s6.close()
        del init6

    # ---- adjoint: 64^3, 3 groups, 8 sources, GLF, FP64; forward with a checkpoint
    # every 20 steps, then the backward pass (recompute + hand-written VJPs) ----
    if not args.no_adjoint:
        from paper_1304_7126_gb300 import adjoint as A
        from paper_1304_7126_gb300 import workloads as W
        w5 = W.adjoint64()
        k5 = args.adjoint_steps
        s5 = R.RT.from_workload(w5)
        dt5 = s5.courant_dt()
        st5 = {k: torch.from_numpy(v).cuda() for k, v in w5.state().items()}
        Ld = torch.from_numpy(w5.src_L).cuda()

        def fwd_bwd(k):
            nH = st5["nH"].clone().requires_grad_(True)
            L = Ld.clone().requires_grad_(True)
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record()
            out = A.run(s5, dt5, k, w5.src_ijk, nH, L, st5, every=20)
            loss = A.neutral_hydrogen_mass(out, w5.dx)
            e1.record()
            loss.backward()
            e2.record()
            e2.synchronize()
            return e0.elapsed_time(e1) / 1e3, e1.elapsed_time(e2) / 1e3, nH.grad, L.grad

        fwd_bwd(3)
        barrier()
        tf, tb, gnh, gl = fwd_bwd(k5)
        tf, tb = max_over_ranks(tf, ws, "cuda"), max_over_ranks(tb, ws, "cuda")
        cg5 = w5.ncells * w5.G
        variants["adjoint64"] = {
            "value": job_units(cg5 * k5, ws) / (tf + tb), "unit": UNIT + " (forward + backward)", "steps": k5,
            "checkpoint_every": 20, "forward_s": tf, "backward_s": tb, "backward_over_forward": tb / tf,
            "grad_L_per_source": (gl * (Ld / Ld.sum(dim=1, keepdim=True))).sum(dim=1).tolist(),
            "grad_nH_abs_max": float(gnh.abs().max()),
            "workload": "64^3, 3 groups, H+He, seed 7, 8 sources of 1e52/s, GLF, FP64; d M_HI / d(n_H, L)"}
        s5.close()

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, args.steps)
        from paper_1304_7126_gb300 import workloads as W
        vcpu = {"stromgren32": (W.stromgren32(32), 500, 500, None),
                "cosmo256": (W.cosmo256(), 2, 1, None),
                "batched%d" % args.batched_boxes: (None, 1, 1, W.batched(16)),
                "adjoint64": (W.adjoint64(), 10, 2, None)}
        for name, (wv, na, n1, bx) in vcpu.items():
            if name in variants:
                variants[name]["cpu_baseline"] = variant_cpu_baseline(wv, na, n1, boxes=bx)

    if rank == 0:
        cfg = _config(w)
        cfg["parallelism"] = "replicas x%d" % ws if ws > 1 else "single GPU"
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": cfg, "roofline": roof, "transport_roofline": transport_roof, "fp_peaks": fp_peaks,
                "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": sum(KERNELS_PER_PHASE[k] * v[1] for k, v in prof.items()), "clocks": clocks,
                "phases": phases,
                "variants": variants,
                "thermo_attempts": {"per_step": attempts / args.steps, "max_per_cell": att_max,
                                    "queued_cells_per_step": queued / args.steps,
                                    "cells_past_first_drain_per_step": long_cells / args.steps,
                                    "first_pass_attempts_by_step": pass1_att,
                                    "queued_attempts_per_step": queued_att / args.steps}}
        print(json.dumps(line), flush=True)
    sim.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
