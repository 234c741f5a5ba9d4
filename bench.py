#!/usr/bin/env python3
"""Benchmark of the relaxing-TVD patch-group hydro path on GB300.

A step is one pass of the whole hot path over the workload: by default
(--mode pair) one gamer_hydro_step_pair call, the xyz and the zyx sweep set
of every patch group with one dt (ghost gather + x/y/z then z/y/x sweeps,
two cell-updates per cell, one persistent FP32 launch for one level), then
the diagnostics (CFL time step and the conservation / positivity check,
FP64 reductions) whose dt feeds the next step; --mode step times single
sweep sets (gamer_hydro_step).  The default workload is the periodic 128^3
smooth k^-2 random field (4096 patches of 8^3 = 512 patch groups).  It fits
in L2, so L2 is flushed (a 256 MiB write) before every timed step, outside
the timed interval.

Prints ONE JSON line (rank 0).  See --help for options.  ``--impl
reference`` times the FP64 CPU oracle instead (on a bounded sample of the
same workload per step).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s and % of HBM roofline, FP32 batched vs plain FP64, at stated L1 err"
UNIT = "cell-updates/s"
GAMMA = 5.0 / 3.0
CFL = 0.5
BYTES_PER_CELL_F32 = (22 ** 3 + 16 ** 3) * 5 * 4 / 16 ** 3   # 72.0: padded read + interior write
BYTES_PER_CELL_F64 = 2 * BYTES_PER_CELL_F32


def parse():
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default="uniform128", choices=sorted(WORKLOADS))
    p.add_argument("--quick", action="store_true",
                   help="device-timed value only (no e2e, FP64, L1, CPU baseline, clocks); for profiling")
    p.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU time of the oracle sample")
    p.add_argument("--mode", choices=["pair", "step"], default="pair",
                   help="pair: one call = gamer_hydro_step_pair (xyz + zyx sweep sets with one dt, one launch); "
                        "step: one call = gamer_hydro_step (one sweep set)")
    p.add_argument("--time-steps", choices=["uniform", "individual"], default="uniform",
                   help="multi-level workloads, --mode pair: one dt for all levels, or every level "
                        "halving its parent's dt (a call then advances level l by 2^(l+1) steps)")
    p.add_argument("--regrid-kernels", action="store_true",
                   help="instead of timing steps: the flag step (three criteria) and the refinement fill of "
                        "the refinement-map rebuild on the workload's level 0, HBM GB/s per launch")
    p.add_argument("--poisson", action="store_true",
                   help="instead of timing steps: the red-black SOR Poisson solver on as many patch groups as "
                        "the workload's level 0 (random potential and density, a fixed iteration count)")
    p.add_argument("--gravity", action="store_true",
                   help="instead of timing steps: the gravity operator G on the workload's level 0 (HBM GB/s "
                        "per launch, FP32 and FP64) and one xyzGGzyx double step against the fused pair step")
    p.add_argument("--no-configs", action="store_true",
                   help="skip the other north-star workloads (3-level AMR, 512^3) that the default run adds "
                        "under 'configs'")
    p.add_argument("--precision", choices=["fp32", "fp64"], default="fp32",
                   help="with --quick: time the FP32 path (default) or the plain FP64 path (one sweep set per "
                        "step through gamer_hydro_step); for profiling the FP64 kernel")
    p.add_argument("--launch-groups", type=int, default=0,
                   help="with --precision fp64: patch groups per kernel launch (gamer_hydro_set_launch_groups; "
                        "1 = one group per launch; 0 = the library default)")
    p.add_argument("--accuracy", action="store_true",
                   help="instead of timing: per-field L1 / max error of the FP32 path against the FP64 path "
                        "(bit-identical to the FP64 oracle) on every workload, plus positivity and conservation")
    return p.parse_args()


# ------------------------------------------------------------ workloads

def _wl_uniform(n, kind):
    def make():
        from paper_0907_3390_gb300 import workloads as W
        if kind == "smooth":
            u, npg = W.smooth_grf(n, seed=1001)
        else:
            u, npg = W.lognormal_grf(n, seed=1003)
        H, st = W.single_level(u, npg)
        return H, st
    return make


def _wl_amr(kind):
    def make():
        from paper_0907_3390_gb300 import workloads as W
        if kind == "amr3":
            return W.amr_grf()
        if kind == "amr4sedov":
            return W.amr_stress("sedov")
        return W.amr_stress("lognormal")
    return make


WORKLOADS = {
    "uniform128": ("smooth k^-2 Gaussian random fields (density contrast 10, rms Mach 1), periodic "
                   "128^3, 4096 patches of 8^3 (512 patch groups), gamma 5/3, CFL 0.5", _wl_uniform(128, "smooth")),
    "uniform256": ("smooth k^-2 Gaussian random fields, periodic 256^3, 32768 patches", _wl_uniform(256, "smooth")),
    "uniform512": ("lognormal k^-2 density (sigma 1.5), rms Mach 3, periodic 512^3, 262144 patches",
                   _wl_uniform(512, "lognormal")),
    "amr3": ("3 levels over a 128^3 base, 4096/9000/21000 patches, lognormal k^-2 density", _wl_amr("amr3")),
    "amr4": ("4 levels, 32768 patches, lognormal sigma 2.5 density, converging flows up to Mach 20",
             _wl_amr("amr4")),
    "amr4sedov": ("4 levels, 32768 patches, Sedov point blast (E = 1 in one finest cell, rho 1, P 1e-5)",
                  _wl_amr("amr4sedov")),
}


STEP_PAIR = ("gamer_hydro_step_pair: the xyz and the zyx sweep set of every patch group with one dt "
             "(2 cell-updates per cell), each set = ghost gather + 3 sweeps, then the CFL dt and the "
             "conservation/positivity check; one CUDA graph of ONE persistent kernel (a group's zyx set starts "
             "when its and its neighbours' xyz results are published; the last CTA reduces the diagnostics and "
             "writes dt and the result to mapped host memory)")
STEP_ONE = ("gamer_hydro_step: one sweep set (gather + 3 sweeps) + CFL dt + conservation/positivity check "
            "(one CUDA graph: persistent sweep kernel with fused diagnostics; its last CTA reduces them and "
            "writes dt and the result to mapped host memory)")


# ------------------------------------------------------------ helpers

def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_source_sha():
    h = hashlib.sha256()
    for f in ("sweep_f32.cu", "common.cuh", "step_reduce.cuh", "lane_maps.h"):
        with open(os.path.join(ROOT, "paper_0907_3390_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profile_per_cell(key="dram_bytes_per_cell", kernel="sweep_f32"):
    """Per-cell-update figure of an FP32 sweep kernel (DRAM bytes, warp
    instructions; kernel 'sweep_f32' = k_sweep_f32, 'sweep_pair' =
    k_sweep_pair) from the committed ncu summary, if it was taken on the
    current kernel source."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    if d.get("source_sha") != kernel_source_sha() or key not in d:
        return None
    return float(d[key])


FP64_PEAK_TF = 1.25       # nominal GB300 FP64 rate (TFLOP/s)


def profile_fp64():
    """FP64 floating-point operations per cell-update of the plain FP64
    kernel (DADD + DMUL + 2 DFMA per thread, from an ncu capture of
    k_pg_f64), if the capture was taken on the current FP64 kernel source."""
    path = os.path.join(ROOT, "profiles", "sweep_f64_counters.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    h = hashlib.sha256()
    for name in ("sweep_f64.cu", "common.cuh"):
        with open(os.path.join(ROOT, "paper_0907_3390_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    if d.get("source_sha") != h.hexdigest()[:16]:
        return None
    return {"flops_per_cell": float(d["fp64_flops_per_cell"]), "source": "profiles/sweep_f64_counters.json"}


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.path = os.path.join("/tmp", f"bench_clocks_{os.getpid()}.csv")
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.5)     # let nvidia-smi start sampling before the timed region
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.remove(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def cpu_oracle_rate(H, states, seconds, threads, max_groups=None):
    """Oracle (plain FP64 C, OpenMP over patch groups) on a bounded sample of
    the workload: sweep sets of level 0 (or of its first max_groups patch
    groups), repeated until about `seconds` of CPU work.  Returns
    cell-updates/s, the sample description and seconds."""
    import oracle
    oracle.set_threads(threads)
    O = oracle.OracleLevels(H, [np.asarray(s, dtype=np.float64) for s in states])
    dt = O.cfl_dt(GAMMA, CFL)
    n = H.levels[0].n_groups if max_groups is None else min(max_groups, H.levels[0].n_groups)
    groups = np.arange(n)
    done, el, k = 0, 0.0, 0
    while el < seconds:
        t0 = time.perf_counter()
        O.advance_level(0, GAMMA, dt, k % 2, groups=groups)
        el += time.perf_counter() - t0
        done += n
        k += 1
    what = f"all {n}" if n == H.levels[0].n_groups else f"the first {n}"
    return done * 4096 / el, f"{k} sweep sets of {what} patch groups of level 0", el


# ------------------------------------------------------------ reference arm

def run_reference(args, rank, world):
    if rank != 0:
        return 0
    desc, make = WORKLOADS[args.workload]
    H, st = make()
    import oracle
    threads = os.cpu_count() or 1
    oracle.set_threads(threads)
    O = oracle.OracleLevels(H, st)
    dt = O.cfl_dt(GAMMA, CFL)
    n = H.levels[0].n_groups
    # each step: a bounded sample of the workload (whole groups), sized so the
    # whole --steps/--warmup run ends within a few minutes
    probe = min(n, max(threads, 8))
    t0 = time.perf_counter()
    O.advance_level(0, GAMMA, dt, 0, groups=np.arange(probe))
    t1 = time.perf_counter() - t0
    per_step_s = max(1.0, 150.0 / max(args.steps + args.warmup, 1))
    count = int(min(n, max(probe, probe * per_step_s / max(t1, 1e-6))))
    groups = np.arange(count)
    for w in range(args.warmup):
        O.advance_level(0, GAMMA, dt, w % 2, groups=groups)
    el = 0.0
    for s in range(args.steps):
        t0 = time.perf_counter()
        O.advance_level(0, GAMMA, dt, s % 2, groups=groups)
        el += time.perf_counter() - t0
    rate = count * 4096 * args.steps / el
    sample = f"{count} of {n} patch groups per step (one sweep set each)"
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": desc, "sample": sample},
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------ our arm

def sweep_kernel_ms(B, torch, S, D, flush, K, pair, n_levels, cfl=None):
    """Average device time of the sweep launches of one step, from events
    the library records around them (gamer_hydro_set_profiling; such steps
    launch directly, events cannot be timed inside graphs), L2 flushed
    before each step.  A one-level pair is one launch; a multi-level pair
    runs as two steps, so its two sweep sets are timed as two
    gamer_hydro_step calls."""
    cfl = CFL if cfl is None else cfl
    kev = (_timing_event(torch), _timing_event(torch))
    torch.cuda.synchronize()
    B.gamer_hydro_set_profiling(S.h, kev[0], kev[1])
    out = []
    for k in range(K):
        if pair and n_levels == 1:
            flush.fill_(float(k))
            B.gamer_hydro_step_pair(S.h, D, cfl)
            torch.cuda.synchronize()
            out.append(kev[0].elapsed_time(kev[1]))
        else:
            t = 0.0
            for _ in range(2 if pair else 1):
                flush.fill_(float(k))
                B.gamer_hydro_step(S.h, D, cfl)
                D.swap()
                torch.cuda.synchronize()
                t += kev[0].elapsed_time(kev[1])
            out.append(t)
    B.gamer_hydro_set_profiling(S.h, None, None)
    return float(np.mean(out))



def _timing_event(torch):
    e = torch.cuda.Event(enable_timing=True)
    e.record()          # materialise the underlying cudaEvent_t
    return e


def run_fp64_quick(args):
    """--quick --precision fp64: sweep sets of the plain FP64 path (one per
    step, gamer_hydro_advance_all with a fixed dt), for profiling k_pg_f64."""
    import torch
    from paper_0907_3390_gb300 import binding as B
    desc, make = WORKLOADS[args.workload]
    H, st = make()
    cells = sum(lv.n_groups for lv in H.levels) * 4096
    S = B.Solver(GAMMA, B.GAMER_LIMITER_VANLEER, B.GAMER_FP64)
    if args.launch_groups > 0:
        B.gamer_hydro_set_launch_groups(S.h, args.launch_groups)
    D = B.DeviceHierarchy(H, st, torch.float64)
    dt = B.gamer_hydro_cfl_dt(S.h, D, CFL)
    for _ in range(args.warmup):
        S.step(D, dt)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        S.step(D, dt)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    print(json.dumps({"metric": METRIC, "value": cells / (ms / 1e3), "unit": UNIT, "n_gpus": 1,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                      "dtype": "f64", "data": "synthetic",
                      "config": {"workload": desc, "step": "one FP64 sweep set (gamer_hydro_advance_all)",
                                 "groups_per_launch": args.launch_groups or "library default"}}), flush=True)
    S.close()
    return 0


def run_ours(args, rank, world, dist):
    import torch
    from paper_0907_3390_gb300 import binding as B
    from paper_0907_3390_gb300 import replicas as R

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    desc, make = WORKLOADS[args.workload]
    H, st = make()
    cells = sum(lv.n_groups for lv in H.levels) * 4096
    stream = torch.cuda.current_stream()

    def barrier():
        R.barrier(dist)

    S = B.Solver(GAMMA, B.GAMER_LIMITER_VANLEER, B.GAMER_FP32, stream=stream)
    D = B.DeviceHierarchy(H, st, torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    sets = 2 if args.mode == "pair" else 1   # sweep sets (cell-updates per cell) per call
    individual = args.time_steps == "individual" and len(H.levels) > 1
    if args.time_steps == "individual" and args.mode != "pair":
        raise SystemExit("--time-steps individual needs --mode pair")
    if individual:
        B.gamer_hydro_set_time_steps(S.h, B.GAMER_TIME_STEPS_INDIVIDUAL)
    # cell-updates per call: level l takes 2^(l+1) steps per call with individual time steps
    updates = (sum(lv.n_groups * 4096 * 2 ** (l + 1) for l, lv in enumerate(H.levels)) if individual
               else cells * sets)

    def step():
        if args.mode == "pair":
            B.gamer_hydro_step_pair(S.h, D, CFL)   # xyz + zyx sets, CFL dt, check: one graph replay
        else:
            B.gamer_hydro_step(S.h, D, CFL)        # one sweep set, CFL dt, check: one graph replay
            D.swap()

    s0, _ = B.gamer_hydro_check(S.h, D)
    clocks = None if args.quick else ClockSampler(local)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # timed region: K whole steps, each bracketed by events on the launch
    # stream, L2 flushed before each
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    for s in range(args.steps):
        flush.fill_(float(s))                       # evict L2 (outside the timed interval)
        ev[s][0].record(stream)
        step()
        ev[s][1].record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop() if clocks else None
    dt_used, dt_next, sums, n_bad = B.gamer_hydro_step_result(S.h)
    step_ms = sum(a.elapsed_time(b) for a, b in ev)

    # the dominant kernel: the same steps again with profiling events around
    # the sweep launches
    if individual:
        kev = (_timing_event(torch), _timing_event(torch))
        torch.cuda.synchronize()
        B.gamer_hydro_set_profiling(S.h, kev[0], kev[1])
        kern_ms = []
        for s in range(args.steps):
            flush.fill_(float(s))
            step()
            torch.cuda.synchronize()
            kern_ms.append(kev[0].elapsed_time(kev[1]))
        B.gamer_hydro_set_profiling(S.h, None, None)
    else:
        kern_ms = [sweep_kernel_ms(B, torch, S, D, flush, args.steps, args.mode == "pair", len(H.levels))]
    value, t_max = R.whole_job_rate(updates * args.steps, step_ms / 1e3, dist, dev)
    res = {"value": value, "ms_per_step": 1e3 * t_max / args.steps, "sets_per_step": sets,
           "updates_per_step": updates, "time_steps": "individual" if individual else "uniform"}
    # kernels per step: one level = the persistent sweep launch alone (it runs
    # the end-of-step reduction in its last CTA); more levels = the sweep
    # launch, one fix-up per coarse level, the diagnostics and the reduction
    n_lev = len(H.levels)
    if individual:
        # sweeps 2^(l+1) per level, fix-ups 2^(l+1) per coarse level, diagnostics, reduction
        res["launches_per_step"] = sum(2 ** (l + 1) for l in range(n_lev)) + \
            sum(2 ** (l + 1) for l in range(n_lev - 1)) + 2
    else:
        res["launches_per_step"] = 1 if n_lev == 1 else sets * (n_lev + 2)

    hbm, peak_kind = measured_peaks()
    k_avg = float(np.mean(kern_ms)) / 1e3
    achieved = BYTES_PER_CELL_F32 * updates / k_avg / 1e9
    kname = "sweep_pair" if sets == 2 and n_lev == 1 else "sweep_f32"
    tpc = profile_per_cell("dram_bytes_per_cell", kname)
    res["roofline"] = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                       "frac": achieved / hbm, "peak_kind": f"{peak_kind} copy bandwidth",
                       "traffic": None if tpc is None or n_lev > 1 else tpc * updates,
                       "kernel": ("k_sweep_pair (xyz and zyx sets of every group: gathers, 2 x 3 sweeps, stores, "
                                  "fused diagnostics and end-of-step reduction, one persistent launch)"
                                  if kname == "sweep_pair" else
                                  "k_sweep_f32 (gather + 3 sweeps + store + fused diagnostics and end-of-step "
                                  "reduction, one persistent launch)"),
                       "kernel_ms": 1e3 * k_avg, "algorithmic_bytes": BYTES_PER_CELL_F32 * updates}
    # the bound that actually limits the kernel: instruction issue (FP32
    # arithmetic of the scheme).  Peak from the unit counts and the clock:
    # SMs x 4 warp schedulers x 1 warp instruction per cycle x max SM clock.
    ipc = profile_per_cell("warp_instructions_per_cell", kname)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = (clk or {}).get("sm_max_mhz") or 2070.0
    issue_peak = sms * 4 * mhz * 1e6 / 1e12
    res["roofline_alu"] = None if ipc is None or n_lev > 1 else {
        "bound": "alu", "achieved": ipc * updates / k_avg / 1e12, "peak": issue_peak, "unit": "T warp-instr/s",
        "frac": ipc * updates / k_avg / 1e12 / issue_peak,
        "peak_kind": f"derived: {sms} SMs x 4 schedulers x 1 warp-instr/cycle x {mhz:.0f} MHz",
        "instructions_per_cell": ipc}
    res["clocks"] = clk
    res["conservation_drift_rel"] = float(np.max(np.abs(sums - s0) / (np.abs(s0) + 1e-30)))
    res["n_bad"] = n_bad
    extras = {}
    if not args.quick:
        # e2e on every rank at once (max over ranks); the rest on rank 0
        extras["e2e"] = run_e2e(args, B, R, torch, H, st, dev, stream, updates, dist)
        if rank == 0:
            extras.update(run_extras(args, B, torch, H, st, cells, dev, stream, updates, world))
        if rank == 0 and world == 1 and not args.no_configs:
            extras["configs"] = run_configs(args, B, torch, dev, stream)
    S.close()
    return res, extras, cells, desc


def run_e2e(args, B, R, torch, H, st, dev, stream, updates, dist):
    # ---- e2e through the C ABI with host buffers.  Every step takes its
    # input state from pinned host memory, advances it through the same
    # call as the timed step (whose last kernel writes the step result to
    # mapped host memory) and copies the new state back to pinned host
    # memory.  NB independent states are in flight (one handle each): the
    # copy-in of step k+1 (own stream) overlaps the compute of step k (the
    # launch stream) and the copy-out of step k-1 (own stream), as a serving
    # loop over independent states would run; with three states a buffer's
    # copy-out and its next copy-in do not hold up the step in between.
    sets = 2 if args.mode == "pair" else 1
    s_in = torch.cuda.Stream(device=dev)
    s_out = torch.cuda.Stream(device=dev)
    NB = 3
    solvers = [B.Solver(GAMMA, B.GAMER_LIMITER_VANLEER, B.GAMER_FP32, stream=stream) for _ in range(NB)]
    if args.time_steps == "individual" and len(H.levels) > 1:
        for S in solvers:
            B.gamer_hydro_set_time_steps(S.h, B.GAMER_TIME_STEPS_INDIVIDUAL)
    bufs = [B.DeviceHierarchy(H, st, torch.float32, device=dev) for _ in range(NB)]
    host_in = [x.cpu().pin_memory() for x in bufs[0].u]
    host_out = [[torch.empty_like(x).pin_memory() for x in host_in] for _ in range(NB)]
    ev_in = [torch.cuda.Event() for _ in range(NB)]
    ev_step = [torch.cuda.Event() for _ in range(NB)]
    ev_out = [torch.cuda.Event() for _ in range(NB)]
    n_e2e = max(4, min(2 * args.steps, 20))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    warm = 2 * NB
    for it in range(warm + n_e2e):
        if it == warm:
            torch.cuda.synchronize()
            R.barrier(dist)
            e0.record(stream)
            s_in.wait_stream(stream)             # the first timed copy-in starts after e0
        b = it % NB
        S, D = solvers[b], bufs[b]
        if it >= NB:
            s_in.wait_event(ev_step[b])          # the previous step on this buffer is done with u
            s_in.wait_event(ev_out[b])           # and its result has been copied out
        with torch.cuda.stream(s_in):
            for l in range(len(D.u)):
                D.u[l].copy_(host_in[l], non_blocking=True)
            ev_in[b].record(s_in)
        stream.wait_event(ev_in[b])
        if it >= NB:
            stream.wait_event(ev_out[b])
        if sets == 2:
            B.gamer_hydro_step_pair(S.h, D, CFL)  # result back in u
            res_bufs = D.u
        else:
            B.gamer_hydro_step(S.h, D, CFL)       # result in u_out
            res_bufs = D.u_out
        ev_step[b].record(stream)
        s_out.wait_event(ev_step[b])
        with torch.cuda.stream(s_out):
            for l in range(len(D.u)):
                host_out[b][l].copy_(res_bufs[l], non_blocking=True)
            ev_out[b].record(s_out)
    for b in range(NB):
        stream.wait_event(ev_out[b])
    e1.record(stream)
    torch.cuda.synchronize()
    R.barrier(dist)
    for S in solvers:
        B.gamer_hydro_step_result(S.h)
    rate, _ = R.whole_job_rate(updates * n_e2e, e0.elapsed_time(e1) / 1e3, dist, dev)
    nbytes = sum(x.numel() * 4 for x in host_in)
    for S in solvers:
        S.close()
    return {"value": rate, "unit": UNIT, "h2d_bytes_per_step": nbytes,
            "d2h_bytes_per_step": nbytes + 88,      # + the step result (11 x 8 B)
            "pipeline": f"{NB} independent states in flight per GPU; copy-in, step and copy-out on 3 streams"}


def run_extras(args, B, torch, H, st, cells, dev, stream, updates, world):
    out = {}

    # ---- plain FP64 GPU path (one block per patch group, same whole-step
    # API) and the per-field L1 error of one FP32 sweep set against it (the
    # FP64 path is bit-identical to the FP64 oracle in the parity tests)
    S64 = B.Solver(GAMMA, B.GAMER_LIMITER_VANLEER, B.GAMER_FP64, stream=stream)
    D64 = B.DeviceHierarchy(H, st, torch.float64, device=dev)
    dt = B.gamer_hydro_cfl_dt(S64.h, D64, CFL)
    S32 = B.Solver(GAMMA, B.GAMER_LIMITER_VANLEER, B.GAMER_FP32, stream=stream)
    D32 = B.DeviceHierarchy(H, st, torch.float32, device=dev)
    S32.step(D32, dt)
    S64.step(D64, dt)
    ref = D64.u[0].double()
    got = D32.u[0].double()
    scale = ref.reshape(5, -1).abs().max(dim=1).values
    l1 = ((got - ref).reshape(5, -1).abs().mean(dim=1) / scale).cpu().numpy()
    n64 = 3
    B.gamer_hydro_step(S64.h, D64, CFL)
    D64.swap()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(n64):
        B.gamer_hydro_step(S64.h, D64, CFL)
        D64.swap()
    e1.record(stream)
    torch.cuda.synchronize()
    ms64 = e0.elapsed_time(e1) / n64
    out["fp64_plain"] = {"value": cells / (ms64 / 1e3), "unit": UNIT, "ms_per_step": ms64,
                         "note": "batched FP64 path: one sweep set per step (gamer_hydro_step), one thread block "
                                 "per patch group and every group of the level in one launch, FP64 throughout; "
                                 "this is not the one-group-per-launch layout (see fp64_per_launch)"}
    # the plain layout: one patch group per kernel launch
    B.gamer_hydro_set_launch_groups(S64.h, 1)
    n1 = 2
    B.gamer_hydro_advance_all(S64.h, D64, dt)
    D64.swap()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(n1):
        B.gamer_hydro_advance_all(S64.h, D64, dt)
        D64.swap()
    e1.record(stream)
    torch.cuda.synchronize()
    ms1 = e0.elapsed_time(e1) / n1
    n_groups = sum(lv.n_groups for lv in H.levels)
    out["fp64_per_launch"] = {"value": cells / (ms1 / 1e3), "unit": UNIT, "ms_per_set": ms1,
                              "launches_per_set": n_groups,
                              "note": "plain FP64 path, one patch group per kernel launch "
                                      "(gamer_hydro_set_launch_groups(h, 1)), one sweep set per call"}
    f64 = profile_fp64()
    if f64 is not None:
        achieved = f64["flops_per_cell"] * cells / (ms64 / 1e3) / 1e12
        out["fp64_plain"]["roofline"] = {
            "bound": "fp64", "achieved": achieved, "peak": FP64_PEAK_TF, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TF, "peak_kind": "nominal GB300 FP64 (no measured FP64 peak)",
            "flops_per_cell": f64["flops_per_cell"], "source": f64["source"]}
    out["l1_rel_err_fp32_vs_fp64"] = {"fields": ["rho", "mx", "my", "mz", "e"], "value": [float(x) for x in l1],
                                      "after": "one sweep set"}
    S64.close()
    S32.close()

    # ---- the oracle on the host cores, bounded sample (one process only:
    # under torchrun the host cores are shared by the ranks)
    if world > 1:
        return out
    threads = os.cpu_count() or 1
    rate, sample, secs = cpu_oracle_rate(H, st, args.cpu_seconds, threads)
    rate1, sample1, secs1 = cpu_oracle_rate(H, st, max(1.0, args.cpu_seconds / 4), 1, max_groups=16)
    out["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample,
                           "seconds": secs, "value_1core": rate1, "sample_1core": sample1}
    return out


# ------------------------------------------------------------ other workloads

# the other spec workloads that fit one GPU, run after the main line:
# (workload, timed pair steps)
CONFIG_RUNS = (("amr3", 10), ("uniform512", 5))


def run_configs(args, B, torch, dev, stream):
    """The uneven 3-level AMR batch (uniform dt) and the 262,144-patch 512^3
    batch, each with the main line's step (gamer_hydro_step_pair: xyz + zyx
    with one dt, CFL dt and check), L2 flushed before every timed step; the
    sweep kernels' own time from events around their launches; per-field L1
    error of one FP32 pair against the FP64 path from the same state with the
    same dt (worst level, relative to the field's largest magnitude)."""
    hbm, peak_kind = measured_peaks()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    out = {}
    for name, K in CONFIG_RUNS:
        desc, make = WORKLOADS[name]
        t0 = time.perf_counter()
        H, st = make()
        gen_s = time.perf_counter() - t0
        cells = sum(lv.n_groups for lv in H.levels) * 4096
        updates = 2 * cells
        S = B.Solver(GAMMA, B.GAMER_LIMITER_VANLEER, B.GAMER_FP32, stream=stream)
        D = B.DeviceHierarchy(H, st, torch.float32, device=dev)
        for _ in range(3):
            B.gamer_hydro_step_pair(S.h, D, CFL)
        torch.cuda.synchronize()
        clocks = ClockSampler(dev.index or 0)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        for k in range(K):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            B.gamer_hydro_step_pair(S.h, D, CFL)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop()
        step_ms = sum(a.elapsed_time(b) for a, b in ev) / K
        _, _, _, n_bad = B.gamer_hydro_step_result(S.h)
        k_ms = sweep_kernel_ms(B, torch, S, D, flush, K, True, H.n_levels)
        S.close()
        del D
        achieved = BYTES_PER_CELL_F32 * updates / (k_ms / 1e3) / 1e9
        # accuracy of one pair against the FP64 path, same state and dt
        S64 = B.Solver(GAMMA, B.GAMER_LIMITER_VANLEER, B.GAMER_FP64, stream=stream)
        D64 = B.DeviceHierarchy(H, st, torch.float64, device=dev)
        dt = B.gamer_hydro_cfl_dt(S64.h, D64, CFL)
        S32 = B.Solver(GAMMA, B.GAMER_LIMITER_VANLEER, B.GAMER_FP32, stream=stream)
        D32 = B.DeviceHierarchy(H, st, torch.float32, device=dev)
        for _ in range(2):
            S64.step(D64, dt)
            S32.step(D32, dt)
        l1 = np.zeros(5)
        for l in range(H.n_levels):
            ref = D64.u[l].reshape(5, -1)
            d = (D32.u[l].double().reshape(5, -1) - ref).abs()
            scale = ref.abs().max(dim=1).values.clamp_min(1e-300)
            l1 = np.maximum(l1, (d.mean(dim=1) / scale).cpu().numpy())
        S64.close()
        S32.close()
        del D64, D32
        torch.cuda.empty_cache()
        out[name] = {
            "workload": desc, "patches": cells // 512, "levels": H.n_levels, "cells": cells,
            "value": updates / (step_ms / 1e3), "unit": UNIT, "ms_per_step": step_ms, "steps": K,
            "kernel_ms": k_ms,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                         "peak_kind": f"{peak_kind} copy bandwidth",
                         "kernel": "the step's sweep launches (k_sweep_pair for one level; k_sweep_f32 per sweep "
                                   "set over all levels otherwise)"},
            "l1_rel_err_fp32_vs_fp64": dict(zip(["rho", "mx", "my", "mz", "e"], [float(x) for x in l1])),
            "l1_after": "one xyz + zyx pair with the FP64 path's dt",
            "n_bad_cells": n_bad, "clocks": clk, "input_generation_s": gen_s,
        }
        del H, st
    return out


# ------------------------------------------------------------ accuracy

def _acc_cases(W):
    def sod_x():
        u, npg, bc = W.sod(0)
        return W.single_level(u, npg, bc=bc)
    return [
        ("cell-wise lognormal 32^3 (64 patches)", lambda: W.single_level(*W.lognormal_cells(32)), 20),
        ("Sod tube along x, 128x16x16, outflow ends", sod_x, 20),
        ("smooth k^-2 fields 128^3 (4096 patches)", lambda: W.single_level(*W.smooth_grf(128, seed=1001)), 100),
        ("3-level AMR, 4096/9000/21000 patches", lambda: W.amr_grf(), 20),
        ("lognormal sigma 1.5, rms Mach 3, 512^3 (262144 patches)",
         lambda: W.single_level(*W.lognormal_grf(512, seed=1003, dtype=np.float32)), 50),
        ("4-level stress, lognormal sigma 2.5, Mach <= 20 (32768 patches)", lambda: W.amr_stress("lognormal"), 20),
        ("4-level stress, Sedov point blast (32768 patches)", lambda: W.amr_stress("sedov"), 20),
    ]


def run_accuracy(args):
    """FP64 path for K steps (dt from Eq. CFL on the device), then the FP32
    path over the same dt sequence; errors per field relative to the
    field's largest magnitude, the worst level reported."""
    import torch
    from paper_0907_3390_gb300 import binding as B
    from paper_0907_3390_gb300 import workloads as W
    fields = ["rho", "mx", "my", "mz", "e"]
    res = []
    for name, make, K in _acc_cases(W):
        H, st = make()
        S64 = B.Solver(GAMMA, B.GAMER_LIMITER_VANLEER, B.GAMER_FP64)
        D64 = B.DeviceHierarchy(H, st, torch.float64)
        s0, nb0 = B.gamer_hydro_check(S64.h, D64)
        dts = []
        for _ in range(K):
            B.gamer_hydro_step(S64.h, D64, CFL)
            D64.swap()
            dts.append(B.gamer_hydro_step_result(S64.h)[0])
        s64, nb64 = B.gamer_hydro_check(S64.h, D64)
        S32 = B.Solver(GAMMA, B.GAMER_LIMITER_VANLEER, B.GAMER_FP32)
        D32 = B.DeviceHierarchy(H, st, torch.float32)
        for dt in dts:
            B.gamer_hydro_advance_all(S32.h, D32, dt)
            D32.swap()
        s32, nb32 = B.gamer_hydro_check(S32.h, D32)
        l1 = np.zeros(5)
        mx = np.zeros(5)
        for l in range(H.n_levels):
            ref = D64.u[l].reshape(5, -1)
            d = (D32.u[l].double().reshape(5, -1) - ref).abs()
            scale = ref.abs().max(dim=1).values.clamp_min(1e-300)
            l1 = np.maximum(l1, (d.mean(dim=1) / scale).cpu().numpy())
            mx = np.maximum(mx, (d.max(dim=1).values / scale).cpu().numpy())
        drift = lambda s: [float(abs(a - b) / (abs(b) + 1e-30)) for a, b in zip(s, s0)]
        res.append({"workload": name, "patches": sum(lv.n_groups for lv in H.levels) * 8, "steps": K,
                    "l1_rel": dict(zip(fields, l1.tolist())), "max_rel": dict(zip(fields, mx.tolist())),
                    "n_bad_initial": int(nb0), "n_bad_fp64": int(nb64), "n_bad_fp32": int(nb32),
                    "mass_energy_drift_fp64": [drift(s64)[0], drift(s64)[4]],
                    "mass_energy_drift_fp32": [drift(s32)[0], drift(s32)[4]]})
        print(json.dumps(res[-1]), file=sys.stderr, flush=True)
        S64.close()
        S32.close()
        del D64, D32
        torch.cuda.empty_cache()
    print(json.dumps({"accuracy": res, "reference": "FP64 GPU path (bit-identical to the FP64 oracle)",
                      "cfl": CFL, "limiter": "van Leer"}), flush=True)
    return 0


def run_regrid_kernels(args):
    """Device time per launch (CUDA events, L2 flushed before each) of
    gamer_hydro_flag for the three criteria and of gamer_hydro_refine_fill
    (every level-0 patch refined, half inherited, half interpolated) on the
    workload's level 0.  Algorithmic bytes: the flag step reads rho (4 B
    per cell in FP32) or all five variables (20 B) once and writes one word
    per patch; the fill writes 8 fine cells x 20 B per coarse cell and reads
    the coarse cell (20 B) or the inherited fine data (160 B)."""
    import torch
    from paper_0907_3390_gb300 import binding as B
    from paper_0907_3390_gb300 import hierarchy as hm
    desc, make = WORKLOADS[args.workload]
    H, st = make()
    H0 = hm.Hierarchy(levels=[H.levels[0]], base_npg=H.base_npg, L=H.L)
    S = B.Solver(GAMMA, B.GAMER_LIMITER_VANLEER, B.GAMER_FP32)
    D = B.DeviceHierarchy(H0, [st[0]], torch.float32)
    n = H.levels[0].n_groups
    cells = n * 4096
    hbm, kind = measured_peaks()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    masks = torch.empty(8 * n, dtype=torch.int32, device="cuda")

    def timed(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        out = []
        for r in range(reps):
            flush.fill_(r)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            out.append(e0.elapsed_time(e1) / 1e3)
        return float(np.median(out))

    res = {}
    for name, crit, thr, byt in (("flag_density_gradient", 0, 0.03, 4), ("flag_pressure_gradient", 1, 1.0, 20),
                                 ("flag_density", 2, 2.0, 4)):
        t = timed(lambda: B.gamer_hydro_flag(S.h, D, 0, crit, thr, 8, masks))
        res[name] = {"ms": 1e3 * t, "algorithmic_GBps": byt * cells / t / 1e9,
                     "frac_of_hbm": byt * cells / t / 1e9 / hbm, "bytes_per_cell": byt}
    # refinement fill of every patch of level 0: groups alternate inherit / interpolate
    nn = 8 * n
    parent = torch.arange(nn, dtype=torch.int32, device="cuda")
    inherit = torch.where(parent % 2 == 0, parent, torch.full_like(parent, -1))
    u_old = torch.zeros((5, 8 * nn, 8, 8, 8), dtype=torch.float32, device="cuda")
    u_new = torch.empty_like(u_old)
    t = timed(lambda: B.gamer_hydro_refine_fill(S.h, D, 0, parent, inherit, u_old, u_new), reps=3)
    fine = nn * 4096
    byt = fine * 20 + (fine // 2) * 20 + (cells // 2) * 20
    res["refine_fill"] = {"ms_with_host_checks": 1e3 * t, "algorithmic_bytes": byt, "fine_cells": fine,
                          "note": "the call checks parents and nesting on the host (synchronously) before its "
                                  "launch; the kernel's own time is in the ncu launch list"}
    print(json.dumps({"regrid_kernels": res, "workload": desc, "cells": cells, "peak_GBps": hbm,
                      "peak_kind": kind, "precision": "FP32 state and criteria"}), flush=True)
    S.close()
    return 0


def run_poisson(args):
    """gamer_poisson_sor on the workload's number of level-0 patch groups,
    20 iterations (tol = 0), FP32 and FP64; cell-updates/s = 16^3 cells x
    groups x iterations / device time (CUDA events, L2 flushed before).  The
    block stays in shared memory for all iterations and each thread keeps its
    own x-row in registers, so the bound is shared-memory bandwidth: the four
    y and z neighbours read and the new value written per cell update (20 B
    in FP32, 40 B in FP64) against SMs x 128 B per cycle x the max SM clock."""
    import torch
    from paper_0907_3390_gb300 import binding as B
    desc, make = WORKLOADS[args.workload]
    H, st = make()
    n = H.levels[0].n_groups
    iters = 20
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    smem_peak = sms * 128 * 2070e6 / 1e9            # GB/s
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    gen = torch.Generator(device="cuda").manual_seed(7)
    out = {}
    for name, prec, dt, b in (("fp32", B.GAMER_FP32, torch.float32, 20), ("fp64", B.GAMER_FP64, torch.float64, 40)):
        phi0 = torch.randn((n, 18, 18, 18), generator=gen, device="cuda", dtype=dt)
        rho = torch.randn((n, 16, 16, 16), generator=gen, device="cuda", dtype=dt)
        phi = phi0.clone()
        B.gamer_poisson_sor(prec, rho, phi, 0.5, 1.7, iters, 0.0)
        times = []
        for r in range(5):
            phi.copy_(phi0)
            flush.fill_(r)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            B.gamer_poisson_sor(prec, rho, phi, 0.5, 1.7, iters, 0.0)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
        t = float(np.median(times))
        upd = n * 4096 * iters
        out[name] = {"ms": 1e3 * t, "cell_updates_per_s": upd / t, "smem_GBps": upd * b / t / 1e9,
                     "smem_frac": upd * b / t / 1e9 / smem_peak}
    # inputs of the finest level's SOR problems (multi-level workloads):
    # potential blocks interpolated from the coarser level, density blocks
    prep = None
    if len(H.levels) > 1:
        l = len(H.levels) - 1
        nf, nc = H.levels[l].n_groups, H.levels[l - 1].n_groups
        S = B.Solver(GAMMA, B.GAMER_LIMITER_VANLEER, B.GAMER_FP32)
        D = B.DeviceHierarchy(H, st, torch.float32)
        phi_c = torch.randn((8 * nc, 8, 8, 8), generator=gen, device="cuda")
        pb = torch.empty((nf, 18, 18, 18), device="cuda")
        rb = torch.empty((nf, 16, 16, 16), device="cuda")
        B.gamer_poisson_prepare(S.h, D, l, phi_c, pb, rb)
        times = []
        for r in range(5):
            flush.fill_(r)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            B.gamer_poisson_prepare(S.h, D, l, phi_c, pb, rb)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
        t = float(np.median(times))
        byt = nf * 4 * (18 ** 3 + 16 ** 3 + 16 ** 3 + 8 ** 3)   # blocks written, density and parent patch read
        hbm, kind = measured_peaks()
        prep = {"level": l, "groups": nf, "ms": 1e3 * t, "algorithmic_GBps": byt / t / 1e9,
                "frac_of_hbm": byt / t / 1e9 / hbm, "note": "FP32; includes the host-side map check of the call"}
        S.close()
    print(json.dumps({"poisson_sor": out, "prepare_fp32": prep, "groups": n, "iterations": iters, "workload": desc,
                      "smem_peak_GBps": smem_peak,
                      "smem_peak_kind": f"derived: {sms} SMs x 128 B/cycle x 2070 MHz"}), flush=True)
    return 0


def run_gravity(args):
    """gamer_gravity_update on the workload's level 0 in a smooth periodic
    potential, FP32 and FP64 (CUDA events, L2 flushed before each launch).
    Algorithmic bytes per cell: the state read (5 values), momentum and
    energy written (4 values) and the group's potential block once (18^3 /
    16^3 values): 41.7 B in FP32, 83.4 B in FP64.  Then one xyzGGzyx double
    step in FP32 (xyz set, G of twice the step, zyx set: three graph or
    kernel launches) against the fused pair step on the same state, both as
    cell-updates/s (2 per cell)."""
    import torch
    from paper_0907_3390_gb300 import binding as B
    from paper_0907_3390_gb300 import workloads as W
    desc, make = WORKLOADS[args.workload]
    H, st = make()
    lv = H.levels[0]
    n, dh = lv.n_groups, lv.dh
    cells = n * 4096
    npg = H.base_npg
    hbm, kind = measured_peaks()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    nd = npg[0] * 16
    kx = 2 * np.pi * np.arange(nd) / nd
    field = 0.01 * (np.sin(kx)[None, None, :] + np.cos(2 * kx)[None, :, None] + np.sin(3 * kx)[:, None, None])
    phi_h = W.periodic_potential_blocks(field, npg)

    def timed(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        out = []
        for r in range(reps):
            flush.fill_(r)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            out.append(e0.elapsed_time(e1) / 1e3)
        return float(np.median(out))

    res = {}
    for name, prec, tdt, b in (("fp32", B.GAMER_FP32, torch.float32, 4), ("fp64", B.GAMER_FP64, torch.float64, 8)):
        u = torch.tensor(np.asarray(st[0]), dtype=tdt, device="cuda")
        phi = torch.tensor(phi_h, dtype=tdt, device="cuda")
        t = timed(lambda: B.gamer_gravity_update(prec, u, phi, dh, 1e-4))
        byt = cells * b * 9 + n * 18 ** 3 * b
        res["gravity_" + name] = {"ms": 1e3 * t, "bytes_per_cell": byt / cells, "GBps": byt / t / 1e9,
                                  "frac_of_hbm": byt / t / 1e9 / hbm}
    # coupled double step against the pair step, FP32
    S = B.Solver(GAMMA, B.GAMER_LIMITER_VANLEER, B.GAMER_FP32)
    D = B.DeviceHierarchy(H, st, torch.float32)
    phi = torch.tensor(phi_h, dtype=torch.float32, device="cuda")
    dt = B.gamer_hydro_cfl_dt(S.h, D, CFL)

    def coupled():
        S.step(D, dt)
        B.gamer_gravity_update(B.GAMER_FP32, D.u[0], phi, dh, 2 * dt)
        S.step(D, dt)
    t_c = timed(coupled)
    S.close()
    S2 = B.Solver(GAMMA, B.GAMER_LIMITER_VANLEER, B.GAMER_FP32)
    D2 = B.DeviceHierarchy(H, st, torch.float32)
    t_p = timed(lambda: B.gamer_hydro_step_pair(S2.h, D2, CFL))
    S2.close()
    res["xyzGGzyx_fp32"] = {"ms": 1e3 * t_c, "cell_updates_per_s": 2 * cells / t_c,
                            "calls": "gamer_hydro_step (xyz), gamer_gravity_update (2 dt), gamer_hydro_step (zyx)"}
    res["pair_fp32"] = {"ms": 1e3 * t_p, "cell_updates_per_s": 2 * cells / t_p,
                        "calls": "gamer_hydro_step_pair (xyz + zyx in one launch, no gravity)"}
    print(json.dumps({"gravity": res, "workload": desc, "cells": cells, "peak_GBps": hbm, "peak_kind": kind}),
          flush=True)
    return 0


def main():
    args = parse()
    if args.accuracy:
        return run_accuracy(args)
    if args.poisson:
        return run_poisson(args)
    if args.gravity:
        return run_gravity(args)
    if args.regrid_kernels:
        return run_regrid_kernels(args)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist_mod
        from paper_0907_3390_gb300 import replicas
        replicas.init(dist_mod, "nccl" if args.impl == "ours" else "gloo")
        dist = dist_mod
    if args.quick and args.precision == "fp64" and args.impl == "ours":
        return run_fp64_quick(args)
    if args.impl == "reference":
        rc = run_reference(args, rank, world)
        if dist is not None:
            dist.destroy_process_group()
        return rc
    res, extras, cells, desc = run_ours(args, rank, world, dist)
    if rank == 0:
        steps = args.steps
        line = {
            "metric": METRIC, "value": res["value"], "unit": UNIT, "n_gpus": world, "steps": steps,
            "warmup": args.warmup, "ms_per_step": res["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": desc, "cells_per_gpu": cells, "precision": "FP32 batched, FP64 reductions",
                       "step": (STEP_PAIR if args.mode == "pair" else STEP_ONE),
                       "sweep_sets_per_step": res["sets_per_step"],
                       "time_steps": res["time_steps"],
                       "cell_updates_per_step": res["updates_per_step"],
                       "l2": "flushed before every timed step (256 MiB write, outside the timed interval)",
                       "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
            "roofline": res["roofline"],
            "roofline_alu": res["roofline_alu"],
            "gpu_launches": res["launches_per_step"] * steps,
            "clocks": res["clocks"],
            "n_bad_cells": res["n_bad"],
            "conservation_drift_rel": res["conservation_drift_rel"],
        }
        for k in ("e2e", "cpu_baseline", "fp64_plain", "fp64_per_launch", "l1_rel_err_fp32_vs_fp64", "configs"):
            if k in extras:
                line[k] = extras[k]
        if "fp64_plain" in extras:
            line["fp32_over_fp64_plain"] = res["value"] / world / extras["fp64_plain"]["value"]
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
