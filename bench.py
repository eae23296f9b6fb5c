#!/usr/bin/env python
"""Benchmark: one low-storage RK3 step of the compressible Navier-Stokes residual on the
256^3 periodic Taylor-Green vortex in binary64, per algorithm family (Jammy, Jacobs &
Sandham, arXiv 1610.09146: Sections 2-4; the paper times this loop in Table 1).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

A "step" is one full RK3 step (three stages: primitives, derivatives, residual, update)
over all 256^3 points; the metric is point-updates/s = points x steps / seconds.  Each
family (store-all BL, store-some SS, recompute-all RA, recompute-some RS, store-none SN)
is timed separately in binary64, and store-some also in the mixed binary64 / double-word
form (dtype f64dw, held to the same 1e-12 parity with the binary64 oracle); the line's
`value` is the fastest of these.  Beside it: the df64 and binary32 families, a compact
record of the 64-instance batched ensemble and of the serving stream (first 40 requests),
and the end-to-end rate through the C ABI with host buffers (two solvers overlapping
their copies, and one solver alone).  Inputs: the analytic Taylor-Green initial condition
(synthetic, no dataset), 671 MB of state per buffer, far above the 129 MB L2, so no
flush is needed between steps.  Under torchrun (N > 1) every rank advances its own
256^3 instance (replicas; the single-instance path has no exchange step) and `value`
is the sum over ranks divided by the slowest rank's time.

`--impl reference` times the FP64 CPU oracle (the checker of the CUDA path) on the
host cores, one RK3 step of the full 256^3 grid per step (about 7 s each on 16 cores).
"""
from __future__ import annotations

import argparse
import datetime as _dt
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_GRID = 256
RE, MACH, PR, GAMMA = 1600.0, 0.1, 0.71, 1.4
METRIC = "point-updates/s"
VARIANTS = ["store_all", "store_some", "recompute_all", "recompute_some", "store_none"]
SHORT = {"store_all": "BL", "store_some": "SS", "recompute_all": "RA", "recompute_some": "RS", "store_none": "SN",
         "recompute_all_inline": "RAI"}

# Table 1 (Section 4): run-time in seconds of 500 iterations at 256^3 on one 24-core
# ARCHER node (24 MPI ranks, Cray C -O3, binary64).  Context only, another machine.
PAPER_256_SECONDS = {"store_all": 1561.52, "recompute_all": 765.42, "recompute_some": 802.76, "store_none": 693.66,
                     "store_some": 685.25}

MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
# binary64 arithmetic peak of GB300, nominal: 152 SMs x 2 FP64 FMA lanes per SM per clock
# x 2 flop x 2.07 GHz maximum SM clock = 1.26 TFLOP/s.  The line uses the rate measured in
# the same run (fd_fp64_peak: a binary64 FMA loop) and falls back to this one.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# Issue-slot peak: 152 SMs x 4 schedulers x one 32-thread instruction per clock x 2.07 GHz,
# in thread instructions per second; the roof of the mixed binary64 / double-word kernel,
# whose binary32 and binary64 work runs on two pipes that share these slots.
ISSUE_PEAK_TINST = 152 * 4 * 32 * 2.07e9 / 1e12
HBM_FALLBACK_GBS = 6800.0

# Algorithmic cost per grid point of one launch, by (dtype, family, kernel class):
# (flops with FMA = 2, HBM bytes at ideal reuse, FP64 pipe instructions), each averaged
# over the three stages.  Counted from the kernel source (see the kernel table of the
# design notes); the fused kernels include the primitives of the next stage, which they
# write with the update (so "prims" runs only after a state is set).
COST = {
    # binary64 SS: the gradient pass also stores the three pair sums of the diagonal
    # gradients; the fused residual weights every tap through one FMA and starts each
    # momentum residual as Q hd + v_i (ncu at 160^3: fused 226/226/221 FP64 instructions
    # and 405/405/395 flops by stage, grad 39)
    ("f64", "store_some", "fused"): (401.7, 309.3, 224.3),
    ("f64", "store_some", "grad"): (48, 120, 39),
    # binary64 RA, tap-weighted (ncu at 160^3: 344/344/339 instructions, 562/562/552 flops)
    ("f64", "recompute_all", "fused"): (558.7, 213.3, 342.3),
    ("f64", "store_all", "fused"): (177, 701.3, 140),
    ("f64", "store_all", "deriv1"): (225, 576, 180),
    ("f64", "store_all", "deriv2"): (114, 200, 84),
    ("f64", "store_all", "products"): (18, 216, 18),
    ("f64", "*", "prims"): (14, 80, 20),
    # RS and SN: the derivative set of the paper as written (BL's arithmetic per derivative);
    # RS re-evaluates the viscous terms in the energy equation, SN the inner derivatives of
    # the six mixed derivatives at the shifted taps; same bytes as SS / RA.  Flops and
    # instructions are ncu's DADD + DMUL + 2 DFMA (resp. their sum) per point, 64^3 grid
    ("f64", "recompute_some", "fused"): (669.7, 285.3, 518.3),
    ("f64", "recompute_some", "grad"): (48, 120, 39),
    ("f64", "store_none", "fused"): (710.7, 213.3, 553.3),
    # binary32 mode: the state and its RK update are double-words (no FP64 instructions)
    ("f32", "store_some", "fused"): (415.7, 222.7, 0),
    ("f32", "store_some", "grad"): (45, 48, 0),
    ("f32", "recompute_all", "fused"): (562.7, 186.7, 0),
    ("f32", "recompute_some", "fused"): (669.7, 222.7, 0),
    ("f32", "recompute_some", "grad"): (45, 48, 0),
    ("f32", "store_none", "fused"): (710.7, 186.7, 0),
    ("f32", "store_all", "fused"): (183, 430.7, 0),
    ("f32", "store_all", "deriv1"): (225, 288, 0),
    ("f32", "store_all", "deriv2"): (114, 100, 0),
    ("f32", "store_all", "products"): (18, 108, 0),
    ("f32", "*", "prims"): (14, 80, 0),
    # df64: the binary64 algorithm's flops, done in double-word arithmetic on the binary32
    # pipe (no FP64 instructions); state and fields are 8-byte double-words
    ("df64", "store_some", "fused"): (409.7, 338.7, 0),
    ("df64", "store_some", "grad"): (45, 96, 0),
    ("df64", "recompute_all", "fused"): (556.7, 266.7, 0),
    ("df64", "recompute_some", "fused"): (669.7, 338.7, 0),
    ("df64", "recompute_some", "grad"): (45, 96, 0),
    ("df64", "store_none", "fused"): (710.7, 266.7, 0),
    ("df64", "store_all", "fused"): (177, 781.3, 0),
    ("df64", "store_all", "deriv1"): (225, 576, 0),
    ("df64", "store_all", "deriv2"): (114, 200, 0),
    ("df64", "store_all", "products"): (18, 216, 0),
    ("df64", "*", "prims"): (14, 120, 0),
    # mixed binary64 / double-word store-some (dtype f64dw): flops are the binary64 algorithm's
    # (the binary64 SS kernels' fused pass and gradient pass).  A stage is two kernels: the first
    # reads the conserved fields, u_i and p (9 double-words) and the binary64 u_i, and writes the
    # diagonal gradients G_ii, div u and its five convective residuals Rc (168 bytes per point);
    # the second reads u_i, p, T (5 double-words), G_ii (3), Rc, div u and the saved register,
    # and writes the state, the saved register (stages 0 and 1), F (10 double-words) and W64 =
    # (u, v, w) of the next stage (322.7 bytes).  Binary64 instructions per point from ncu at
    # 160^3
    # binary64 recompute-all with the primitives recomputed at every tap (no primitive arrays):
    # bytes per point read the state taps once and the saved register, write the state and
    # the saved register; flops / instructions from ncu at 160^3 (DADD + DMUL + 2 DFMA)
    ("f64", "recompute_all_inline", "fused"): (3095.7, 133.3, 1774.3),
    ("f64dw", "store_some", "fused"): (460.7, 490.7, 43.3),
    ("f64dw", "*", "prims"): (14, 144, 17),  # reads Q (40 B), writes F (80) and W64 (24)
}
# Thread instructions per point of one fused pass (all pipes): ncu's smsp__thread_inst_executed
# of the two kernels at 160^3, the diagonal gradients with the convective part 1527 per point and
# the rest 2723, 2719, 2689 (stages 0-2, mean 2710.3); the issue-slot cost of the mixed pass.  Its
# binary64 instructions (first kernel DADD 6, DMUL 1, DFMA 5; second DADD 9, DMUL 5, DFMA
# 19/19/14 per point) give the 43.3 of the cost table.
ISSUE_COST = {("f64dw", "store_some", "fused"): 4237.3}
# Kernels launched per timed pass of a class, where a pass is more than one launch.
KERNELS_PER_PASS = {("f64dw", "store_some", "fused"): 2}
# FP64 pipe issue peak: 2 instructions per SM per clock.
FP64_PEAK_INSTR = 152 * 2 * 2.07e9


def cost_of(dtype, alg, kclass):
    return COST.get((dtype, alg, kclass)) or COST.get((dtype, "*", kclass))


# ---------------------------------------------------------------- utilities


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate_over_ranks(local_ms, points_per_rank, steps, dist=None, device=None):
    """Whole-job throughput: the slowest rank's time (max over ranks of the timed region)
    and the points all ranks advanced.  Returns (value, max_ms)."""
    ws = 1
    ms = float(local_ms)
    if dist is not None and dist.is_initialized():
        import torch
        ws = dist.get_world_size()
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ws * points_per_rank * steps / (ms / 1e3), ms


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples every 200 ms while running."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.windows = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None

    def mark(self, t0, t1):
        self.windows.append((t0, t1))

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        rows = []
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = _dt.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                continue
            rows.append((ts, parts))
        inwin = [p for ts, p in rows if any(a <= ts <= b for a, b in self.windows)] or [p for _, p in rows]
        sm = [float(p[2]) for p in inwin if p[2].replace(".", "", 1).isdigit()]
        smax = [float(p[3]) for p in inwin if p[3].replace(".", "", 1).isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for p in inwin for i in range(4) if p[6 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(inwin)}


def measured_peaks():
    try:
        d = json.load(open(MEASURED_PEAKS))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


# ------------------------------------------------------------- our CUDA path


def time_family(fd, torch, alg, dtype, n, steps, warmup, stream, barrier, clocks):
    from paper_1610_09146_gb300 import native
    s = fd.Solver(n, Re=RE, Mach=MACH, Pr=PR, gamma=GAMMA, dt=fd.dt_for_grid(n), algorithm=alg, dtype=dtype,
                  stream=stream)
    s.step(warmup)
    torch.cuda.synchronize()
    native.fd_profile(s.h, 1)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    t0 = time.time()
    e0.record(stream)
    s.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    t1 = time.time()
    barrier()
    clocks.mark(t0, t1)
    ms = e0.elapsed_time(e1)
    kern = {}
    for c, name in enumerate(native.KERNEL_CLASS_NAMES):
        tot, cnt = native.fd_profile_read(s.h, c)
        if cnt:
            kern[name] = {"ms_total": tot, "launches": cnt, "ms_avg": tot / cnt}
    native.fd_profile(s.h, 0)
    finite = s.check_finite()
    ke, ens = s.diagnostics()
    return s, ms, kern, finite, (ke, ens)


def roofline_of(dtype, alg, kern, n, hbm_peak, hbm_src, fp64_peak=None):
    """Roofline entry of the kernel with the largest share of the step.  fp64_peak: the
    measured binary64 rate in TFLOP/s (None: the nominal one)."""
    name, k = max(kern.items(), key=lambda kv: kv[1]["ms_total"])
    flops_pt, bytes_pt, instr_pt = cost_of(dtype, alg, name)
    sec = k["ms_avg"] / 1e3
    gbs = bytes_pt * n / sec / 1e9
    tflops = flops_pt * n / sec / 1e12
    p64 = fp64_peak or FP64_PEAK_TFLOPS
    p64_src = ("measured in this run (fd_fp64_peak: binary64 FMA loop)" if fp64_peak
               else "FP64 nominal: 152 SMs x 4 flop/clk x 2.07 GHz")
    if dtype == "f64dw" and (dtype, alg, name) in ISSUE_COST:
        tinst = ISSUE_COST[(dtype, alg, name)] * n / sec / 1e12
        entry = {"kernel": f"{SHORT[alg]}:{name}", "bound": "alu", "achieved": round(tinst, 3),
                 "peak": round(ISSUE_PEAK_TINST, 3), "unit": "Tinst/s", "frac": round(tinst / ISSUE_PEAK_TINST, 4),
                 "peak_source": "issue slots: 152 SMs x 4 schedulers x 32 threads x 2.07 GHz",
                 "binary64_equivalent_tflops": round(tflops, 4), "vs_fp64_peak": round(tflops / p64, 4),
                 "fp64_peak_tflops": round(p64, 4), "fp64_peak_source": p64_src,
                 "fp64_pipe_frac": round(instr_pt * n / sec / (p64 * 1e12 / 2), 4),
                 "hbm_achieved_gbs": round(gbs, 1), "hbm_frac": round(gbs / hbm_peak, 4)}
    elif dtype in ("f64", "df64", "f64dw"):
        entry = {"kernel": f"{SHORT[alg]}:{name}", "bound": "alu", "achieved": round(tflops, 4),
                 "peak": round(p64, 4), "unit": "TFLOP/s", "frac": round(tflops / p64, 4),
                 "peak_source": p64_src,
                 "fp64_pipe_frac": round(instr_pt * n / sec / (p64 * 1e12 / 2), 4),
                 "hbm_achieved_gbs": round(gbs, 1), "hbm_frac": round(gbs / hbm_peak, 4)}
    else:
        entry = {"kernel": f"{SHORT[alg]}:{name}", "bound": "hbm", "achieved": round(gbs, 1),
                 "peak": hbm_peak, "unit": "GB/s", "frac": round(gbs / hbm_peak, 4),
                 "peak_source": f"{hbm_src} (MEASURED_PEAKS.json hbm_gbs)" if hbm_src == "measured" else "fallback"}
    entry["share"] = round(k["ms_total"] / sum(v["ms_total"] for v in kern.values()), 4)
    bpp = TRAFFIC_BPP.get((dtype, alg, name))
    entry["traffic"] = round(bpp * n) if bpp is not None else None
    entry["algorithmic_per_point"] = {"flops": flops_pt, "bytes": bytes_pt, "fp64_instr": instr_pt}
    return entry


# DRAM traffic per point of one launch, dram__bytes_read.sum + dram__bytes_write.sum from one
# ncu capture of every kernel of the 160^3 bench line (bench.py --grid 160 --steps 2 --warmup 3
# --no-cpu-baseline --no-extras; mean over the stages' launches), the traffic of a launch being
# this times the points (the stencil kernels' traffic is proportional to the point count: the
# binary32 RA kernel gives 180.0 B/point at 160^3 and 187.4 at 256^3; its entry is the 256^3 capture
# of the kernel's current 36 x 12 staging box).  The roofline entry's `traffic` is this times the
# points of the run.  The mixed store-some entries are a later capture
# of the same 160^3 grid through the public API (fused pass: both kernels, 154.1 + 325.6).
TRAFFIC_BPP = {
    ("f64", "store_some", "fused"): 304.5, ("f64", "store_some", "grad"): 105.9,
    ("f64", "recompute_all", "fused"): 205.9, ("f64", "recompute_some", "fused"): 281.0,
    ("f64", "recompute_some", "grad"): 105.9, ("f64", "store_none", "fused"): 206.2,
    ("f64", "store_all", "fused"): 696.1, ("f64", "store_all", "deriv1"): 578.2,
    ("f64", "store_all", "deriv2"): 187.6, ("f64", "store_all", "products"): 200.4,
    ("f64", "recompute_all_inline", "fused"): 125.3,
    ("f64dw", "store_some", "fused"): 479.7,
    ("f32", "store_some", "fused"): 213.4, ("f32", "store_some", "grad"): 34.5,
    ("f32", "recompute_all", "fused"): 187.4, ("f32", "recompute_some", "fused"): 214.1,
    ("f32", "recompute_some", "grad"): 34.5, ("f32", "store_none", "fused"): 175.9,
    ("f32", "store_all", "fused"): 423.0, ("f32", "store_all", "deriv1"): 277.4,
    ("f32", "store_all", "deriv2"): 86.7, ("f32", "store_all", "products"): 93.1,
    ("df64", "store_some", "fused"): 332.1, ("df64", "store_some", "grad"): 81.9,
    ("df64", "recompute_all", "fused"): 261.1, ("df64", "recompute_some", "fused"): 333.0,
    ("df64", "recompute_some", "grad"): 81.9, ("df64", "store_none", "fused"): 258.0,
    ("df64", "store_all", "fused"): 747.6, ("df64", "store_all", "deriv1"): 573.5,
    ("df64", "store_all", "deriv2"): 187.0, ("df64", "store_all", "products"): 201.5,
}


def e2e_run(fd, torch, alg, dtype, n, steps, nsolvers=2):
    """Same metric through the public API with host buffers: every step copies a state in
    from pinned host memory, advances one RK3 step and copies the state back out.  With two
    solvers on two streams taking the steps in turn (fd_set_state_async / fd_step /
    fd_get_state_async), one solve's copies overlap the other's step, as a user streaming
    independent states through the library would run it; with one solver nothing overlaps
    (copy in, step, copy out, in sequence)."""
    from paper_1610_09146_gb300 import native
    nel = 5 * n**3
    streams = [torch.cuda.Stream() for _ in range(nsolvers)]
    solvers = [fd.Solver(n, Re=RE, Mach=MACH, Pr=PR, gamma=GAMMA, dt=fd.dt_for_grid(n), algorithm=alg,
                         dtype=dtype, stream=st) for st in streams]
    hin = torch.empty(nel, dtype=torch.float64, pin_memory=True)
    hout = [torch.empty(nel, dtype=torch.float64, pin_memory=True) for _ in streams]
    native.fd_get_state(solvers[0].h, hin.data_ptr(), nel, 0)

    def one(k):
        s, o = solvers[k % nsolvers], hout[k % nsolvers]
        native.fd_set_state_async(s.h, hin.data_ptr(), nel, 0)
        native.fd_step(s.h, 1)
        native.fd_get_state_async(s.h, o.data_ptr(), nel, 0)

    for k in range(nsolvers):  # warm-up: one step on each solver
        one(k)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(steps):
        one(k)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    ok = all(s.check_finite() for s in solvers)
    for s in solvers:
        s.close()
    how = ("two solvers on two streams taking the steps in turn" if nsolvers == 2
           else "one solver: copy in, step, copy out, in sequence")
    return {"value": n**3 * steps / (t1 - t0), "unit": METRIC, "h2d_bytes_per_step": nel * 8,
            "d2h_bytes_per_step": nel * 8, "steps": steps, "finite": ok, "family": SHORT[alg], "dtype": dtype,
            "path": "per step: fd_set_state_async(pinned host) + fd_step(1) + fd_get_state_async(pinned host), "
                    + how}


def cpu_baseline_full(n):
    """The oracle as it stands: one RK3 step of the full n^3 Taylor-Green grid."""
    import oracle
    Q = oracle.tgv_ic(n, n, n, GAMMA, MACH)
    t0 = time.perf_counter()
    oracle.run(Q, 1, dt=3.385e-3 * 64 / n, Re=RE, Mach=MACH, Pr=PR, gamma=GAMMA)
    t = time.perf_counter() - t0
    return {"value": n**3 / t, "unit": METRIC, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"1 RK3 step of the full {n}^3 grid ({t:.1f} s)"}


def run_ours(args):
    import torch

    import paper_1610_09146_gb300 as fd
    from paper_1610_09146_gb300 import native
    ws, rank, local = dist_env()
    dist = None
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    else:
        torch.cuda.set_device(0)
    fd.build()
    if ws > 1:
        dist.barrier()

    def barrier():
        if dist is not None:
            dist.barrier()

    n = args.grid
    npts = n**3
    stream = torch.cuda.Stream()
    hbm_peak, hbm_src = measured_peaks()
    try:
        fp64_peak = native.fd_fp64_peak() / 1e12
    except Exception:
        fp64_peak = None
    clocks = ClockSampler(local)
    clocks.start()
    # the binary64 families, and the mixed binary64 / double-word store-some form, which is
    # held to the same parity bound (1e-12 against the binary64 oracle)
    cases = [(alg, args.dtype) for alg in args.variants]
    if args.dtype == "f64" and "store_some" in args.variants and not args.no_f64dw:
        cases.append(("store_some", "f64dw"))
    results = {}
    best = None
    for alg, dtype in cases:
        s, ms, kern, finite, diag = time_family(fd, torch, alg, dtype, n, args.steps, args.warmup, stream,
                                                barrier, clocks)
        value, ms = aggregate_over_ranks(ms, npts, args.steps, dist, "cuda")
        launches = sum(k["launches"] * KERNELS_PER_PASS.get((dtype, alg, c), 1) for c, k in kern.items())
        key = SHORT[alg] if dtype == args.dtype else f"{SHORT[alg]}_{dtype}"
        results[key] = {"value": value, "ms_per_step": ms / args.steps, "finite": finite, "gpu_launches": launches,
                        "kernels": kern, "dtype": dtype, "family": alg,
                        "roofline": roofline_of(dtype, alg, kern, npts, hbm_peak, hbm_src, fp64_peak),
                        "ke": diag[0], "enstrophy": diag[1],
                        "paper_table1_256_point_updates_per_s": npts * 500 / PAPER_256_SECONDS[alg]}
        s.close()
        if best is None or value > results[best]["value"]:
            best = key
    # binary64-accurate double-word families (FD_DF64): reported beside the binary64 line
    p64 = fp64_peak or FP64_PEAK_TFLOPS
    df64 = {}
    if args.dtype == "f64" and not args.no_df64:
        for alg in args.variants:
            s, ms, kern, finite, diag = time_family(fd, torch, alg, "df64", n, args.steps, args.warmup, stream,
                                                    barrier, clocks)
            s.close()
            value, ms = aggregate_over_ranks(ms, npts, args.steps, dist, "cuda")
            name, k = max(kern.items(), key=lambda kv: kv[1]["ms_total"])
            flops_pt = cost_of("f64", alg, name)[0]
            eq = flops_pt * npts / (k["ms_avg"] / 1e3) / 1e12
            df64[SHORT[alg]] = {"value": value, "ms_per_step": ms / args.steps, "finite": finite,
                                "dominant_kernel": name, "kernels": {kk: round(vv["ms_avg"], 4) for kk, vv in kern.items()},
                                "binary64_equivalent_tflops": round(eq, 4),
                                "vs_fp64_peak": round(eq / p64, 4), "ke": diag[0]}
    # binary32-stencil mode (FD_F32_ACCDW) families, beside the binary64 line
    f32 = {}
    if args.dtype == "f64" and not args.no_df64:
        for alg in args.variants:
            s, ms, kern, finite, diag = time_family(fd, torch, alg, "f32", n, args.steps, args.warmup, stream,
                                                    barrier, clocks)
            s.close()
            value, ms = aggregate_over_ranks(ms, npts, args.steps, dist, "cuda")
            f32[SHORT[alg]] = {"value": value, "ms_per_step": ms / args.steps, "finite": finite,
                               "kernels": {kk: round(vv["ms_avg"], 4) for kk, vv in kern.items()},
                               "roofline": roofline_of("f32", alg, kern, npts, hbm_peak, hbm_src),
                               "ke_rel_vs_binary64": abs(diag[0] - results[SHORT[alg]]["ke"])
                               / results[SHORT[alg]]["ke"]}
    cl = clocks.stop()
    r = results[best]
    e2e_steps = max(4, min(args.steps, 40))
    e2e = e2e_run(fd, torch, r["family"], r["dtype"], n, e2e_steps)
    e2e["value"], _ = aggregate_over_ranks(1e3 * npts * e2e["steps"] / e2e["value"], npts, e2e["steps"], dist,
                                           "cuda")
    e2e1 = e2e_run(fd, torch, r["family"], r["dtype"], n, e2e_steps, nsolvers=1)
    e2e1["value"], _ = aggregate_over_ranks(1e3 * npts * e2e1["steps"] / e2e1["value"], npts, e2e1["steps"], dist,
                                            "cuda")
    dtype_label = {"f64": "f64", "f64dw": "f64dw (binary64 state, pressure, div u, RK; double-word stencils)"}
    line = {
        "metric": METRIC, "value": r["value"], "unit": METRIC, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": r["value"] / r["paper_table1_256_point_updates_per_s"],
        "dtype": dtype_label.get(r["dtype"], r["dtype"]),
        "data": "synthetic (analytic Taylor-Green vortex initial condition)",
        "config": {"workload": f"Taylor-Green vortex {n}^3, binary64 results (parity 1e-12 with the binary64 "
                               "oracle), one low-storage RK3 step per step, each algorithm family timed separately; "
                               "value = fastest family",
                   "family": f"{r['family']} ({SHORT[r['family']]})", "grid": [n, n, n], "Re": RE, "Mach": MACH,
                   "Pr": PR, "gamma": GAMMA, "dt": fd.dt_for_grid(n),
                   "l2": f"inputs larger than L2 ({40 * npts / 1e6:.0f} MB state per buffer vs 129 MB L2); no flush",
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "roofline": r["roofline"], "gpu_launches": r["gpu_launches"], "e2e": e2e, "e2e_one_solver": e2e1,
        "clocks": cl,
        "fp64_peak_measured_tflops": round(fp64_peak, 4) if fp64_peak else None,
        "variants": {a: {k: v for k, v in results[a].items() if k != "kernels"} | {
            "kernels": {kk: round(vv["ms_avg"], 4) for kk, vv in results[a]["kernels"].items()}}
            for a in results},
        "variants_df64": df64,
        "variants_f32": f32,
        "variants_f32_note": "dtype f32: binary32 stencils on perturbation fields, compensated (double-word) state "
                             "and RK update; roofline against the measured HBM copy rate",
        "variants_df64_note": "dtype df64: double-word arithmetic on the binary32 pipe; binary64_equivalent_tflops "
                              "counts the binary64 algorithm's flops",
    }
    if rank == 0 and ws == 1 and not args.no_extras:
        line["batched"] = batched_extra(fd, args)
        line["serve"] = serve_extra(fd, args)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_full(n)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def batched_extra(fd, args):
    """Compact record of the 64-instance ensemble (binary32 batch with recompute-all, the
    autotuner's choice for every grid on GB300, vs the binary64 per-solve loop and batch)."""
    from paper_1610_09146_gb300 import workloads
    specs = workloads.ensemble(count=64, steps=100)
    tuned = [dict(sp, algorithm="recompute_all", tile_points=0) for sp in specs]
    r = batched_summary(fd, specs, 100, tuned)
    return {"workload": "64 Taylor-Green solves, grids {32,48,64,96,128}^3, Re U[400,3200], Mach U[0.1,0.4], "
                        "100 RK3 steps, seed 1610; binary32 batch (recompute-all)",
            "solves_per_s": r["value"], "fp64_loop_solves_per_s": r["fp64_loop"]["solves_per_s"],
            "fp64_batched_solves_per_s": r["fp64_batched"]["solves_per_s"],
            "f64dw_batched_solves_per_s": r["f64dw_batched"]["solves_per_s"],
            "fp64_batched_equals_loop": r["fp64_batched"]["ke_bitwise_equal_to_loop"],
            "speedup_vs_fp64_loop": r["speedup_vs_fp64_loop"], "ke_rel_err_vs_fp64_max": r["ke_rel_err_vs_fp64"]["max"]}


def serve_extra(fd, args):
    """Compact serving record: the first args.serve_requests requests of the seeded stream
    (mean 20 requests/s), binary32 requests on recompute-all and binary64 on store-some."""
    from paper_1610_09146_gb300 import workloads
    reqs = workloads.requests(count=args.serve_requests, rate=20.0)
    for q in reqs:
        q["algorithm"] = "recompute_all" if q["dtype"] == "f32" else "store_some"
        if q["dtype"] == "f64":  # binary64 requests run the mixed form (binary64 parity, 2x faster)
            q["dtype"] = "f64dw"
        q["tile_points"] = 0
        q["tag"] = q["id"]
    r = serve_summary(fd, reqs, 20.0, 64, 256)
    return {"workload": f"first {len(reqs)} requests of the Poisson stream (mean 20/s, seed 9146), grids 48^3-192^3, "
                        "50-500 RK3 steps, f32 (RA) or f64 (mixed binary64 / double-word SS) per request",
            "solves_per_s": r["value"], "latency_p50_s": r["latency_s"]["p50"],
            "latency_p99_s": r["latency_s"]["p99"], "offered_over_capacity": r["offered_over_capacity"],
            "completed_ok": r["completed_ok"], "span_s": r["span_s"]}


# ------------------------------------------------------------ batched ensemble


def batched_summary(fd, specs, steps, tuned):
    """The ensemble in one binary32 batch (families / tiles of `tuned`), against the plain
    binary64 per-solve loop and the binary64 batch of the same solves.  A solve = create +
    steps + diagnostics; seconds are wall time with the device synchronised."""
    import numpy as np
    import torch

    def batched(dtype, sp):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with fd.Batch(sp, dtype=dtype) as b:
            b.step(steps)
            ke, en = b.diagnostics()
        t1 = time.perf_counter()
        return t1 - t0, ke, en

    def loop64():
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ke = []
        for s in specs:
            with fd.Solver(s["n"], Re=s["Re"], Mach=s["Mach"], dt=s["dt"], algorithm="store_some",
                           dtype="f64") as sol:
                sol.step(steps)
                ke.append(sol.diagnostics()[0])
        torch.cuda.synchronize()
        return time.perf_counter() - t0, np.array(ke)

    batched("f32", tuned[:4])  # warm-up: module load, allocator pools
    tb, ke32, _ = batched("f32", tuned)
    tb2, _, _ = batched("f32", tuned)
    tb = min(tb, tb2)
    tl, ke64 = loop64()
    # binary64 batch of the same solves (store-some everywhere): bitwise the loop's results
    t64b, ke64b, _ = batched("f64", [dict(s, algorithm="store_some", tile_points=1024) for s in specs])
    # the mixed binary64 / double-word batch (binary64 parity) of the same solves
    tdw, kedw, _ = batched("f64dw", [dict(s, algorithm="store_some", tile_points=1024) for s in specs])
    kerr = np.abs(ke32 - ke64) / ke64
    pts = sum(s["n"] ** 3 for s in specs)
    return {
        "metric": "solves/s", "value": len(specs) / tb, "unit": "solves/s", "higher_is_better": True,
        "dtype": "f32 stencils / compensated-f32 (double-word) accumulation",
        "seconds": tb, "point_updates_per_s": pts * steps / tb,
        "fp64_loop": {"solves_per_s": len(specs) / tl, "seconds": tl, "family": "store_some"},
        "fp64_batched": {"solves_per_s": len(specs) / t64b, "seconds": t64b,
                         "ke_bitwise_equal_to_loop": bool(np.array_equal(ke64b, ke64))},
        "f64dw_batched": {"solves_per_s": len(specs) / tdw, "seconds": tdw,
                          "ke_rel_err_vs_fp64_max": float(np.max(np.abs(kedw - ke64) / ke64))},
        "speedup_vs_fp64_loop": tl / tb,
        "ke_rel_err_vs_fp64": {"max": float(kerr.max()), "median": float(np.median(kerr))},
    }


def run_batched(args):
    """64 uneven Taylor-Green solves (grids from {32,48,64,96,128}^3, Re in [400,3200],
    Mach in [0.1,0.4], 100 RK3 steps): binary32-stencil batch in one persistent launch per
    family and stage (family and tile size per grid from the autotuner) against the plain
    binary64 per-solve loop on the same GPU.  A solve = create + steps + diagnostics."""
    import torch

    import paper_1610_09146_gb300 as fd
    from paper_1610_09146_gb300 import autotune, workloads
    torch.cuda.set_device(0)
    fd.build()
    specs = workloads.ensemble(count=args.instances, steps=args.solve_steps)
    tuned, choice = autotune.choose(specs, "f32")
    line = {"workload": f"batched ensemble: {len(specs)} Taylor-Green solves, grids {{32,48,64,96,128}}^3, "
                        f"Re U[400,3200], Mach U[0.1,0.4], {args.solve_steps} RK3 steps, seed 1610"}
    line |= batched_summary(fd, specs, args.solve_steps, tuned)
    line["autotune"] = {str(n): {"family": f, "tile_points": t, "ms_per_instance_step": round(m, 4)}
                        for n, (f, t, m) in choice.items()}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------- 512^3 mixed precision


def run_mixed512(args):
    """Taylor-Green 512^3: binary32-stencil / binary64-accumulate recompute-all and store-some
    against the binary64 store-some run on the GPU, after 100 and after 200 RK3 steps
    (per conserved variable relative L2 error, kinetic energy and enstrophy error), with
    each run's throughput.  The binary64 GPU path is itself checked against the oracle
    (relative L-inf, 10 steps of 64^3) in the same run."""
    import numpy as np
    import torch

    import oracle
    import paper_1610_09146_gb300 as fd
    from paper_1610_09146_gb300 import native
    torch.cuda.set_device(0)
    fd.build()
    n, steps = args.grid, args.solve_steps
    dt = fd.dt_for_grid(n)
    half = steps // 2

    def run(alg, dtype):
        out = {}
        with fd.Solver(n, dt=dt, algorithm=alg, dtype=dtype) as s:
            native.fd_profile(s.h, 1)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s.step(half)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            out["Q_half"] = s.state()
            out["diag_half"] = s.diagnostics()
            t2 = time.perf_counter()
            s.step(steps - half)
            torch.cuda.synchronize()
            t3 = time.perf_counter()
            out["Q"] = s.state()
            out["diag"] = s.diagnostics()
            fused_ms, fused_n = native.fd_profile_read(s.h, native.FD_KERNEL_FUSED)
        out["ms_per_step"] = 1e3 * ((t1 - t0) + (t3 - t2)) / steps
        out["fused_ms"] = fused_ms / max(fused_n, 1)
        return out

    def rel_l2(a, b):
        return [float(np.linalg.norm(a[v] - b[v]) / np.linalg.norm(b[v])) for v in range(5)]

    # binary64 path vs oracle at 64^3, 10 steps
    m = 64
    ref = oracle.run(oracle.tgv_ic(m, m, m, GAMMA, MACH), 10, dt=fd.dt_for_grid(m))
    with fd.Solver(m, dt=fd.dt_for_grid(m), algorithm="store_some", dtype="f64") as s:
        s.step(10)
        Qm = s.state()
    val64 = max(float(np.abs(Qm[v] - ref[v]).max() / np.abs(ref[v]).max()) for v in range(5))
    base = run("store_some", "f64")
    res = {}
    for alg in ("recompute_all", "store_some"):
        r = run(alg, "f32")
        res[SHORT[alg]] = {
            "ms_per_step": r["ms_per_step"], "point_updates_per_s": n**3 / (r["ms_per_step"] / 1e3),
            "fused_ms_per_launch": r["fused_ms"],
            f"rel_l2_per_var_{half}_steps": rel_l2(r["Q_half"], base["Q_half"]),
            f"rel_l2_per_var_{steps}_steps": rel_l2(r["Q"], base["Q"]),
            f"ke_rel_err_{half}_steps": abs(r["diag_half"][0] - base["diag_half"][0]) / base["diag_half"][0],
            f"ke_rel_err_{steps}_steps": abs(r["diag"][0] - base["diag"][0]) / base["diag"][0],
            f"enstrophy_rel_err_{steps}_steps": abs(r["diag"][1] - base["diag"][1]) / base["diag"][1],
        }
        del r
    line = {
        "workload": f"Taylor-Green {n}^3, binary32 stencils / compensated binary32 (double-word) RK accumulation, binary64 reductions, "
                    f"{steps} RK3 steps, vs the binary64 GPU run",
        "metric": METRIC, "unit": METRIC, "higher_is_better": True, "grid": [n, n, n], "dt": dt,
        "value": max(v["point_updates_per_s"] for v in res.values()),
        "fp64_reference": {"family": "SS", "ms_per_step": base["ms_per_step"],
                           "point_updates_per_s": n**3 / (base["ms_per_step"] / 1e3),
                           "ke": base["diag"][0], "enstrophy": base["diag"][1],
                           "validated_vs_oracle_64cube_10steps_rel_linf": val64},
        "f32": res,
        "bounds": {"rel_l2_state": 1e-5, "ke_rel": 1e-6},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- size sweep


def run_sweep(args):
    """Roofline sweep over grid sizes (128^3, 256^3, 384^3 by default): every family in
    binary64 and the fastest binary32 / df64 families, each timed in three windows of K steps
    after a warm-up (CUDA events on the solver's stream; the median window is reported), with
    the dominant kernel placed on its roofline as in the single-grid line."""
    import numpy as np
    import torch

    import paper_1610_09146_gb300 as fd
    from paper_1610_09146_gb300 import native
    torch.cuda.set_device(0)
    fd.build()
    hbm_peak, hbm_src = measured_peaks()
    stream = torch.cuda.Stream()
    cases = [("f64", a) for a in VARIANTS] + [("f64", "recompute_all_inline"), ("f64dw", "store_some"),
                                              ("f32", "recompute_all"), ("f32", "store_some"),
                                              ("df64", "store_some"), ("df64", "store_none")]
    out = {}
    for n in args.sizes:
        npts = n**3
        steps = max(2, int(round(args.steps * (256 / n) ** 3)))
        res = {}
        for dtype, alg in cases:
            with fd.Solver(n, Re=RE, Mach=MACH, Pr=PR, gamma=GAMMA, dt=fd.dt_for_grid(n), algorithm=alg,
                           dtype=dtype, stream=stream) as s:
                s.step(args.warmup)
                windows, kerns = [], []
                for _ in range(3):
                    torch.cuda.synchronize()
                    native.fd_profile(s.h, 1)
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    s.step(steps)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    windows.append(e0.elapsed_time(e1) / steps)
                    kern = {}
                    for c, name in enumerate(native.KERNEL_CLASS_NAMES):
                        tot, cnt = native.fd_profile_read(s.h, c)
                        if cnt:
                            kern[name] = {"ms_total": tot, "launches": cnt, "ms_avg": tot / cnt}
                    native.fd_profile(s.h, 0)
                    kerns.append(kern)
                finite = s.check_finite()
            i = int(np.argsort(windows)[1])  # the median window
            ms = windows[i]
            rl = roofline_of("f64" if dtype == "df64" else dtype, alg, kerns[i], npts, hbm_peak, hbm_src)
            res[f"{dtype}:{SHORT[alg]}"] = {
                "ms_per_step": round(ms, 4), "point_updates_per_s": npts / (ms / 1e3), "finite": finite,
                "windows_ms": [round(w, 4) for w in windows],
                "kernels_ms": {k: round(v["ms_avg"], 4) for k, v in kerns[i].items()},
                "roofline": {k: rl[k] for k in ("kernel", "bound", "achieved", "unit", "frac", "share")}
                            | ({"fp64_pipe_frac": rl["fp64_pipe_frac"], "hbm_frac": rl["hbm_frac"]}
                               if dtype == "f64" else {}),
            }
        out[str(n)] = {"steps_per_window": steps, "results": res}
    line = {"workload": "roofline sweep over grid sizes, Taylor-Green vortex, every family", "metric": METRIC,
            "unit": METRIC, "sizes": args.sizes, "hbm_peak_gbs": hbm_peak,
            "fp64_peak_tflops": round(FP64_PEAK_TFLOPS, 4),
            "note": "df64 rooflines count the binary64 algorithm's flops against the FP64 peak", "sweep": out}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------ long-time history


def run_history(args):
    """Taylor-Green vortex (Re 1600, M 0.1) integrated to t = args.t_end on one grid, in one
    precision mode and family, sampling the kinetic energy and enstrophy every
    args.sample_dt time units (Section 3, Fig. 3 shows these two curves).  The reference
    curves of Wang et al. 2013 are not available, so the run checks what the equations fix
    instead: at low Mach number the kinetic energy decays at the rate 2 nu Omega (the
    incompressible energy identity, with O(M^2) compressible corrections), and a second
    grid or precision mode must give the same curves."""
    import numpy as np
    import torch

    import paper_1610_09146_gb300 as fd
    torch.cuda.set_device(0)
    fd.build()
    n = args.grid
    alg = args.variants[0]
    dt = fd.dt_for_grid(n)
    per = max(1, int(round(args.sample_dt / dt)))
    nsamp = int(np.ceil(args.t_end / (per * dt)))
    with fd.Solver(n, dt=dt, algorithm=alg, dtype=args.dtype) as s:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        t, ke, en = s.history(per, nsamp)
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        finite = s.check_finite()
    nu = 1.0 / RE
    eps = -(ke[2:] - ke[:-2]) / (t[2:] - t[:-2])       # -dKE/dt, central differences
    two_nu_omega = 2 * nu * en[1:-1]
    ip = int(np.argmax(eps))
    ie = int(np.argmax(en))
    line = {
        "workload": f"Taylor-Green vortex {n}^3 to t = {args.t_end}, Re {RE:g}, M {MACH:g}, "
                    f"{SHORT[alg]} family, dtype {args.dtype}",
        "metric": METRIC, "unit": METRIC, "higher_is_better": True,
        "value": n**3 * per * nsamp / sec, "seconds": sec, "grid": [n, n, n], "dt": dt,
        "steps": per * nsamp, "dtype": args.dtype, "family": SHORT[alg], "finite": finite,
        "summary": {
            "ke_final": float(ke[-1]),
            "enstrophy_peak": {"t": float(t[ie]), "value": float(en[ie])},
            "dissipation_peak": {"t": float(t[1 + ip]), "value": float(eps[ip])},
            "eps_minus_2nu_omega_at_peak_rel": float((eps[ip] - two_nu_omega[ip]) / eps[ip]),
            "eps_minus_2nu_omega_max_rel": float(np.max(np.abs(eps - two_nu_omega)) / eps[ip]),
        },
        "series": {"t": [round(float(x), 6) for x in t], "ke": [float(x) for x in ke],
                   "enstrophy": [float(x) for x in en]},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ serving


def serve_summary(fd, reqs, rate, arena_gb, max_active):
    """Serve `reqs` (dicts with arrival time t, grid, steps, dtype, algorithm, tile_points)
    through the continuous-batching server: each request is submitted when its arrival time
    passes on the wall clock; ticks run while any solve is queued or active.  Latency =
    completion (the tick that retired it) - arrival."""
    import numpy as np
    work = sum(r["n"] ** 3 * r["steps"] for r in reqs)
    with fd.Server(arena_gb * (1 << 30), max_active=max_active) as srv:
        # warm-up outside the measurement: one tiny solve of each dtype
        for dt_ in ("f32", "f64"):
            srv.submit(dict(n=16, steps=2, dtype=dt_, tag=-1))
        while srv.stats()["completed"] < 2:
            srv.tick()
        srv.poll()
        t0 = time.perf_counter()
        nxt, done, active_hist = 0, {}, []
        busy = 0.0
        while len(done) < len(reqs):
            now = time.perf_counter() - t0
            while nxt < len(reqs) and reqs[nxt]["t"] <= now:
                srv.submit(reqs[nxt])
                nxt += 1
            st = srv.stats()
            if st["active"] == 0 and st["queued"] == 0:
                if nxt < len(reqs):
                    time.sleep(max(0.0, min(0.002, reqs[nxt]["t"] - now)))
                continue
            ta = time.perf_counter()
            active_hist.append(srv.tick())
            tb = time.perf_counter()
            busy += tb - ta
            for res in srv.poll():
                done[res["tag"]] = (tb - t0, res)
        t_end = max(v[0] for v in done.values())
        stats = srv.stats()
    lat = np.array([done[r["id"]][0] - r["t"] for r in reqs])
    ok = sum(1 for v in done.values() if v[1]["status"] == fd.FD_OK)
    span = t_end - reqs[0]["t"]
    offered = rate * work / len(reqs)
    return {
        "metric": "solves/s", "value": len(reqs) / span, "unit": "solves/s", "higher_is_better": True,
        "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                      "mean": float(lat.mean()), "max": float(lat.max())},
        "completed_ok": ok, "requests": len(reqs), "span_s": span,
        "point_updates_per_s": work / span,
        "capacity_point_updates_per_busy_s": work / busy,
        "offered_point_updates_per_s": offered,
        "offered_over_capacity": offered / (work / busy),
        "mean_active_per_tick": float(np.mean(active_hist)), "ticks": stats["ticks"],
        "arena_gb": arena_gb, "max_active": max_active,
    }


def run_serve(args):
    """Poisson stream (mean 20 requests/s, seeded) of Taylor-Green solves, grids the multiples
    of 16 in [48, 192], 50-500 steps, Re in [400, 3200], Mach in [0.1, 0.4], binary32 or
    binary64 with equal odds, served by the continuous-batching server: requests are
    submitted when their arrival time passes on the wall clock, admitted by device
    footprint, advanced together (time-sliced ticks).  Latency = completion - arrival."""
    import torch

    import paper_1610_09146_gb300 as fd
    from paper_1610_09146_gb300 import autotune, workloads
    torch.cuda.set_device(0)
    fd.build()
    reqs = workloads.requests(count=args.requests, rate=args.rate)
    # family and tile per (grid, dtype) from the autotuner (cached between runs)
    best = {}
    for r in reqs:
        r["tag"] = r["id"]
        if r["dtype"] == "f64" and not args.plain_f64:
            # binary64 requests run the mixed form (binary64 parity, store-some only)
            r["dtype"], r["algorithm"], r["tile_points"] = "f64dw", "store_some", 0
            continue
        k = (r["n"], r["dtype"])
        if k not in best:
            fam, tile, ms = autotune.tune(r["n"], r["dtype"])
            best[k] = (fam, tile, ms)
        r["algorithm"], r["tile_points"] = best[k][0], best[k][1]
    line = {"workload": f"serving: {len(reqs)} Poisson requests (mean {args.rate}/s, seed 9146), grids 48^3-192^3, "
                        "50-500 RK3 steps, Re U[400,3200], Mach U[0.1,0.4], f32 or f64 per request"
                        + (" (f64 on the plain binary64 kernels)" if args.plain_f64 else
                           " (f64 on the mixed binary64 / double-word store-some kernels)")}
    line |= serve_summary(fd, reqs, args.rate, args.arena_gb, args.max_active)
    line["autotune"] = {f"{n}|{d}": {"family": f, "tile_points": t} for (n, d), (f, t, _) in sorted(best.items())}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------ reference arm


def run_reference(args):
    """The oracle (the plain binary64 CPU solver that checks the CUDA path) on the host
    cores, on the same workload as the CUDA line: one RK3 step of the full grid per step."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    n = args.grid
    dt = 3.385e-3 * 64 / max(n, 64)  # the time-step rule of the CUDA line (Section 3)
    Q = oracle.tgv_ic(n, n, n, GAMMA, MACH)
    times = []
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        Q = oracle.run(Q, 1, dt=dt, Re=RE, Mach=MACH, Pr=PR, gamma=GAMMA)
        t1 = time.perf_counter()
        if it >= args.warmup:
            times.append(t1 - t0)
    pts = n**3
    ms = 1e3 * sum(times) / len(times)
    value = pts / (ms / 1e3)
    sample = f"one RK3 step of the full {n}^3 grid per step ({ms / 1e3:.2f} s each)"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic (analytic Taylor-Green vortex initial condition)",
        "config": {"workload": f"Taylor-Green vortex {n}^3, binary64 results (parity 1e-12 with the binary64 "
                               "oracle), one low-storage RK3 step per step",
                   "grid": [n, n, n], "Re": RE, "Mach": MACH, "Pr": PR, "gamma": GAMMA, "dt": dt},
        "cpu_baseline": {"value": value, "unit": METRIC, "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--grid", type=int, default=N_GRID)
    ap.add_argument("--dtype", choices=["f64", "f32", "df64", "f64dw"], default="f64",
                    help="arithmetic of the line's families (f64 also times the mixed f64dw store-some form); "
                         "f64dw: the mixed form alone (store-some)")
    ap.add_argument("--variants", nargs="+", default=VARIANTS, choices=VARIANTS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-df64", action="store_true", help="skip the df64 and binary32 families beside the line")
    ap.add_argument("--no-f64dw", action="store_true", help="skip the mixed binary64 / double-word store-some form")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched and serving records of the line")
    ap.add_argument("--serve-requests", type=int, default=40, help="requests in the line's serving record")
    ap.add_argument("--plain-f64", action="store_true",
                    help="serve binary64 requests with the plain binary64 kernels instead of the mixed form")
    ap.add_argument("--workload", choices=["single", "batched", "serve", "mixed512", "history", "sweep"],
                    default="single",
                    help="single: the 256^3 line (default); batched / serve / mixed512: the ensemble, "
                         "serving and 512^3 mixed-precision runs; history: KE / enstrophy to --t-end; "
                         "sweep: every family at --sizes")
    ap.add_argument("--instances", type=int, default=64)
    ap.add_argument("--solve-steps", type=int, default=100)
    ap.add_argument("--requests", type=int, default=120)
    ap.add_argument("--rate", type=float, default=20.0)
    ap.add_argument("--arena-gb", type=int, default=64)
    ap.add_argument("--max-active", type=int, default=256)
    ap.add_argument("--t-end", type=float, default=20.0)
    ap.add_argument("--sizes", type=int, nargs="+", default=[128, 256, 384])
    ap.add_argument("--sample-dt", type=float, default=0.1)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "mixed512":
        if args.grid == N_GRID:
            args.grid = 512
        if args.solve_steps == 100:
            args.solve_steps = 200
        run_mixed512(args)
    elif args.workload == "sweep":
        if args.steps == 100:
            args.steps = 10
        run_sweep(args)
    elif args.workload == "history":
        if args.dtype == "f64dw":
            args.variants = ["store_some"]
        if args.variants == VARIANTS:
            args.variants = ["recompute_all" if args.dtype == "f32" else "store_some"]
        run_history(args)
    else:
        if args.dtype == "f64dw":  # the mixed form exists for the store-some family only
            args.variants = ["store_some"]
        run_ours(args)


if __name__ == "__main__":
    main()
