#!/usr/bin/env python3
"""Throughput of the GB300 micro-continuum DBS-VOF time step (cell-steps/s).

Default workload: the 3-D 128^3 fractured porous block (log-normal
permeability, Gaussian random field with correlation length 8 cells,
sigma_lnk 1, mean k 1e-13 m^2, porosity 0.2-0.6 tied to k, a 6-cell solid-free
fracture, water injected into oil with viscosity ratio 10, gravity on),
pressure residual 1e-8, FP64 (value) and the FP32-preconditioned variant
(``mixed``).  A step is one full pressure-velocity step (saturation update,
properties, momentum predictor, two PISO correctors with GMG-PCG).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank advances its own replica of the workload:
the single-domain step has no data-parallel split, so the GPUs run
independent replicas (weak scaling) and the job throughput is the sum.  The
batched and serving workloads deal their independent domains / requests to
the ranks instead (no collective on the data path).

The default line also carries, on stated reduced configurations: the error of
one step of every precision against the oracle (``error_vs_oracle``), the
V-cycle-wide roofline, a 64-domain batch, a 3 s serving trace (p50/p99), the
512 x 128 x 256 wave tank (mixed + BF16 and FP64) and the 2-D 64^2 case.
``--impl reference`` times the FP64 CPU oracle on bounded samples of the same
workload (one serial oracle process per host core, each on its own 16-layer
slab), on rank 0 only.  ``--workload wave_tank --steps 2000`` runs configuration
3 (the 512 x 128 x 256 tank) at its full length.
"""
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
sys.path.insert(0, ROOT)

METRIC = "cell-steps/s FP64 vs mixed precision at 1e-8 residual; p50/p99 request latency"
UNIT = "cell-steps/s"
DOMINANT = "smooth_fine"  # red-black Gauss-Seidel half sweep on the finest level
SLAB = (56, 72)  # z layers of the bounded CPU sample


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mdbs", choices=["mdbs", "reference"])
    ap.add_argument("--n", type=int, default=128, help="cells per axis of the workload")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--workload", default="grf128", choices=["grf128", "batched", "serving", "buckley_leverett", "wave_tank"])
    ap.add_argument("--columns", type=int, default=512, help="buckley_leverett: columns in the batch")
    ap.add_argument("--rate", type=float, default=20.0, help="serving: arrivals per second")
    ap.add_argument("--duration", type=float, default=10.0, help="serving: arrival window [s]")
    ap.add_argument("--max-side", type=int, default=96, help="serving: largest cube side")
    ap.add_argument("--req-steps", type=int, default=100, help="serving: steps per request")
    ap.add_argument("--domains", type=int, default=512, help="batched workload: number of domains")
    ap.add_argument("--precision", type=int, default=0, help="batched workload: 0 FP64, 1 mixed")
    ap.add_argument("--tank-precision", type=int, default=2,
                    help="wave_tank workload: 0 FP64, 1 mixed, 2 mixed with BF16 coarse coefficients")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default multigrid schedule")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched and serving sub-objects")
    ap.add_argument("--extra-domains", type=int, default=64, help="batched sub-object: domains")
    ap.add_argument("--extra-duration", type=float, default=3.0, help="serving sub-object: arrival window [s]")
    ap.add_argument("--extra-max-side", type=int, default=64, help="serving sub-object: largest cube side")
    ap.add_argument("--extra-req-steps", type=int, default=50, help="serving sub-object: steps per request")
    ap.add_argument("--wave-steps", type=int, default=10, help="wave tank sub-object: timed steps")
    ap.add_argument("--schedule", default=None,
                    help="fixed multigrid schedule instead of autotuning, e.g. rows=1,tail=4096,snake=0,kz=8,ctas=1,coop=0,vec=0")
    return ap.parse_args()


def workload(n):
    from paper_2003_08374_gb300 import workloads as W
    return W.grf_3d(n=n, seed=2, p_tol=1e-8, max_cg=200)


def slab_of(case):
    """Layers SLAB of the workload as a stand-alone case (same recipe, same fields)."""
    from paper_2003_08374_gb300 import workloads as W
    z0, z1 = SLAB
    nx, ny, nz = case.nx, case.ny, case.nz
    z0, z1 = min(z0, nz - 1), min(z1, nz)
    s = case.replace(nz=z1 - z0, name=case.name + "_slab%d_%d" % (z0, z1))
    cut = lambda a: a.reshape(nz, ny, nx)[z0:z1].ravel().copy()
    s.porosity, s.permeability, s.alpha, s.p = (cut(a) for a in (case.porosity, case.permeability,
                                                                 case.alpha, case.p))
    W._zero_fields(s)
    s.ux[:] = case.inlet_u
    return s


def time_oracle(case, steps, warmup):
    from oracle.api import OracleSim
    o = OracleSim(case)
    for _ in range(warmup):
        o.step(1)
    t0 = time.perf_counter()
    for _ in range(steps):
        o.step(1)
    dt = time.perf_counter() - t0
    return case.cells * steps / dt, dt


def _oracle_slab_worker(n, z0, steps, warmup, barrier, out):
    """One process of the all-cores oracle baseline: its own 16-layer slab of the
    workload, `warmup` untimed then `steps` timed oracle steps, the timed ones
    started together with the other processes."""
    global SLAB
    SLAB = (z0, z0 + 16)
    sample = slab_of(workload(n))
    from oracle.api import OracleSim
    o = OracleSim(sample)
    if warmup:
        o.step(warmup)
    barrier.wait()
    t0 = time.perf_counter()
    o.step(steps)
    out.put((sample.cells * steps, time.perf_counter() - t0))
    o.close()


def time_oracle_all_cores(n, steps, warmup=0):
    """The oracle as it stands (serial) on every host core at once: one process per core,
    each stepping its own slab (spawned: no CUDA state is inherited).  Returns the
    aggregate cell-steps/s (all cells over the slowest process's time), the processes
    and that time."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    barrier, out = ctx.Barrier(cores), ctx.Queue()
    span = max(1, n - 16)
    procs = [ctx.Process(target=_oracle_slab_worker, args=(n, (SLAB[0] + 8 * q) % span, steps, warmup, barrier, out))
             for q in range(cores)]
    for pr in procs:
        pr.start()
    res = [out.get() for _ in procs]
    for pr in procs:
        pr.join()
    secs = max(r[1] for r in res)
    return sum(r[0] for r in res) / secs, cores, secs


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x, world, device):
    """The maximum of x over the ranks of the process group (x itself on one rank)."""
    if world == 1:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def shard_by_cells(cells, world):
    """Independent units (domains, requests) of the given cell counts dealt to `world` ranks:
    largest first to the rank with the fewest cells so far (ties: lowest rank), so every
    rank's share is within one unit of the mean.  Returns one index list per rank."""
    load = [0] * world
    out = [[] for _ in range(world)]
    for i in sorted(range(len(cells)), key=lambda i: (-cells[i], i)):
        r = min(range(world), key=lambda q: (load[q], q))
        out[r].append(i)
        load[r] += cells[i]
    return [sorted(o) for o in out]


def gather_lists(values, world):
    """Concatenation of every rank's host list (statistics only; no device data)."""
    if world == 1:
        return list(values)
    import torch.distributed as dist
    parts = [None] * world
    dist.all_gather_object(parts, list(values))
    return [v for part in parts for v in part]


def replicas_value(cells, steps, world, ms):
    """Whole-job cell-steps/s of `world` independent replicas of a `cells`-cell workload
    that all finished `steps` steps within `ms` milliseconds (the slowest rank's time)."""
    return cells * steps * world / (ms / 1e3)


def reference_arm(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return 0
    case = workload(args.n)
    sample = slab_of(case)
    # the oracle as it stands on every host core: one serial process per core, each on
    # its own 16-layer slab of the workload
    value, cores, secs = time_oracle_all_cores(args.n, args.steps, args.warmup)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": case.name + " (FP64 CPU oracle, bounded sample)", "cells": sample.cells * cores,
                   "p_tol": case.p_tol},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "%d oracle processes at once, one per host core, each %d steps of its own "
                                   "16-layer slab (%dx%dx16 cells) of the %s workload"
                                   % (cores, args.steps, sample.nx, sample.ny, case.name)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms.  The sampler is
    running (its first sample in) before the bracketed region starts, and only the
    samples taken inside the region are summarised."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None
        self.t0 = self.t1 = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            wait_until = time.perf_counter() + 3.0
            while not self.rows and time.perf_counter() < wait_until and self.proc.poll() is None:
                time.sleep(0.01)
        except OSError:
            self.proc = None
        self.t0 = time.perf_counter()
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append((time.perf_counter(), parts))

    def __exit__(self, *a):
        self.t1 = time.perf_counter()
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        inside = [r for t, r in self.rows if self.t0 is not None and self.t0 <= t <= (self.t1 or t)]
        if not inside and self.rows:  # a region shorter than one interval: the sample just before it
            before = [r for t, r in self.rows if self.t0 is not None and t < self.t0]
            inside = before[-1:]
        self.rows_inside = inside
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in inside if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in inside if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in inside for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(inside)}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


def kernel_source_hash():
    """Hash of the half-sweep kernel's source (smooth_cell, smooth_cell_corr, k_smooth)."""
    src = open(os.path.join(ROOT, "paper_2003_08374_gb300", "csrc", "pressure.cu")).read()
    a = src.index("// One red-black Gauss-Seidel update of cell c")
    b = src.index("// ------------------------------------------------------------------ fused red-black sweep (FP32)")
    return hashlib.sha256(src[a:b].encode()).hexdigest()[:12]


def measured_traffic(kernel, precision_tag, cells):
    """DRAM bytes per launch from the committed ncu summary, scaled to `cells`, if the kernel
    source is unchanged since the capture; else None."""
    path = os.path.join(ROOT, "profiles", "%s_%s.md" % (kernel, precision_tag))
    try:
        txt = open(path).read()
    except OSError:
        return None
    kv = {}
    for line in txt.splitlines():
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            kv[k.strip()] = v.strip().strip("`")
    if kv.get("source_hash") != kernel_source_hash():
        return None
    try:
        per_cell = float(kv["dram_bytes_per_launch"]) / float(kv["cells"])
    except (KeyError, ValueError):
        return None
    return per_cell * cells


FP64_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12  # SMs x FP64 flop/clk/SM x max SM clock (GB300: 1.26)


def level_sizes(n):
    """Multigrid hierarchy: every axis longer than 4 cells is halved (rounding up)."""
    out = [tuple(n)]
    while True:
        c = tuple((a + 1) // 2 if a > 4 else a for a in out[-1])
        if c == out[-1]:
            return out
        out.append(c)


def fused_sweeps(tuning, word):
    return bool(tuning) and tuning.get("sweep_kz", 0) > 0 and word == 4


def roofline(prof, cells, word, fp64, tuning=None, nu=(2, 2)):
    """Roofline of the finest-level red-black sweeps.  Split schedule: per V-cycle the finest
    level runs 2 (nu1 + nu2) half sweeps; the first post-smoothing one also applies the
    prolongation and is timed with it, so `smooth_fine` holds the others: 1 from a zero guess
    (b, 1/diag, x written on half the cells: 1.5 words per cell) and the rest full (b, 1/diag,
    x written and the other colour's x read on half the cells, the three face-coefficient
    arrays in full: 5 words per cell).  Flops per updated cell: 6 fused multiply-adds and one
    multiply (13), 1 for the zero-guess sweep.  Fused schedule (FP32 levels, sweep_kz > 0):
    each launch is a sweep pair reading b, 1/diag, T x3 and x_in and writing x_out, 7 words
    per cell, 13 flops per cell and colour."""
    if DOMINANT not in prof:
        return None
    tot_ms, cnt = prof[DOMINANT]
    avg_s = tot_ms / cnt / 1e3
    halves = 2 * (nu[0] + nu[1])
    if fused_sweeps(tuning, word):
        alg_bytes = 7 * word * cells
        flops = 13.0 * cells
    else:
        alg_bytes = ((halves - 2) * 5 * word + 1.5 * word) / (halves - 1) * cells
        flops = ((halves - 2) * 13 + 1) / (halves - 1) * cells / 2
    pk = peaks()
    hbm_peak = pk["hbm_gbs"] if pk else 6800.0
    gbs = alg_bytes / avg_s / 1e9
    tfl = flops / avg_s / 1e12
    hbm = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
           "traffic": measured_traffic(DOMINANT, "fp64_grf128" if fp64 else "fp32_grf128", cells),
           "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if pk else "fallback 6800 GB/s"}
    out = dict(hbm)
    if fp64:
        alu = {"bound": "alu", "achieved": tfl, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
               "frac": tfl / FP64_PEAK_TFLOPS, "traffic": hbm["traffic"],
               "peak_source": "FP64 pipe: 152 SMs x 4 flop/clk x 2.07 GHz (nominal 1.25 TFLOP/s)"}
        if alu["frac"] > hbm["frac"]:
            out = dict(alu)
            out["hbm"] = {"achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak}
        else:
            out["alu"] = {"achieved": tfl, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                          "frac": tfl / FP64_PEAK_TFLOPS}
    out.update({"kernel": DOMINANT + ("_fp64" if fp64 else "_fp32"), "launches": cnt, "avg_us": avg_s * 1e6,
                "alg_bytes_per_launch": alg_bytes, "flops_per_launch": flops,
                # traffic is the ncu DRAM figure of one full half sweep: compare it with this
                "alg_bytes_full_sweep": (7 if fused_sweeps(tuning, word) else 5) * word * cells,
                "timing": "CUDA events around every kernel launch in an eager pass of the same K steps"})
    return out


VCYCLE_KERNELS = ("smooth_fine", "smooth_coarse", "restrict_fine", "restrict_coarse", "prolong_fine",
                  "prolong_coarse", "tail_vcycle", "coarse_coop", "zero")


def vcycle_bytes(n, word, tuning, nu=(2, 2), bf16_coarse=False):
    """Algorithmic HBM bytes of one V-cycle, level by level (each array read or written once
    per sweep; neighbours from cache).  Per level of N cells with word w (coefficients wt):
    split half sweeps -- one from a zero guess 1.5w, full ones 2w + 3wt, the first
    post-smoothing one also reads the coarse correction (+ w/8); fused pairs 4w + 3wt plus a
    separate prolongation 2w + w/8; the residual restriction 2w + 3wt + w/8 (x of every
    cell, b and diag of the colour-0 cells whose residual it forms, the face coefficients,
    the coarse b).  The coarsest
    level's exact solve reads its dense inverse (N^2 words)."""
    levels = level_sizes(n)
    out = []
    for l, sz in enumerate(levels):
        N = sz[0] * sz[1] * sz[2]
        w = word
        wt = 2 if (bf16_coarse and l >= 1) else w
        if l == len(levels) - 1:
            out.append((N, (N * N + 2 * N) * w))
            continue
        halves = 2 * (nu[0] + nu[1])
        if fused_sweeps(tuning, word) and N > tuning.get("tail_cells", 0):
            b = (nu[0] + nu[1]) * (4 * w + 3 * wt) + 2 * w + w / 8
        else:
            b = 1.5 * w + (halves - 2) * (2 * w + 3 * wt) + (2 * w + 3 * wt + w / 8)
        b += 2 * w + 3 * wt + w / 8
        out.append((N, b * N))
    return out


def vcycle_fp64_instructions(n, nu=(2, 2)):
    """FP64 instructions of one split-sweep V-cycle, level by level: per updated cell a full
    half sweep issues 7 (6 fused multiply-adds, 1 multiply), the zero-guess one 1, the
    prolonging one 13 (6 more adds of the coarse correction); the masked restriction 9 per
    colour-0 fine cell (diag x, 6 fused multiply-adds, b - Ax, the sum into the coarse
    cell); the coarsest level's dense product N^2."""
    levels = level_sizes(n)
    out = []
    halves = 2 * (nu[0] + nu[1])
    for l, sz in enumerate(levels):
        N = sz[0] * sz[1] * sz[2]
        if l == len(levels) - 1:
            out.append(N * N)
            continue
        out.append(N / 2 * (1 + (halves - 2) * 7 + 13) + N / 2 * 9)
    return out


def vcycle_roofline(prof, n, word, tuning, graph_ms, nu=(2, 2), bf16_coarse=False):
    """HBM roofline of the whole preconditioner: algorithmic bytes of every V-cycle run in
    the eager pass over the summed CUDA-event time of the V-cycle kernels, and the same with
    those kernels' time scaled by graph step time / eager kernel time (the share of the
    captured step they take)."""
    if not prof or "smooth_fine" not in prof:
        return None
    levels = vcycle_bytes(n, word, tuning, nu, bf16_coarse)
    per_cycle = sum(b for _, b in levels)
    halves = 2 * (nu[0] + nu[1])
    per_cycle_launches = (nu[0] + nu[1]) if fused_sweeps(tuning, word) else halves - 1
    cycles = prof["smooth_fine"][1] / per_cycle_launches
    vc_ms = sum(prof[k][0] for k in VCYCLE_KERNELS if k in prof)
    all_ms = sum(v[0] for v in prof.values())
    pk = peaks()
    peak = pk["hbm_gbs"] if pk else 6800.0
    gbs = per_cycle * cycles / (vc_ms / 1e3) / 1e9
    scaled_ms = vc_ms * graph_ms / all_ms
    gbs_g = per_cycle * cycles / (scaled_ms / 1e3) / 1e9
    out = {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
           "graph_scaled": {"achieved": gbs_g, "frac": gbs_g / peak, "vcycle_ms": scaled_ms,
                            "share_of_step": vc_ms / all_ms},
           "alg_bytes_per_vcycle": per_cycle, "vcycles": cycles, "kernel_ms": vc_ms,
            "levels": [{"cells": c, "alg_bytes": b} for c, b in levels],
            "kernels": [k for k in VCYCLE_KERNELS if k in prof],
           "timing": "sum of CUDA-event kernel times in the eager pass; graph_scaled multiplies them by "
                     "graph step time / eager kernel time"}
    if word == 8 and not fused_sweeps(tuning, word):
        # FP64 levels: each level is bound by the larger of its HBM time and its FP64-pipe
        # time (GB300 issues FP64 at 2 lanes per clock per SM)
        instr = vcycle_fp64_instructions(n, nu)
        rate = FP64_PEAK_TFLOPS * 1e12 / 2  # FP64 instructions per second
        roof_s = sum(max(b / (peak * 1e9), i / rate) for (_, b), i in zip(levels, instr)) * cycles
        out["fp64"] = {"instructions_per_vcycle": sum(instr),
                       "pipe_frac": sum(instr) * cycles / rate / (vc_ms / 1e3),
                       "time_at_roof_ms": roof_s * 1e3,
                       "frac_of_roof": roof_s / (vc_ms / 1e3),
                       "graph_scaled_frac_of_roof": roof_s / (scaled_ms / 1e3),
                       "roof": "per level the larger of algorithmic bytes / measured HBM and FP64 "
                               "instructions / (152 SMs x 2 lanes x 2.07 GHz)"}
    return out


def error_vs_oracle(case, precisions):
    """Error of one benchmark step (pressure residual case.p_tol) against the FP64 oracle's
    step solved to 1e-15, on the bounded slab of the workload: relative L2 of alpha, p, u."""
    from oracle.api import OracleSim
    from paper_2003_08374_gb300 import mdbs
    sample = slab_of(case)
    t0 = time.perf_counter()
    o = OracleSim(sample.replace(p_tol=1e-15, max_cg=1000))
    o.step(1)
    fo = o.fields()
    secs = time.perf_counter() - t0
    out = {"sample": "one step of z-layers %d-%d (%dx%dx%d cells) from the workload's initial state; oracle "
                     "solved to 1e-15 (%.1f s)" % (SLAB[0], SLAB[1], sample.nx, sample.ny, sample.nz, secs)}
    uo = np.concatenate([fo["ux"], fo["uy"], fo["uz"]])
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    for name, prec in precisions:
        g = mdbs.Simulation(sample.replace(precision=prec))
        g.step(1)
        fg = g.fields()
        g.close()
        ug = np.concatenate([fg["ux"], fg["uy"], fg["uz"]])
        out[name] = {"alpha": rel(fg["alpha"], fo["alpha"]), "p": rel(fg["p"], fo["p"]), "u": rel(ug, uo),
                     "p_tol": case.p_tol}
    return out


def batched_summary(args, precision, count, steps, warmup, stream, clock_index):
    """A batch of `count` uneven domains (the batched recipe: 3/4 3-D with sides log-uniform in
    [32, 96], 1/4 2-D in [64, 256]) in one launch per phase, autotuned; cell-steps/s."""
    import torch
    from paper_2003_08374_gb300 import mdbs
    from paper_2003_08374_gb300 import workloads as W
    cases = W.batched_domains(count=count, seed=4, p_tol=1e-8, max_cg=200, precision=precision)
    cells = sum(c.cells for c in cases)
    sims = [mdbs.Simulation(c) for c in cases]
    b = mdbs.Batch(sims)
    b.set_stream(stream.cuda_stream)
    tuning, _ = pick_schedule(b, args, trial_steps=1)
    for _ in range(warmup):
        b.step(1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        b.step(1)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    iters = [s.stats()["cg_iters"] for s in sims]
    b.close()
    for s in sims:
        s.close()
    return {"value": cells * steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps, "steps": steps,
            "domains": count, "cells": cells, "precision": ["fp64", "mixed", "mixed_bf16"][precision],
            "cg_iters_max": int(max(max(i) for i in iters)), "tuning": tuning}


def timed_steps(sim, steps, warmup, stream):
    import torch
    for _ in range(warmup):
        sim.step(1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        sim.step(1)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def field_errors(fg, fo):
    rel = lambda a, b: float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
    ug = np.concatenate([fg["ux"], fg["uy"], fg["uz"]])
    uo = np.concatenate([fo["ux"], fo["uy"], fo["uz"]])
    return {"alpha": rel(fg["alpha"], fo["alpha"]), "p": rel(fg["p"], fo["p"]), "u": rel(ug, uo)}


def wave_tank_summary(args, steps, warmup, stream):
    """The wave tank of section 5.1's stand-in (512 x 128 x 256 cells, porous barrier, solitary
    wave, CFL 0.5): mixed precision with BF16 coarse coefficients (its configuration) and
    FP64, autotuned, over a stated number of steps from the initial state; the error of one
    step of a 2-cell-wide span of the same tank (it is uniform along y) against the oracle."""
    from oracle.api import OracleSim
    from paper_2003_08374_gb300 import mdbs
    from paper_2003_08374_gb300 import workloads as W
    out = {"workload": "wave_tank_512x128x256 (16.8 M cells, CFL 0.5, dt_max 2e-3 s)", "p_tol": 1e-8}
    for name, prec in (("mixed_bf16", W.MIXED_BF16), ("fp64", W.FP64)):
        case = W.wave_tank(p_tol=1e-8, max_cg=200, precision=prec)
        sim = mdbs.Simulation(case)
        sim.set_stream(stream.cuda_stream)
        tuning, _ = pick_schedule(sim, args, trial_steps=1)
        sim.set_fields(case.alpha, case.ux, case.uy, case.uz, case.p)
        ms = timed_steps(sim, steps, warmup, stream)
        st = sim.stats()
        out[name] = {"value": case.cells * steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps,
                     "steps": steps, "warmup": warmup, "dt_after": st["dt"], "time_after": st["time"],
                     "cg_iters_last_step": st["cg_iters"], "tuning": tuning}
        sim.close()
    out["mixed_bf16"]["speedup_vs_fp64"] = out["mixed_bf16"]["value"] / out["fp64"]["value"]
    # error of one step against the oracle on the same recipe at a quarter of the length and
    # depth and a 2-cell span (a full-size span already needs about 500 oracle CG iterations
    # at 1e-15: the free surface at a density ratio of 1000 makes the pressure system stiff)
    small = W.wave_tank(nx=128, ny=2, nz=64, depth=20, x0=32, barrier=(80, 96, 24), p_tol=1e-8, max_cg=500)
    t0 = time.perf_counter()
    o = OracleSim(small.replace(p_tol=1e-15, max_cg=2000, precision=W.FP64))
    o.step(1)
    fo = o.fields()
    secs = time.perf_counter() - t0
    out["error_vs_oracle"] = {"sample": "one step of the tank recipe at quarter length and depth with a 2-cell span "
                                        "(128 x 2 x 64), oracle at 1e-15 (%.1f s)" % secs}
    for name, prec in (("mixed_bf16", W.MIXED_BF16), ("fp64", W.FP64)):
        g = mdbs.Simulation(small.replace(precision=prec))
        g.step(1)
        out["error_vs_oracle"][name] = field_errors(g.fields(), fo)
        g.close()
    return out


def wave_tank_arm(args):
    """Configuration 3 at full size and length: the 512 x 128 x 256 wave tank (porous
    barrier, solitary wave, CFL 0.5, walls and an open top), autotuned, --warmup untimed
    and --steps timed steps from the initial state.  Besides throughput it reports the
    run's state: simulated time and dt, CG iterations (last step, mean and the largest per
    corrector), the liquid volume against its initial value (the open top is the only
    boundary it can cross), the saturation bounds, and unconverged solves."""
    import torch
    from paper_2003_08374_gb300 import mdbs
    from paper_2003_08374_gb300 import workloads as W
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    prec = {0: W.FP64, 1: W.MIXED, 2: W.MIXED_BF16}[args.tank_precision]
    case = W.wave_tank(p_tol=1e-8, max_cg=200, precision=prec)
    sim = mdbs.Simulation(case)
    sim.set_stream(stream.cuda_stream)
    tuning, _ = pick_schedule(sim, args, trial_steps=1)
    sim.set_fields(case.alpha, case.ux, case.uy, case.uz, case.p)
    mass0 = sim.stats()["mass"]
    for _ in range(args.warmup):
        sim.step(1)
    torch.cuda.synchronize()
    it0 = sim.stats()["cg_iters_total"]
    iters_max = [0] * case.n_corr
    amin, amax = 1.0, 0.0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    chunk = 50  # statistics every chunk steps; the device time covers only the steps
    ms = 0.0
    done = 0
    with ClockSampler(0) as clk:
        while done < args.steps:
            k = min(chunk, args.steps - done)
            e0.record(stream)
            sim.step(k)
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
            done += k
            st = sim.stats()
            iters_max = [max(a, b) for a, b in zip(iters_max, st["cg_iters"])]
            amin, amax = min(amin, st["alpha_min"]), max(amax, st["alpha_max"])
    st = sim.stats()
    line = {"metric": METRIC, "value": case.cells * args.steps / (ms / 1e3), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {0: "f64", 1: "f64 (FP32 V-cycle)", 2: "f64 (FP32 V-cycle, BF16 coarse coefficients)"}[
                args.tank_precision], "data": "synthetic",
            "config": {"workload": "wave_tank_512x128x256 (16.8 M cells, CFL 0.5, dt_max 2e-3 s)", "cells": case.cells,
                       "p_tol": case.p_tol, "tuning": tuning,
                       "timing": "device time of the steps, in chunks of %d with statistics read between" % chunk},
            "run": {"time_s": st["time"], "dt_last": st["dt"], "cg_iters_last_step": st["cg_iters"],
                    "cg_iters_max": iters_max,
                    "cg_iters_mean_per_corrector": (st["cg_iters_total"] - it0) / (args.steps * case.n_corr),
                    "unconverged_solves": st["not_converged"],
                    "liquid_volume_rel_change": (st["mass"] - mass0) / mass0,
                    "alpha_min": amin, "alpha_max": amax},
            "clocks": clk.summary()}
    sim.close()
    print(json.dumps(line), flush=True)
    return 0


def fracture_2d_summary(args, stream):
    """The 2-D 64 x 64 fracture case (dx 10 um, dt 1e-6 s, FP64, 100 steps): a launch-bound
    step, autotuned like the other workloads; its error after the 100 steps against the
    oracle at 1e-15, the case at 1e-8."""
    from oracle.api import OracleSim
    from paper_2003_08374_gb300 import mdbs
    from paper_2003_08374_gb300 import workloads as W
    out = {"workload": "fracture_2d_64x64 (FP64, 100 steps)"}
    ref = OracleSim(W.fracture_2d(nx=64, ny=64, p_tol=1e-15, max_cg=500))
    ref.step(100)
    fo = ref.fields()
    for p_tol in (1e-8, 1e-15):
        case = W.fracture_2d(nx=64, ny=64, p_tol=p_tol, max_cg=500)
        sim = mdbs.Simulation(case)
        sim.set_stream(stream.cuda_stream)
        tuning = sim.tuning() if args.no_autotune else sim.autotune(trial_steps=2)[0]
        ms = timed_steps(sim, 100, 0, stream)
        st = sim.stats()
        key = "p_tol_%.0e" % p_tol
        out[key] = {"value": case.cells * 100 / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / 100,
                    "launches_per_step": st["kernel_launches"] / 100.0, "cg_iters_last_step": st["cg_iters"],
                    "tuning": tuning}
        out[key]["error_vs_oracle_1e-15"] = field_errors(sim.fields(), fo)
        sim.close()
    return out


def serving_summary(precision, rate, duration, max_side, req_steps, stream):
    """Continuous batching of a seeded Poisson trace of fractured-porous requests: served
    cell-steps/s and p50/p99 request latency."""
    from paper_2003_08374_gb300 import workloads as W
    from paper_2003_08374_gb300.serve import Request, Server, fractured_request_case
    trace = W.poisson_requests(rate=rate, duration=duration, seed=5, lo=32, hi=max_side)
    reqs = [Request(rid=i, arrival=t["t"], steps=req_steps,
                    case=fractured_request_case(t["side"], t["ca"], t["seed"], precision=precision, p_tol=1e-8,
                                                max_cg=200))
            for i, t in enumerate(trace)]
    offered = sum(r.case.cells * r.steps for r in reqs) / duration
    srv = Server(max_active=256, round_steps=10, keep_fields=False, stream_handle=stream.cuda_stream)
    summ = srv.run(reqs)
    summ.update({"precision": ["fp64", "mixed", "mixed_bf16"][precision], "offered_cell_steps_per_s": offered,
                 "trace": "Poisson %.0f req/s for %.0f s, cube sides log-uniform in [32, %d], capillary number "
                          "log-uniform in [1e-5, 1e-2], %d steps each" % (rate, duration, max_side, req_steps)})
    return summ


def pick_schedule(obj, args, trial_steps):
    """The multigrid schedule of a simulation or batch: given (--schedule), default
    (--no-autotune) or autotuned.  Returns (schedule, per-trial ms per step)."""
    if args.schedule:
        kv = dict(item.split("=") for item in args.schedule.split(","))
        obj.set_tuning({"smooth_rows": int(kv.get("rows", 1)), "tail_cells": int(kv.get("tail", 4096)),
                        "snake": int(kv.get("snake", 0)), "sweep_kz": int(kv.get("kz", 0)),
                        "tail_ctas": int(kv.get("ctas", 1)), "coarse_coop": int(kv.get("coop", 0)),
                        "vec_sweeps": int(kv.get("vec", 0))})
        return obj.tuning(), []
    if args.no_autotune:
        return obj.tuning(), []
    return obj.autotune(trial_steps=trial_steps)


def gpu_arm(args):
    import torch
    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2003_08374_gb300.build import build_library
    build_library()
    from paper_2003_08374_gb300 import mdbs
    from paper_2003_08374_gb300 import workloads as W

    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def rank_max(x):
        return max_over_ranks(x, world, "cuda")

    def timed(sim, steps, warmup, profile_kernel=None):
        for _ in range(warmup):
            sim.step(1)
        if profile_kernel:
            sim.profile(True, only=None if profile_kernel == "*" else profile_kernel)
        l0 = sim.stats()["kernel_launches"]
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clk:
            e0.record(stream)
            for _ in range(steps):
                sim.step(1)
            e1.record(stream)
            torch.cuda.synchronize()
        barrier()
        ms = e0.elapsed_time(e1)
        prof = sim.profile_read() if profile_kernel else {}
        if profile_kernel:
            sim.profile(False)
        st = sim.stats()
        return ms, prof, clk.summary(), st["kernel_launches"] - l0, st

    case = workload(args.n)
    if args.precision == 1:  # the mixed variant alone (profiling runs)
        case = case.replace(precision=W.MIXED)
        args.no_mixed = True
    sim = mdbs.Simulation(case)
    sim.set_stream(stream.cuda_stream)
    # schedule of the multigrid kernels picked by timing real steps (state restored after)
    tuning, tune_ms = pick_schedule(sim, args, trial_steps=2)
    # headline: every step is one CUDA-graph launch (CG loops as device-side WHILE nodes)
    ms, _, clocks, launches, st = timed(sim, args.steps, args.warmup)
    ms = rank_max(ms)
    value = replicas_value(case.cells, args.steps, world, ms)
    cg_iters = st["cg_iters"]
    # the same number of steps again with CUDA events around each launch of the dominant
    # kernel (event timing needs individually launched kernels, so this pass runs eagerly)
    sim.set_fields(case.alpha, case.ux, case.uy, case.uz, case.p)
    _, prof, _, _, _ = timed(sim, args.steps, args.warmup, "*")
    breakdown = {k: round(v[0] / args.steps, 4) for k, v in sorted(prof.items(), key=lambda kv: -kv[1][0])}

    nu = (case.mg_nu1, case.mg_nu2)
    word = 8 if args.precision == 0 else 4
    roof = roofline(prof, case.cells, word, fp64=args.precision == 0, tuning=tuning, nu=nu)
    roof_vc = vcycle_roofline(prof, (case.nx, case.ny, case.nz), word, tuning, ms, nu=nu,
                              bf16_coarse=args.precision == 2)

    def variant(precision):
        """The same workload with the FP32 V-cycle (precision 1) or FP32 with BF16 coarse-level
        coefficients (precision 2) inside FP64 flexible CG."""
        vcase = case.replace(precision=precision)
        vsim = mdbs.Simulation(vcase)
        vsim.set_stream(stream.cuda_stream)
        vtuning = pick_schedule(vsim, args, trial_steps=2)[0]
        it0 = vsim.stats()["cg_iters_total"]
        for _ in range(args.warmup):
            vsim.step(1)
        it1 = vsim.stats()["cg_iters_total"]
        vms, _, _, _, vst = timed(vsim, args.steps, 0)
        vms = rank_max(vms)
        vval = replicas_value(case.cells, args.steps, world, vms)
        out = {"value": vval, "ms_per_step": vms / args.steps, "speedup_vs_fp64": vval / value,
               "tuning": vtuning, "cg_iters_last_step": vst["cg_iters"],
               "cg_iters_timed": vst["cg_iters_total"] - it1, "cg_iters_warmup": it1 - it0}
        vsim.set_fields(case.alpha, case.ux, case.uy, case.uz, case.p)
        _, vprof, _, _, _ = timed(vsim, args.steps, args.warmup, "*")
        out["roofline"] = roofline(vprof, case.cells, 4, fp64=False, tuning=vtuning, nu=nu)
        out["roofline_vcycle"] = vcycle_roofline(vprof, (case.nx, case.ny, case.nz), 4, vtuning, vms, nu=nu,
                                                 bf16_coarse=precision == 2)
        out["kernel_ms_per_step"] = {k: round(v[0] / args.steps, 4)
                                     for k, v in sorted(vprof.items(), key=lambda kv: -kv[1][0])}
        vsim.close()
        return out

    mixed = bf16 = None
    if not args.no_mixed:
        mixed = variant(W.MIXED)
        bf16 = variant(W.MIXED_BF16)
        # BF16 coarse coefficients are kept only while the CG iteration count grows < 10 %
        growth = bf16["cg_iters_timed"] / max(mixed["cg_iters_timed"], 1) - 1.0
        bf16["cg_iters_growth_vs_mixed"] = growth
        bf16["kept"] = growth < 0.10
        mixed["bf16_coarse"] = bf16

    # end to end through the public API with host buffers: each step copies the state in
    # from pinned host memory (mdbs_set_fields), steps, and reads it back (mdbs_get_fields)
    pin = lambda n: torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()
    host = {k: pin(v.size) for k, v in sim.fields().items() if v.size}
    for k, v in sim.fields().items():
        if v.size:
            host[k][:] = v
    nbytes = sum(v.nbytes for v in host.values())
    lib = mdbs.lib()
    P = mdbs._ptr
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        sim._check(lib.mdbs_set_fields(sim.h, P(host["alpha"]), P(host["ux"]), P(host["uy"]), P(host["uz"]),
                                       P(host["p"])))
        sim.step(1)
        sim._check(lib.mdbs_get_fields(sim.h, P(host["alpha"]), P(host["ux"]), P(host["uy"]), P(host["uz"]),
                                       P(host["p"])))
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ems = rank_max(e0.elapsed_time(e1))
    e2e = {"value": replicas_value(case.cells, args.steps, world, ems), "unit": UNIT,
           "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes}
    sim.close()

    cpu = None
    errors = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sample = slab_of(case)
        cval, csec = time_oracle(sample, 2, 0)
        cpu = {"value": cval, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "2 oracle steps on z-layers %d-%d (%dx%dx%d cells) of the workload, %.1f s"
                         % (SLAB[0], SLAB[1], sample.nx, sample.ny, sample.nz, csec)}
        aval, acores, asec = time_oracle_all_cores(args.n, 2)
        cpu["all_cores"] = {"value": aval, "unit": UNIT, "cores": acores, "kind": "oracle",
                            "sample": "%d oracle processes at once, one per host core, each 2 steps of its own "
                                      "16-layer slab of the workload (%.1f s); the oracle is serial, so one "
                                      "domain's step uses one core" % (acores, asec)}
        # the error of each timed configuration against the FP64 oracle
        errors = error_vs_oracle(case, [("fp64", W.FP64)] + ([] if args.no_mixed else
                                                             [("mixed", W.MIXED), ("mixed_bf16", W.MIXED_BF16)]))
    # reduced batched and serving configurations (stated in each object), FP64 and mixed
    batched = serving = wave = frac2d = None
    if not args.no_extras and world == 1:
        wave = wave_tank_summary(args, args.wave_steps, args.warmup, stream)
        frac2d = fracture_2d_summary(args, stream)
        batched = {name: batched_summary(args, prec, args.extra_domains, args.steps, args.warmup, stream, local)
                   for name, prec in (("fp64", W.FP64), ("mixed", W.MIXED))}
        serving = {name: serving_summary(prec, args.rate, args.extra_duration, args.extra_max_side,
                                         args.extra_req_steps, stream)
                   for name, prec in (("fp64", W.FP64), ("mixed", W.MIXED))}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": case.name + ("" if args.precision == 0 else " (mixed)"), "cells": case.cells, "p_tol": case.p_tol, "n_corr": case.n_corr,
                       "mom_sweeps": case.mom_sweeps, "parallelism": "replicas" if world > 1 else "single",
                       "l2": "inputs larger than L2 (%.1f GB device state)" % (mdbs.bytes_required(case) / 1e9),
                       "cg_iters_last_step": cg_iters, "tuning": tuning,
                       "autotune_ms_per_trial": [round(t, 3) for t in tune_ms]},
            "mixed": mixed, "roofline": roof, "roofline_vcycle": roof_vc, "error_vs_oracle": errors,
            "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
            "gpu_launches": launches,
            "kernel_ms_per_step": breakdown,
            "batched": batched, "serving": serving, "wave_tank": wave, "fracture_2d": frac2d,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def init_ranks(torch):
    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return rank, world, local


def batched_arm(args):
    """Many uneven independent domains advanced as one batch (one launch per step phase,
    one CUDA graph per step): sides log-uniform in [32, 96] (3-D) or [64, 256] (2-D).
    Under torchrun the seeded set of `domains` x N domains is dealt to the N ranks by cell
    count (every rank about `domains` domains: weak scaling); each rank advances its own
    batch, nothing crosses ranks but the timing and the statistics."""
    import torch
    rank, world, local = init_ranks(torch)
    from paper_2003_08374_gb300.build import build_library
    build_library()
    from paper_2003_08374_gb300 import mdbs
    from paper_2003_08374_gb300 import workloads as W
    all_cases = W.batched_domains(count=args.domains * world, seed=4, p_tol=1e-8, max_cg=200,
                                  precision=args.precision)
    mine = shard_by_cells([c.cells for c in all_cases], world)[rank]
    cases = [all_cases[i] for i in mine]
    cells_all = sum(c.cells for c in all_cases)
    stream = torch.cuda.current_stream()
    sims = [mdbs.Simulation(c) for c in cases]
    b = mdbs.Batch(sims)
    b.set_stream(stream.cuda_stream)
    tuning, tune_ms = pick_schedule(b, args, trial_steps=1)
    for _ in range(args.warmup):
        b.step(1)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            b.step(1)
        e1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ms = max_over_ranks(e0.elapsed_time(e1), world, "cuda")
    iters = gather_lists([max(s.stats()["cg_iters"]) for s in sims], world)
    if rank == 0:
        line = {"metric": METRIC, "value": cells_all * args.steps / (ms / 1e3), "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic",
                "config": {"workload": "batched_%d_domains" % len(all_cases), "cells": cells_all,
                           "precision": "fp64" if args.precision == 0 else "mixed",
                           "parallelism": "domains dealt to %d ranks by cell count" % world if world > 1 else "single",
                           "cg_iters_max": int(max(iters)), "cg_iters_mean": float(np.mean(iters)),
                           "tuning": tuning, "autotune_ms_per_trial": [round(t, 2) for t in tune_ms]},
                "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    b.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def bl_columns(count, nx=2000):
    """Darcy-scale columns of sections 4.1.1-4.1.2 (4 m, 2000 cells), cycling through water
    into oil / air, Brooks-Corey / Van Genuchten and gravity off / on."""
    from paper_2003_08374_gb300 import workloads as W
    kinds = [(d, m, g) for g in (False, True) for m in (W.BROOKS_COREY, W.VAN_GENUCHTEN) for d in ("oil", "air")]
    return [W.buckley_leverett(nx=nx, displaced=kinds[i % 8][0], kr_model=kinds[i % 8][1], gravity=kinds[i % 8][2])
            for i in range(count)]


def bl_arm(args):
    """The 1-D Buckley-Leverett column: one column alone (latency of a step: a 2000-cell
    step is bound by launch and dependency latency, not by memory) and a batch of
    columns advanced together (the whole-job number)."""
    import torch
    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    from paper_2003_08374_gb300.build import build_library
    build_library()
    from paper_2003_08374_gb300 import mdbs
    stream = torch.cuda.current_stream()

    def run(obj, steps, warmup):
        for _ in range(warmup):
            obj.step(1)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            obj.step(1)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    def single(precision):
        """One column alone, autotuned: graph steps, then an eager pass with events per kernel."""
        c = bl_columns(1)[0].replace(precision=precision)
        one = mdbs.Simulation(c)
        one.set_stream(stream.cuda_stream)
        tun = pick_schedule(one, args, trial_steps=2)[0]
        l0 = one.stats()["kernel_launches"]
        ms1 = run(one, args.steps, args.warmup)
        st1 = one.stats()
        out = {"precision": "fp64" if precision == 0 else "mixed", "ms_per_step": ms1 / args.steps,
               "cell_steps_per_s": c.cells * args.steps / (ms1 / 1e3),
               "gpu_launches_per_step": (st1["kernel_launches"] - l0) / (args.steps + args.warmup),
               "cg_iters_last_step": st1["cg_iters"], "tuning": tun}
        one.profile(True, only=None)
        run(one, args.steps, 0)
        prof = one.profile_read()
        one.profile(False)
        one.close()
        out["kernel_ms_per_step"] = {k: round(v[0] / args.steps, 4)
                                     for k, v in sorted(prof.items(), key=lambda kv: -kv[1][0])}
        return out, prof

    case = bl_columns(1)[0]
    single64, prof = single(0)
    single32, _ = single(1)
    top, (top_ms, top_n) = max(prof.items(), key=lambda kv: kv[1][0])

    cases = bl_columns(args.columns)
    cells = sum(c.cells for c in cases)
    sims = [mdbs.Simulation(c) for c in cases]
    b = mdbs.Batch(sims)
    b.set_stream(stream.cuda_stream)
    tuning, tune_ms = pick_schedule(b, args, trial_steps=1)
    with ClockSampler(local) as clk:
        ms = run(b, args.steps, args.warmup)
    iters = [s.stats()["cg_iters"] for s in sims]
    b.close()

    cpu = None
    if not args.no_cpu_baseline:
        cval, csec = time_oracle(case, 200, 0)
        cpu = {"value": cval, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "200 oracle steps of one 2000-cell column (water into oil, Brooks-Corey), %.1f s" % csec}
    pk = peaks()
    hbm_peak = pk["hbm_gbs"] if pk else 6800.0
    line = {"metric": METRIC, "value": cells * args.steps / (ms / 1e3), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "buckley_leverett_%d_columns_2000_cells" % len(cases), "cells": cells,
                       "cg_iters_max": max(max(i) for i in iters), "tuning": tuning,
                       "l2": "inputs smaller than L2 (a latency-bound workload)"},
            "single_column": single64, "single_column_mixed": single32,
            "roofline": {"bound": "hbm", "kernel": top, "avg_us": top_ms / top_n * 1e3,
                         "achieved": None, "peak": hbm_peak, "unit": "GB/s", "frac": None, "traffic": None,
                         "note": "a 2000-cell step moves about 1 MB: latency-bound, no memory roofline applies"},
            "cpu_baseline": cpu, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    return 0


def serving_arm(args):
    """Continuous batching of a seeded Poisson trace of fractured-porous requests (sides
    log-uniform in [32, max_side], capillary number log-uniform in [1e-5, 1e-2]).  Under
    torchrun the trace arrives at N times the rate and its requests are dealt to the N
    ranks round robin in arrival order (weak scaling); each rank serves its own; the
    latencies are gathered on the host for p50/p99 over all requests."""
    import torch
    rank, world, local = init_ranks(torch)
    from paper_2003_08374_gb300.build import build_library
    build_library()
    from paper_2003_08374_gb300 import workloads as W
    from paper_2003_08374_gb300.serve import Request, Server, fractured_request_case
    trace = W.poisson_requests(rate=args.rate * world, duration=args.duration, seed=5, lo=32, hi=args.max_side)
    reqs = [Request(rid=i, arrival=t["t"], steps=args.req_steps,
                    case=fractured_request_case(t["side"], t["ca"], t["seed"], precision=args.precision,
                                                p_tol=1e-8, max_cg=200))
            for i, t in enumerate(trace) if i % world == rank]
    offered = sum(c["side"] ** 3 for c in trace) * args.req_steps / args.duration
    srv = Server(max_active=256, round_steps=10, keep_fields=False,
                 stream_handle=torch.cuda.current_stream().cuda_stream)
    if world > 1:
        torch.distributed.barrier()
    with ClockSampler(local) as clk:
        summary = srv.run(reqs)
    lat = gather_lists([r.finished - r.arrival for r in reqs if r.finished is not None], world)
    served = gather_lists([srv.cell_steps], world)
    wall = max_over_ranks(summary["wall_s"], world, "cuda")
    if world > 1:
        summary.update({"completed": len(lat), "requests": len(trace), "wall_s": wall,
                        "p50_latency_s": float(np.percentile(lat, 50)) if lat else None,
                        "p99_latency_s": float(np.percentile(lat, 99)) if lat else None,
                        "served_cell_steps_per_s": sum(served) / wall})
    if rank == 0:
        line = {"metric": METRIC, "value": summary["served_cell_steps_per_s"], "unit": UNIT, "n_gpus": world,
                "steps": args.req_steps, "warmup": 0, "ms_per_step": None, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": "serving_poisson_%.0fps_%.0fs_side32-%d_%dsteps" % (
                    args.rate * world, args.duration, args.max_side, args.req_steps),
                    "precision": "fp64" if args.precision == 0 else "mixed",
                    "parallelism": "requests dealt to %d ranks round robin" % world if world > 1 else "single",
                    "offered_cell_steps_per_s": offered},
                "serving": summary, "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.workload == "serving" and args.impl != "reference":
        return serving_arm(args)
    if args.impl == "reference":
        return reference_arm(args)
    if args.workload == "batched":
        return batched_arm(args)
    if args.workload == "buckley_leverett":
        return bl_arm(args)
    if args.workload == "wave_tank":
        return wave_tank_arm(args)
    return gpu_arm(args)


if __name__ == "__main__":
    sys.exit(main())
