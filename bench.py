"""Benchmark of the batched projection columns (batched AP solves) on GB300.

One step = one mdp_project_batch over every basis column of every subdomain of the workload
(extension, ring residual, sine transforms, per-mode tridiagonal solves, trace gather: the
whole forward hot path), inputs resident in HBM. Prints ONE JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload dd8x8] [--impl ours|reference]

The headline workload is the largest single-GPU one, the 8 x 8 decomposition (64 subdomains,
257^2 / 513^2 / 1025^2 grids, 32768 columns); the other workloads are measured more briefly
and reported in the same line under "configs".

--impl reference times the CPU oracle (SciPy SuperLU, the test oracle) on the host cores on a
bounded sample of the same workload; it is the deliberately slow baseline, not a target.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "batched AP solves/s (FP64 complex), % HBM roofline vs per-RHS path at <=1e-10"
UNIT = "AP solves/s"
NOMINAL_FP64_GFLOPS = 152 * 2 * 2 * 2.070  # SMs x DFMA/clk/SM x flops/DFMA x max GHz = 1258.6
L2_FLUSH_BYTES = 512 << 20
HEADLINE = "dd8x8"
SUB_CONFIGS = ("single_129", "dd2x2_257", "checker2x2", "strip4x1")


def hbm_peak():
    """(GB/s, source) of the HBM roofline: the measured copy bandwidth when the measured-peaks
    file is present, else the recipe's fallback figure."""
    try:
        v = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
        return v, "measured"
    except (OSError, ValueError, KeyError, TypeError):
        return 6800.0, "fallback"


# ------------------------------------------------------------------ oracle timing (CPU)
def _oracle_worker_init(sub_dict):
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    global _ORACLE
    from oracle.projection import APSystem
    _ORACLE = APSystem(W.Subdomain(**sub_dict))


def _oracle_worker_cols(cols):
    t = time.perf_counter()
    _ORACLE.columns(cols=cols)
    return len(cols), time.perf_counter() - t


def grid_classes(wl):
    """{nx: (index of the first subdomain with that grid, number of subdomains)}."""
    cls = {}
    for i, s in enumerate(wl.subdomains):
        first, cnt = cls.get(s.nx, (i, 0))
        cls[s.nx] = (first, cnt + 1)
    return dict(sorted(cls.items()))


def class_workers(cls, workers):
    """Host processes per grid class: about in proportion to the class's share of the oracle's
    work (columns x n^2 log n), at least one each, at most 6 on the largest grids (a SuperLU
    factorisation of a 1025^2 AP holds about 5 GB)."""
    import math
    wt = {nx: cnt * nx * nx * math.log2(nx) for nx, (_, cnt) in cls.items()}
    tot = sum(wt.values())
    alloc = {nx: 1 for nx in cls}
    spare = max(0, workers - len(cls))
    for nx in sorted(cls, key=lambda n: -wt[n]):
        extra = min(spare, int(round(spare * wt[nx] / tot)) if tot else 0)
        alloc[nx] += extra
    big = max(cls)
    cap = {nx: (6 if nx >= 1025 and len(cls) > 1 else workers) for nx in cls}
    if alloc[big] > cap[big]:
        alloc[big] = cap[big]
    # what rounding or the cap left over goes to the heaviest class below its cap
    while sum(alloc.values()) < workers:
        open_ = [n for n in cls if alloc[n] < cap[n]]
        if not open_:
            break
        alloc[max(open_, key=lambda n: wt[n] / alloc[n])] += 1
    return alloc


class OracleClasses:
    """One spawned process pool per grid class of a workload, each worker holding one SuperLU
    factorisation of the class's first subdomain (made in the pool's initializer: untimed, like
    plan creation). `round(cols_per_worker)` solves that many basis columns in every worker of
    every class at once and returns the per-class busy seconds and column counts."""

    def __init__(self, wl, workers):
        import dataclasses
        self.wl = wl
        self.cls = grid_classes(wl)
        self.alloc = class_workers(self.cls, workers)
        ctx = mp.get_context("spawn")
        self.pools = {nx: ctx.Pool(self.alloc[nx], initializer=_oracle_worker_init,
                                   initargs=(dataclasses.asdict(wl.subdomains[first]),))
                      for nx, (first, _) in self.cls.items()}
        self.next = {nx: 0 for nx in self.cls}
        warm = [self.pools[nx].map_async(_oracle_worker_cols, [[0]] * self.alloc[nx]) for nx in self.cls]
        for w in warm:
            w.get()

    @property
    def cores(self):
        return sum(self.alloc.values())

    def round(self, cols_per_worker=1):
        jobs = {}
        for nx, (first, _) in self.cls.items():
            ncol = 8 * self.wl.subdomains[first].n_modes
            chunks = []
            for _ in range(self.alloc[nx]):
                chunks.append([(self.next[nx] + j) % ncol for j in range(cols_per_worker)])
                self.next[nx] += cols_per_worker
            jobs[nx] = self.pools[nx].map_async(_oracle_worker_cols, chunks)
        res = {}
        for nx, j in jobs.items():
            r = j.get()
            res[nx] = (sum(x[1] for x in r), sum(x[0] for x in r))
        return res

    def close(self):
        for p in self.pools.values():
            p.close()
            p.join()


def extrapolated_rate(wl, busy, cores):
    """Columns/s of the whole workload on `cores` host cores from the per-class seconds per
    column (busy[nx] = (seconds, columns) summed over that class's workers): the single-core
    time of every column of the workload, divided over the cores."""
    total = 0.0
    for nx, (_, cnt) in grid_classes(wl).items():
        sec, cols = busy[nx]
        first = grid_classes(wl)[nx][0]
        total += cnt * 8 * wl.subdomains[first].n_modes * sec / cols
    return wl.n_columns * cores / total


def oracle_baseline(wl, workers, min_seconds=10.0):
    """cpu_baseline: the oracle on a bounded sample of the workload (one subdomain per grid
    class, one column per worker per round, rounds until min_seconds of wall time), the rate
    extrapolated to the workload's mix of grids."""
    oc = OracleClasses(wl, workers)
    busy = {nx: (0.0, 0) for nx in oc.cls}
    t = time.perf_counter()
    while time.perf_counter() - t < min_seconds:
        for nx, (s, c) in oc.round(1).items():
            busy[nx] = (busy[nx][0] + s, busy[nx][1] + c)
    wall = time.perf_counter() - t
    oc.close()
    value = extrapolated_rate(wl, busy, oc.cores)
    per = ", ".join(f"{nx}^2: {busy[nx][1]} columns on {oc.alloc[nx]} processes, "
                    f"{1e3 * busy[nx][0] / busy[nx][1]:.1f} ms/column" for nx in oc.cls)
    multi = len(oc.cls) > 1
    sample = (f"{'extrapolated: ' if multi else ''}one subdomain per grid class of {wl.name} ({per}); "
              f"SuperLU factorisation per process untimed; {wall:.1f} s wall"
              + ("; rate = the workload's columns x cores / its single-core time at the measured "
                 "per-class seconds per column" if multi else ""))
    return value, oc.cores, sample


# ------------------------------------------------------------------ clocks
class ClockSampler:
    def __init__(self, index):
        self.index = index
        self.proc = None
        import tempfile
        self.path = os.path.join(tempfile.gettempdir(), f"mdp_bench_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(1.0)   # nvidia-smi's start-up (driver queries) stays out of the timed region
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        load = [r for r in rows if r[2] > 250.0] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in load for i, v in enumerate(r[3]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in load), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(load), "power_w_max": max(r[2] for r in rows)}


# ------------------------------------------------------------------ cost model
def kernel_flops(plan, items):
    """Algorithmic FP64 flops (FMA = 2, mul/add = 1) per kernel for a list of (sub, ncols)
    work items, from each subdomain's geometry (plan.sub_info): the arithmetic of the
    ring-sparse formulation as the kernels perform it -- complex factor rows cost complex
    multiply-adds, rows whose LU factors are real cost real-by-complex ones, and a centred
    subdomain pairs m with Nx - m in the sine transforms."""
    tot = {}

    def add(k, v):
        tot[k] = tot.get(k, 0.0) + v

    for sub, nc in items:
        g = plan.sub_info(sub)
        Px, Py, Nq, Nt, i0, cx, R, Nx = g["Px"], g["Py"], g["Nq"], g["Nt"], g["i0"], g["cplx"], g["R"], g["Nx"]
        xs = g["xsym"]
        # the projection sweeps rows i0 .. nhi+1 (rows above are condensed into the last pivot),
        # pivot-scaled: forward = scaled right-hand side + recurrence, back = x - u1 x' (no 1/d)
        nb = Py + 2
        nf = nb - 1
        if cx:
            f = g["complex_rows"] / float(Nq * nb)
            fwd = f * (6 + 8) + (1 - f) * ((3 if xs else 8) + 4)
            tri = nf * fwd + nb * (8 * f + 4 * (1 - f))
            inv = 4
        else:
            tri = nf * ((3 if xs else 8) + 2) + nb * 2
            inv = 2
        add("k_tri", nc * Nq * tri)
        add("k_inv_cols", nc * (Py - 2) * Nq * (2 if xs else 4) * inv)
        fft_rows = (Nx & (Nx - 1)) == 0 and 8 <= Nx <= 2048
        if fft_rows:
            # DST-I of a dense row by one complex FFT of length Nx: the twist of the input pairs
            # (two complex adds and four FMA per pair, 6 Nx), two multiply-free stages (4 Nx),
            # log2(Nx) - 2 stages of Nx/2 butterflies (complex multiply 6 + two complex adds 4),
            # the even outputs and the odd terms (4 Nx) and the segmented scan over Nx/2 terms
            # (Nx flops per step, log2(min(32, Nx/2)) steps)
            lg = Nx.bit_length() - 1
            dst = 6 * Nx + 4 * Nx + 5 * Nx * (lg - 2) + 4 * Nx + Nx * min(5, lg - 1)
            add("k_inv_rows", nc * 4 * (dst + 2 * (Px + 2)))
        else:
            add("k_inv_rows", nc * 4 * ((Px // 2 + 2) if xs else (Px + 2)) * Nq * inv)
        if fft_rows:
            # one DST-I per row pair of a column (real data packed as re/im)
            add("k_fwd_rows", nc * 2 * dst)
        else:
            add("k_fwd_rows", nc * (Nx // 2) * 4 * ((Px + 1) // 2 if xs else Px) * 2)
        add("k_residual", nc * R * 9 * 2)
    return tot


# ------------------------------------------------------------------ ncu traffic record
def kernel_source_sha():
    import hashlib
    h = hashlib.sha256()
    for f in ("kernels.cu", "kernels_tc.cu", "kernels_common.cuh", "mdp_internal.h"):
        h.update(open(os.path.join(ROOT, "paper_2103_12172_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def recorded_traffic(kernel, workload):
    """DRAM bytes per step of `kernel` on `workload` from profiles/traffic.json (an ncu capture
    of every launch of one step, or a smaller capture scaled by the units processed, as recorded
    there), or None when absent or taken on a different kernel source. Per step, not per launch:
    the plan's workspace budget decides how many waves (launches) a step takes; the record is
    taken with the plan the autotuner picks, whose packing also sets how many table rows come
    from L2."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path))[workload][kernel]
    except (OSError, ValueError, KeyError):
        return None
    return rec["dram_bytes_per_step"] if rec.get("source_sha256") == kernel_source_sha() else None


# ------------------------------------------------------------------ reference arm
def run_reference(args, wl):
    """The oracle on the host cores: every step solves one basis column per process of one
    subdomain per grid class (factorisations untimed); value = the per-class seconds per
    column extrapolated to the workload's mix (a single grid class: plain columns/s)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    workers = max(1, min(16, os.cpu_count() or 1))
    oc = OracleClasses(wl, workers)
    busy = {nx: (0.0, 0) for nx in oc.cls}
    times = []
    for s in range(args.warmup + args.steps):
        t = time.perf_counter()
        r = oc.round(1)
        dt = time.perf_counter() - t
        if s >= args.warmup:
            times.append(dt)
            for nx, (sec, c) in r.items():
                busy[nx] = (busy[nx][0] + sec, busy[nx][1] + c)
    oc.close()
    value = extrapolated_rate(wl, busy, oc.cores)
    cols = sum(c for (_, c) in busy.values())
    multi = len(oc.cls) > 1
    sample = (f"{'extrapolated: ' if multi else ''}one basis column per process per step of one subdomain per "
              f"grid class of {wl.name} (" + ", ".join(f"{nx}^2 on {oc.alloc[nx]} processes" for nx in oc.cls)
              + f"), {cols} columns timed; SuperLU factorisation per process outside the timed region")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "description": wl.description,
                       "columns_per_step": cols // max(1, args.steps)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oc.cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ DD pipeline legs
def dd_legs(reps=5):
    """Timings of the layered strip (4 x 129^2, k = 40, M* = 24, impedance data of a plane wave):
    one coupled solve to the receivers, one loss + k-gradient step, the field of every layer,
    and a solve with a source in every layer. Milliseconds per call (CUDA events, after
    warm-up); the projection columns are recomputed inside every call."""
    import math
    import numpy as np
    import torch
    from paper_2103_12172_gb300.strip import LayeredStrip, incident_impedance_bc, receiver_row
    subs = list(W.strip4x1().subdomains)
    rows = [receiver_row(s) for s in subs]
    strip = LayeredStrip(subs, incident_impedance_bc(0.3), rows)
    k0 = [s.k for s in subs]
    targets = [u.clone() for u in strip.receivers(torch.tensor(W.strip_targets(), dtype=torch.float64))]

    def timed(fn):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    def solve():
        with torch.no_grad():
            strip.receivers(torch.tensor(k0, dtype=torch.float64))

    def grad_step():
        k = torch.tensor(k0, dtype=torch.float64, requires_grad=True)
        loss = sum(torch.sum(torch.abs(u - t) ** 2) for u, t in zip(strip.receivers(k), targets))
        loss.backward()

    def field():
        strip.field(torch.tensor(k0, dtype=torch.float64))

    al, be = 40.0 * math.cos(0.3), 40.0 * math.sin(0.3) * 1.1

    def src(j):
        def fun(x, y):
            f = (40.0 ** 2 - al ** 2 - be ** 2) * np.exp(1j * (al * x + be * y))
            return f, 1j * al * f, 1j * be * f, -al ** 2 * f, -be ** 2 * f
        return fun
    sstrip = LayeredStrip(subs, incident_impedance_bc(0.3), rows, source=src)

    def solve_src():
        sstrip._src_cache = {}   # recompute the source terms every call
        with torch.no_grad():
            sstrip.receivers(torch.tensor(k0, dtype=torch.float64))

    out = {"workload": W.strip4x1().name, "solve_ms": timed(solve), "grad_step_ms": timed(grad_step),
           "field_ms": timed(field), "solve_with_source_ms": timed(solve_src)}
    strip.plan.close()
    sstrip.plan.close()
    return out


# ------------------------------------------------------------------ our arm
def event_time(fn, reps, stream):
    """Mean milliseconds of fn() over reps calls on `stream` (CUDA events, after one warm call)."""
    import torch
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def measure(mdp, wl, steps, warmup, world=1, barrier=None, clocks=None, full=True):
    """Throughput of one workload: `steps` timed mdp_project_batch passes over every column
    (CUDA events on the launching stream, L2 flushed between steps, per-kernel events for the
    roofline), then the side legs: end to end through host buffers, the gradient pass, the
    per-RHS comparator and (full) the graph-replayed and deduplicated variants."""
    import torch

    from paper_2103_12172_gb300.autotune import plan_kwargs, tune_plan

    dev = torch.device("cuda", torch.cuda.current_device())
    subs = list(wl.subdomains)
    n_cols = wl.n_columns
    tuned = tune_plan(subs)                    # untimed: tile and kernel variants for this GPU and shape
    kw = plan_kwargs(tuned)
    tile = kw["tile_cols"]
    plan = mdp.Plan(subs, **kw)
    out = torch.empty(plan.output_size, dtype=torch.complex128, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        plan.project(out=out)
    torch.cuda.synchronize()
    plan.status()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    plan.profile(True)
    if barrier:
        barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for i in range(steps):
        flush.fill_(float(i))                  # evict L2 between timed steps (not timed)
        starts[i].record(stream)
        plan.project(out=out)
        ends[i].record(stream)
    torch.cuda.synchronize()
    if barrier:
        barrier()
    wall = time.perf_counter() - wall0
    plan.profile(False)
    prof = plan.profile_read()
    plan.status()
    total_ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([total_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    value = world * n_cols * steps / (total_ms / 1e3)
    # host cost of issuing one step (profiling off, nothing waited for): the timed loop's wall
    # time minus its device time is this issue time, the L2 fills, and the per-launch event
    # records of the profiling
    t0 = time.perf_counter()
    plan.project(out=out)
    issue_ms = 1e3 * (time.perf_counter() - t0)
    torch.cuda.synchronize()

    # roofline of the dominant kernel (live CUDA events around its launches, timed region)
    flops = kernel_flops(plan, [(s, 8 * subs[s].n_modes) for s in range(len(subs))])
    dom = max(prof, key=lambda k: prof[k][0])
    dom_ms, dom_launches = prof[dom]
    launches_per_step = dom_launches / steps
    flops_per_launch = flops.get(dom, 0.0) / launches_per_step
    launch_s = dom_ms / dom_launches / 1e3
    achieved = flops_per_launch / launch_s / 1e12
    peak = NOMINAL_FP64_GFLOPS / 1e3
    step_traffic = recorded_traffic(dom, wl.name)
    traffic = step_traffic / launches_per_step if step_traffic else None
    hbm, hbm_src = hbm_peak()
    roof = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": traffic,
            "peak_note": "FP64 FMA: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (derived from unit counts and "
                         "clock; the DFMA rate per SM is measured by the probe)",
            "step_flop_frac": sum(flops.values()) / (total_ms / steps / 1e3) / 1e12 / peak,
            "launches_per_step": launches_per_step}
    if traffic:
        roof["dram_gbs"] = traffic / launch_s / 1e9
        roof["dram_frac"] = roof["dram_gbs"] / hbm
        roof["dram_peak_gbs"] = hbm
        roof["dram_peak_note"] = f"{hbm_src} HBM copy bandwidth; DRAM fraction is context, the path is FP64-bound"
    res = {"value": value, "unit": UNIT, "ms_per_step": total_ms / steps, "columns_per_step": n_cols,
           "tile_cols": tile, "tuned": kw, "roofline": roof,
           "kernels_ms_per_step": {k: v[0] / steps for k, v in sorted(prof.items())},
           "gpu_launches": sum(n for (_, n) in prof.values()),
           "wall_s_timed": wall, "host_issue_ms_per_step": issue_ms}

    # end to end through the public API with host buffers: new wavenumbers from host memory
    # (every mode refactored on the GPU), all columns, every step's result read back to pinned
    # host memory. Three streams form a pipeline: step i+1's upload and refactorisation run on
    # a factor stream into the plan's second table set (mdp_plan_update_k_async) while step i
    # projects on the compute stream, and step i's read-back runs on a copy stream (two output
    # buffers, so a projection never overwrites columns still being copied); the timed region
    # ends when the last copy has landed.
    host_out = [torch.empty(plan.output_size, dtype=torch.complex128, pin_memory=True) for _ in range(2)]
    outs = [out, torch.empty_like(out)]
    cs, xs, fs = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    copied = [None, None]
    ks = [s.k for s in subs]
    e2e_steps = max(3, min(steps, 10))

    def e2e_step(i):
        b = i % 2
        plan.update_k_async([k * (1.0 + 1e-9 * (i + 1)) for k in ks], stream=fs)
        if copied[b] is not None:
            cs.wait_event(copied[b])             # the copy of step i-2 has left outs[b]
        plan.project(out=outs[b], stream=cs)     # waits for step i's tables
        done = torch.cuda.Event()
        done.record(cs)
        xs.wait_event(done)
        with torch.cuda.stream(xs):
            host_out[b].copy_(outs[b], non_blocking=True)
        copied[b] = torch.cuda.Event()
        copied[b].record(xs)

    e2e_step(-1)                                 # untimed warm-up of the same step
    torch.cuda.synchronize()
    plan.status()                                # the warm-up's refactorisation met no singular mode
    copied = [None, None]
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        e2e_step(i)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    plan.status()                                # sticky: no timed step met a singular mode either
    plan.update_k(ks)
    update_bytes = int(plan.L.mdp_plan_update_bytes(plan.handle))
    res["e2e"] = {"value": world * n_cols * e2e_steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": update_bytes,
                  "d2h_bytes_per_step": int(plan.output_size * 16),
                  "what": "update_k (new k up, every mode refactored on the GPU) + project + D2H of all columns "
                          "to pinned host memory; pipelined: step i+1's update and refactorisation (second table "
                          "set) and step i's D2H overlap step i's projection"}
    del host_out, outs

    # adjoint: dLoss/dk for every subdomain through mdp_ap_adjoint (forward recompute + G^H)
    cot = out.clone()
    gk = torch.zeros(len(subs), dtype=torch.float64, device=dev)
    adj_ms = event_time(lambda: plan.adjoint(cot, grad_xi=False, grad_k=gk), max(2, min(steps, 5)), stream)
    plan.status()
    res["adjoint_grad_k"] = {"value": n_cols / (adj_ms / 1e3), "unit": UNIT, "ms_per_step": adj_ms}
    del cot

    # per-RHS comparator: the same kernels, one column per launch sequence, no batching; per grid
    # class on its first subdomain, extrapolated to the workload's mix
    per_col_ms = {}
    for nx, (first, cnt) in grid_classes(wl).items():
        one = torch.empty(plan.layout(first)[0], dtype=torch.complex128, device=dev)
        ncol = 8 * subs[first].n_modes
        reps = 16 if nx <= 513 else 8
        c = [0]

        def one_col():
            plan.project_columns(first, c[0] % ncol, 1, out=one)
            c[0] += 37

        per_col_ms[nx] = event_time(one_col, reps, stream)
    t_per_rhs = sum(cnt * 8 * subs[first].n_modes * per_col_ms[nx] for nx, (first, cnt) in grid_classes(wl).items())
    per_rhs = n_cols / (t_per_rhs / 1e3)
    res["per_rhs"] = {"value": per_rhs, "unit": UNIT, "speedup_batched": value / world / per_rhs,
                      "ms_per_column": per_col_ms}

    if full:
        # the same step replayed as one CUDA graph (library graph mode): the difference is what
        # the per-kernel, per-wave launches cost
        gplan = mdp.Plan(subs, graph=True, **kw)
        gs = torch.cuda.Stream()
        with torch.cuda.stream(gs):
            graph_ms = event_time(lambda: gplan.project(out=out), max(3, min(steps, 10)), gs)
        gplan.close()
        res["graph"] = {"ms_per_step": graph_ms, "launches_per_step": 1, "tile_cols": tile,
                        "launch_overhead_frac": max(0.0, 1.0 - graph_ms / res["ms_per_step"])}
        # identical subdomains solved once (MDP_PLAN_DEDUPE), reported separately: the same columns
        # of every subdomain, the distinct problems solved and their blocks copied
        dplan = mdp.Plan(subs, dedupe=True, **kw)
        n_distinct = len(set(dplan.leaders()))
        if n_distinct < len(subs):
            dedupe_ms = event_time(lambda: dplan.project(out=out), max(3, min(steps, 10)), stream)
            res["dedupe"] = {"value": world * n_cols / (dedupe_ms / 1e3), "unit": UNIT, "ms_per_step": dedupe_ms,
                             "distinct_subdomains": n_distinct,
                             "what": "identical subdomains solved once, blocks copied (not the headline value)"}
        dplan.close()
    plan.close()
    del out, flush
    torch.cuda.empty_cache()
    return res


def run_ours(args, wl):
    import torch
    import torch.distributed as dist

    import paper_2103_12172_gb300 as mdp
    from paper_2103_12172_gb300 import _build

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    _build.build()

    def barrier():
        if world > 1:
            dist.barrier()

    fp64_probe = mdp.probe_fp64_gflops()
    dmma_probe = mdp.probe_dmma_gflops()         # the FP64 tensor-core path, for comparison
    with ClockSampler(local) as clk:
        head = measure(mdp, wl, args.steps, args.warmup, world=world, barrier=barrier, full=True)
    line = {
        "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "description": wl.description, "columns_per_step": head["columns_per_step"],
                   "tile_cols": head["tile_cols"], "tuned": head["tuned"],
                   "l2": "flushed between timed steps (512 MiB write, untimed); every wave's workspace also "
                         "exceeds L2", "parallelism": f"replicas{world}"},
        "roofline": dict(head["roofline"], fp64_probe_tflops=fp64_probe / 1e3,
                         fp64_dmma_probe_tflops=dmma_probe / 1e3),
        "kernels_ms_per_step": head["kernels_ms_per_step"],
        "gpu_launches": head["gpu_launches"],
        "per_rhs": head["per_rhs"],
        "graph": head.get("graph"),
        "adjoint_grad_k": head["adjoint_grad_k"],
        "e2e": head["e2e"],
        "wall_s_timed": head["wall_s_timed"],
        "host_issue_ms_per_step": head["host_issue_ms_per_step"],
        "wall_note": "wall_s_timed spans the timed loop on the host: the device time of the timed steps, "
                     "the untimed L2-flush fills between them and, where the host is slower than the GPU, "
                     "the issue of each step (host_issue_ms_per_step, measured with profiling off)",
    }
    if "dedupe" in head:
        line["dedupe"] = head["dedupe"]
    line["clocks"] = clk.summary()

    if not args.no_configs and world == 1:
        cfgs = {}
        for name in SUB_CONFIGS:
            if W.WORKLOADS[name]().name == wl.name:
                continue
            sub_wl = W.WORKLOADS[name]()
            r = measure(mdp, sub_wl, max(5, min(args.steps, 10)), 3, full=False)
            cfgs[name] = {"workload": sub_wl.name, "value": r["value"], "unit": UNIT,
                          "ms_per_step": r["ms_per_step"], "columns_per_step": r["columns_per_step"],
                          "tile_cols": r["tile_cols"], "tuned": r["tuned"], "roofline_kernel": r["roofline"]["kernel"],
                          "roofline_frac": r["roofline"]["frac"],
                          "step_flop_frac": r["roofline"]["step_flop_frac"],
                          "dram_frac": r["roofline"].get("dram_frac"),
                          "kernels_ms_per_step": r["kernels_ms_per_step"],
                          "adjoint_grad_k": r["adjoint_grad_k"]["value"], "e2e": r["e2e"]["value"],
                          "per_rhs_speedup": r["per_rhs"]["speedup_batched"]}
        line["configs"] = cfgs
    if rank == 0 and not args.no_dd_legs:
        line["dd_pipeline"] = dd_legs()

    # CPU baseline: the oracle as it stands, on the host cores, bounded sample (rank 0 at N=1)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        workers = max(1, min(16, os.cpu_count() or 1))
        cps, cores, sample = oracle_baseline(wl, workers)
        line["cpu_baseline"] = {"value": cps, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default=HEADLINE, choices=sorted(W.WORKLOADS))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-dd-legs", action="store_true", help="skip the layered-strip pipeline timings")
    ap.add_argument("--no-configs", action="store_true", help="skip the other workloads' sub-lines")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    wl = W.WORKLOADS[args.workload]()
    if args.impl == "reference":
        return run_reference(args, wl)
    return run_ours(args, wl)


if __name__ == "__main__":
    sys.exit(main())
