"""Benchmark of the batched projection columns (batched AP solves) on GB300.

One step = one mdp_project_batch over every basis column of every subdomain of the workload
(extension, ring residual, sine transforms, per-mode tridiagonal solves, trace gather: the
whole forward hot path), inputs resident in HBM. Prints ONE JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload dd2x2_257] [--impl ours|reference]

--impl reference times the CPU oracle (SciPy SuperLU, the test oracle) on the host cores on a
bounded sample of the same workload; it is the deliberately slow baseline, not a target.
"""
from __future__ import annotations

import argparse
import json
import math
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


def oracle_throughput(sub, workers, min_seconds=10.0):
    """Columns/s of the oracle over `workers` spawned processes, each factoring `sub` once
    (untimed, like plan creation) and solving basis columns in rounds of one column per
    worker until at least `min_seconds` of wall time have passed."""
    import dataclasses
    ctx = mp.get_context("spawn")
    ncol = 8 * sub.n_modes
    with ctx.Pool(workers, initializer=_oracle_worker_init, initargs=(dataclasses.asdict(sub),)) as pool:
        pool.map(_oracle_worker_cols, [[0]] * workers)  # warm: factor in every worker
        done, c = 0, 0
        t = time.perf_counter()
        while time.perf_counter() - t < min_seconds:
            chunks = [[(c + i) % ncol] for i in range(workers)]
            c += workers
            done += sum(r[0] for r in pool.map(_oracle_worker_cols, chunks))
        wall = time.perf_counter() - t
    return done / wall, done, wall


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
        time.sleep(0.3)
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
    for f in ("kernels.cu", "kernels_common.cuh", "mdp_internal.h"):
        h.update(open(os.path.join(ROOT, "paper_2103_12172_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def recorded_traffic(kernel, workload):
    """DRAM bytes per launch of `kernel` on `workload` from profiles/traffic.json (an ncu
    capture), or None when absent or taken on a different kernel source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path))[workload][kernel]
    except (OSError, ValueError, KeyError):
        return None
    return rec["dram_bytes_per_launch"] if rec.get("source_sha256") == kernel_source_sha() else None


# ------------------------------------------------------------------ reference arm
def run_reference(args, wl):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    sub = wl.subdomains[0]
    workers = max(1, min(16, os.cpu_count() or 1))
    per_step = workers * max(1, int(os.environ.get("MDP_REF_COLS_PER_WORKER", "2")))
    import dataclasses
    ctx = mp.get_context("spawn")
    times, cols = [], 0
    with ctx.Pool(workers, initializer=_oracle_worker_init, initargs=(dataclasses.asdict(sub),)) as pool:
        pool.map(_oracle_worker_cols, [[0]] * workers)
        for s in range(args.warmup + args.steps):
            chunks = [[(s * per_step + i + j * workers) % (8 * sub.n_modes) for j in range(per_step // workers)]
                      for i in range(workers)]
            t = time.perf_counter()
            res = pool.map(_oracle_worker_cols, chunks)
            dt = time.perf_counter() - t
            if s >= args.warmup:
                times.append(dt)
                cols += sum(r[0] for r in res)
    total = sum(times)
    value = cols / total
    sample = (f"{per_step} basis columns per step of subdomain 0 ({sub.nx}x{sub.ny}, k={sub.k}) of {wl.name}; "
              f"SuperLU factorisation per worker outside the timed region")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "description": wl.description, "columns_per_step": per_step},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle", "sample": sample},
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
    dev = torch.device("cuda", local)

    subs = list(wl.subdomains)
    from paper_2103_12172_gb300.autotune import tune_tile
    tile = tune_tile(subs)                     # untimed: columns per work item for this GPU and shape
    plan = mdp.Plan(subs, tile_cols=tile)
    n_cols = sum(8 * s.n_modes for s in subs)
    out = torch.empty(plan.output_size, dtype=torch.complex128, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()

    fp64_probe = mdp.probe_fp64_gflops()
    for _ in range(args.warmup):
        plan.project(out=out)
    torch.cuda.synchronize()
    plan.status()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    plan.profile(True)
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        wall0 = time.perf_counter()
        for i in range(args.steps):
            flush.fill_(float(i))                  # evict L2 between timed steps (not timed)
            starts[i].record(stream)
            plan.project(out=out)
            ends[i].record(stream)
        torch.cuda.synchronize()
        barrier()
        wall = time.perf_counter() - wall0
    plan.profile(False)
    prof = plan.profile_read()
    plan.status()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([total_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    value = world * n_cols * args.steps / (total_ms / 1e3)

    # roofline of the dominant kernel (live CUDA events around its launches, timed region)
    items = []
    for s in range(len(subs)):
        items.append((s, 8 * subs[s].n_modes))
    flops = kernel_flops(plan, items)
    dom = max(prof, key=lambda k: prof[k][0])
    dom_ms, dom_launches = prof[dom]
    launches_per_step = dom_launches / args.steps
    flops_per_launch = flops.get(dom, 0.0) / launches_per_step
    achieved = flops_per_launch / (dom_ms / dom_launches / 1e3) / 1e12
    peak = NOMINAL_FP64_GFLOPS / 1e3
    gpu_launches = sum(n for (_, n) in prof.values())

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
    e2e_steps = max(3, min(args.steps, 10))

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
    copied = [None, None]
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        e2e_step(i)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    plan.status()                                # no step met a singular mode
    plan.update_k(ks)
    update_bytes = int(plan.L.mdp_plan_update_bytes(plan.handle))
    e2e = {"value": world * n_cols * e2e_steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": update_bytes,
           "d2h_bytes_per_step": int(plan.output_size * 16),
           "what": "update_k (new k up, every mode refactored on the GPU) + project + D2H of all columns "
                   "to pinned host memory; pipelined: step i+1's update and refactorisation (second table set) "
                   "and step i's D2H overlap step i's projection"}

    # the same step replayed as one CUDA graph (library graph mode)
    gplan = mdp.Plan(subs, tile_cols=tile, graph=True)
    gs = torch.cuda.Stream()
    with torch.cuda.stream(gs):
        for _ in range(2):
            gplan.project(out=out)
        ge0, ge1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ge0.record(gs)
        for _ in range(args.steps):
            gplan.project(out=out)
        ge1.record(gs)
    gs.synchronize()
    graph_ms = ge0.elapsed_time(ge1) / args.steps
    gplan.close()

    # identical subdomains solved once (MDP_PLAN_DEDUPE), reported separately: the same columns
    # of every subdomain, the distinct problems solved and their blocks copied
    dplan = mdp.Plan(subs, tile_cols=tile, dedupe=True)
    n_distinct = len(set(dplan.leaders()))
    for _ in range(2):
        dplan.project(out=out)
    de0, de1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    de0.record(stream)
    for _ in range(args.steps):
        dplan.project(out=out)
    de1.record(stream)
    torch.cuda.synchronize()
    dedupe_ms = de0.elapsed_time(de1) / args.steps
    dplan.close()

    # adjoint: dLoss/dk for every subdomain through mdp_ap_adjoint (forward recompute + G^H)
    cot = out.clone()
    gk = torch.zeros(len(subs), dtype=torch.float64, device=dev)
    for _ in range(2):
        plan.adjoint(cot, grad_xi=False, grad_k=gk)
    ae0, ae1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ae0.record(stream)
    for _ in range(args.steps):
        plan.adjoint(cot, grad_xi=False, grad_k=gk)
    ae1.record(stream)
    torch.cuda.synchronize()
    adj_ms = ae0.elapsed_time(ae1) / args.steps

    # per-RHS comparator: the same kernels one column per launch sequence, no batching
    per_rhs_cols = min(64, n_cols)
    one = torch.empty(plan.layout(0)[0], dtype=torch.complex128, device=dev)
    for c in range(4):
        plan.project_columns(0, c, 1, out=one)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for c in range(per_rhs_cols):
        plan.project_columns(0, c % (8 * subs[0].n_modes), 1, out=one)
    e1.record(stream)
    torch.cuda.synchronize()
    per_rhs = per_rhs_cols / (e0.elapsed_time(e1) / 1e3)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "description": wl.description, "columns_per_step": n_cols,
                   "tile_cols": tile,
                   "l2": "flushed between timed steps (512 MiB write, untimed)", "parallelism": f"replicas{world}"},
        "roofline": {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": recorded_traffic(dom, wl.name),
                     "peak_note": "FP64 FMA: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (DFMA rate per SM measured)",
                     "fp64_probe_tflops": fp64_probe / 1e3},
        "kernels_ms_per_step": {k: v[0] / args.steps for k, v in sorted(prof.items())},
        "gpu_launches": gpu_launches,
        "per_rhs": {"value": per_rhs, "unit": UNIT, "speedup_batched": value / world / per_rhs},
        "graph": {"ms_per_step": graph_ms, "launches_per_step": 1, "tile_cols": tile},
        "dedupe": {"value": world * n_cols / (dedupe_ms / 1e3), "unit": UNIT, "ms_per_step": dedupe_ms,
                   "distinct_subdomains": n_distinct,
                   "what": "identical subdomains solved once, blocks copied (not the headline value)"},
        "adjoint_grad_k": {"value": n_cols / (adj_ms / 1e3), "unit": UNIT, "ms_per_step": adj_ms},
        "e2e": e2e,
        "wall_s_timed": wall,
    }
    if rank == 0 and not args.no_dd_legs:
        line["dd_pipeline"] = dd_legs()

    # CPU baseline: the oracle as it stands, on the host cores, bounded sample (rank 0 at N=1)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        workers = max(1, min(16, os.cpu_count() or 1))
        sub = subs[0]
        cps, done, wall_c = oracle_throughput(sub, workers)
        line["cpu_baseline"] = {"value": cps, "unit": UNIT, "cores": workers, "kind": "oracle",
                                "sample": f"{done} basis columns of subdomain 0 ({sub.nx}x{sub.ny}, k={sub.k}) over "
                                          f"{workers} spawned processes, SuperLU factor per process untimed, "
                                          f"{wall_c:.2f} s wall"}
    line["clocks"] = clk.summary()
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
    ap.add_argument("--workload", default="dd2x2_257", choices=sorted(W.WORKLOADS))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-dd-legs", action="store_true", help="skip the layered-strip pipeline timings")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    wl = W.WORKLOADS[args.workload]()
    if args.impl == "reference":
        return run_reference(args, wl)
    return run_ours(args, wl)


if __name__ == "__main__":
    sys.exit(main())
