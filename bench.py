#!/usr/bin/env python3
"""Benchmark of the tau = 1 lattice Boltzmann step on GB300.

Workload (default): the 2-D shock tube on the square lattice, 4096 x 512
nodes, x-only Sod jump at mid-length, transmissive x ends, reflecting y walls,
run toward t = 0.2 (820 steps), synthetic initial state (Section V.C).

One benchmark step = one tau = 1 step of the whole grid: the fused step
kernel (window records, migration, summation, the new nodes' equilibria,
reach and FP64 partial totals) and a one-block finalize kernel (FP64 totals,
reach hand-off).  The state (67 MB in FP32, plus 100 MB of equilibrium
records) is about the size of the 129 MB L2, so L2 is flushed by a 256 MB
write between timed steps and every step is timed alone with CUDA events on
the solver's stream.

  value      node-updates/s of the FP32 path (device-resident state)
  fp64       the same for the FP64 path (bit-exact with the oracle)
  e2e        node-updates/s of whole solves through the C ABI from pinned
             host buffers: set moments (H2D), 820 steps, moments (D2H)
  roofline   step: algorithmic bytes (4 fields read + 4 written per node) /
             mean step time (both kernels), against the measured HBM copy
             rate
  alu_check  the arrivals' multiply-adds (256 flop per node update) of the
             FP32 and FP64 steps against this GPU's measured FMA peaks
  cpu_baseline  the FP64 oracle on this host's cores, bounded sample

Other workloads (one JSON line each): --workload cylinder2d (8192^2 periodic
cylinder), sod1d (1-D Sod time to solution, plain and CUDA-graph), tubes
(4096 batched 1-D tubes vs plain FP64 one at a time), serve (continuous
batching: capacity and Poisson sweep vs plain FP64 one at a time).

--impl reference times the oracle alone (the CPU reference arm).
Multi-GPU (torchrun): independent replicas, one per rank (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NX, NY = 4096, 512
T_END = 0.2
WORKLOAD = "sod_2d_4096x512_transmissive_x_reflecting_y"
# profiling case: the periodic cylinder box, state larger than L2
WORKLOADS = {
    "sod2d": dict(nx=4096, ny=512, name=WORKLOAD),
    "cylinder2d": dict(nx=8192, ny=8192, name="cylinder_2d_8192x8192_periodic"),
}
METRIC = "node-updates/s"
L2_FLUSH_BYTES = 256 << 20


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


def max_over_ranks(values, world, device):
    """Element-wise maximum of per-rank timings over all ranks (identity on
    one rank).  Works with the NCCL (CUDA tensors) and gloo (CPU) groups."""
    if world <= 1:
        return [float(v) for v in values]
    import torch
    t = torch.tensor(values, dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def job_rate(units_per_rank, world, t_max):
    """Whole-job throughput of independent replicas: all ranks' units over
    the slowest rank's time."""
    return world * units_per_rank / t_max


def measured_traffic(nodes):
    """DRAM bytes per launch of the FP32 2-D step kernel from the committed
    ncu summary, scaled by nodes; None unless the kernel sources are the
    ones that summary was taken from."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "step2d_f32_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        rec = json.load(f)
    h = hashlib.sha256()
    for src in rec["sources"]:
        with open(os.path.join(ROOT, src), "rb") as g:
            h.update(g.read())
    if h.hexdigest() != rec["sha256"]:
        return None
    return rec["dram_bytes_per_node"] * nodes


def steps_and_lambda(t_end, dx):
    n = max(1, int(math.ceil(t_end / dx - 1e-9)))
    return n, t_end / (n * dx)


# --------------------------------------------------------------------------
# clocks sampled during the timed region
# --------------------------------------------------------------------------
class Clocks:
    """nvidia-smi samples (every 20 ms) collected from its output pipe by a
    reader thread while the timed region runs."""

    def __init__(self, gpu_index: int):
        import threading
        self.proc = None
        self.lines = []
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={q}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return

        def read():
            for line in self.proc.stdout:
                self.lines.append(line)

        self.reader = threading.Thread(target=read, daemon=True)
        self.reader.start()

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.reader.join(timeout=5)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        for line in list(self.lines):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------
def run_ours(args, rank, world):
    import torch
    from paper_1602_02675_gb300 import lbm as L

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream()
    wl = WORKLOADS[args.workload]
    nx, ny = wl["nx"], wl["ny"]
    dx = 1.0 / nx
    nsolve, lam = steps_and_lambda(T_END, dx)
    if args.workload == "cylinder2d":
        lam = 1.0
    N = nx * ny
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def make(prec, cons_every=1):
        if args.workload == "cylinder2d":
            cfg = L.make_config(2, nx, ny, dt=lam * dx, precision=prec,
                                bc_x=L.PERIODIC, bc_y=L.PERIODIC,
                                kahan=args.kahan, cons_every=cons_every,
                                stream=stream.cuda_stream)
            s = L.Solver(cfg)
            s.init_riemann((1.0, 0.0, 0.0, 1.0), (0.125, 0.0, 0.0, 0.1),
                           L.CIRCLE, 0.5, 0.5, 0.4)
            return s
        cfg = L.make_config(2, nx, ny, dt=lam * dx, precision=prec,
                            bc_x=L.TRANSMISSIVE, bc_y=L.REFLECTING,
                            kahan=args.kahan, cons_every=cons_every,
                            stream=stream.cuda_stream)
        s = L.Solver(cfg)
        s.init_riemann((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), L.PLANAR_X, 0.5)
        return s

    def timed_steps(s, K, W):
        with torch.cuda.stream(stream):
            s.step(W)
            stream.synchronize()
            ev = [(torch.cuda.Event(enable_timing=True),
                   torch.cuda.Event(enable_timing=True)) for _ in range(K)]
            if world > 1:
                torch.distributed.barrier()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for a, b in ev:
                flush.fill_(1.0)          # evict the state from L2
                a.record(stream)
                s.step(1)
                b.record(stream)
            stream.synchronize()
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
        ms = [a.elapsed_time(b) for a, b in ev]
        s.synchronize()
        return ms, wall

    # FP32 (headline)
    s32 = make(L.F32)
    clocks = Clocks(dev)
    ms32, wall32 = timed_steps(s32, args.steps, args.warmup)
    clk = clocks.stop()
    s32.close()
    # FP64 (oracle-exact path)
    k64 = max(3, args.steps // 4)
    ms64 = [float("nan")]
    if args.precision == "both":
        s64 = make(L.F64)
        ms64, _ = timed_steps(s64, k64, max(3, args.warmup))
        s64.close()

    t32, t64 = max_over_ranks([sum(ms32) / 1e3, sum(ms64) / 1e3], world,
                              "cuda")
    value = job_rate(N * args.steps, world, t32)
    v64 = job_rate(N * k64, world, t64)

    # e2e: whole solves through the C ABI from pinned host memory
    e2e = (run_e2e(args, L, torch, stream, lam, nsolve, world)
           if args.e2e_solves > 0 and args.workload == "sod2d" else None)

    peak, peak_kind = load_peaks()
    mean_ms = t32 / args.steps * 1e3
    bytes_per_launch = 8 * 4 * N            # 4 fields read + 4 written, FP32
    achieved = bytes_per_launch / (mean_ms / 1e3) / 1e9
    roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
            "unit": "GB/s", "frac": round(achieved / peak, 4),
            "traffic": (args.traffic if args.traffic is not None else
                        (measured_traffic(N) if args.kahan == 0 else None)),
            "peak_kind": peak_kind,
            "kernel": ("lbm::fast::step2d_f32" if args.kahan == 0
                       else "step_kernel<float,2,true>"),
            "bytes_per_launch": bytes_per_launch,
            "nominal_peak": 7900.0,
            "frac_of_nominal": round(achieved / 7900.0, 4),
            "duration": ("CUDA events around lbm_step: step kernel + "
                         "one-block finalize kernel" if args.kahan == 0 else
                         "CUDA events around lbm_step: one step kernel")}
    mean64 = t64 / k64 * 1e3
    # Arithmetic roof: the gather's 32 arrivals x 4 fields of multiply-adds
    # (256 flop per node update, a lower bound on the method's arithmetic)
    # against this GPU's measured FMA throughput.
    peak32 = L.lbm_measure_fma_peak(L.F32, stream.cuda_stream)
    peak64 = L.lbm_measure_fma_peak(L.F64, stream.cuda_stream)
    alu = {"flop_per_node_update": 256,
           "basis": "32 packet arrivals x 4 fields, multiply + add each",
           "fp32_fma_peak_tflops": round(peak32 / 1e12, 2),
           "fp64_fma_peak_tflops": round(peak64 / 1e12, 3),
           "fp32_frac": round(value * 256 / peak32, 4),
           "fp64_frac": (round(v64 * 256 / peak64, 4)
                         if args.precision == "both" else None)}
    line = {
        "metric": METRIC, "value": value, "unit": "node-updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(mean_ms, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (Sod initial state, Section V.C)",
        "config": {"workload": wl["name"], "nx": nx, "ny": ny, "nodes": N,
                   "lambda": lam, "steps_to_t0.2": nsolve,
                   "l2": "flushed (256 MB write) before every timed step",
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
        "fp64": {"value": v64, "unit": "node-updates/s", "steps": k64,
                 "ms_per_step": round(mean64, 5),
                 "hbm_frac": round((16 * 4 * N) / (mean64 / 1e3) / 1e9 / peak, 4),
                 # FP64 on this GPU is bound by its FP64 pipe: the arrivals'
                 # 256 flop per node update against the measured FP64 rate
                 "roofline": ({"bound": "alu",
                               "achieved": round(v64 * 256 / 1e12, 4),
                               "peak": round(peak64 / 1e12, 4),
                               "unit": "TFLOP/s",
                               "frac": round(v64 * 256 / peak64, 4),
                               "peak_kind": "measured (lbm_measure_fma_peak)"}
                              if args.precision == "both" else None),
                 "parity": "bit-exact with the FP64 oracle (tests)"},
        "e2e": e2e,
        "roofline": roof,
        "alu_check": alu,
        "clocks": clk,
        "gpu_launches": args.steps * (2 if args.kahan == 0 else 1),
        "wall_s_timed_fp32": round(wall32, 4),
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
    if rank == 0 and not args.no_l1:
        line["l1_vs_oracle"] = l1_vs_oracle(L)
    return line


def run_e2e(args, L, torch, stream, lam, nsolve, world):
    """Whole solves: H2D of the initial moments from pinned host memory,
    nsolve steps, D2H of the final moments and pressure."""
    import numpy as np
    N = NX * NY
    dx = 1.0 / NX
    # the initial state, as a user would hold it on the host (physical units)
    x = (np.arange(NX) + 0.5) * dx
    left = np.tile(x < 0.5, NY)
    pin = lambda: torch.empty(N, dtype=torch.float64, pin_memory=True).numpy()
    rho, mx, my, rhoE = pin(), pin(), pin(), pin()
    rho[:] = np.where(left, 1.0, 0.125)
    mx[:] = 0.0
    my[:] = 0.0
    rhoE[:] = np.where(left, 1.0, 0.1) / 0.4
    outs = {k: pin() for k in ("rho", "mx", "my", "rhoE", "p")}
    cfg = L.make_config(2, NX, NY, dt=lam * dx, precision=L.F32,
                        bc_x=L.TRANSMISSIVE, bc_y=L.REFLECTING,
                        kahan=args.kahan, stream=stream.cuda_stream)
    times = []
    with L.Solver(cfg) as s:
        for rep in range(1 + args.e2e_solves):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s.set_moments(rho, mx, my, rhoE)
            s.step(nsolve)
            s.moments(outs)
            dt = time.perf_counter() - t0
            if rep > 0:
                times.append(dt)
    t = statistics.median(times)
    return {"value": world * N * nsolve / t, "unit": "node-updates/s",
            "h2d_bytes_per_step": 4 * 8 * N, "d2h_bytes_per_step": 5 * 8 * N,
            "step": f"one solve to t=0.2 ({nsolve} lattice steps)",
            "solve_ms_p50": round(1e3 * t, 3),
            "solves": len(times)}


# --------------------------------------------------------------------------
# the oracle on the host: CPU baseline and reference arm
# --------------------------------------------------------------------------
def _oracle_sod_steps(nsteps, ny=NY):
    from oracle import oracle as O
    dx = 1.0 / NX
    _, lam = steps_and_lambda(T_END, dx)
    P = O.Params(dim=2, nx=NX, ny=ny, bc_x=O.TRANSMISSIVE, bc_y=O.REFLECTING)
    s = O.riemann_planar(P, 0.0, 1.0, 0.5, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1),
                         lam)
    t0 = time.perf_counter()
    O.run(P, s, nsteps)
    return time.perf_counter() - t0, NX * ny * nsteps


def cpu_baseline(seconds: float) -> dict:
    # calibrate on one step of a 4096 x 8 strip, then size the sample
    t, nu = _oracle_sod_steps(1, ny=8)
    rate = nu / t
    rows = max(8, min(NY, int(seconds * rate / NX)))
    t, nu = _oracle_sod_steps(1, ny=rows)
    return {"value": nu / t, "unit": "node-updates/s", "cores": 1,
            "kind": "oracle",
            "sample": f"1 step of a 4096 x {rows} strip of the 4096 x 512 Sod "
                      f"lattice (FP64, single thread), {t:.1f} s"}


def l1_vs_oracle(L) -> dict:
    """FP32 and FP64 paths against the FP64 oracle on the benchmark workload:
    a whole 4096 x 512 solve to t = 0.2 (820 steps), mean |error| / field
    range of every row against the oracle's row stored in
    tests/golden/sod2d_row_4096_t0.2.txt (written from oracle/ alone; the
    data vary along x only, so every row is that row)."""
    import numpy as np
    ref = np.loadtxt(os.path.join(ROOT, "tests", "golden",
                                  "sod2d_row_4096_t0.2.txt"))
    o = {"rho": ref[:, 0], "mx": ref[:, 1], "rhoE": ref[:, 2]}
    nsolve, lam = steps_and_lambda(T_END, 1.0 / NX)
    out = {}
    for prec, kahan, name in ((L.F32, 0, "f32"), (L.F32, 1, "f32_kahan"),
                              (L.F64, 1, "f64")):
        cfg = L.make_config(2, NX, NY, dt=lam / NX, precision=prec,
                            bc_x=L.TRANSMISSIVE, bc_y=L.REFLECTING,
                            kahan=kahan)
        with L.Solver(cfg) as s:
            s.init_riemann((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), L.PLANAR_X, 0.5)
            s.step(nsolve)
            g = s.moments()
        out[name] = {f: float(np.mean(np.abs(g[f].reshape(NY, NX) - o[f])) /
                              (o[f].max() - o[f].min()))
                     for f in ("rho", "mx", "rhoE")}
        out[name]["my_max_abs"] = float(np.max(np.abs(g["my"])))
    out["case"] = ("sod_2d_4096x512, 820 steps to t = 0.2, every row; f32: "
                   "register kernel (plain FP32 sums), f32_kahan: compensated "
                   "exact-order kernel")
    return out


def run_tubes(args):
    """Batched 1-D tubes (4096 seeded tubes, 256..16384 nodes, pressure
    ratio 2..100, density ratio 1..10, at rest, t = 0.2): solves/s of the
    batched FP32 path (one persistent launch per step, CUDA graphs) against
    the plain FP64 path that solves one tube at a time through a handle."""
    import torch
    from paper_1602_02675_gb300 import inputs as I
    from paper_1602_02675_gb300 import lbm as L
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    specs = I.tubes_batch(args.tubes)
    tubes, nus = [], 0
    for t in specs:
        ns, lam = t.steps_and_lambda(T_END)
        tubes.append(L.make_tube(t.n, ns, lam / t.n, t.left, t.right))
        nus += t.n * ns
    stream = torch.cuda.Stream()
    times = []
    for rep in range(1 + args.batch_reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with L.Batch(tubes, precision=L.F32, kahan=1,
                     stream=stream.cuda_stream) as b:   # tunes the tile
            b.run()
            b.sync()
            tuning = b.tuning()
        dt = time.perf_counter() - t0
        if rep > 0:
            times.append(dt)
    tb = statistics.median(times)
    # plain FP64 one tube at a time, seeded subsample
    rng = __import__("random").Random(20260)
    sub = rng.sample(range(len(specs)), min(args.seq_tubes, len(specs)))
    t64, nus64, lat = 0.0, 0, []
    for j in sub:
        t = specs[j]
        ns, lam = t.steps_and_lambda(T_END)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cfg = L.make_config(1, t.n, dt=lam / t.n, precision=L.F64,
                            bc_x=L.TRANSMISSIVE, stream=stream.cuda_stream)
        with L.Solver(cfg) as s:
            s.init_riemann(t.left, t.right, L.PLANAR_X, 0.5)
            s.step(ns)
            s.moments()
        d = time.perf_counter() - t0
        t64 += d
        lat.append(d)
        nus64 += t.n * ns
    solves_b = len(specs) / tb
    solves_64 = len(sub) / t64
    lat.sort()
    return {
        "metric": "solves/s", "value": solves_b, "unit": "solves/s",
        "workload": f"tubes_batch_{len(specs)}", "dtype": "f32",
        "batched": {"solves_per_s": solves_b, "node_updates_per_s": nus / tb,
                    "wall_s": tb, "node_updates": nus, "tubes": len(specs),
                    "tile_tuning": tuning,
                    "timed": "creation (tile tuning included) to results"},
        "plain_fp64_one_at_a_time": {
            "solves_per_s": solves_64, "node_updates_per_s": nus64 / t64,
            "sample_tubes": len(sub),
            "latency_ms_p50": 1e3 * lat[len(lat) // 2],
            "latency_ms_p99": 1e3 * lat[min(len(lat) - 1, int(0.99 * len(lat)))]},
        "speedup_solves_per_s": solves_b / solves_64,
    }


def run_serve(args):
    """Serving: a seeded mix (70 % 1-D tubes of 512..65536 nodes, 30 % 2-D
    grids, random Riemann states, t_end in [0.05, 0.25]) through the
    continuous-batching server (FP32) within a device-memory budget.
    Capacity: every request arrives at once.  Then Poisson arrivals at 50,
    90 and 120 % of that capacity (solves/s and latency percentiles).  The
    plain FP64 path serves a seeded subsample one solve at a time."""
    import numpy as np
    import torch
    from paper_1602_02675_gb300 import lbm as L
    from paper_1602_02675_gb300 import serve as S
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    reqs = S.mixed_requests(args.requests, seed=20264,
                            n2=(256, args.max_side))
    budget = int(args.budget_gb * (1 << 30))
    # warm-up: compile caches, allocator
    w = S.Server(budget=budget, precision=L.F32)
    for r in S.mixed_requests(6, seed=7, n1=(512, 2048), n2=(256, 300)):
        w.submit(r)
    w.drain()
    w.close()

    def trace(arrivals):
        srv = S.Server(budget=budget, precision=L.F32)
        try:
            st = S.run_trace(srv, S.mixed_requests(args.requests, seed=20264,
                                                   n2=(256, args.max_side)),
                             arrivals)
            st["peak_admitted_gb"] = srv.peak_used / (1 << 30)
        finally:
            srv.close()
        return st

    cap = trace(np.zeros(len(reqs)))
    capacity = cap["solves_per_s"]
    sweep = []
    for frac in (0.5, 0.9, 1.2):
        rate = frac * capacity
        st = trace(S.poisson_arrivals(len(reqs), rate, seed=20265))
        sweep.append({"rate_frac_of_capacity": frac, "rate": rate, **st})
    rng = __import__("random").Random(20266)
    sub = rng.sample(range(len(reqs)), min(args.seq_tubes, len(reqs)))
    t_seq, lat = 0.0, []
    for j in sub:
        r = reqs[j]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S.solve_alone(r, L.F64)
        d = time.perf_counter() - t0
        t_seq += d
        lat.append(d)
    base = {"solves_per_s": len(sub) / t_seq, "sample": len(sub),
            "service_ms_p50": float(1e3 * np.percentile(lat, 50)),
            "service_ms_p99": float(1e3 * np.percentile(lat, 99))}
    return {"metric": "solves/s", "value": capacity, "unit": "solves/s",
            "workload": f"serve_{len(reqs)}_mixed", "dtype": "f32",
            "capacity": cap, "poisson_sweep": sweep,
            "budget_gb": args.budget_gb, "max_2d_side": args.max_side,
            "plain_fp64_one_at_a_time": base,
            "speedup_solves_per_s": capacity / base["solves_per_s"],
            "accuracy": "each served solve equals the same solve alone "
                        "(tests); FP32 vs FP64 oracle within 1e-5 of range"}


def run_sod1d(args):
    """The 1-D Sod tube (Section V.C): 1000 nodes, FP64, lambda = 1, 200
    steps to t = 0.2.  Time to solution (initial state + 200 steps, device
    time by CUDA events) over `--repeats` solves, once with plain launches
    through the C ABI and once replaying one CUDA graph that holds the whole
    solve; 201 launches per solve make it launch-bound."""
    import numpy as np
    import torch
    from paper_1602_02675_gb300 import lbm as L
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    stream = torch.cuda.Stream()
    n = 1000
    nsteps, lam = steps_and_lambda(T_END, 1.0 / n)
    cfg = L.make_config(1, n, dt=lam / n, precision=L.F64,
                        bc_x=L.TRANSMISSIVE, stream=stream.cuda_stream)
    solver = L.Solver(cfg)

    def solve():
        solver.init_riemann((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), L.PLANAR_X,
                            0.5)
        solver.step(nsteps)

    def timed(run):
        ms = []
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                run()
            stream.synchronize()
            for _ in range(args.repeats):
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                run()
                b.record(stream)
                b.synchronize()
                ms.append(a.elapsed_time(b))
        return {"p50_ms": float(np.percentile(ms, 50)),
                "p99_ms": float(np.percentile(ms, 99)),
                "mean_ms": float(np.mean(ms))}

    plain = timed(solve)
    rho_plain = solver.moments()["rho"].copy()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        solve()
    stream.synchronize()
    graphed = timed(graph.replay)
    rho_graph = solver.moments()["rho"]
    solver.close()
    return {"metric": "time to solution", "value": graphed["p50_ms"],
            "unit": "ms", "higher_is_better": False, "dtype": "f64",
            "data": "synthetic (Sod initial state, Section V.C)",
            "config": {"workload": "sod_1d_1000", "nodes": n,
                       "steps": nsteps, "lambda": lam,
                       "repeats": args.repeats},
            "graph": graphed, "plain": plain,
            "gpu_launches_per_solve": 2 + nsteps,
            "graph_equals_plain": bool(np.array_equal(rho_plain, rho_graph))}


def run_reference(args, rank, world):
    """The CPU oracle as it stands: K bounded samples of the workload."""
    if rank != 0:
        return None
    times, nus = [], []
    rows = args.ref_rows
    for _ in range(args.warmup):
        _oracle_sod_steps(1, ny=rows)
    for _ in range(args.steps):
        t, nu = _oracle_sod_steps(1, ny=rows)
        times.append(t)
        nus.append(nu)
    value = sum(nus) / sum(times)
    return {
        "metric": METRIC, "value": value, "unit": "node-updates/s",
        "impl": "reference", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(1e3 * sum(times) / len(times), 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic (Sod initial state, Section V.C)",
        "config": {"workload": WORKLOAD, "nx": NX, "ny": NY,
                   "sample_rows": rows},
        "cpu_baseline": {"value": value, "unit": "node-updates/s",
                         "cores": 1, "kind": "oracle",
                         "sample": f"each step: 1 lattice step of a 4096 x {rows} "
                                   "strip of the Sod lattice (FP64, 1 thread)"},
        "e2e": {"value": value, "unit": "node-updates/s",
                "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-solves", type=int, default=2)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-rows", type=int, default=16)
    ap.add_argument("--traffic", type=float, default=None,
                    help="ncu dram bytes per step-kernel launch, if measured")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-l1", action="store_true")
    ap.add_argument("--workload", default="sod2d",
                    choices=sorted(WORKLOADS) + ["tubes", "serve", "sod1d"])
    ap.add_argument("--repeats", type=int, default=100,
                    help="sod1d: solves timed")
    ap.add_argument("--requests", type=int, default=300)
    ap.add_argument("--budget-gb", type=float, default=120.0)
    ap.add_argument("--max-side", type=int, default=1024)
    ap.add_argument("--tubes", type=int, default=4096)
    ap.add_argument("--batch-reps", type=int, default=2)
    ap.add_argument("--seq-tubes", type=int, default=48)
    ap.add_argument("--precision", default="both", choices=["both", "f32"])
    ap.add_argument("--kahan", type=int, default=0, choices=[0, 1],
                    help="FP32 kernel: 0 register kernel, 1 compensated "
                         "exact-order kernel")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.workload == "tubes":
        print(json.dumps(run_tubes(args)))
        return
    if args.workload == "serve":
        print(json.dumps(run_serve(args)))
        return
    if args.workload == "sod1d":
        print(json.dumps(run_sod1d(args)))
        return
    if args.impl == "reference":
        line = run_reference(args, rank, world)
        if line is not None:
            print(json.dumps(line))
        return
    if world > 1:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        torch.distributed.init_process_group("nccl")
    line = run_ours(args, rank, world)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
