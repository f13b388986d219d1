#!/usr/bin/env python3
"""Benchmark of the tau = 1 lattice Boltzmann step on GB300.

Workload (default): the large 2-D cylindrical Riemann problem on the square
lattice, 8192 x 8192 nodes on [0, 1]^2, inside a circle of radius 0.4 about
(0.5, 0.5) (rho, p) = (1, 1), outside (0.125, 0.1), at rest, gamma = 1.4,
periodic box, lambda = 1, 2000 steps (Section V.C's Riemann problem on a 2-D
grid); synthetic initial state.

One benchmark step = one tau = 1 step of the whole grid: the fused FP32
step kernel (window equilibria, deposit, shifted gather, the new nodes'
reach and compensated partial totals) and a one-block finalize kernel
(FP64 totals, reach hand-off).  The timed region is the whole solve from
its initial state (K steps, 2000 by default), timed in blocks of up to 100
steps with CUDA events on the solver's stream; the state (1.07 GB per set
in FP32) is far larger than the 129 MB L2, so no flush is needed.

  value      node-updates/s of the FP32 path over the timed solve
  windows    ms per step of the first, middle and last block of the solve
             (the lattice-scale structure of the flow grows with time)
  fp64       the FP64 path (bit-exact with the oracle) over the first steps
  e2e        node-updates/s of whole solves through the C ABI from pinned
             host buffers: set moments (H2D), K steps, moments (D2H)
  roofline   step: algorithmic bytes (4 fields read + 4 written per node) /
             mean step time (both kernels), against the measured HBM copy
             rate
  alu_check  the arrivals' multiply-adds (256 flop per node update) of the
             FP32 and FP64 steps against this GPU's measured FMA peaks
  precision  FP32 against FP64 on the full grid after the first steps, and
             at the end of the timed solve
  sod2d      the 2-D shock tube (4096 x 512, transmissive x, reflecting y),
             L2 flushed before every timed step, with FP32 / FP64 errors
             against the oracle's stored row
  bgk2d      the relaxation-time step (tau = 1.5) on the 2048^2 cylinder
  cpu_baseline  the FP64 oracle on this host's cores, bounded sample

Other workloads (one JSON line each): --workload sod2d (the shock tube as
the main line), sod1d (1-D Sod time to solution, plain and CUDA-graph),
tubes (4096 batched 1-D tubes vs plain FP64 one at a time), serve
(continuous batching: capacity and Poisson sweep vs plain FP64 one at a
time), patch2d, batch2d, bgk2d (the relaxation-time step, tau != 1, on its
per-packet state).

--impl reference times the oracle alone (the CPU reference arm).
Multi-GPU (torchrun): independent replicas, one per rank (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import platform
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NX, NY = 4096, 512
T_END = 0.2
WORKLOAD = "sod_2d_4096x512_transmissive_x_reflecting_y"
CYL_N, CYL_STEPS = 8192, 2000
CYL_NAME = "cylinder_2d_8192x8192_periodic"
WORKLOADS = {
    "sod2d": dict(nx=4096, ny=512, name=WORKLOAD),
    "cylinder2d": dict(nx=CYL_N, ny=CYL_N, name=CYL_NAME),
}
METRIC = "node-updates/s"
L2_FLUSH_BYTES = 256 << 20
CYL_IN = (1.0, 0.0, 0.0, 1.0)
CYL_OUT = (0.125, 0.0, 0.0, 0.1)


def host_info() -> dict:
    """Host cores and CPU model of the machine running the oracle."""
    model = platform.processor() or platform.machine()
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True,
                             timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model,
            "arch": platform.machine()}


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


def measured_traffic(nodes, name="step2d_ds_traffic.json"):
    """DRAM bytes per launch of the FP32 2-D step kernel from the committed
    ncu summary, scaled by nodes; None unless the kernel sources are the
    ones that summary was taken from."""
    import hashlib
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    with open(path) as f:
        rec = json.load(f)
    h = hashlib.sha256()
    for src in rec["sources"]:
        p = os.path.join(ROOT, src)
        if not os.path.exists(p):
            return None
        with open(p, "rb") as g:
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
def fp32_kernel_name(kahan):
    return "lbm::ds::step2d_ds_fused<%s>" % ("false" if kahan == 0 else "true")


# launches of ours per 2-D FP32 step: the persistent deposit kernel and the
# finalize kernel
DS_LAUNCHES_PER_STEP = 2


def run_cylinder(args, rank, world):
    """The 8192^2 periodic cylinder: the whole FP32 solve from its initial
    state, the FP64 path over its first steps, FP32 against FP64, e2e."""
    import numpy as np
    import torch
    from paper_1602_02675_gb300 import lbm as L

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream()
    n = CYL_N
    N = n * n
    K = args.steps if args.steps > 0 else CYL_STEPS

    def make(prec, kahan=args.kahan):
        cfg = L.make_config(2, n, n, dt=1.0 / n, precision=prec,
                            bc_x=L.PERIODIC, bc_y=L.PERIODIC, kahan=kahan,
                            cons_every=1, stream=stream.cuda_stream)
        return L.Solver(cfg)

    def init(s):
        s.init_riemann(CYL_IN, CYL_OUT, L.CIRCLE, 0.5, 0.5, 0.4)

    def timed_solve(s, k, w, block=100):
        """w untimed steps, back to the initial state, then k steps timed
        in blocks with CUDA events on the solver's stream."""
        with torch.cuda.stream(stream):
            init(s)
            s.step(w)
            init(s)
            stream.synchronize()
            nb = [min(block, k - i) for i in range(0, k, block)]
            ev = [(torch.cuda.Event(enable_timing=True),
                   torch.cuda.Event(enable_timing=True)) for _ in nb]
            if world > 1:
                torch.distributed.barrier()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for (a, b), m in zip(ev, nb):
                a.record(stream)
                s.step(m)
                b.record(stream)
            stream.synchronize()
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
        ms = [a.elapsed_time(b) for a, b in ev]
        return ms, nb, wall

    s32 = make(L.F32)
    clocks = Clocks(dev)
    ms32, nb32, wall32 = timed_solve(s32, K, args.warmup)
    clk = clocks.stop()
    s32.synchronize()
    diag32 = s32.diagnostics()
    reach32 = s32.reach()
    end32 = s32.moments()
    s32.close()
    per_step = [m / k for m, k in zip(ms32, nb32)]
    windows = {"first": {"steps": f"1-{nb32[0]}", "ms_per_step": round(per_step[0], 5)},
               "middle": {"steps": f"{sum(nb32[:len(nb32) // 2]) + 1}-"
                                   f"{sum(nb32[:len(nb32) // 2 + 1])}",
                          "ms_per_step": round(per_step[len(nb32) // 2], 5)},
               "last": {"steps": f"{K - nb32[-1] + 1}-{K}",
                        "ms_per_step": round(per_step[-1], 5)}}

    # FP64 (oracle-exact path) over the first steps
    k64 = max(3, args.fp64_steps)
    ms64 = [float("nan")]
    if args.precision == "both":
        s64 = make(L.F64, kahan=1)
        ms64, _, _ = timed_solve(s64, k64, 3, block=k64)
        s64.close()

    t32, t64 = max_over_ranks([sum(ms32) / 1e3, sum(ms64) / 1e3], world,
                              "cuda")
    value = job_rate(N * K, world, t32)
    v64 = job_rate(N * k64, world, t64)
    mean_ms = t32 / K * 1e3
    mean64 = t64 / k64 * 1e3

    peak, peak_kind = load_peaks()
    bytes_per_launch = 8 * 4 * N            # 4 fields read + 4 written, FP32
    achieved = bytes_per_launch / (mean_ms / 1e3) / 1e9
    roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
            "unit": "GB/s", "frac": round(achieved / peak, 4),
            "traffic": (args.traffic if args.traffic is not None else
                        (measured_traffic(N) if args.kahan == 0 else None)),
            "peak_kind": peak_kind,
            "kernel": fp32_kernel_name(args.kahan),
            "bytes_per_launch": bytes_per_launch,
            "nominal_peak": 7900.0,
            "frac_of_nominal": round(achieved / 7900.0, 4),
            "duration": "CUDA events around lbm_step over the whole timed "
                        "solve: the deposit kernel and the finalize kernel"}
    peak32 = L.lbm_measure_fma_peak(L.F32, stream.cuda_stream)
    peak64 = L.lbm_measure_fma_peak(L.F64, stream.cuda_stream)
    alu = {"flop_per_node_update": 256,
           "basis": "32 packet arrivals x 4 fields, multiply + add each",
           "fp32_fma_peak_tflops": round(peak32 / 1e12, 2),
           "fp64_fma_peak_tflops": round(peak64 / 1e12, 3),
           "fp32_frac": round(value * 256 / peak32, 4),
           "fp64_frac": (round(v64 * 256 / peak64, 4)
                         if args.precision == "both" else None)}

    e2e = (run_e2e_cylinder(args, L, torch, stream, K, world)
           if args.e2e_solves > 0 else None)
    precision = (cylinder_precision(args, L, stream, end32, K)
                 if rank == 0 and args.precision == "both" and not args.no_l1
                 else None)
    line = {
        "metric": METRIC, "value": value, "unit": "node-updates/s",
        "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": round(mean_ms, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (cylindrical Riemann problem, Section V.C states)",
        "config": {"workload": CYL_NAME, "nx": n, "ny": n, "nodes": N,
                   "lambda": 1.0, "steps_of_solve": CYL_STEPS,
                   "timed": f"steps 1-{K} of the solve from its initial state",
                   "l2": "state (1.07 GB per set) larger than the 129 MB L2; "
                         "no flush",
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
        "windows": windows,
        "ms_per_step_blocks": [round(x, 5) for x in per_step],
        "fp32_end_state": {"reach": reach32, "diagnostics": diag32},
        "fp64": {"value": v64, "unit": "node-updates/s", "steps": k64,
                 "timed": f"steps 1-{k64} of the solve",
                 "ms_per_step": round(mean64, 5),
                 "hbm_frac": round((16 * 4 * N) / (mean64 / 1e3) / 1e9 / peak, 4),
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
        "gpu_launches": DS_LAUNCHES_PER_STEP * K,
        "wall_s_timed_fp32": round(wall32, 4),
        "precision": precision,
    }
    if rank == 0 and not args.no_sod:
        line["sod2d"] = run_sod2d(args, L, torch, stream, world, rank,
                                  secondary=True)
    if rank == 0 and not args.no_bgk:
        b = run_bgk2d(args)
        line["bgk2d"] = {k: b[k] for k in ("value", "unit", "ms_per_step",
                                           "steps", "warmup", "roofline",
                                           "gpu_launches",
                                           "conservation_drift", "clocks")}
        line["bgk2d"]["workload"] = b["config"]["workload"]
        line["bgk2d"]["tau"] = b["config"]["tau"]
        line["bgk2d"]["parity"] = ("FP64 bit-exact with the FP64 oracle, FP32 "
                                   "within 1e-5 of each field's range (tests)")
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds,
                                            cpu_procs(args.cpu_procs))
    return line


def cylinder_precision(args, L, stream, end32, K):
    """FP32 against FP64 on the full 8192^2 grid: mean |FP32 - FP64| / range
    of the FP64 field after the first steps (FP64 is bit-exact with the
    oracle in the tests), and the FP32 state at the end of the timed solve
    against the FP64 state after the same number of steps when that is
    short enough to run here."""
    import numpy as np
    n = CYL_N
    steps = min(args.precision_steps, K)

    def run(prec, kahan, k):
        cfg = L.make_config(2, n, n, dt=1.0 / n, precision=prec,
                            bc_x=L.PERIODIC, bc_y=L.PERIODIC, kahan=kahan,
                            stream=stream.cuda_stream)
        with L.Solver(cfg) as s:
            s.init_riemann(CYL_IN, CYL_OUT, L.CIRCLE, 0.5, 0.5, 0.4)
            s.step(k)
            return s.moments()

    ref = run(L.F64, 1, steps)
    out = {"steps": steps, "metric": "mean |x - x_FP64| / (max - min of x_FP64)"}
    for name, kahan in (("f32", 0), ("f32_kahan", 1)):
        g = run(L.F32, kahan, steps)
        out[name] = {f: float(np.mean(np.abs(g[f] - ref[f])) /
                              max(float(ref[f].max() - ref[f].min()), 1e-300))
                     for f in ("rho", "mx", "my", "rhoE")}
    if K == steps:
        out["end_of_timed_solve_is_this_state"] = True
    out["note"] = ("the square-lattice step amplifies round-off (design "
                   "notes): the oracle itself, rounding its state to FP32 "
                   "each step, departs from FP64 by the amounts in "
                   "tests/golden/cylinder_fp32_storage_floor.txt")
    return out


def run_e2e_cylinder(args, L, torch, stream, K, world):
    """Whole solves: H2D of the initial moments from pinned host memory, K
    steps, D2H of the final moments and pressure."""
    import numpy as np
    n = CYL_N
    N = n * n
    x = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(x, x)
    inside = ((X - 0.5) ** 2 + (Y - 0.5) ** 2 < 0.16).ravel()
    pin = lambda: torch.empty(N, dtype=torch.float64, pin_memory=True).numpy()
    rho, mx, my, rhoE = pin(), pin(), pin(), pin()
    rho[:] = np.where(inside, 1.0, 0.125)
    mx[:] = 0.0
    my[:] = 0.0
    rhoE[:] = np.where(inside, 1.0, 0.1) / 0.4
    outs = {k: pin() for k in ("rho", "mx", "my", "rhoE", "p")}
    cfg = L.make_config(2, n, n, dt=1.0 / n, precision=L.F32,
                        bc_x=L.PERIODIC, bc_y=L.PERIODIC, kahan=args.kahan,
                        stream=stream.cuda_stream)
    times = []
    with L.Solver(cfg) as s:
        for rep in range(1 + args.e2e_solves):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s.set_moments(rho, mx, my, rhoE)
            s.step(K if rep > 0 else 2)
            s.moments(outs)
            dt = time.perf_counter() - t0
            if rep > 0:
                times.append(dt)
    t = statistics.median(times)
    return {"value": world * N * K / t, "unit": "node-updates/s",
            "h2d_bytes_per_step": 4 * 8 * N, "d2h_bytes_per_step": 5 * 8 * N,
            "step": f"one solve ({K} lattice steps) with its host transfers",
            "solve_ms_p50": round(1e3 * t, 3), "solves": len(times)}


def run_sod2d(args, L, torch, stream, world, rank, secondary=False):
    """The 2-D shock tube, 4096 x 512: each timed step alone after a 256 MB
    L2 flush, FP32 (and FP64), errors against the oracle's stored row."""
    dx = 1.0 / NX
    nsolve, lam = steps_and_lambda(T_END, dx)
    N = NX * NY
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    K = args.sod_steps if secondary else args.steps

    def make(prec, kahan):
        cfg = L.make_config(2, NX, NY, dt=lam * dx, precision=prec,
                            bc_x=L.TRANSMISSIVE, bc_y=L.REFLECTING,
                            kahan=kahan, cons_every=1,
                            stream=stream.cuda_stream)
        s = L.Solver(cfg)
        s.init_riemann((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), L.PLANAR_X, 0.5)
        return s

    def timed_steps(s, k, w):
        with torch.cuda.stream(stream):
            s.step(w)
            stream.synchronize()
            ev = [(torch.cuda.Event(enable_timing=True),
                   torch.cuda.Event(enable_timing=True)) for _ in range(k)]
            if world > 1 and not secondary:
                torch.distributed.barrier()
            torch.cuda.synchronize()
            for a, b in ev:
                flush.fill_(1.0)          # evict the state from L2
                a.record(stream)
                s.step(1)
                b.record(stream)
            stream.synchronize()
            torch.cuda.synchronize()
        ms = [a.elapsed_time(b) for a, b in ev]
        s.synchronize()
        return ms

    s32 = make(L.F32, args.kahan)
    clocks = None if secondary else Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    ms32 = timed_steps(s32, K, args.warmup)
    clk = clocks.stop() if clocks else None
    s32.close()
    k64 = max(3, K // 4)
    s64 = make(L.F64, 1)
    ms64 = timed_steps(s64, k64, 3)
    s64.close()
    t32, t64 = (sum(ms32) / 1e3, sum(ms64) / 1e3)
    if not secondary:
        t32, t64 = max_over_ranks([t32, t64], world, "cuda")
    value = job_rate(N * K, world if not secondary else 1, t32)
    mean_ms = t32 / K * 1e3
    peak, peak_kind = load_peaks()
    achieved = 32 * N / (mean_ms / 1e3) / 1e9
    out = {"workload": WORKLOAD, "value": value, "unit": "node-updates/s",
           "steps": K, "ms_per_step": round(mean_ms, 5),
           "timed": f"steps {args.warmup + 1}-{args.warmup + K} of the "
                    f"{nsolve}-step solve, each alone after an L2 flush",
           "roofline": {"bound": "hbm", "achieved": round(achieved, 1),
                        "peak": peak, "unit": "GB/s",
                        "frac": round(achieved / peak, 4),
                        "peak_kind": peak_kind,
                        "kernel": fp32_kernel_name(args.kahan)},
           "fp64": {"ms_per_step": round(t64 / k64 * 1e3, 5),
                    "value": N * k64 / t64}}
    if clk is not None:
        out["clocks"] = clk
    if rank == 0 and not args.no_l1:
        out["l1_vs_oracle"] = l1_vs_oracle(L)
    return out


def run_batch2d(args):
    """--workload batch2d: many small 2-D grids (sides log-uniform 64..512,
    planar Riemann jumps with the served requests' states: left (1, 0, 1),
    pressure ratio log-uniform 2..100, density ratio 1..10, end time
    0.05..0.25; transmissive x, reflecting y; FP32) solved to their end
    times, once as one lbm_batch2d (two launches per lattice step for the
    whole batch) and once grid by grid through lbm_step on one stream (the
    one-solve-at-a-time path).  Both timed with CUDA events, creation and
    initial states excluded."""
    import torch
    from paper_1602_02675_gb300 import lbm as L
    from paper_1602_02675_gb300 import serve as S
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    stream = torch.cuda.Stream()
    count = args.grids
    reqs = S.mixed_requests(count, seed=20271, n2=(64, 512),
                            frac_1d=0.0)
    specs = []
    for r in reqs:
        steps, lam = r.steps_and_lambda()
        cfg = L.make_config(2, r.n, r.ny, dt=lam / r.n, precision=L.F32,
                            bc_x=L.TRANSMISSIVE, bc_y=L.REFLECTING,
                            kahan=args.kahan, stream=stream.cuda_stream)
        specs.append((cfg, r, steps))
    nu = sum(r.n * r.ny * k for _, r, k in specs)
    grids = [L.make_grid2d(c, r.left, r.right, L.PLANAR_X, r.x_d, 0.5, 0.0, k)
             for c, r, k in specs]

    def timed(fn):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            stream.synchronize()
            a.record(stream)
            fn()
            b.record(stream)
            stream.synchronize()
        return a.elapsed_time(b) / 1e3

    with L.Batch2D(grids, stream=stream.cuda_stream) as b:
        t_batch = timed(b.run)
        steps_batch = b.steps()
    solvers = []
    for c, r, k in specs:
        s = L.Solver(c)
        s.init_riemann(r.left, r.right, L.PLANAR_X, r.x_d)
        solvers.append((s, k))
    t_alone = timed(lambda: [s.step(k) for s, k in solvers])
    for s, _ in solvers:
        s.close()
    return {"metric": METRIC, "value": nu / t_batch, "unit": "node-updates/s",
            "n_gpus": 1, "higher_is_better": True, "dtype": "f32",
            "data": "synthetic (served 2-D requests' states, sides 64..512)",
            "config": {"workload": f"batch2d_{count}_grids_64_512",
                       "grids": count, "node_updates": nu,
                       "batch_steps": steps_batch},
            "solves_per_s": count / t_batch, "s_batch": round(t_batch, 4),
            "one_at_a_time": {"value": nu / t_alone, "s": round(t_alone, 4),
                              "solves_per_s": count / t_alone},
            "speedup": round(t_alone / t_batch, 3),
            "gpu_launches": DS_LAUNCHES_PER_STEP * steps_batch}


PATCH_N = 4096
PATCH_N = 4096


def run_patch2d(args):
    """--workload patch2d: a 4096 x 4096 periodic patchwork state (squares
    of 7 nodes, each with its own velocity, |V| < 0.9, and p/rho in
    0.3 .. 2.2; inputs.patch_prims): every window holds several level
    speeds and lattice shifts of both signs, so every tile after the first
    step takes the mixed-window kernel (the reach stays within 6 over the
    first steps).  FP32, K steps after W warm-up steps, timed as one block
    with CUDA events (state 268 MB per set, larger than L2)."""
    import torch
    from paper_1602_02675_gb300 import inputs as I
    from paper_1602_02675_gb300 import lbm as L
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    stream = torch.cuda.Stream()
    n = PATCH_N
    K = args.steps if args.steps > 0 else 20
    cfg = L.make_config(2, n, n, dt=1.0 / n, precision=L.F32,
                        bc_x=L.PERIODIC, bc_y=L.PERIODIC, kahan=args.kahan,
                        cons_every=1, stream=stream.cuda_stream)
    prims = I.patch_prims(n, n, seed=7, u_max=0.9, p_over_rho=(0.3, 2.2))
    with L.Solver(cfg) as s, torch.cuda.stream(stream):
        s.set_primitives(*prims)
        s.step(args.warmup)
        stream.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
        a.record(stream)
        s.step(K)
        b.record(stream)
        stream.synchronize()
        clk = clocks.stop()
        ms = a.elapsed_time(b)
        s.synchronize()
        diag, reach = s.diagnostics(), s.reach()
    mean_ms = ms / K
    peak, peak_kind = load_peaks()
    achieved = 32 * n * n / (mean_ms / 1e3) / 1e9
    return {"metric": METRIC, "value": n * n * K / (ms / 1e3),
            "unit": "node-updates/s", "n_gpus": 1, "steps": K,
            "warmup": args.warmup, "ms_per_step": round(mean_ms, 5),
            "higher_is_better": True, "dtype": "f32",
            "data": "synthetic (patchwork of uniform squares, |V| < 0.9, "
                    "p/rho 0.3 .. 2.2)",
            "config": {"workload": "patchwork_2d_4096x4096_periodic",
                       "nx": n, "ny": n, "timed": f"steps {args.warmup + 1}-"
                       f"{args.warmup + K}", "l2": "state larger than L2"},
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1),
                         "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4),
                         "peak_kind": peak_kind},
            "gpu_launches": DS_LAUNCHES_PER_STEP * K,
            "end_state": {"reach": reach, "diagnostics": diag},
            "clocks": clk}


BGK_N = 2048


def run_bgk2d(args):
    """--workload bgk2d: the relaxation-time step (tau != 1, eqs 4-5) on
    its per-packet state: the periodic cylinder of Section V.C on a 2048 x
    2048 grid (circle r < 0.4 about the centre, inner (1, 0, 0, 1), outer
    (0.125, 0, 0, 0.1)), tau = --tau, FP32.  K steps after W warm-up steps,
    timed as one block with CUDA events around lbm_bgk_step (max_reach 4:
    one launch per step); the state, 537 MB per packet set, is larger than
    L2.  Algorithmic bytes: 8 slots x 4 fields x 4 bytes read and written,
    256 B per node update."""
    import torch
    from paper_1602_02675_gb300 import lbm as L
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    stream = torch.cuda.Stream()
    n = BGK_N
    K = args.steps if args.steps > 0 else 100
    # max_reach 4: the one-launch step (window collided in shared memory);
    # --bgk-max-reach 6 takes the collision and gather kernels
    cfg = L.make_config(2, n, n, dt=1.0 / n, precision=L.F32,
                        bc_x=L.PERIODIC, bc_y=L.PERIODIC,
                        max_reach=args.bgk_max_reach,
                        stream=stream.cuda_stream)
    one = args.bgk_max_reach <= 4
    with L.Bgk(cfg, args.tau) as g, torch.cuda.stream(stream):
        g.init_riemann((1.0, 0.0, 0.0, 1.0), (0.125, 0.0, 0.0, 0.1),
                       L.CIRCLE, 0.5, 0.5, 0.4)
        t0 = g.conservation()
        g.step(args.warmup)
        stream.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
        a.record(stream)
        g.step(K)
        b.record(stream)
        stream.synchronize()
        clk = clocks.stop()
        ms = a.elapsed_time(b)
        g.synchronize()
        diag = g.diagnostics()
        t1 = g.conservation()
    mean_ms = ms / K
    peak, peak_kind = load_peaks()
    achieved = 256 * n * n / (mean_ms / 1e3) / 1e9
    drift = [float(abs(x - y) / max(abs(t0[0]), abs(t0[3])))
             for x, y in zip(t1, t0)]
    return {"metric": METRIC, "value": n * n * K / (ms / 1e3),
            "unit": "node-updates/s", "n_gpus": 1, "steps": K,
            "warmup": args.warmup, "ms_per_step": round(mean_ms, 5),
            "higher_is_better": True, "dtype": "f32",
            "data": "synthetic (cylindrical Riemann problem, Section V.C "
                    "states)",
            "config": {"workload": f"bgk_cylinder_2d_{n}x{n}_periodic",
                       "tau": args.tau, "nx": n, "ny": n,
                       "max_reach": args.bgk_max_reach,
                       "timed": f"steps {args.warmup + 1}-{args.warmup + K}",
                       "l2": "state (537 MB per packet set) larger than L2; "
                             "no flush"},
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1),
                         "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4),
                         "peak_kind": peak_kind,
                         "bytes_per_node_update": 256,
                         "kernel": ("lbm::bgk::step2d<float>" if one else
                                    "lbm::bgk::collide<float,2> + "
                                    "gather<float,2>"),
                         "duration": "CUDA events around lbm_bgk_step"},
            "gpu_launches": (1 if one else 2) * K,
            "conservation_drift": drift,
            "end_state": diag, "clocks": clk}


# --------------------------------------------------------------------------
# the oracle on the host: CPU baseline and reference arm
# --------------------------------------------------------------------------
def _oracle_cylinder_rows(rows, nsteps=1):
    """nsteps oracle steps of a periodic strip of the cylinder's initial
    state: all 8192 columns, `rows` rows through the circle's centre (the
    same arithmetic per node as the full grid; the strip closes on itself
    along y).  Returns (seconds, node updates)."""
    import numpy as np
    from oracle import oracle as O
    n = CYL_N
    P = O.Params(dim=2, nx=n, ny=rows, bc_x=O.PERIODIC, bc_y=O.PERIODIC)
    x = (np.arange(n) + 0.5) / n
    y = 0.5 + (np.arange(rows) - rows // 2 + 0.5) / n
    X, Y = np.meshgrid(x, y)
    inside = ((X - 0.5) ** 2 + (Y - 0.5) ** 2 < 0.16).ravel()
    pick = lambda i: np.where(inside, CYL_IN[i], CYL_OUT[i])
    s = O.prims_to_lattice(1.4, 1.0, pick(0), pick(1), pick(2), pick(3))
    t0 = time.perf_counter()
    O.run(P, s, nsteps)
    return time.perf_counter() - t0, n * rows * nsteps


def _oracle_rows_task(rows):
    return _oracle_cylinder_rows(rows)


def _oracle_on_cores(rows, procs, timeout=60.0):
    """One oracle step of the strip in each of `procs` processes at once
    (spawned, so that no process is forked from one that holds a GPU
    context; a first round loads the library in each): (wall seconds of the
    concurrent round, node updates of all processes), or None when the pool
    fails or runs out of time (the caller then times one thread)."""
    import multiprocessing as mp
    try:
        with mp.get_context("spawn").Pool(procs) as pool:
            pool.map_async(_oracle_rows_task, [1] * procs).get(timeout)
            t0 = time.perf_counter()
            res = pool.map_async(_oracle_rows_task, [rows] * procs).get(timeout)
            wall = time.perf_counter() - t0
    except Exception:
        return None
    return wall, sum(nu for _, nu in res)


def cpu_procs(requested: int) -> int:
    """Processes of the oracle timing: as requested, else one per host core
    (at most 64)."""
    return max(1, requested if requested > 0 else min(64, os.cpu_count() or 1))


def cpu_baseline(seconds: float, procs: int = 1) -> dict:
    # calibrate on one step of an 8192 x 4 strip, then size the sample:
    # about `seconds` of CPU work over all processes together
    t, nu = _oracle_cylinder_rows(4)
    rate = nu / t
    rows = max(4, min(CYL_N, int(seconds * rate / (procs * CYL_N))))
    got = _oracle_on_cores(rows, procs) if procs > 1 else None
    if got is None:
        procs = 1
        rows = max(4, min(CYL_N, int(seconds * rate / CYL_N)))
        t, nu = _oracle_cylinder_rows(rows)
    else:
        t, nu = got
    return {"value": nu / t, "unit": "node-updates/s", "cores": procs,
            "kind": "oracle", "host": host_info(),
            "sample": f"1 step of an 8192 x {rows} periodic strip through the "
                      f"centre of the cylinder's initial state in each of "
                      f"{procs} processes at once (FP64 oracle as it stands, "
                      f"one thread each), {t:.1f} s"}


def l1_vs_oracle(L) -> dict:
    """FP32 and FP64 paths against the FP64 oracle on the shock tube: a
    whole 4096 x 512 solve to t = 0.2 (820 steps), mean |error| / field
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
                   "deposit kernel, f32_kahan: deposit kernel with the "
                   "compensated gather")
    return out


def run_tubes(args, rank=0, world=1):
    """Batched 1-D tubes (4096 seeded tubes, 256..16384 nodes, pressure
    ratio 2..100, density ratio 1..10, at rest, t = 0.2): solves/s of the
    batched FP32 path (one persistent launch per step, CUDA graphs) against
    the plain FP64 path that solves one tube at a time through a handle.
    With several ranks the tubes are split between them by work (each rank
    one batch of its tubes, no exchange), the time is the slowest rank's."""
    import torch
    from paper_1602_02675_gb300 import inputs as I
    from paper_1602_02675_gb300 import lbm as L
    from paper_1602_02675_gb300 import partition as Pt
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    specs = I.tubes_batch(args.tubes)
    work = [t.n * t.steps_and_lambda(T_END)[0] for t in specs]
    mine = Pt.assign(work, world)[rank]
    tubes, nus = [], 0
    for j in mine:
        t = specs[j]
        ns, lam = t.steps_and_lambda(T_END)
        tubes.append(L.make_tube(t.n, ns, lam / t.n, t.left, t.right))
    nus = sum(work)
    stream = torch.cuda.Stream()
    times = []
    for rep in range(1 + args.batch_reps):
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        with L.Batch(tubes, precision=L.F32, kahan=1,
                     stream=stream.cuda_stream) as b:   # tunes the tile
            b.run()
            b.sync()
            tuning = b.tuning()
        dt = time.perf_counter() - t0
        if rep > 0:
            times.append(dt)
    tb = max_over_ranks([statistics.median(times)], world, "cuda")[0]
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
        "n_gpus": world,
        "scaling": "strong" if world > 1 else None,
        "partition": ("tubes split by work between ranks, one batch per "
                      "rank, no exchange" if world > 1 else None),
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
    """The CPU oracle as it stands: K bounded samples of the workload (each
    a step of a periodic strip of the cylinder's initial state)."""
    if rank != 0:
        return None
    times, nus = [], []
    rows = args.ref_rows
    K = args.steps if args.steps > 0 else 5
    procs = cpu_procs(args.cpu_procs)

    def one():
        got = _oracle_on_cores(rows, procs) if procs > 1 else None
        return got if got is not None else _oracle_cylinder_rows(rows)

    for _ in range(args.warmup):
        one()
    for _ in range(K):
        t, nu = one()
        times.append(t)
        nus.append(nu)
    used = procs if nus[0] == CYL_N * rows * procs else 1
    value = sum(nus) / sum(times)
    sample = (f"each step: 1 lattice step of an 8192 x {rows} periodic strip "
              "through the centre of the cylinder's initial state in each of "
              f"{used} processes at once (FP64 oracle as it stands, one thread "
              "each)")
    return {
        "metric": METRIC, "value": value, "unit": "node-updates/s",
        "impl": "reference", "n_gpus": world, "steps": K,
        "warmup": args.warmup,
        "ms_per_step": round(1e3 * sum(times) / len(times), 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic (cylindrical Riemann problem, Section V.C states)",
        "config": {"workload": CYL_NAME, "nx": CYL_N, "ny": CYL_N,
                   "sample_rows": rows},
        "cpu_baseline": {"value": value, "unit": "node-updates/s",
                         "cores": used, "kind": "oracle",
                         "host": host_info(), "sample": sample},
        "e2e": {"value": value, "unit": "node-updates/s",
                "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=0,
                    help="timed steps (cylinder: 0 = the whole 2000-step "
                         "solve; sod2d: 0 = 200)")
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-solves", type=int, default=1)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--cpu-procs", type=int, default=0,
                    help="oracle timing: processes run at once (0 = one per "
                         "host core)")
    ap.add_argument("--ref-rows", type=int, default=8)
    ap.add_argument("--traffic", type=float, default=None,
                    help="ncu dram bytes per step-kernel launch, if measured")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-l1", action="store_true")
    ap.add_argument("--no-sod", action="store_true",
                    help="cylinder: skip the shock-tube sub-measurement")
    ap.add_argument("--no-bgk", action="store_true",
                    help="cylinder: skip the tau != 1 sub-measurement")
    ap.add_argument("--sod-steps", type=int, default=200)
    ap.add_argument("--fp64-steps", type=int, default=10)
    ap.add_argument("--precision-steps", type=int, default=100)
    ap.add_argument("--workload", default="cylinder2d",
                    choices=sorted(WORKLOADS) + ["tubes", "serve", "sod1d",
                                                 "patch2d", "batch2d",
                                                 "bgk2d"])
    ap.add_argument("--tau", type=float, default=1.5,
                    help="bgk2d: relaxation time (eqs 4-5)")
    ap.add_argument("--bgk-max-reach", type=int, default=4,
                    help="bgk2d: reach limit (<= 4: one-launch step)")
    ap.add_argument("--repeats", type=int, default=100,
                    help="sod1d: solves timed")
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--budget-gb", type=float, default=120.0)
    ap.add_argument("--max-side", type=int, default=2048)
    ap.add_argument("--tubes", type=int, default=4096)
    ap.add_argument("--grids", type=int, default=256,
                    help="batch2d: grids in the batch")
    ap.add_argument("--batch-reps", type=int, default=2)
    ap.add_argument("--seq-tubes", type=int, default=48)
    ap.add_argument("--precision", default="both", choices=["both", "f32"])
    ap.add_argument("--kahan", type=int, default=0, choices=[0, 1],
                    help="FP32 deposit kernel: 0 plain gather, 1 "
                         "compensated gather")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.workload == "tubes":
        if world > 1:
            import torch
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
            torch.distributed.init_process_group("nccl")
        line = run_tubes(args, rank, world)
        if rank == 0:
            print(json.dumps(line))
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    if args.workload == "serve":
        print(json.dumps(run_serve(args)))
        return
    if args.workload == "sod1d":
        print(json.dumps(run_sod1d(args)))
        return
    if args.workload == "patch2d":
        print(json.dumps(run_patch2d(args)))
        return
    if args.workload == "batch2d":
        print(json.dumps(run_batch2d(args)))
        return
    if args.workload == "bgk2d":
        print(json.dumps(run_bgk2d(args)))
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
    if args.workload == "cylinder2d":
        line = run_cylinder(args, rank, world)
    else:
        line = run_sod2d_main(args, rank, world)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


def run_sod2d_main(args, rank, world):
    """--workload sod2d: the shock tube as the main line."""
    import torch
    from paper_1602_02675_gb300 import lbm as L
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    stream = torch.cuda.Stream()
    if args.steps <= 0:
        args.steps = args.sod_steps
    sub = run_sod2d(args, L, torch, stream, world, rank, secondary=False)
    line = {"metric": METRIC, "value": sub["value"], "unit": "node-updates/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": sub["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (Sod initial state, Section V.C)",
            "config": {"workload": WORKLOAD, "nx": NX, "ny": NY,
                       "l2": "flushed (256 MB write) before every timed step",
                       "parallelism": (f"replicas x{world}" if world > 1
                                       else "1 GPU")},
            "roofline": sub["roofline"], "clocks": sub.get("clocks"),
            "gpu_launches": DS_LAUNCHES_PER_STEP * args.steps,
            "sod2d": sub}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds,
                                            cpu_procs(args.cpu_procs))
    return line


if __name__ == "__main__":
    main()
