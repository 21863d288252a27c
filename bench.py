#!/usr/bin/env python
"""Benchmark of the MEG7-prim TVD-RK3 step on one GB300.

Workload (headline): the 2D Riemann problem of Example 9 (Schulz-Rinne four
quadrants, split at (0.8, 0.8)) on a 4096 x 4096 grid with transmissive
boundaries, CFL 0.5, FP64 (the plain method), run to t = 0.3. The timed
window starts mid-run: before the warm-up the state is advanced from t = 0 to
t = 0.15 (setup, untimed; on 4096^2 by the FP32 form, which reaches the window
in a few seconds), so the timed steps see the shocks, contacts and slip lines
of a typical step rather than the nearly flat initial data.
One step = one TVD-RK3 step = three fused residual + stage-update passes,
three ghost fills and the CFL wavespeed reduction, with dt formed on the
device. Metric: cell-updates/s, one cell-update = one interior cell through
one RK stage. The FP32 form (stencil arithmetic in FP32, FP64 stage
accumulation) and the FP32 form with the learned sensor are timed on the same
workload and window and reported beside it; the 1024^2 grid of the same
problem is reported as an extra key.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gbr|reference]
Under torchrun (N > 1) the grid is split along y into N slabs, one per rank
and GPU (strong scaling): before every RK stage each slab receives six rows
from each neighbour, and after every step the CFL wavespeed is max-reduced
over the ranks (NCCL). The wall time is the max over ranks; the value is the
whole grid's cell-updates over it.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s"
N_DEFAULT = 4096  # the 4096^2 Riemann problem (the FP64 target grid)
N_SMALL = 1024    # the 1024^2 grid of the same problem (extra key)
CFL = 0.5
T_WINDOW = 0.15   # start of the timed window (run end time 0.3)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["gbr", "reference"], default="gbr")
    ap.add_argument("--n", type=int, default=N_DEFAULT, help="grid size (cells per side)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--no-small", action="store_true", help="skip the 1024^2 extra key")
    ap.add_argument("--t-window", type=float, default=T_WINDOW, help="start time of the timed window")
    ap.add_argument("--state-cache", default=None,
                    help="npz file holding the window's start state: read if present, else written")
    ap.add_argument("--profile-only", action="store_true",
                    help="only the FP64 steps of the headline workload, bracketed by cudaProfilerStart/Stop "
                         "(for ncu --profile-from-start off); prints a short JSON line")
    ap.add_argument("--profile-precision", type=int, default=64, choices=[32, 64])
    ap.add_argument("--profile-sensor", type=int, default=0, choices=[0, 1, 2],
                    help="with --profile-only: the learned sensor as a decision pass (1) or fused (2)")
    ap.add_argument("--profile-timed", action="store_true",
                    help="bracket the headline forms' timed steps with cudaProfilerStart/Stop "
                         "(for ncu --profile-from-start off)")
    ap.add_argument("--prelude-precision", type=int, default=None, choices=[32, 64],
                    help="precision of the untimed prelude (default: 32 above 2048 cells per side, else 64)")
    ap.add_argument("--ensemble-cases", type=int, default=64)
    ap.add_argument("--ensemble-steps", type=int, default=50)
    ap.add_argument("--paper-table", action="store_true",
                    help="instead of the benchmark: the runs of the paper's Table speed (whole runs, CFL 0.2)")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the scheme variants and the viscous shock-tube workload")
    return ap.parse_args()


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# Algorithmic work per cell-update (one interior cell through one RK stage)
# of the plain smooth-region path comes from paper_2305_00762_gb300.costs,
# which derives it term by term.
FP64_PEAK_NOMINAL = 1250.0    # GB300 FP64 (non-tensor): 152 SMs x 2 FMA/clk x 2 flop x 2.07 GHz
FP32_PEAK_NOMINAL = 80550.0   # 152 SMs x 128 FP32 lanes x 2 flop (FMA) x 2.07 GHz
# DRAM bytes (read + write) per launch of the FP64 stage kernel, mean over the
# three stages of a step in the timed window, from ncu captures
# (dram__bytes_read.sum + dram__bytes_write.sum) of
# `bench.py --profile-only --n N --steps 2 --warmup 1 --state-cache ...`.
# Re-measure when the kernel changes (None: not measured for this kernel).
F64_STAGE_DRAM_BYTES = {1024: 59.58e6, 4096: 1405.94e6}


def fma_peaks():
    """Measured FP64 and FP32 fused multiply-add throughput (GFLOP/s) of the
    current device, from the FMA-chain probe library (built beside libgbr),
    or None if it cannot run."""
    import ctypes
    from paper_2305_00762_gb300 import build as B
    try:
        L = ctypes.CDLL(B.PROBE_LIB)
        f = L.gbr_probe_fma_gflops
        f.restype = ctypes.c_int
        f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
        out = {}
        for prec, iters in ((64, 4096), (32, 65536)):
            g = ctypes.c_double(0.0)
            if f(prec, iters, ctypes.byref(g)) != 0:
                return None
            out[prec] = g.value
        return out
    except OSError:
        return None


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        if not getattr(self, "lines", None):
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except (ValueError, IndexError):
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() in ("active", "1"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl"
        dist.init_process_group(backend=backend)
        return dist, rank, ws, local
    return None, 0, 1, 0


def barrier(dist, torch):
    if dist is not None:
        dist.barrier()
    if torch.cuda.is_available():
        torch.cuda.synchronize()


def allmax(dist, torch, x):
    """Maximum of x over the ranks (x itself without a process group)."""
    if dist is None:
        return x
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(dist, torch, units_per_rank, seconds, ws):
    """Every rank runs an independent replica of the same workload: the
    whole-job rate is the units all ranks processed over the slowest rank's
    time."""
    return units_per_rank * ws / allmax(dist, torch, seconds)


def cpu_baseline(case, small_case, budget_s=12.0, single_budget_s=8.0):
    """The oracle, as it stands, on the host cores: whole RK3 steps of the
    workload's window state until about budget_s seconds have passed, with
    all the cores the oracle uses (OpenMP over rows); then on one core, on
    the 1024^2 window state of the same problem (one 4096^2 step would take
    about a minute on one core; the rate per cell does not depend on the
    grid size)."""
    import oracle as O
    O.build()

    def rate(c, budget):
        cfg = O.Config(c.nx, c.ny, c.dx, c.dy, c.gamma, c.mu, c.Pr, c.bc)
        dt = CFL / O.max_wavespeed(cfg, c.Q)
        Q = c.Q.copy()
        t0 = time.perf_counter()
        n = 0
        while True:
            Q, rc = O.rk3_step(cfg, Q, dt)
            n += 1
            el = time.perf_counter() - t0
            if el >= budget or el / n * (n + 1) > 2.5 * budget:
                return 3.0 * c.nx * c.ny * n / el, n, el
    cores = O.num_threads()
    v, n, el = rate(case, budget_s)
    O.set_num_threads(1)
    try:
        v1, n1, el1 = rate(small_case, single_budget_s)
    finally:
        O.set_num_threads(cores)
    return {"value": v, "unit": METRIC, "cores": cores, "kind": "oracle",
            "sample": f"{n} RK3 step(s) of the {case.nx}x{case.ny} Riemann window state, FP64, {el:.1f} s",
            "single_core": {"value": v1, "cores": 1,
                            "sample": f"{n1} RK3 step(s) of the {small_case.nx}x{small_case.ny} window state, "
                                      f"{el1:.1f} s"}}

def oracle_window_state(O, case, cfl=CFL, t_start=T_WINDOW):
    """Advance the workload from t = 0 to t_start with the oracle (setup)."""
    cfg = O.Config(case.nx, case.ny, case.dx, case.dy, case.gamma, case.mu, case.Pr, case.bc)
    Q, t, n = O.run(cfg, case.Q, t_start, cfl)
    return cfg, Q, t


def run_reference(args):
    """--impl reference: the oracle (plain FP64 C, OpenMP over rows) on the
    host cores. Each step is one RK3 step of a bounded sample of the same
    workload: the same Riemann problem and window on a 256 x 256 grid, its
    start state prepared by the oracle itself (untimed)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O
    from paper_2305_00762_gb300 import cases
    O.build()
    n = 256
    cfg, Q, t0_sim = oracle_window_state(O, cases.riemann_2d(n), t_start=args.t_window)
    for _ in range(args.warmup):
        Q, _ = O.rk3_step(cfg, Q, CFL / O.max_wavespeed(cfg, Q))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        Q, _ = O.rk3_step(cfg, Q, CFL / O.max_wavespeed(cfg, Q))
    el = time.perf_counter() - t0
    v = 3.0 * n * n * args.steps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": METRIC, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"riemann_2d_{args.n}x{args.n}_fp64", "sample": f"{n}x{n}",
                   "cfl": CFL, "window_t_start": round(t0_sim, 6)},
        "cpu_baseline": {"value": v, "unit": METRIC, "cores": O.num_threads(), "kind": "oracle",
                         "sample": f"{args.steps} RK3 steps of the {n}x{n} Riemann problem from t = {t0_sim:.3f}"},
        "e2e": {"value": v, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)

def run_ensemble(args, torch, gbr, cases, st, sensor_w=None):
    """The batched form: the seeded ensemble of independent vortex / shear
    layer grids (sizes from {256^2, 512^2, 1024^2, 2048^2}), FP32 arithmetic
    with the learned sensor, autotuned tile shape, the timed steps replayed
    from one CUDA graph (args.ensemble_steps steps, each grid at its own
    dt). The states (about 2.8 GB for 64 grids) exceed L2, so no flush is
    needed."""
    table = cases.ensemble(args.ensemble_cases)
    ens = [cases.make_ensemble_case(kind, n, prm) for kind, n, prm in table]
    b = gbr.Batch(ens, precision=32, stream=st.cuda_stream)
    if sensor_w is not None:
        b.set_sensor(sensor_w)
    for k, c in enumerate(ens):
        b.set_state(k, torch.from_numpy(c.Q).cuda())
    del ens
    steps = args.ensemble_steps
    choice, shape = b.autotune(trials=3)
    b.step_cfl(CFL, args.warmup)
    b.step_cfl(CFL, steps)   # capture now, replay below
    b.sync()
    cells = sum(n * n for _, n, _ in table)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    b.step_cfl(CFL, steps)
    e1.record(st)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    rc = b.sync(allow=(gbr.GBR_ERR_NONPHYSICAL,))
    t, dt = b.times(allow=(gbr.GBR_ERR_NONPHYSICAL,))
    b.close()
    acc = ensemble_accuracy(torch, gbr, cases, table, st, sensor_w, steps)
    return {"value": 3.0 * cells * steps / (ms * 1e-3), "unit": METRIC, "grids": len(table),
            "cells": cells, "steps": steps, "ms_per_step": ms / steps, "precision": "fp32",
            "learned_sensor": sensor_w is not None,
            "tile": list(shape), "graph": True, "dt_min": float(dt.min()), "dt_max": float(dt.max()),
            "status": gbr.error_string(rc),
            "sizes": {str(n): sum(1 for _, m, _ in table if m == n) for n in (256, 512, 1024, 2048)},
            "density_l1_vs_oracle": acc}



def ensemble_accuracy(torch, gbr, cases, table, st, sensor_w, nsteps, per_size=4):
    """Per-case density L1 error of the batched FP32 (+ learned sensor) form
    against the FP64 oracle: the batch takes nsteps CFL steps from t = 0
    (each grid at its own dt), then the oracle runs the first `per_size`
    256^2 and 512^2 members to the time each reached (CFL 0.5, last step
    clipped to land on it), on the host cores. The larger members are left
    out to keep the oracle's share of the run bounded (a 2048^2 member would
    take minutes)."""
    import oracle as O
    O.build()
    ens = [cases.make_ensemble_case(kind, n, prm) for kind, n, prm in table]
    b = gbr.Batch(ens, precision=32, stream=st.cuda_stream)
    if sensor_w is not None:
        b.set_sensor(sensor_w)
    for k, c in enumerate(ens):
        b.set_state(k, torch.from_numpy(c.Q).cuda())
    b.step_cfl(CFL, nsteps)
    t, _ = b.times()
    picked = {256: [], 512: []}
    for k, (_, n, _) in enumerate(table):
        if n in picked and len(picked[n]) < per_size:
            picked[n].append(k)
    out = {}
    t0 = time.perf_counter()
    for n, ks in picked.items():
        for k in ks:
            c = ens[k]
            cfg = O.Config(c.nx, c.ny, c.dx, c.dy, c.gamma, c.mu, c.Pr, c.bc)
            Qo, to, no = O.run(cfg, c.Q, float(t[k]), CFL)
            r32 = b.get_state(k)[0]
            out[str(k)] = {"n": n, "kind": table[k][0], "t": float(t[k]), "oracle_steps": no,
                           "l1": float(np.abs(r32 - Qo[0]).sum() / np.abs(Qo[0]).sum())}
    b.close()
    l1 = [v["l1"] for v in out.values()]
    return {"per_case": out, "max": max(l1), "median": float(np.median(l1)), "steps": nsteps,
            "oracle_s": time.perf_counter() - t0}

def run_variants(torch, gbr, case, q_start, st, flush, plain_rate, steps=10, warmup=3):
    """The scheme's other members on the benchmark's workload and window
    state, FP64: MEG7-cons, the fourth-order member of the family, and the
    shock-stable HLLC-LM Riemann solver."""
    cells = case.nx * case.ny
    out = {}
    for name, kw in (("meg7_cons", {"cons": True}), ("order4", {"order": 4}), ("hllc_lm", {"riemann": 1})):
        s = gbr.Solver.for_case(case, stream=st.cuda_stream, precision=64, **kw)
        s.set_state(q_start)
        for _ in range(warmup):
            s.step_cfl(CFL)
        s.sync()
        ms = time_steps(torch, s, steps, flush)
        rc = s.sync(allow=(gbr.GBR_ERR_NONPHYSICAL,))
        s.close()
        rate = 3.0 * cells * steps / (ms * 1e-3)
        out[name] = {"value": rate, "unit": METRIC, "ms_per_step": ms / steps, "vs_plain_fp64": rate / plain_rate,
                     "status": gbr.error_string(rc)}
    return out


def run_viscous(torch, gbr, cases, st, flush, prelude=50, warmup=3, steps=200):
    """The viscous shock tube on 2048 x 1024 cells (Re 1000, Pr 0.73, no-slip
    walls, symmetry top) at the paper's CFL 0.2 (the viscous bound decides dt
    on this grid, and CFL 0.5 is beyond the stability limit of the viscous
    operator there): FP64 and FP32 forms timed over a fixed 200-step window
    from a common state after `prelude` FP64 steps, and the FP32 form's
    density L1 against FP64 after 20 steps of a common fixed dt."""
    c = cases.viscous_shock_tube(2048, 1024)
    cells = c.nx * c.ny
    pre = gbr.Solver.for_case(c, stream=st.cuda_stream, precision=64)
    pre.set_state(torch.from_numpy(c.Q).cuda())
    for _ in range(prelude):
        pre.step_cfl(c.cfl)
    q0 = torch.empty((4, c.ny, c.nx), dtype=torch.float64, device="cuda")
    gbr.gbr_get_state(pre.ctx, q0, c.nx, c.ny)
    t0 = pre.time()
    dt = 0.8 * c.cfl / pre.max_wavespeed()
    pre.close()
    out = {"workload": "viscous_shock_tube_2048x1024", "unit": METRIC, "cfl": c.cfl, "t_start": t0,
           "prelude_fp64_steps": prelude, "timed_steps": steps}
    rho = {}
    for prec in (64, 32):
        s = gbr.Solver.for_case(c, stream=st.cuda_stream, precision=prec)
        s.set_state(q0)
        for _ in range(warmup):
            s.step_cfl(c.cfl)
        s.sync()
        ms = time_steps(torch, s, steps, flush, cfl=c.cfl)
        rc = s.sync(allow=(gbr.GBR_ERR_NONPHYSICAL,))
        s.close()
        out[f"fp{prec}"] = {"value": 3.0 * cells * steps / (ms * 1e-3), "ms_per_step": ms / steps,
                            "status": gbr.error_string(rc)}
        s = gbr.Solver.for_case(c, stream=st.cuda_stream, precision=prec)
        s.set_state(q0)
        for _ in range(20):
            s.step(dt)
        rho[prec] = s.get_state()[0]
        s.close()
    out["density_l1_fp32_vs_fp64_20_steps"] = float(np.abs(rho[32] - rho[64]).sum() / np.abs(rho[64]).sum())
    return out

def run_to(solver, t_end, cfl, chunk=50):
    """Advance to t_end at the given CFL with dt formed on the device: chunks
    of `chunk` unbounded steps while the time left exceeds three chunks at the
    last mean dt, then single steps with dt_max = the time left (one host read
    of the time per chunk or step). Returns the number of steps."""
    steps, t, mean_dt = 0, solver.time(), None
    while t < t_end * (1 - 1e-14):
        left = t_end - t
        if mean_dt is not None and left > 3.0 * chunk * mean_dt:
            for _ in range(chunk):
                solver.step_cfl(cfl)
            n = chunk
        else:
            solver.step_cfl(cfl, left)
            n = 1
        t_new = solver.time()
        steps += n
        mean_dt = (t_new - t) / n
        t = t_new
    return steps


def run_paper_table(torch, gbr, cases):
    """The paper's Table speed runs (whole runs at the paper's CFL 0.2,
    MEG7-prim and MEG7-cons in FP64, and MEG7-prim in the FP32 form):
    wall-clock seconds on this GPU, host loop included, beside the paper's
    serial CPU times (unnamed hardware, unstated precision: context only)."""
    import numpy as np
    runs = [("riemann_2d_400x400_t0.8", lambda: cases.riemann_2d(400, t_end=0.8), 0.8,
             {"prim": 1025.0, "cons": 1031.0}),
            ("double_mach_1024x256_t0.2", lambda: cases.double_mach(1024, 256), 0.2,
             {"prim": 1806.0, "cons": 1946.0}),
            ("viscous_shock_tube_1280x640_t1", lambda: cases.viscous_shock_tube(1280, 640), 1.0,
             {"prim": 35455.0, "cons": 38062.0})]
    out = {}
    for name, make, t_end, paper in runs:
        c = make()
        row = {"paper_serial_cpu_s": paper}
        for form, kw in (("fp64_prim", {}), ("fp64_cons", {"cons": True}), ("fp32_prim", {"precision": 32})):
            s = gbr.Solver.for_case(c, **kw)
            s.set_state(torch.from_numpy(c.Q).cuda())
            s.step_cfl(0.2, 1e-12)   # warm-up launch (kernel set-up), then restart from t = 0
            s.set_state(torch.from_numpy(c.Q).cuda())
            s.set_time(0.0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            steps = run_to(s, t_end, 0.2)
            rc = s.sync(allow=(gbr.GBR_ERR_NONPHYSICAL,))
            wall = time.perf_counter() - t0
            t = s.time()
            Q = s.get_state()
            s.close()
            row[form] = {"wall_s": wall, "steps": steps, "t": t, "t_end_overshoot": t > t_end * (1 + 1e-12),
                         "status": gbr.error_string(rc),
                         "rho_min": float(Q[0].min()), "rho_max": float(Q[0].max()),
                         "cell_updates_per_s": 3.0 * c.nx * c.ny * steps / wall}
        out[name] = row
    return out


def time_steps(torch, solver, steps, flush, profile=False, cfl=CFL):
    """Device time of `steps` RK3 steps, L2 flushed between steps (outside
    the events); per-step events on the library's stream."""
    st = torch.cuda.current_stream()
    total = 0.0
    if profile:
        torch.cuda.cudart().cudaProfilerStart()
    for _ in range(steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(st)
        solver.step_cfl(cfl)
        b.record(st)
        b.synchronize()
        total += a.elapsed_time(b)
    if profile:
        torch.cuda.cudart().cudaProfilerStop()
    return total


def window_state(torch, gbr, case, st, t_window, precision, cache=None):
    """Untimed prelude: CFL steps (chunks of 50, dt formed on the device) from
    t = 0 until t >= t_window, in the given precision. Returns the state on
    the device, its time and the step count. With `cache` (an .npz path) the
    state is read from there when it matches, else written there."""
    shape = (4, case.ny, case.nx)
    if cache and os.path.exists(cache):
        z = np.load(cache)
        if (tuple(z["Q"].shape) == shape and float(z["t_window"]) == t_window
                and int(z["precision"]) == precision):
            return torch.from_numpy(z["Q"]).cuda(), float(z["t"]), int(z["steps"])
    pre = gbr.Solver.for_case(case, stream=st.cuda_stream, precision=precision)
    pre.set_state(torch.from_numpy(case.Q).cuda())
    steps = 0
    while steps < 100000 and pre.time() < t_window:
        for _ in range(50):
            pre.step_cfl(CFL)
        steps += 50
    t = pre.time() if steps else 0.0
    q = torch.empty(shape, dtype=torch.float64, device="cuda")
    gbr.gbr_get_state(pre.ctx, q, case.nx, case.ny)
    pre.close()
    if cache:
        np.savez(cache, Q=q.cpu().numpy(), t=t, steps=steps, t_window=t_window, precision=precision)
    return q, t, steps


def time_forms(args, torch, gbr, case, q_start, forms, st, flush, dist, ws, local, sensor_w):
    """Device time of args.steps RK3 steps of each (precision, learned) form
    from the window state, after args.warmup untimed steps; per-launch
    events of the library (GBR_OPT_TIMING) for the roofline."""
    cells = case.nx * case.ny
    results = {}
    for prec, learned in forms:
        s = gbr.Solver.for_case(case, stream=st.cuda_stream, precision=prec)
        s.set_state(q_start)
        if learned:
            s.set_sensor(sensor_w)
        for _ in range(args.warmup):
            s.step_cfl(CFL)
        s.sync()
        s.timing(True)
        barrier(dist, torch)
        with ClockSampler(local) as clk:
            ms = time_steps(torch, s, args.steps, flush, profile=args.profile_timed)
        barrier(dist, torch)
        tm, dropped = s.get_timing()
        s.timing(False)
        rate = whole_job_rate(dist, torch, 3.0 * cells * args.steps, ms * 1e-3, ws)
        ms = allmax(dist, torch, ms)
        rc = s.sync(allow=(gbr.GBR_ERR_NONPHYSICAL,))
        results[(prec, learned)] = {"ms": ms, "rate": rate, "timing": tm, "clocks": clk.summary(), "status": rc}
        s.close()
    return results


def form_accuracy(gbr, case, q_start, forms, st, sensor_w, nsteps=20):
    """Density L1 error of each form against the FP64 path (which matches the
    oracle to 1e-12 per step) after the same nsteps fixed-dt steps from the
    window state."""
    acc = {}
    ref = None
    dt_fix = None
    for prec, learned in forms:
        s = gbr.Solver.for_case(case, stream=st.cuda_stream, precision=prec)
        s.set_state(q_start)
        if learned:
            s.set_sensor(sensor_w)
        if dt_fix is None:
            dt_fix = 0.8 * CFL / s.max_wavespeed()
        for _ in range(nsteps):
            s.step(dt_fix)
        rho = s.get_state()[0]
        s.close()
        if ref is None:
            ref = rho
        else:
            acc[(prec, learned)] = float(np.abs(rho - ref).sum() / np.abs(ref).sum())
    return acc


def stage_avg_ms(r):
    ms, n = r["timing"]["stage"]
    return ms / max(n, 1)


def roofline(costs, cells, r64, fma, hbm_peak, n):
    """The FP64 stage kernel against the FP64 ALU peak: algorithmic flops per
    launch (flop per cell-update x cells) over its mean launch time."""
    stage_s = stage_avg_ms(r64) * 1e-3
    flop_cell = costs.fp64_flop_per_cell_update()
    achieved = flop_cell * cells / stage_s / 1e9
    hbm = costs.hbm_bytes_per_cell_update() * cells / stage_s / 1e9
    measured = fma[64] if fma else None
    peak = measured if measured else FP64_PEAK_NOMINAL
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "GFLOP/s", "frac": achieved / peak,
            "traffic": F64_STAGE_DRAM_BYTES.get(n), "traffic_unit": "bytes/launch",
            "peak_source": ("measured: FP64 FMA-chain probe on this GPU (bench_alu_peak.cu)" if measured
                            else "nominal: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz (probe unavailable)"),
            "peak_nominal": FP64_PEAK_NOMINAL, "frac_of_nominal": achieved / FP64_PEAK_NOMINAL,
            "kernel": "stage_kernel<double> (fused residual + RK stage)",
            "flop_per_cell_update": flop_cell, "stage_ms_avg": stage_s * 1e3,
            "hbm_achieved_gbs": hbm, "hbm_peak_gbs": hbm_peak, "hbm_frac": hbm / hbm_peak}


def fp32_entry(r, r64, costs, cells, fma, hbm_peak, acc):
    st_s = stage_avg_ms(r) * 1e-3
    alu = costs.fp64_flop_per_cell_update() * cells / st_s / 1e9
    return {"value": r["rate"], "ms_per_step": r["ms"] / max(1, r.get("steps", 1)),
            "speedup_vs_fp64": r64["ms"] / r["ms"], "stage_ms_avg": st_s * 1e3,
            "hbm_frac": costs.hbm_bytes_per_cell_update() * cells / st_s / 1e9 / hbm_peak,
            "alu_frac_fp32_of_nominal": alu / FP32_PEAK_NOMINAL,
            "alu_peak_fp32_measured": fma[32] if fma else None,
            "alu_frac_fp32": alu / fma[32] if fma else None,
            "clocks": r["clocks"], "density_l1_vs_fp64_20_steps": acc}


def run_slabs(args, torch, gbr, cases, dist, rank, ws, local):
    """N > 1: the workload's grid split along y into ws slabs, one per rank
    (paper_2305_00762_gb300.slab.DistSlab). Every rank prepares the same
    window state (the untimed prelude on the whole grid), keeps its rows and
    steps them with halo exchanges before each stage and a max all-reduce of
    the wavespeed after each step; the timed steps are bracketed by a barrier
    and a synchronize on both sides, and the time is the max over ranks."""
    from paper_2305_00762_gb300 import slab as S
    case = cases.riemann_2d(args.n)
    st = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    pre_precision = args.prelude_precision or (32 if args.n > 2048 else 64)
    q_start, t_start, pre_steps = window_state(torch, gbr, case, st, args.t_window, pre_precision,
                                               args.state_cache)
    transport = "device" if dist.get_backend() == "nccl" else "host"
    sl = S.DistSlab(case, rank, ws, transport=transport, precision=64)
    q_local = q_start[:, sl.i0:sl.i1, :].contiguous()
    del q_start
    sl.set_state(q_local)
    for _ in range(args.warmup):
        sl.step_cfl(CFL)
    sl.solver.timing(True)
    barrier(dist, torch)
    with ClockSampler(local) as clk:
        total = 0.0
        for _ in range(args.steps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(st)
            sl.step_cfl(CFL)
            b.record(st)
            b.synchronize()
            total += a.elapsed_time(b)
    barrier(dist, torch)
    tm, _ = sl.solver.get_timing()
    sl.solver.timing(False)
    ms = allmax(dist, torch, total)
    cells = case.nx * case.ny
    rc = sl.solver.sync(allow=(gbr.GBR_ERR_NONPHYSICAL,))
    # end to end: each rank's slab in from pinned host memory and out again
    hq = q_local.cpu().pin_memory()
    hout = torch.empty_like(hq).pin_memory()
    barrier(dist, torch)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        gbr.gbr_set_state(sl.solver.ctx, hq.numpy(), sl.solver.nx, sl.solver.ny)
        sl._reduce_lambda()
        sl.step_cfl(CFL)
        gbr.gbr_get_state(sl.solver.ctx, hout.numpy(), sl.solver.nx, sl.solver.ny)
    barrier(dist, torch)
    e2e = 3.0 * cells * args.steps / allmax(dist, torch, time.perf_counter() - t0)
    slab_bytes = 32 * sl.solver.nx * sl.solver.ny
    sl.close()
    if rank == 0:
        line = {
            "metric": METRIC, "value": 3.0 * cells * args.steps / (ms * 1e-3), "unit": METRIC, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"riemann_2d_{args.n}x{args.n}_fp64", "nx": args.n, "ny": args.n,
                       "cfl": CFL, "bc": "transmissive", "l2": "flushed between steps (256 MB write)",
                       "window_t_start": round(t_start, 6), "prelude_steps": pre_steps,
                       "prelude_precision": f"fp{pre_precision}", "parallelism": f"y-slabs x{ws}",
                       "halo": f"6 rows x 4 fields per neighbour per stage ({dist.get_backend()} send/recv, "
                               f"{transport} buffers)",
                       "wavespeed": f"max all-reduce per step ({dist.get_backend()})"},
            "e2e": {"value": e2e, "unit": METRIC, "h2d_bytes_per_step": slab_bytes * ws,
                    "d2h_bytes_per_step": slab_bytes * ws},
            "gpu_launches": int(sum(n for _, n in tm.values())),
            "clocks": clk.summary(), "status": gbr.error_string(rc),
        }
        print(json.dumps(line), flush=True)
    dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    dist, rank, ws, local = dist_init()
    torch.cuda.set_device(local)
    from paper_2305_00762_gb300 import build, cases, costs, gbr
    build.build()
    gbr.load()
    if ws > 1 and not args.paper_table:
        return run_slabs(args, torch, gbr, cases, dist, rank, ws, local)
    if args.paper_table:
        if rank == 0:
            print(json.dumps({"paper_table_speed": run_paper_table(torch, gbr, cases), "cfl": 0.2,
                              "note": "whole runs, host loop included; the paper's times are serial CPU runs "
                                      "on unnamed hardware (context only)"}), flush=True)
        if dist is not None:
            dist.destroy_process_group()
        return
    case = cases.riemann_2d(args.n)
    st = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > L2 (129 MB)
    cells = case.nx * case.ny
    pre_precision = args.prelude_precision or (32 if args.n > 2048 else 64)
    q_start, t_start, pre_steps = window_state(torch, gbr, case, st, args.t_window, pre_precision,
                                               args.state_cache)
    torch.cuda.synchronize()

    if args.profile_only:
        s = gbr.Solver.for_case(case, stream=st.cuda_stream, precision=args.profile_precision)
        s.set_state(q_start)
        if args.profile_sensor:
            from paper_2305_00762_gb300 import sensor_train
            s.set_sensor(sensor_train.load_weights())
            gbr.gbr_set_option(s.ctx, gbr.GBR_OPT_SENSOR, args.profile_sensor)
        for _ in range(args.warmup):
            s.step_cfl(CFL)
        s.sync()
        ms = time_steps(torch, s, args.steps, flush, profile=True)
        rc = s.sync(allow=(gbr.GBR_ERR_NONPHYSICAL,))
        s.close()
        if rank == 0:
            print(json.dumps({"profile_only": True, "n": args.n, "precision": args.profile_precision,
                              "window_t_start": t_start, "steps": args.steps, "ms_per_step": ms / args.steps,
                              "status": gbr.error_string(rc)}), flush=True)
        if dist is not None:
            dist.destroy_process_group()
        return

    from paper_2305_00762_gb300 import sensor_train
    try:
        sensor_w = sensor_train.load_weights()
    except OSError:
        sensor_w = None
    forms = [(64, False), (32, False)] + ([(32, True)] if sensor_w is not None else [])
    results = time_forms(args, torch, gbr, case, q_start, forms, st, flush, dist, ws, local, sensor_w)
    for r in results.values():
        r["steps"] = args.steps
    acc = form_accuracy(gbr, case, q_start, forms, st, sensor_w)

    # End to end through the public API with host buffers: every step copies
    # the state in from pinned host memory and the new state back out.
    s = gbr.Solver.for_case(case, stream=st.cuda_stream, precision=64)
    hq = q_start.cpu().pin_memory()
    hout = torch.empty_like(hq).pin_memory()
    for _ in range(args.warmup):
        gbr.gbr_set_state(s.ctx, hq.numpy(), case.nx, case.ny)
        s.step_cfl(CFL)
        gbr.gbr_get_state(s.ctx, hout.numpy(), case.nx, case.ny)
    barrier(dist, torch)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        gbr.gbr_set_state(s.ctx, hq.numpy(), case.nx, case.ny)
        s.step_cfl(CFL)
        gbr.gbr_get_state(s.ctx, hout.numpy(), case.nx, case.ny)
    barrier(dist, torch)
    e2e_rate = whole_job_rate(dist, torch, 3.0 * cells * args.steps, time.perf_counter() - t0, ws)
    s.close()
    del hq, hout

    # The 1024^2 grid of the same problem (extra key; window state from FP64).
    small = None
    if not args.no_small and args.n != N_SMALL:
        sc = cases.riemann_2d(N_SMALL)
        qs, ts, ps = window_state(torch, gbr, sc, st, args.t_window, 64)
        rs = time_forms(args, torch, gbr, sc, qs, forms, st, flush, dist, ws, local, sensor_w)
        small = (sc, qs, ts, ps, rs)

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    r64 = results[(64, False)]
    pk = peaks()
    hbm_peak = pk.get("hbm_gbs", 6800.0)
    fma = fma_peaks()   # after the timed regions
    line = {
        "metric": METRIC, "value": r64["rate"], "unit": METRIC, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r64["ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"riemann_2d_{args.n}x{args.n}_fp64", "nx": args.n, "ny": args.n,
                   "cfl": CFL, "bc": "transmissive", "l2": "flushed between steps (256 MB write)",
                   "window_t_start": round(t_start, 6), "prelude_steps": pre_steps,
                   "prelude_precision": f"fp{pre_precision}", "replicas": ws},
        "roofline": roofline(costs, cells, r64, fma, hbm_peak, args.n),
        "fp32_form": fp32_entry(results[(32, False)], r64, costs, cells, fma, hbm_peak, acc.get((32, False))),
        "e2e": {"value": e2e_rate, "unit": METRIC,
                "h2d_bytes_per_step": 32 * cells, "d2h_bytes_per_step": 32 * cells},
        "gpu_launches": int(sum(n for _, n in r64["timing"].values())),
        "clocks": r64["clocks"],
        "status": gbr.error_string(r64["status"]),
    }
    if (32, True) in results:
        e = fp32_entry(results[(32, True)], r64, costs, cells, fma, hbm_peak, acc.get((32, True)))
        e["sensor"] = ("MLP 50-32-32-1, BF16 tcgen05.mma (FP32 accumulators in tensor memory), "
                       "fallback band [0.3, 0.7]")
        line["fp32_learned_form"] = e
    if small is not None:
        sc, qs, ts, ps, rs = small
        s64 = rs[(64, False)]
        line[f"riemann_{N_SMALL}"] = {
            "workload": f"riemann_2d_{N_SMALL}x{N_SMALL}", "window_t_start": round(ts, 6),
            "prelude_fp64_steps": ps, "fp64": {"value": s64["rate"], "ms_per_step": s64["ms"] / args.steps,
                                               "roofline": roofline(costs, sc.nx * sc.ny, s64, fma, hbm_peak,
                                                                    N_SMALL)},
            **{("fp32" if not l else "fp32_learned"): {"value": r["rate"], "ms_per_step": r["ms"] / args.steps,
                                                       "stage_ms_avg": stage_avg_ms(r)}
               for (p_, l), r in rs.items() if p_ == 32}}
        if not args.no_variants:
            line["variants_fp64"] = run_variants(torch, gbr, sc, qs, st, flush, s64["rate"])
    if not args.no_variants:
        line["viscous"] = run_viscous(torch, gbr, cases, st, flush)
    if not args.no_ensemble:
        line["ensemble"] = run_ensemble(args, torch, gbr, cases, st, sensor_w)
    if not args.no_cpu_baseline:
        big = cases.Case(case.name, q_start.cpu().numpy(), case.dx, case.dy, case.gamma, case.mu, case.Pr, case.bc)
        if small is not None:
            sc, qs = small[0], small[1]
            little = cases.Case(sc.name, qs.cpu().numpy(), sc.dx, sc.dy, sc.gamma, sc.mu, sc.Pr, sc.bc)
        else:
            little = big
        line["cpu_baseline"] = cpu_baseline(big, little)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
