#!/usr/bin/env python3
"""Benchmark of the HWENO hot path on B300.

Headline workload: 2D Euler four-quadrant Riemann problem on [0,1]^2,
4096 x 4096 cells, seeded quadrant states (rho, p ~ U[0.1, 1.5], |u|, |v| <= 1,
seed 2024), transmissive boundaries, characteristic-wise nonlinear HWENO in
FP64 (the paper's precision).  A step is one SSP-RK3 step (three fused stage
kernels plus the device-resident time-step control); the metric is
cell-updates per RK stage per second.  The FP32 and mixed-precision arms, the
learned-indicator arms and two scheme variants are timed on the same state
and reported under "arms", each with its relative L1 error against the FP64
path and against the CPU oracle on the 256^2 version of the problem.  The
default line also carries "shock_entropy_learned": the shock / entropy-wave family
at 2048^2 with the plain FP64, plain mixed and learned mixed paths timed and
compared with the oracle (the learned indicator's gain at matched L1).

Every workload line (--workload) carries a roofline: the algorithmic flops of
a cell update in one stage (the method's formulas in plain evaluation, the
same count for every precision) times the cells of a stage launch, over the
stage kernel's average launch time measured with CUDA events on its stream.

Prints ONE JSON line (rank 0).  --impl reference times the CPU oracle on the
host cores (bounded samples of the same workload).  Under torchrun the
batched workloads are sharded across ranks by cells (no exchange) and the
single-grid workloads are split into slabs of rows with a 2-row halo
exchange per RK stage and one max-allreduce of alpha per step (weak scaling:
every rank owns a slab of the single-GPU size); the barrier and the max over
ranks bracket the timed region.
"""
from __future__ import annotations

import argparse
import functools
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "HWENO cell-updates/s per RK stage & HBM GB/s; learned/FP32 vs plain at matched L1"
UNIT = "cell-updates/s"
N_GRID = 4096
SEED = 2024
W2D = (0.99, 0.0025, 0.0025, 0.0025, 0.0025)

# Algorithmic flops of one cell update in one RK stage: every formula of
# Sec. 2.1 / 2.2 Steps 1-4 and Remark 1 in plain evaluation (products with a
# constant 0 dropped, with +-1 free; each cell reconstructed once per stage,
# per pass for characteristic 2D Euler; each cell's right and top face; alpha
# once per step).  Written by `python -m oracle.flops` (composed from the
# coefficient maps and checked exactly against the instrumented oracle by
# tests/test_flop_count.py); one count per scheme, whatever the precision.
ALGO_FLOPS = {
    "advection1d": 163.0,
    "burgers1d": 165.0,
    "euler1d_char": 704.3333,
    "euler1d_component": 536.3333,
    "burgers2d": 1469.0,
    "euler2d_char": 10732.6667,
    "euler2d_char_typical": 11100.6667,
    "euler2d_component": 6468.6667,
}
ALGO_SOURCE = ("algorithmic: the method's formulas in plain evaluation per cell and stage "
               "(oracle/flops.py, equal to the instrumented oracle's count)")
# What the 2D Euler characteristic-wise stage kernel executes per interior
# cell-stage (ncu FP op counters, 2 per FMA and 2 per paired FP32 lane, at
# 1536^2, the ring-lane
# redundancy removed; profiles/stage2d_euler_char_counters_1536.md): the
# kernel evaluates the same formulas with fewer operations (centre-shifted
# maps, face restrictions shared by the Gauss points, symmetric Gauss pairs).
EXEC_FLOPS = {("euler2d_char", "f64"): 4999.0, ("euler2d_char", "f32"): 4801.0}
MIXED_FP64_FLOPS_PER_CELL_STAGE = 10.2  # executed, early-time 1536^2 state; data dependent
# DRAM bytes per cell of the 2D Euler stage kernel, mean of the three stage
# launches at 2048^2 (state larger than L2), scaled to the grid by cells;
# None once the kernel has changed since the capture.
TRAFFIC_PER_CELL = {"fp64": 268.7, "fp32": 130.8, "fp32_ind64": 135.0}
TRAFFIC_NOTE = "mean DRAM bytes of the three stage launches at 2048^2, scaled to the grid by cells"
# Stored fields F and limited-derivative fields D per cell: stage 1 reads F
# and writes F + D, stages 2-3 read 2F and write F -> (8F + D)/3 words per
# cell-stage.
FIELDS = {"euler2d": (12, 8), "burgers2d": (3, 2), "euler1d": (6, 3), "scalar1d": (2, 1)}
# ALU peaks from the unit counts and the clock: per SM and clock 128 FP32
# FMA lanes and 2 FP64 FMA (B300's FP64 rate is 1/64 of FP32), 2 flops per
# FMA, 148 SMs, the measured maximum SM clock.
FMA_PER_SM_CLK = {"f32": 128, "f64": 2}

# Arms of the single-grid 2D Euler workloads: (name, precision, learned
# indicator, scheme options).
ARMS = [("fp64", "FP64", False, {}), ("fp32", "FP32", False, {}), ("fp32_ind64", "FP32_IND64", False, {}),
        ("fp32_learned", "FP32", True, {}), ("fp32_ind64_learned", "FP32_IND64", True, {}),
        ("fp32_ind64_typical", "FP32_IND64", False, {"smoothness": "BETA_TYPICAL"}),
        ("fp32_ind64_component", "FP32_IND64", False, {"charwise": 0})]
DTYPE = {"FP64": "f64", "FP32": "f32", "FP32_IND64": "f32 (f64 indicators/weights)"}


def host_cpu() -> str:
    """Model name of the host CPU the oracle runs on (from /proc/cpuinfo)."""
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def words_per_cell_stage(kind: str) -> float:
    F, D = FIELDS[kind]
    return (8 * F + D) / 3.0


def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return json.load(fh)
    except OSError:
        return {}


def alu_peak_tflops(kind: str, sms: int, mhz: float) -> float:
    return sms * FMA_PER_SM_CLK[kind] * 2 * mhz * 1e6 / 1e12


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.gpu), "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        try:
            with open(self.path) as fh:
                for line in fh:
                    p = [x.strip() for x in line.split(",")]
                    if len(p) < 9:
                        continue
                    try:
                        sm.append(float(p[1]))
                        mx.append(float(p[2]))
                    except ValueError:
                        continue
                    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
                    for name, v in zip(names, p[5:9]):
                        if v.lower() == "active":
                            reasons.add(name)
            os.unlink(self.path)
        except OSError:
            pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def merge_clocks(parts) -> dict:
    parts = [c for c in parts if c and c.get("samples")]
    if not parts:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
    return {"sm_mhz": statistics.median([c["sm_mhz"] for c in parts]),
            "sm_max_mhz": max(c["sm_max_mhz"] for c in parts),
            "reasons": sorted(set(r for c in parts for r in c["reasons"])),
            "samples": sum(c["samples"] for c in parts)}


# ----------------------------------------------------------------- workloads
@functools.lru_cache(maxsize=2)
def quadrant_state(n: int) -> np.ndarray:
    """The four-quadrant initial state (built once per grid size; callers
    only read it)."""
    from paper_2607_24325_b300 import workloads as W
    return W.quadrant_2d(W.quadrant_states(SEED), 0.5, 0.5, 0.0, 1.0, 0.0, 1.0, n, n)


def window_problem(m: int):
    """An m x m window of the 4096^2 workload centred on the quadrant corner
    (same cell size, transmissive sides): the CPU oracle's bounded sample."""
    from paper_2607_24325_b300 import workloads as W
    import oracle
    h = 1.0 / N_GRID
    lo = 0.5 - 0.5 * m * h
    U = W.quadrant_2d(W.quadrant_states(SEED), 0.5, 0.5, lo, lo + m * h, lo, lo + m * h, m, m)
    prob = oracle.Problem(dim=2, equation=oracle.EQ_EULER, nx=m, ny=m, xlo=lo, xhi=lo + m * h, ylo=lo,
                          yhi=lo + m * h, lin_w=W2D, bc=(oracle.BC_OUTFLOW,) * 4)
    return prob, U


def cpu_oracle_rate(m: int, steps: int = 1) -> dict:
    """Cell-updates per RK stage per second of the oracle (serial C, one core)."""
    import oracle
    prob, U = window_problem(m)
    ax, ay = oracle.alpha(prob, U)
    dt = oracle.dt(prob, ax, ay)
    t0 = time.perf_counter()
    for _ in range(steps):
        U = oracle.step(prob, U, dt, ax, ay)
    el = time.perf_counter() - t0
    return {"value": m * m * 3 * steps / el, "unit": UNIT, "cores": 1, "cpu": host_cpu(), "kind": "oracle",
            "sample": f"{steps} SSP-RK3 step(s) of the serial FP64 C oracle on a {m}x{m} window of the "
                      f"4096^2 four-quadrant state ({el:.1f} s)"}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x: float) -> float:
    """The largest x over all ranks (a job's time is its slowest rank's);
    x itself when no process group is running."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_rate(units_per_rank: float, seconds: float, world: int) -> float:
    """Whole-job throughput of `world` ranks doing equal work: all ranks'
    units over the slowest rank's time (every rank calls it: it reduces
    across ranks)."""
    return world * units_per_rank / max_over_ranks(seconds)


def headline_config(ng, world, head_name):
    """The headline workload, as both arms report it (the reference arm times
    a window of it: its cpu_baseline.sample says which)."""
    return {"workload": f"2D Euler four-quadrant Riemann {ng}^2, transmissive, characteristic-wise "
                        f"nonlinear HWENO, SSP-RK3, arm {head_name}",
            "nx": ng, "ny": ng * world, "cells": ng * ng * world, "stages_per_step": 3,
            "l2": "inputs larger than L2 (state 1.6 GB FP64, 0.8 GB FP32 at 4096^2)",
            "parallelism": f"slabs of rows over {world} GPUs (2-row halo exchange per stage)" if world > 1
            else "single GPU"}


def run_reference(args, world, rank):
    if rank != 0:
        return
    import oracle
    oracle.build()
    m = 96
    prob, U = window_problem(m)
    ax, ay = oracle.alpha(prob, U)
    dt = oracle.dt(prob, ax, ay)
    for _ in range(args.warmup):
        oracle.step(prob, U, dt, ax, ay)
    t0 = time.perf_counter()
    V = U
    for _ in range(args.steps):
        V = oracle.step(prob, V, dt, ax, ay)
    el = time.perf_counter() - t0
    value = m * m * 3 * args.steps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded four-quadrant Riemann states)",
        "config": headline_config(args.grid, 1, "fp64"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "cpu": host_cpu(), "kind": "oracle",
                         "sample": f"one SSP-RK3 step of the serial C oracle on a {m}x{m} window per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------ timed running
def time_steps(obj, torch, steps, flush=None, clock_gpu=0):
    """Advance `steps` steps of a Solver or Batch with stage profiling on
    (CUDA events around every stage launch on the object's stream); each step
    alone after an L2 flush when `flush` is given, else all steps in one
    call.  Returns (ms over the timed steps, mean stage-launch ms, stage
    launches, kernels launched, clocks)."""
    stream = torch.cuda.ExternalStream(obj.stream)
    obj.set_profiling(True)
    torch.cuda.synchronize()
    if torch.distributed.is_available() and torch.distributed.is_initialized():
        torch.distributed.barrier()
    total = 0.0
    with ClockSampler(clock_gpu) as clk:
        left = steps
        while left > 0:
            k = 1 if flush is not None else left
            if flush is not None:
                flush.fill_(1.0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            obj.advance(1e30, max_steps=k)
            e1.record(stream)
            torch.cuda.synchronize()
            total += e0.elapsed_time(e1)
            left -= k
    stage_ms, stage_n, launches = obj.profile()
    obj.set_profiling(False)
    return total, stage_ms / max(stage_n, 1), stage_n, launches, clk.summary()


def roofline(algo_key, cells_per_launch, stage_ms, kind, sms, mhz, precision_name, traffic_per_cell=None,
             probe=None):
    """The ALU roofline of the stage kernel: algorithmic flops of a launch
    over its mean measured duration against the unit-count peak (and against
    the FMA microbenchmark's measured rate, `probe` in TFLOP/s)."""
    peak = alu_peak_tflops(kind, sms, mhz)
    fl = ALGO_FLOPS[algo_key]
    achieved = fl * cells_per_launch / (stage_ms * 1e-3) / 1e12
    out = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
           "traffic": None if traffic_per_cell is None else traffic_per_cell * cells_per_launch,
           "avg_launch_ms": stage_ms, "flops_per_cell_stage": fl, "flops_source": ALGO_SOURCE,
           "peak_source": f"{sms} SMs x {FMA_PER_SM_CLK[kind]} {kind.upper()} FMA/clk x 2 flop x {mhz:.0f} MHz "
                          f"(unit counts and the measured maximum SM clock)",
           "pipe": f"{kind.upper()} FMA ({precision_name})"}
    if traffic_per_cell is not None:
        out["traffic_unit"] = "bytes per launch"
        out["traffic_note"] = TRAFFIC_NOTE
    if probe:
        out["peak_probe"] = probe
        out["frac_of_probe"] = achieved / probe
        out["probe_source"] = f"hweno_peak_fma: independent {kind.upper()} FMA chains on every SM, timed with CUDA events"
    ex = EXEC_FLOPS.get((algo_key, kind))
    if ex is not None:
        out["frac_executed"] = ex * cells_per_launch / (stage_ms * 1e-3) / 1e12 / peak
        out["executed_flops_per_cell_stage"] = ex
    return out


def hbm_fraction(kind, esz, cells, stage_ms, hbm_peak, hbm_src):
    b = words_per_cell_stage(kind) * esz
    gbs = b * cells / (stage_ms * 1e-3) / 1e9
    return {"achieved_gbs": gbs, "peak_gbs": hbm_peak, "frac": gbs / hbm_peak, "peak_source": hbm_src,
            "bytes_per_cell_stage": b}


def device_facts(torch, local, hw):
    """SM count, clock, HBM peak, and the FMA microbenchmark's FP32 and FP64
    rates (TFLOP/s) measured now on this GPU."""
    props = torch.cuda.get_device_properties(local)
    peaks = measured_peaks()
    mhz = float(peaks.get("sm_max_mhz") or 2032.0)
    hbm = peaks.get("hbm_gbs")
    probe = {"f32": hw.hweno_peak_fma(hw.FP32) / 1e12, "f64": hw.hweno_peak_fma(hw.FP64) / 1e12}
    return {"sms": props.multi_processor_count, "mhz": mhz, "hbm": float(hbm or 6400.0),
            "hbm_src": "of measured" if hbm else "of fallback", "probe": probe}


def rel_l1(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).mean() / np.abs(b).mean())


# --------------------------------------------------- the single 2D grids
def euler_cfg(hw, n, precision, extra=None, bc=None, bc_state=None):
    kw = dict(dim=2, nx=n, ny=n, equation=hw.EQ_EULER, lin_w=W2D, bc=bc or (hw.BC_OUTFLOW,) * 4,
              precision=precision)
    if bc_state is not None:
        kw["bc_state"] = bc_state
    kw.update(extra or {})
    return hw.Config(**kw)


def train_indicator(verbose=False):
    """The learned indicator for the bench: trained on the GPU (outside the
    timed region) on shock / entropy-wave snapshots and on four-quadrant
    problems with other seeds than the bench's."""
    import torch
    from paper_2607_24325_b300 import hweno as hw
    from paper_2607_24325_b300 import indicator as IND
    from paper_2607_24325_b300 import workloads as W
    data = IND.generate(seeds=[1, 2, 3], n=160, times=(0.0, 0.03, 0.06, 0.1))
    feats, devs = [data.feat], [data.dev]
    for seed in (7, 8, 9):
        n = 192
        s = hw.Solver(euler_cfg(hw, n, hw.FP64))
        s.set_state(torch.from_numpy(W.quadrant_2d(W.quadrant_states(seed), 0.5, 0.5, 0, 1, 0, 1, n, n)).cuda())
        for t in (0.0, 0.05, 0.1):
            if t > 0:
                s.advance(t)
            F = torch.empty((n * n, 75), dtype=torch.float32, device="cuda")
            D = torch.empty((n * n,), dtype=torch.float32, device="cuda")
            hw.hweno_indicator_features(s.h, F)
            hw.hweno_indicator_labels(s.h, D)
            feats.append(F)
            devs.append(D)
        s.close()
    full = IND.Dataset(feat=torch.cat(feats), dev=torch.cat(devs), n=sum(f.shape[0] for f in feats))
    theta, losses = IND.train(full, epochs=6, seed=0, verbose=verbose)
    return theta, IND.evaluate(theta, full), losses


def oracle_comparison(hw, torch, make_problem, plan, theta, T):
    """Every arm and the oracle on the 256^2 version of the workload, advanced
    to the same time T: relative L1 of the density against the oracle (and
    the oracle's step count and seconds)."""
    import oracle
    cfg64, U0, prob = make_problem(256)
    t0 = time.perf_counter()
    Uo, to, steps_o = oracle.run(prob, U0, T)
    el = time.perf_counter() - t0
    out = {"grid": "256^2", "t_final": T, "oracle_steps": steps_o, "oracle_seconds": el}
    for name, prec, learned, extra in plan:
        cfg, _, _ = make_problem(256, prec, extra)
        s = hw.Solver(cfg)
        if learned and theta is not None:
            hw.hweno_indicator_load(s.h, theta, 0.5)
        s.set_state(torch.from_numpy(U0).cuda())
        s.advance(T)
        R = s.get_state(device=False).astype(np.float64)
        s.close()
        out[name] = rel_l1(R[0], Uo[0])
    return out


def problem_factory(hw, workload, ng):
    """(make_problem(n, precision, options) -> (config, initial state, oracle
    problem), the oracle-comparison time, the data note, the workload name)
    of a single 2D Euler workload."""
    from paper_2607_24325_b300 import indicator as IND
    from paper_2607_24325_b300 import workloads as W
    import oracle
    if workload == "euler2d_quadrant":
        def make_problem(n, prec=hw.FP64, extra=None):
            U = quadrant_state(n)
            prob = oracle.Problem(dim=2, equation=oracle.EQ_EULER, nx=n, ny=n, lin_w=W2D,
                                  bc=(oracle.BC_OUTFLOW,) * 4, **_oracle_opts(extra))
            return euler_cfg(hw, n, prec, extra), U, prob
        return (make_problem, 0.002, "synthetic (seeded four-quadrant Riemann states, seed 2024)",
                f"2D Euler four-quadrant Riemann {ng}^2, transmissive, characteristic-wise nonlinear HWENO, SSP-RK3")
    se_seed = 11
    states = {}   # the initial state per grid size (it does not depend on the arm)

    def make_problem(n, prec=hw.FP64, extra=None):
        if n not in states:
            states[n] = IND.shock_entropy_problem(se_seed, n, hw.FP64)[1]
        U = states[n]
        cfg = IND.shock_entropy_config(n, prec)   # inflow of the post-shock state on the left
        prm = W.shock_entropy_2d(seed=se_seed).params
        cfg.bc_state = [list(W.prim_to_cons_2d(prm["rho2"], prm["u2"], 0.0, prm["p2"])), [0.0] * 4, [0.0] * 4,
                        [0.0] * 4]
        for k, v in (extra or {}).items():
            setattr(cfg, k, v)
        prob = oracle.Problem(dim=2, equation=oracle.EQ_EULER, nx=n, ny=n, lin_w=W2D,
                              bc=(oracle.BC_INFLOW, oracle.BC_OUTFLOW, oracle.BC_OUTFLOW, oracle.BC_OUTFLOW),
                              bc_state=[list(cfg.bc_state[0]), [0.0] * 4, [0.0] * 4, [0.0] * 4],
                              **_oracle_opts(extra))
        return cfg, U, prob
    prm = W.shock_entropy_2d(seed=se_seed).params
    return (make_problem, 0.004, f"synthetic (shock / entropy-wave family, seed {se_seed})",
            f"2D Euler shock / entropy wave {ng}^2 (Mach {prm['mach']:.2f} shock into rho = 1 + 0.2 "
            f"sin(k x.n), k = {prm['k'] / np.pi:.0f} pi), inflow + transmissive, characteristic-wise "
            f"nonlinear HWENO, SSP-RK3")


def time_solver_arm(hw, torch, cfg, U0, steps, warmup, local, theta=None):
    """One arm on one GPU: autotune, warm-up, then `steps` profiled steps
    from the initial state."""
    s = hw.Solver(cfg)
    if theta is not None:
        hw.hweno_indicator_load(s.h, theta, 0.5)
    U0_dev = torch.from_numpy(U0).cuda()
    s.set_state(U0_dev)
    hw.hweno_autotune(s.h, reps=2)
    s.advance(1e30, max_steps=warmup)
    s.set_state(U0_dev)   # the timed steps start from the workload's initial state
    ms, stage_ms, stage_n, launches, clk = time_steps(s, torch, steps, clock_gpu=local)
    rho = s.get_state()[0].double().clone()
    smooth = None
    if theta is not None:
        sm = torch.empty((cfg.nx * cfg.ny,), dtype=torch.uint8, device="cuda")
        hw.hweno_indicator_mask(s.h, sm, None)
        smooth = float(sm.float().mean().item())
    s.close()
    return {"ms": ms, "stage_ms": stage_ms, "stage_launches": stage_n, "launches": launches, "clocks": clk,
            "rho": rho, "smooth_fraction": smooth}


def shock_entropy_learned(args, hw, torch, local, theta):
    """The learned indicator where it was built for (the shock / entropy-wave
    family, 2048^2): the plain FP64 path, the plain mixed path and the mixed
    path with the learned indicator, each timed on the GPU and compared with
    the oracle on the 256^2 problem (matched L1)."""
    ng = args.grid_se
    make_problem, T_cmp, _, wname = problem_factory(hw, "shock_entropy", ng)
    plan = [("fp64", hw.FP64, False, {}), ("fp32_ind64", hw.FP32_IND64, False, {}),
            ("fp32_ind64_learned", hw.FP32_IND64, True, {})]
    steps = min(args.steps, 5)
    out = {}
    for name, prec, learned, extra in plan:
        cfg, U0, _ = make_problem(ng, prec, extra)
        r = time_solver_arm(hw, torch, cfg, U0, steps, min(args.warmup, 3), local, theta if learned else None)
        out[name] = {"value": ng * ng * 3 * steps / (r["ms"] * 1e-3), "ms_per_step": r["ms"] / steps}
        if r["smooth_fraction"] is not None:
            out[name]["linear_path_fraction"] = r["smooth_fraction"]
    cmp = oracle_comparison(hw, torch, make_problem, plan, theta, T_cmp)
    for name in out:
        out[name]["rel_l1_rho_vs_oracle_256"] = cmp[name]
    le, pm, pf = out["fp32_ind64_learned"], out["fp32_ind64"], out["fp64"]
    return {"workload": wname, "steps": steps, "arms": out,
            "learned_speedup_vs_fp64": le["value"] / pf["value"],
            "learned_speedup_vs_plain_mixed": le["value"] / pm["value"],
            "l1_learned_over_plain_mixed": le["rel_l1_rho_vs_oracle_256"] / pm["rel_l1_rho_vs_oracle_256"],
            "oracle_grid": "256^2", "oracle_t_final": T_cmp}


def run_euler2d(args, hw, torch, world, rank, local, workload):
    """A single 2D Euler grid (the four-quadrant headline or the shock /
    entropy-wave family), every arm timed on the same state; the FP64 arm is
    the headline."""
    torch.cuda.set_device(local)
    dev = device_facts(torch, local, hw)
    ng = args.grid if workload == "euler2d_quadrant" else args.grid_se
    make_problem, T_cmp, data, wname = problem_factory(hw, workload, ng)

    plan = [(name, getattr(hw, prec), learned,
             {k: getattr(hw, v) if isinstance(v, str) else v for k, v in extra.items()})
            for name, prec, learned, extra in ARMS]
    if workload == "shock_entropy":
        plan = [p for p in plan if p[0] in ("fp64", "fp32", "fp32_ind64", "fp32_learned", "fp32_ind64_learned")]
    if args.only is not None:
        plan = [p for p in plan if p[0] == args.only]
    head_name = "fp64" if any(p[0] == "fp64" for p in plan) else plan[0][0]

    theta = ind_eval = None
    if any(p[2] for p in plan):
        theta, ind_eval, _ = train_indicator()

    # the slab of this rank (weak scaling: every rank owns ng rows)
    from paper_2607_24325_b300 import partition as PT
    cfg64, U0_np, _ = make_problem(ng)
    slab = PT.BenchSlab.for_rank(cfg64, U0_np, world, rank) if world > 1 else None

    cells_rank = ng * ng
    arms = {}
    for name, prec, learned, extra in plan:
        cfg, U0, _ = make_problem(ng, prec, extra)
        if slab is not None:
            r = PT.time_slab_arm(hw, torch, PT.BenchSlab.for_rank(cfg, U0, world, rank), args.steps, args.warmup,
                                 local, theta if learned else None)
        else:
            r = time_solver_arm(hw, torch, cfg, U0, args.steps, args.warmup, local, theta if learned else None)
        r.update({"precision": prec, "learned": learned, "extra": extra})
        arms[name] = r
    for name in arms:   # every rank, same order: each arm's time is its slowest rank's
        arms[name]["ms"] = max_over_ranks(arms[name]["ms"])

    # end to end through the public API with host buffers, every step
    e2e = None
    if not args.no_e2e and slab is None:
        prec = arms[head_name]["precision"]
        cfg, U0, _ = make_problem(ng, prec)
        e2e = e2e_run(hw, torch, cfg, U0, args.steps)
    elif not args.no_e2e:
        cfg, U0, _ = make_problem(ng, arms[head_name]["precision"])
        e2e = PT.e2e_slab(hw, torch, PT.BenchSlab.for_rank(cfg, U0, world, rank), args.steps)
        e2e["value"] = world * e2e.pop("units") / max_over_ranks(e2e.pop("seconds"))

    se = None
    if workload == "euler2d_quadrant" and world == 1 and args.only is None and not args.no_shock_entropy:
        se = shock_entropy_learned(args, hw, torch, local, theta)

    cmp = None
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cmp = oracle_comparison(hw, torch, make_problem, plan, theta, T_cmp)
        if workload == "euler2d_quadrant":
            cpu = cpu_oracle_rate(256, steps=2)
        else:
            cpu = {"value": 256 * 256 * 3 * cmp["oracle_steps"] / cmp["oracle_seconds"], "unit": UNIT, "cores": 1, "cpu": host_cpu(),
                   "kind": "oracle", "sample": f"{cmp['oracle_steps']} SSP-RK3 steps of the serial FP64 C oracle on "
                                               f"the 256^2 version of the workload ({cmp['oracle_seconds']:.1f} s)"}

    if rank == 0:
        ref_rho = arms["fp64"]["rho"] if "fp64" in arms else None
        algo_base = "euler2d_char"
        summ = {}
        for name, r in arms.items():
            kind = "f64" if r["precision"] == hw.FP64 else "f32"
            key = algo_base
            if r["extra"].get("smoothness") == hw.BETA_TYPICAL:
                key = "euler2d_char_typical"
            if r["extra"].get("charwise") == 0:
                key = "euler2d_component"
            pname = {hw.FP64: "FP64", hw.FP32: "FP32", hw.FP32_IND64: "FP32_IND64"}[r["precision"]]
            traffic = None
            if workload == "euler2d_quadrant" and not r["learned"] and not r["extra"] and slab is None:
                traffic = TRAFFIC_PER_CELL.get(name)
            roof = roofline(key, r.get("cells_local", cells_rank), r["stage_ms"], kind, dev["sms"], dev["mhz"],
                            pname, traffic, probe=dev["probe"][kind])
            if r["learned"]:
                roof["note"] = ("effective: the plain scheme's algorithmic count; the linear path skips Steps 2-3 "
                                "and the projections on the cells the network clears")
            if r["precision"] == hw.FP32_IND64 and key == "euler2d_char" and workload == "euler2d_quadrant":
                roof["fp64_flops_per_cell_stage"] = MIXED_FP64_FLOPS_PER_CELL_STAGE
                roof["fp64_frac"] = (MIXED_FP64_FLOPS_PER_CELL_STAGE * cells_rank / (r["stage_ms"] * 1e-3) / 1e12
                                     / alu_peak_tflops("f64", dev["sms"], dev["mhz"]))
            a = {"value": world * cells_rank * 3 * args.steps / (r["ms"] * 1e-3), "ms_per_step": r["ms"] / args.steps,
                 "dtype": DTYPE[pname], "roofline": roof,
                 "hbm": hbm_fraction("euler2d", 8 if kind == "f64" else 4, cells_rank, r["stage_ms"], dev["hbm"],
                                     dev["hbm_src"]),
                 "clocks": r["clocks"], "gpu_launches": int(r["launches"])}
            if ref_rho is not None:
                a["rel_l1_rho_vs_fp64"] = rel_l1(r["rho"].cpu().numpy(), ref_rho.cpu().numpy())
                a["speedup_vs_fp64"] = arms["fp64"]["ms"] / r["ms"]
            if cmp is not None and name in cmp:
                a["rel_l1_rho_vs_oracle_256"] = cmp[name]
            if r.get("smooth_fraction") is not None:
                a["linear_path_fraction"] = r["smooth_fraction"]
            if r["extra"]:
                a["variant"] = {k: int(v) for k, v in r["extra"].items()}
            summ[name] = a
        hs = summ[head_name]
        head = arms[head_name]
        line = {
            "metric": METRIC, "value": world * cells_rank * 3 * args.steps / (head["ms"] * 1e-3), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms"] / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": hs["dtype"],
            "data": data,
            "config": (headline_config(ng, world, head_name) if workload == "euler2d_quadrant" else
                       {"workload": f"{wname}, arm {head_name}", "nx": ng, "ny": ng * world,
                        "cells": cells_rank * world, "stages_per_step": 3, "l2": "inputs larger than L2",
                        "parallelism": "single GPU" if world == 1 else f"slabs of rows over {world} GPUs"}),
            "roofline": hs["roofline"],
            "hbm": hs["hbm"],
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": hs["gpu_launches"],
            "clocks": merge_clocks([r["clocks"] for r in arms.values()]),
            "arms": summ,
            "oracle_comparison": cmp,
            "learned_indicator": ind_eval,
        }
        if se is not None:
            line["shock_entropy_learned"] = se
        if "fp32_ind64_learned" in summ and "fp64" in summ:
            la, pa = summ["fp32_ind64_learned"], summ["fp64"]
            line["learned_vs_plain_fp64"] = {
                "speedup": la["value"] / pa["value"],
                "rel_l1_vs_oracle_256": {"learned": la.get("rel_l1_rho_vs_oracle_256"),
                                         "plain_fp64": pa.get("rel_l1_rho_vs_oracle_256"),
                                         "plain_fp32_ind64": summ.get("fp32_ind64", {}).get(
                                             "rel_l1_rho_vs_oracle_256")}}
        print(json.dumps(line), flush=True)


def _oracle_opts(extra):
    import oracle
    out = {}
    for k, v in (extra or {}).items():
        if k == "smoothness":
            out["smoothness"] = oracle.BETA_TYPICAL if int(v) == 1 else oracle.BETA_MOMENT
        elif k == "charwise":
            out["charwise"] = int(v)
    return out


def e2e_run(hw, torch, cfg, U0, steps):
    """End to end through the public API with host buffers, every step: the
    state goes host -> device from pinned memory (hweno_set_state), one
    SSP-RK3 step runs (hweno_advance), and the new state comes back device ->
    host into pinned memory (hweno_get_state), which the next step sends
    again."""
    dtype = torch.float64 if cfg.precision == hw.FP64 else torch.float32
    a = torch.from_numpy(U0).to(dtype).pin_memory()
    b = torch.empty_like(a).pin_memory()
    s = hw.Solver(cfg)
    hw.hweno_set_state(s.h, a)          # warm the path (graph capture, first launches)
    s.advance(1e30, max_steps=1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    src, dst = a, b
    for _ in range(steps):
        hw.hweno_set_state(s.h, src)
        s.advance(1e30, max_steps=1)
        hw.hweno_get_state(s.h, dst)     # synchronises: the host has the step's result
        src, dst = dst, src
    el = time.perf_counter() - t0
    s.close()
    nbytes = a.numel() * a.element_size()
    cells = cfg.nx * cfg.ny
    return {"value": cells * 3 * steps / el, "unit": UNIT, "h2d_bytes_per_step": nbytes,
            "d2h_bytes_per_step": nbytes,
            "what": "per step: the whole state host->device from pinned memory, one SSP-RK3 step, the whole state "
                    "device->host into pinned memory"}


# ------------------------------------------------------- other workloads
def run_single_grid(args, hw, torch, world, rank, local, workload, cfg_kw, U0, arms, flush_l2, algo_key, fkind):
    """Time `arms` [(name, precision)] of one grid from U0 (each step timed
    alone after a 256 MB L2 flush when the state fits in L2); one JSON line,
    the FP64 arm the headline."""
    torch.cuda.set_device(local)
    dev = device_facts(torch, local, hw)
    U0 = torch.from_numpy(U0)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda") if flush_l2 else None
    cells = int(np.prod(U0.shape[1:]))
    out = {}
    clocks = []
    for name, prec in arms:
        s = hw.Solver(hw.Config(precision=prec, **cfg_kw))
        s.set_state(U0.cuda())
        hw.hweno_autotune(s.h, reps=2)
        s.advance(1e30, max_steps=args.warmup)
        s.set_state(U0.cuda())
        ms, stage_ms, _, launches, clk = time_steps(s, torch, args.steps, flush=flush, clock_gpu=local)
        s.close()
        ms = max_over_ranks(ms)   # under torchrun every rank advances its own copy (replicas)
        kind = "f64" if prec == hw.FP64 else "f32"
        pname = {hw.FP64: "FP64", hw.FP32: "FP32", hw.FP32_IND64: "FP32_IND64"}[prec]
        out[name] = {"value": world * cells * 3 * args.steps / (ms * 1e-3), "ms_per_step": ms / args.steps,
                     "dtype": DTYPE[pname],
                     "roofline": roofline(algo_key, cells, stage_ms, kind, dev["sms"], dev["mhz"], pname,
                                          probe=dev["probe"][kind]),
                     "hbm": hbm_fraction(fkind, 8 if kind == "f64" else 4, cells, stage_ms, dev["hbm"],
                                         dev["hbm_src"]),
                     "gpu_launches": int(launches)}
        clocks.append(clk)
    head = "fp64"
    if rank == 0:
        h = out[head]
        line = {"metric": METRIC, "value": h["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": h["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": h["dtype"],
                "data": "synthetic (closed-form initial data)",
                "config": {"workload": workload + ", arm fp64", "cells": cells * world,
                           "l2": "flushed (256 MB write) before every timed step" if flush_l2
                           else "inputs larger than L2",
                           "parallelism": "single GPU" if world == 1 else f"replicas on {world} GPUs"},
                "roofline": h["roofline"], "hbm": h["hbm"], "gpu_launches": h["gpu_launches"],
                "clocks": merge_clocks(clocks), "arms": out}
        print(json.dumps(line), flush=True)


def run_batch(args, hw, torch, world, rank, local, dim):
    """The batched workloads: 256 1D Euler Riemann problems (seed 1234, sizes
    log-uniform in [256, 8192], transmissive, characteristic-wise) or 48
    seeded 2D four-quadrant problems (nx, ny log-uniform in [96, 768]), one
    launch per stage for all instances.  The 1D batch (~28 MB in FP64) fits
    in L2, so L2 is flushed (256 MB write) before every timed step and each
    step is timed alone; the 2D batch exceeds L2.  Under torchrun the
    instances are sharded across ranks by cells (no exchange)."""
    from paper_2607_24325_b300 import partition as PT
    from paper_2607_24325_b300 import workloads as W
    torch.cuda.set_device(local)
    dev = device_facts(torch, local, hw)
    if dim == 1:
        B = W.riemann_batch_1d(n=256, seed=1234)
        sizes = [int(x) for x in B.sizes]
        states = [B.instance(k) for k in range(len(sizes))]
        cells_of = sizes
        mk = lambda k, prec: hw.Config(dim=1, nx=sizes[k], equation=hw.EQ_EULER, bc=(hw.BC_OUTFLOW,) * 4,
                                       precision=prec)
        arms = (("fp64", hw.FP64), ("fp32", hw.FP32), ("fp32_ind64", hw.FP32_IND64))
        flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
        algo_key, fkind = "euler1d_char", "euler1d"
        wname = "256 1D Euler Riemann problems, sizes log-uniform 256-8192, one launch per stage"
        data = "synthetic (seed 1234)"
    else:
        sizes2, states = W.quadrant_batch_2d()
        cells_of = [nx * ny for nx, ny in sizes2]
        mk = lambda k, prec: hw.Config(dim=2, nx=sizes2[k][0], ny=sizes2[k][1], equation=hw.EQ_EULER, lin_w=W2D,
                                       bc=(hw.BC_OUTFLOW,) * 4, precision=prec)
        arms = (("fp64", hw.FP64), ("fp32", hw.FP32), ("fp32_ind64", hw.FP32_IND64))
        flush = None
        algo_key, fkind = "euler2d_char", "euler2d"
        wname = "48 2D Euler four-quadrant problems, nx, ny log-uniform 96-768, one launch per stage"
        data = "synthetic (seed 2025)"
    # weak scaling: every rank advances a full copy's worth of cells, made of
    # its shard of `world` copies of the instance list
    reps = world
    all_idx = [k % len(cells_of) for k in range(len(cells_of) * reps)]
    mine = PT.shard_by_cells([cells_of[k] for k in all_idx], world)[rank]
    idx = [all_idx[j] for j in mine]
    out = {}
    clocks = []
    for name, prec in arms:
        b = hw.Batch([mk(k, prec) for k in idx])
        U = torch.from_numpy(b.pack([states[k] for k in idx])).cuda()
        b.set_state(U)
        shape = hw.hweno_batch_autotune(b.h, reps=3)[1]
        b.advance(1e30, max_steps=args.warmup)
        b.set_state(U)
        ms, stage_ms, _, launches, clk = time_steps(b, torch, args.steps, flush=flush, clock_gpu=local)
        cells = int(b.total)
        b.close()
        ms_max = max_over_ranks(ms)
        total_cells = sum_over_ranks(cells)
        kind = "f64" if prec == hw.FP64 else "f32"
        pname = {hw.FP64: "FP64", hw.FP32: "FP32", hw.FP32_IND64: "FP32_IND64"}[prec]
        out[name] = {"value": total_cells * 3 * args.steps / (ms_max * 1e-3), "ms_per_step": ms_max / args.steps,
                     "cells": int(total_cells), "dtype": DTYPE[pname],
                     "roofline": roofline(algo_key, cells, stage_ms, kind, dev["sms"], dev["mhz"], pname,
                                          probe=dev["probe"][kind]),
                     "hbm": hbm_fraction(fkind, 8 if kind == "f64" else 4, cells, stage_ms, dev["hbm"],
                                         dev["hbm_src"]),
                     "gpu_launches": int(launches), "launch_shape": list(shape)}
        clocks.append(clk)
    if rank == 0:
        h = out["fp64"]
        line = {"metric": METRIC, "value": h["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": h["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": h["dtype"], "data": data,
                "config": {"workload": wname + ", arm fp64", "cells": h["cells"],
                           "l2": "flushed (256 MB write) before every timed step" if flush is not None
                           else "inputs larger than L2",
                           "parallelism": "single GPU" if world == 1 else
                           f"instances sharded by cells over {world} GPUs (no exchange)"},
                "roofline": h["roofline"], "hbm": h["hbm"], "gpu_launches": h["gpu_launches"],
                "clocks": merge_clocks(clocks), "arms": out}
        print(json.dumps(line), flush=True)


def run_dmr(args, hw, torch, world, rank, local):
    """The double Mach reflection on the paper's 1920 x 480 mesh (split
    reflective wall, moving-shock top boundary), from its initial state:
    FP64, FP32 and FP32 with FP64 smoothness indicators.  The FP32 state
    (44 MB) fits in L2, so L2 is flushed (256 MB write) before every timed
    step and each step is timed alone."""
    from paper_2607_24325_b300 import workloads as W
    nx, ny = 1920, 480
    B = W.dmr_boundary()
    cfg_kw = dict(dim=2, nx=nx, ny=ny, xlo=0.0, xhi=4.0, ylo=0.0, yhi=1.0, equation=hw.EQ_EULER, lin_w=W2D,
                  bc=B["bc"], bc_state=B["bc_state"], bc_state2=B["bc_state2"], bc_param=B["bc_param"])
    run_single_grid(args, hw, torch, world, rank, local,
                    "2D Euler double Mach reflection 1920x480, split wall, moving-shock top boundary",
                    cfg_kw, W.dmr_2d(nx, ny), [("fp32", hw.FP32), ("fp32_ind64", hw.FP32_IND64), ("fp64", hw.FP64)],
                    flush_l2=True, algo_key="euler2d_char", fkind="euler2d")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--grid", type=int, default=N_GRID, help="cells per side (profiling runs use a small grid)")
    ap.add_argument("--grid-se", type=int, default=2048, help="cells per side of the shock / entropy-wave workload")
    ap.add_argument("--only", choices=[a[0] for a in ARMS], default=None,
                    help="time one arm only (profiling runs)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-shock-entropy", action="store_true",
                    help="skip the shock / entropy-wave section of the default line")
    ap.add_argument("--workload", choices=["euler2d_quadrant", "shock_entropy", "batch1d", "batch2d", "dmr",
                                           "advection1d", "burgers2d"],
                    default="euler2d_quadrant",
                    help="shock_entropy: the shock / entropy-wave family at 2048^2 with the learned indicator; "
                         "batch1d: 256 seeded 1D Euler Riemann problems of uneven sizes in one batch; "
                         "batch2d: 48 seeded 2D four-quadrant problems of uneven sizes in one batch; "
                         "dmr: the double Mach reflection on the paper's 1920 x 480 mesh; "
                         "advection1d / burgers2d: the throughput runs of Examples 1 and 3")
    args = ap.parse_args()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return

    import torch
    import torch.distributed as dist
    import __graft_entry__
    __graft_entry__.build()
    from paper_2607_24325_b300 import hweno as hw
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    try:
        if args.workload == "batch1d":
            run_batch(args, hw, torch, world, rank, local, 1)
        elif args.workload == "batch2d":
            run_batch(args, hw, torch, world, rank, local, 2)
        elif args.workload == "dmr":
            run_dmr(args, hw, torch, world, rank, local)
        elif args.workload == "advection1d":
            from paper_2607_24325_b300 import workloads as W
            n = 1 << 24
            run_single_grid(args, hw, torch, world, rank, local,
                            "1D linear advection u0 = sin(pi x) on [0,2], periodic, 2^24 cells",
                            dict(dim=1, nx=n, xlo=0.0, xhi=2.0, equation=hw.EQ_ADVECTION, adv_x=1.0),
                            W.sine_1d_cells(n), [("fp32", hw.FP32), ("fp32_ind64", hw.FP32_IND64), ("fp64", hw.FP64)],
                            flush_l2=False, algo_key="advection1d", fkind="scalar1d")
        elif args.workload == "burgers2d":
            from paper_2607_24325_b300 import workloads as W
            n = 4096
            run_single_grid(args, hw, torch, world, rank, local,
                            "2D Burgers u0 = 0.5 + sin(pi (x + y) / 2) on [0,4]^2, periodic, 4096^2 cells",
                            dict(dim=2, nx=n, ny=n, xlo=0.0, xhi=4.0, ylo=0.0, yhi=4.0, equation=hw.EQ_BURGERS,
                                 lin_w=W2D), W.sine_2d_cells(n, n),
                            [("fp32", hw.FP32), ("fp32_ind64", hw.FP32_IND64), ("fp64", hw.FP64)], flush_l2=False,
                            algo_key="burgers2d", fkind="burgers2d")
        else:
            run_euler2d(args, hw, torch, world, rank, local, args.workload)
    finally:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
