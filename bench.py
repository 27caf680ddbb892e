#!/usr/bin/env python
"""Benchmark: batched MLMC level-pair solves of the stochastic Henry problem.

Workload (one step): MLMC levels 0..3 of the Henry problem on [0,2]x[0,1]
(32x16, 64x32, 128x64, 256x128 cells; 24, 48, 96, 192 implicit Euler steps
to T = 43200 s) with 1024 / 256 / 64 / 16 level pairs, each pair a fine solve
at level l and a coarse solve at level l-1 sharing one xi ~ U[-1,1]^3, then
the per-level MLMC statistics of the 22 QoIs. The four levels run
concurrently on four CUDA streams. The headline runs the multigrid in FP64
(the plain FP64 GPU form); the same workload with FP32 multigrid inside FP64
defect correction is reported beside it.

Metric: level-pair solves per second (pairs of all levels / wall time).
Beside it:
  roofline    the dominant kernel (FP64 smoother half-sweep on the level-3
              grid) with the L2 flushed before every timed launch: the
              method's bytes per updated cell over the launch time, against
              the measured HBM copy bandwidth, and its FP64 operations
              against the FP64 FMA rate measured in the same run;
  streaming   the same kernels on the 1024x512 grid (16 samples, operands
              far beyond L2), where the memory roof is the one that binds;
  whole_level per level, the method's bytes of a whole solve (per-cell
              figures x the defect-correction iterations the solve took)
              over its wall time;
  mlmc        the second half of the metric: adaptive MLMC to RMSE 1e-3 on
              c at three points, 6 levels (32x16 .. 1024x512), 6 random
              variables, FP32 multigrid and FP64 multigrid, wall times;
  cpu_baseline the FP64 oracle on every host core.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank runs the workload on its own GPU with its own
sample indices (weak scaling); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

LEVELS = (0, 1, 2, 3)
BATCH = {0: 1024, 1: 256, 2: 64, 3: 16}
METRIC = "Henry solves/s per level; MLMC wall time at target RMSE, FP32-MG vs FP64"
UNIT = "level-pair solves/s"
WORKLOAD = ("henry-mlmc-4lvl-batched: levels 0-3 (32x16..256x128 cells, 24..192 steps, "
            "T=43200 s), 1024/256/64/16 level pairs, 3 random variables, per-level stats")
CONFIG = {"workload": WORKLOAD, "levels": list(LEVELS), "batch": [BATCH[l] for l in LEVELS],
          "n_xi": 3, "T_s": 43200.0, "newton_rtol": 1e-10, "newton_atol": 1e-11,
          "l2": "flushed between timed steps (256 MB write)"}
FLUSH_FLOATS = 64 * 1024 * 1024          # 256 MB, twice the L2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--loop", default="graph", choices=["graph", "host"],
                    help="host: the same solves with the host-side Newton loop (plain kernel "
                         "launches, bitwise the same results); for ncu launch lists, which do "
                         "not enter the conditional graph bodies of the default loop")
    ap.add_argument("--pairs", default="graph", choices=["graph", "streams"],
                    help="graph: all level pairs of a step through henry_sample_levels (one "
                         "graph launch per coarse time step); streams: henry_sample_pairs per "
                         "level on four streams")
    ap.add_argument("--no-fp32", action="store_true", help="skip the FP32-multigrid variant")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the discrete-adjoint timing")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-mlmc", action="store_true", help="skip the adaptive MLMC runs")
    ap.add_argument("--no-extra", action="store_true",
                    help="headline only: skip every line but the timed steps and e2e")
    a = ap.parse_args()
    if a.no_extra:
        a.no_fp32 = a.no_adjoint = a.no_cpu = a.no_mlmc = True
    return a


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for k, n in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(n)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# the method's byte model: bytes per fine cell of each operation
# ---------------------------------------------------------------------------
def vcycle_bytes(T, nu1, nu2):
    """One V(nu1, nu2) per fine cell, T = bytes of the multigrid type: every
    half-sweep reads the operator (20 values), b and the other colour's x
    and writes x (26 values per updated cell, i.e. per cell and sweep); the
    residual + restriction reads A, b, x and writes the coarse r (98 B in
    FP32); the prolongation and correction 18 B; the coarse levels add a
    third (4/3 of the finest level)."""
    return ((nu1 + nu2) * 26 * T + 98 * T / 4 + 18 * T / 4) * 4.0 / 3.0


def dc_iteration_bytes(T, vcycles, nu1, nu2):
    """One defect-correction iteration per fine cell: the V-cycles, the FP64
    residual (p, c, c_old, phi, K read, R written: 56 B), the cast to the
    right-hand side and the state update (about 0.14 KB with FP32 operators,
    0.15 KB with FP64)."""
    return vcycles * vcycle_bytes(T, nu1, nu2) + (140.0 if T == 4 else 150.0)


def step_bytes(T):
    """Once per implicit step and cell: the residual and the Jacobian (40 B
    read, R 16 B and J 20 values written)."""
    return 56.0 + 40.0 + 20 * T


def solve_bytes(ncell, B, nt, iters_total, T, vcycles, nu1, nu2):
    return ncell * (B * nt * step_bytes(T) + iters_total * dc_iteration_bytes(T, vcycles, nu1, nu2))


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def make_inputs(rank, n_xi=3):
    import torch
    from paper_2403_17018_gb300.inputs import xi_batch
    return {l: torch.from_numpy(xi_batch(l, rank * BATCH[l], BATCH[l], n_xi=n_xi)).cuda()
            for l in LEVELS}


class Workload:
    """One context for the four levels, each level with its autotuned
    schedule (henry_set_schedule). pairs="graph": a step is one
    henry_sample_levels call (one CUDA graph launch per coarse time step for
    all level pairs); pairs="streams": henry_sample_pairs per level on four
    streams."""

    def __init__(self, precision, schedules, loop_mode, pairs="graph"):
        import torch
        from paper_2403_17018_gb300 import binding as hb
        self.hb = hb
        self.ctx = hb.Context(hb.default_config(nlevels=4, precision=precision,
                                                loop_mode=loop_mode))
        self.schedules = schedules
        for l in LEVELS:
            self.ctx.set_schedule(l, **schedules[l])
        self.cfg = self.ctx.cfg
        self.T = 8 if precision == hb.PREC_FP64 else 4
        self.pairs = pairs
        self.streams = {l: torch.cuda.Stream() for l in LEVELS}
        self.out = {}

    def launch_count(self):
        return self.ctx.launch_count()

    def close(self):
        self.ctx.close()

    def step(self, xis, host=None):
        """All level pairs, then the per-level statistics (synchronous per
        level). With `host` = dict of pinned buffers, copy xi in from host
        memory and the QoIs back to host memory inside the step."""
        import torch
        main = torch.cuda.current_stream()
        if self.pairs == "graph":
            if host is not None:
                for l in LEVELS:
                    xis[l].copy_(host["xi"][l], non_blocking=True)
            self.out = self.ctx.sample_levels({l: xis[l] for l in LEVELS})
            streams = {l: main for l in LEVELS}
        else:
            ev = torch.cuda.Event()
            ev.record(main)
            for l in LEVELS:
                s = self.streams[l]
                s.wait_event(ev)
                with torch.cuda.stream(s):
                    if host is not None:
                        xis[l].copy_(host["xi"][l], non_blocking=True)
                    self.out[l] = self.ctx.sample_pairs(l, xis[l], stream=s)
            streams = self.streams
        stats = {}
        for l in LEVELS:
            s = streams[l]
            qf, qc, _, _, st = self.out[l]
            S = self.hb.LevelStats()
            self.ctx.level_stats(l, qf, qc, st, S, stream=s)
            stats[l] = S
            if host is not None:
                with torch.cuda.stream(s):
                    host["qf"][l].copy_(qf, non_blocking=True)
                    if qc is not None:
                        host["qc"][l].copy_(qc, non_blocking=True)
                    host["st"][l].copy_(st, non_blocking=True)
        if self.pairs != "graph":
            for l in LEVELS:
                e = torch.cuda.Event()
                e.record(self.streams[l])
                main.wait_event(e)
        return stats


def tune_schedules(precision_name):
    """Autotuned schedule per level: V-cycles per iteration x smoothing sweeps
    x shared-memory V-cycle threshold, then the operator reuse factor, the
    residual tile height and the temporally blocked legs, each timed on one
    solve of the level over the whole horizon. Kept in the autotuner's cache (by GPU, level, precision, batch),
    so a second run on the same machine -- e.g. under a profiler -- reuses
    it; returns (schedules, seconds spent tuning)."""
    import torch
    from paper_2403_17018_gb300 import autotune as A
    A.CANDIDATES = {"vcycles": (2, 3, 4), "nu": ((2, 2), (3, 3)), "small_cells": (128, 512),
                    "jac_lag": (0, 10, 30), "res_rows": (0, 2, 16), "tb_cells": (0, 2048),
                    "keep_lags": (30, 100)}
    t0 = time.perf_counter()
    gpu = torch.cuda.get_device_name(0)
    cache = A.load_cache()
    out = {}
    for l in LEVELS:
        key = A._key(gpu, l, precision_name, BATCH[l], 32, 16) + "|bench-horizon"
        if key not in cache:
            cache[key], _ = A.tune_level(l, BATCH[l], precision_name, steps=None, reps=1,
                                         splits=(1,))
        out[l] = cache[key]
    A.save_cache(cache)
    return out, time.perf_counter() - t0


def sched_str(s):
    return (f"V({s['nu1']},{s['nu2']}) x{s['vcycles']} smem<={s['mg_small_cells']} "
            f"lag={s['jac_lag']}{'+keep' if s.get('jac_keep') else ''} rows={s.get('res_rows', 0)} "
            f"tb<={s.get('mg_tb_cells', 0)}")


def time_steps(wl, xis, K, W, barrier, flush, host=None):
    import torch
    for _ in range(W):
        wl.step(xis, host)
    torch.cuda.synchronize()
    total_ms = 0.0
    per_step = []
    n0 = wl.launch_count()
    stats = None
    for _ in range(K):
        flush()
        torch.cuda.synchronize()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        stats = wl.step(xis, host)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        per_step.append(ms)
        total_ms += ms
    barrier()
    launches = wl.launch_count() - n0
    return total_ms, per_step, launches, stats


def per_level_rates(wl, xis):
    """Level-pair solves/s of each level's batch run alone (device time)."""
    import torch
    rates = {}
    for l in LEVELS:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        wl.ctx.sample_pairs(l, xis[l])
        e1.record()
        torch.cuda.synchronize()
        rates[f"L{l}"] = round(BATCH[l] / (e0.elapsed_time(e1) / 1e3), 2)
    return rates


def whole_level(wl, xis, hbm):
    """Per level: the fine solves of the level's batch run alone; the method's
    bytes of the solve (per-cell figures x the defect-correction iterations
    the solve took, reported by the solver) over its device time."""
    import torch
    out = {}
    ctx = wl.ctx
    for l in LEVELS:
        sc = wl.schedules[l]
        li = ctx.level_info(l)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        res = ctx.solve(l, xis[l], want_iters=True)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        its = int(res["iters"].sum().item())
        by = solve_bytes(li.nx * li.ny, BATCH[l], li.nt, its, wl.T, sc["vcycles"], sc["nu1"],
                         sc["nu2"])
        gbs = by / (ms / 1e3) / 1e9
        out[f"L{l}"] = {"solve_ms": round(ms, 2), "iters_per_step": round(its / BATCH[l] / li.nt, 3),
                        "bytes": by, "achieved_gbs": round(gbs, 1), "frac": round(gbs / hbm, 4)}
    return out


def kernel_line(ctx, level, which, reps, flush, hbm, fp64_tflops, T, name):
    ms, by, fl = ctx.time_kernel(level, 0, which, reps=reps, flush=flush)
    gbs = by / (ms / 1e3) / 1e9
    line = {"kernel": name, "ms_per_launch": round(ms, 5), "bytes_per_launch": by,
            "achieved_gbs": round(gbs, 1), "frac_hbm": round(gbs / hbm, 4)}
    if T == 8 or which == 1:
        tf = fl / (ms / 1e3) / 1e12
        line.update({"fp64_tflops": round(tf, 4), "frac_fp64": round(tf / fp64_tflops, 4)})
    return line


def roofline(ctx, flush, peaks, fp64_tflops):
    """The dominant kernel of the headline step (the FP64 smoother half-sweep
    on the level-3 grid, 16 samples), each launch timed cold (L2 flushed
    before it). Achieved = the method's bytes per updated cell (26 FP64
    values) x the cells of one launch / its duration, against the measured
    HBM copy bandwidth; the FP64 pipe, its co-limit on GB300, beside it."""
    hbm = peaks["hbm_gbs"]
    ms, by, fl = ctx.time_kernel(3, 0, 0, reps=50, flush=flush)
    gbs = by / (ms / 1e3) / 1e9
    tf = fl / (ms / 1e3) / 1e12
    ms2, by2, fl2 = ctx.time_kernel(3, 0, 1, reps=20, flush=flush)
    return {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s",
            "frac": round(gbs / hbm, 4), "traffic": None,
            "peak_source": peaks.get("source", "MEASURED_PEAKS.json hbm_gbs (measured)"),
            "kernel": "k_smooth<double> red half-sweep, level 3 (256x128 cells x 16 samples), "
                      "L2 flushed before each launch",
            "bytes_per_launch": by, "ms_per_launch": round(ms, 5),
            "fp64_pipe": {"achieved_tflops": round(tf, 4), "peak_tflops": round(fp64_tflops, 4),
                          "frac": round(tf / fp64_tflops, 4),
                          "peak_source": "measured in this run (henry_probe_fp64)"},
            "second": {"kernel": "k_resjac<double> (FP64 residual + Jacobian, level 3), cold",
                       "ms_per_launch": round(ms2, 5),
                       "achieved_gbs": round(by2 / (ms2 / 1e3) / 1e9, 1),
                       "fp64_tflops": round(fl2 / (ms2 / 1e3) / 1e12, 4),
                       "frac_fp64": round(fl2 / (ms2 / 1e3) / 1e12 / fp64_tflops, 4)}}


def streaming(flush, hbm, fp64_tflops):
    """The smoother and residual kernels on the 1024x512 grid (level 5 of the
    six-level configuration) with 16 samples: 4.2 M cell updates per
    half-sweep, operands several times the L2. A context whose level 0 is
    that grid (with level 5's time step) runs 2 steps to fill the operators,
    then the kernels are replayed cold."""
    from paper_2403_17018_gb300 import binding as hb
    from paper_2403_17018_gb300.inputs import xi_batch
    import torch
    out = {}
    tau5 = 43200.0 / (24 << 5)
    xi = torch.from_numpy(xi_batch(5, 0, 16)).cuda()
    for prec, name, T in ((hb.PREC_FP32_MG, "fp32mg", 4), (hb.PREC_FP64, "fp64", 8)):
        ctx = hb.Context(hb.default_config(nx0=1024, ny0=512, nt0=2, T=2 * tau5, nlevels=1,
                                           precision=prec))
        ctx.solve(0, xi)
        tname = "float" if T == 4 else "double"
        out[name] = {
            "smoother": kernel_line(ctx, 0, 0, 20, flush, hbm, fp64_tflops, T,
                                    f"k_smooth<{tname}> red half-sweep, 1024x512 x 16, cold"),
            "residual_jacobian": kernel_line(ctx, 0, 1, 10, flush, hbm, fp64_tflops, T,
                                             f"k_resjac<{tname}>, 1024x512 x 16, cold")}
        ctx.close()
    return out


def adjoint_timing(rank, world, B=256, ckpt=8):
    """Discrete adjoint of the configuration with 128x64 cells, 96 steps and
    256 samples (checkpoint every 8 steps): dQ_S/dxi and dQ_S/dlogK for
    every sample, FP32 multigrid inside the FP64 defect corrections, timed
    with CUDA events against the forward solve of the same batch."""
    import torch
    from paper_2403_17018_gb300 import binding as hb
    from paper_2403_17018_gb300.inputs import logk_perturbation, xi_batch
    ctx = hb.Context(hb.default_config(nlevels=3, precision=hb.PREC_FP32_MG, vcycles=3))
    xi = torch.from_numpy(xi_batch(2, rank * B, B)).cuda()
    lk = torch.from_numpy(logk_perturbation(64, 128, B, seed=2403017018 + rank)).cuda()
    ctx.adjoint(2, xi, logk=lk, ckpt_every=ckpt)          # warm-up: workspaces, graphs
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    torch.cuda.synchronize()
    ev[0].record()
    ctx.solve(2, xi, logk=lk)
    ev[1].record()
    q, g, gl, st = ctx.adjoint(2, xi, logk=lk, ckpt_every=ckpt)
    ev[2].record()
    torch.cuda.synchronize()
    fwd, adj = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
    ctx.close()
    return {"config": f"128x64 cells, 96 steps, {B} samples per GPU, checkpoint every {ckpt} "
                      "steps, QoI Q_S, gradients w.r.t. xi and per-cell log K (8192)",
            "gradients_per_s": round(B * world / (adj / 1e3), 2), "adjoint_ms": round(adj, 1),
            "forward_ms": round(fwd, 1), "adjoint_over_forward": round(adj / fwd, 2),
            "failed": int((st != 0).sum().item())}


def mlmc_wall_times():
    """Second half of the metric: adaptive MLMC to RMSE 1e-3 on c at the
    three points, 6 levels (32x16 .. 1024x512 cells, 24..768 steps), 6
    random variables, identical seeds, with FP32 multigrid and with FP64
    multigrid; schedules autotuned first (tuning time reported apart)."""
    from paper_2403_17018_gb300 import mlmc
    cands = {"vcycles": (2, 3), "nu": ((2, 2),), "small_cells": (128, 512), "jac_lag": (0, 30),
             "tb_cells": (0, 2048), "keep_lags": (30, 100)}
    out = {"config": "6 levels 32x16..1024x512, 6 random variables, RMSE 1e-3 on c at "
                     "(1.40,0.05), (1.65,0.25), (1.90,0.50), variance budget eps^2/2, "
                     "levels on concurrent streams"}
    for prec in ("fp32mg", "fp64"):
        r = mlmc.tuned_run(levels=6, eps=1e-3, n_xi=6, precision=prec, tune=True,
                           candidates=cands)
        out[prec] = {"wall_s": round(r["wall_s"], 2), "tuning_s": round(r["tuning_s"], 1),
                     "rmse": [round(r["rmse"][q], 7) for q in (3, 4, 5)],
                     "estimate": [round(r["estimate"][q], 6) for q in (3, 4, 5)],
                     "samples": r["n"], "rounds": r["rounds"], "failed": r["failed"],
                     "seconds_per_pair": [float(f"{x:.3g}") for x in r["seconds_per_pair"]],
                     "schedules": {str(k): sched_str(v) for k, v in r["schedules"].items()}}
    out["fp32mg_speedup"] = round(out["fp64"]["wall_s"] / out["fp32mg"]["wall_s"], 3)
    return out


# ---------------------------------------------------------------------------
# CPU oracle (cpu_baseline of the GPU arm, and the reference arm)
# ---------------------------------------------------------------------------
def _cpu_init():
    # one numpy thread per worker process: the pool supplies the parallelism
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"


def _cpu_solve(level, xi_level, sample, mid, half=False):
    """One whole oracle solve of `level` for sample `sample` of xi_level's
    stream (half: only the first half of the horizon); returns (level,
    seconds, state at step nt/2 or None)."""
    from oracle import henry as H
    from paper_2403_17018_gb300.inputs import xi_batch
    g = H.level_grid(level)
    if half:
        g = H.Grid(g.nx, g.ny, g.nt // 2, g.T / 2)
    t = time.perf_counter()
    r = H.solve(g, H.Physics(), xi_batch(xi_level, sample, 1)[0], keep_states=mid)
    dt = time.perf_counter() - t
    if not mid:
        return level, dt, None
    return level, dt, (r["states"][-1] if half else r["states"][g.nt // 2])


def _cpu_steps(level, xi_level, sample, coarse_state, nsteps):
    """nsteps implicit steps of `level` from the level-(level-1) state at the
    middle of the horizon (c and the non-hydrostatic part of p transferred
    piecewise constant), after one untimed step that settles the transfer;
    returns (level, seconds per step x steps of the level)."""
    import numpy as np
    from oracle import henry as H
    from paper_2403_17018_gb300.inputs import xi_batch
    ph = H.Physics()
    g = H.level_grid(level)
    gc = H.level_grid(level - 1)
    pc, cc = coarse_state
    p = H.hydrostatic_guess(g, ph) + H.prolong_constant(pc - H.hydrostatic_guess(gc, ph))
    c = np.clip(H.prolong_constant(cc), 0.0, 1.0)
    f = H.fields(g, ph, xi_batch(xi_level, sample, 1)[0])
    p, c, _ = H.newton_step(g, ph, f, p, c, c.copy())
    t = time.perf_counter()
    for _ in range(nsteps):
        p, c, _ = H.newton_step(g, ph, f, p, c, c.copy())
    return level, (time.perf_counter() - t) / nsteps * g.nt


def cpu_pool(cores):
    import multiprocessing as mp
    return mp.get_context("spawn").Pool(cores, initializer=_cpu_init)


def pair_rate(solve_s, cores):
    """Level-pair solves/s of the workload from per-solve seconds of each
    level (a pair = fine solve at l + coarse solve at l-1) on `cores` cores."""
    pair = {l: solve_s[l] + (solve_s[l - 1] if l > 0 else 0.0) for l in LEVELS}
    busy = sum(BATCH[l] * pair[l] for l in LEVELS) / cores
    return sum(BATCH.values()) / busy, pair


def cpu_baseline():
    """The FP64 oracle on every core of this host (a process per core):
    whole solves of levels 0, 1 and 2 (one per core each; the level-2 solves
    keep their state at mid-horizon), then 2 implicit steps of level 3 per
    core from those mid-horizon states (after one settling step), scaled to
    the 192 steps of a level-3 solve."""
    cores = len(os.sched_getaffinity(0))
    t0 = time.perf_counter()
    times = {l: [] for l in LEVELS}
    mids = []
    with cpu_pool(cores) as pool:
        jobs = [pool.apply_async(_cpu_solve, (l, 3 if l == 2 else l, s, l == 2))
                for l in (2, 1, 0) for s in range(cores)]
        for j in jobs:
            l, dt, mid = j.get()
            times[l].append(dt)
            if mid is not None:
                mids.append(mid)
        jobs = [pool.apply_async(_cpu_steps, (3, 3, s, mids[s], 2)) for s in range(len(mids))]
        for j in jobs:
            l, dt = j.get()
            times[l].append(dt)
    solve_s = {l: sum(v) / len(v) for l, v in times.items()}
    value, pair = pair_rate(solve_s, cores)
    return {"value": round(value, 6), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": (f"numpy/scipy FP64 oracle, one process per core ({cores}): {cores} whole "
                       f"solves each of levels 0, 1, 2; level 3: 2 steps per core from the "
                       f"level-2 states at mid-horizon, scaled to 192 steps; wall "
                       f"{time.perf_counter() - t0:.1f} s"),
            "solve_seconds": {f"L{l}": round(solve_s[l], 4) for l in LEVELS},
            "pair_seconds": {f"L{l}": round(pair[l], 4) for l in LEVELS}}


def reference_levels(W, K):
    """Levels of the reference arm's warm-up and timed steps: warm-up step w
    runs level w mod 4, timed step k continues the cycle with level
    (W + k) mod 4; the levels neither list reaches are measured once more
    outside the timed steps (the third list)."""
    warm = [w % 4 for w in range(W)]
    timed = [(W + k) % 4 for k in range(K)]
    extra = [l for l in LEVELS if l not in warm and l not in timed]
    return warm, timed, extra


def run_reference(args):
    """The oracle on every host core, on this workload's config and metric:
    warm-up step w runs level w mod 4 and timed step k level (W + k) mod 4
    on every core (levels 0 and 1: whole solves;
    level 2: 12 steps, level 3: 2 steps, each from mid-horizon states of the
    level below prepared in the first warm-up step and scaled to the level's
    step count). value = pairs/s of the workload from the per-level solve
    times of the timed steps."""
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    K, W = args.steps, max(args.warmup, 1)
    cores = len(os.sched_getaffinity(0))
    seen = {l: [] for l in LEVELS}
    step_ms = []
    with cpu_pool(cores) as pool:
        # mid-horizon states: level 1 (for level-2 steps), level 2 (for level 3)
        mids = {}
        for l in (1, 2):
            jobs = [pool.apply_async(_cpu_solve, (l, l + 1, s, True, True)) for s in range(cores)]
            mids[l] = [j.get()[2] for j in jobs]

        def one_step(level):
            if level <= 1:
                jobs = [pool.apply_async(_cpu_solve, (level, level, s, False)) for s in range(cores)]
                return [j.get()[1] for j in jobs]
            n = 12 if level == 2 else 2
            jobs = [pool.apply_async(_cpu_steps, (level, level, s, mids[level - 1][s], n))
                    for s in range(cores)]
            return [j.get()[1] for j in jobs]

        warm_levels, timed_levels, extra_levels = reference_levels(W, K)
        for level in warm_levels:
            seen[level] += one_step(level)
        timed = {l: [] for l in LEVELS}
        for level in timed_levels:
            t0 = time.perf_counter()
            timed[level] += one_step(level)
            step_ms.append((time.perf_counter() - t0) * 1e3)
        for level in extra_levels:
            seen[level] += one_step(level)
    solve_s = {l: (sum(timed[l]) / len(timed[l])) if timed[l] else sum(seen[l]) / len(seen[l])
               for l in LEVELS}
    value, pair = pair_rate(solve_s, cores)
    sample = (f"numpy/scipy FP64 oracle, one process per core ({cores}); warm-up step w: level "
              f"w mod 4, timed step k: level (W + k) mod 4 "
              f"on every core (levels 0, 1 whole solves; level 2: 12 steps, level 3: 2 steps, "
              f"from mid-horizon states, scaled to 96 / 192 steps)")
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT,
            "n_gpus": 0, "steps": K, "warmup": W,
            "ms_per_step": round(sum(step_ms) / max(len(step_ms), 1), 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded SplitMix64 xi ~ U[-1,1]^3)", "config": CONFIG,
            "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": cores,
                             "kind": "oracle", "sample": sample},
            "solve_seconds": {f"L{l}": round(solve_s[l], 4) for l in LEVELS},
            "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    import __graft_entry__
    __graft_entry__.build()
    from paper_2403_17018_gb300 import binding as hb
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
        peaks["source"] = "MEASURED_PEAKS.json hbm_gbs (measured)"
    except OSError:
        peaks = {"hbm_gbs": 6800.0, "source": "fallback 6.8 TB/s (no measured peaks file)"}
    hbm = peaks["hbm_gbs"]
    flush_buf = torch.empty(FLUSH_FLOATS, dtype=torch.float32, device="cuda")
    flush = lambda: flush_buf.add_(1.0)
    xis = make_inputs(rank)
    K, W = args.steps, max(args.warmup, 3)
    pairs_per_step = sum(BATCH.values())
    loop = hb.LOOP_HOST if args.loop == "host" else hb.LOOP_GRAPH

    # ---- headline: FP64 multigrid ------------------------------------------
    sched64, tune64_s = tune_schedules("fp64")
    wl = Workload(hb.PREC_FP64, sched64, loop, args.pairs)
    clocks = ClockSampler(local)
    clocks.start()
    ms, per_step, launches, stats = time_steps(wl, xis, K, W, barrier, flush)
    clk = clocks.stop()
    t_max = ms
    if dist is not None:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_max = float(t.item())
    value = pairs_per_step * world * K / (t_max / 1e3)
    bad = sum(int((wl.out[l][4] != 0).sum().item()) for l in LEVELS)

    # ---- e2e through the public API with pinned host buffers ---------------
    host = {"xi": {l: xis[l].cpu().pin_memory() for l in LEVELS},
            "qf": {l: torch.empty((BATCH[l], hb.NQ), dtype=torch.float64).pin_memory() for l in LEVELS},
            "qc": {l: torch.empty((BATCH[l], hb.NQ), dtype=torch.float64).pin_memory() for l in LEVELS},
            "st": {l: torch.empty((BATCH[l],), dtype=torch.int32).pin_memory() for l in LEVELS}}
    ms_e2e, _, _, _ = time_steps(wl, xis, K, 1, barrier, flush, host=host)
    h2d = sum(BATCH[l] * 3 * 8 for l in LEVELS)
    d2h = sum(BATCH[l] * (hb.NQ * 8 * (2 if l > 0 else 1) + 4) for l in LEVELS)
    e2e_value = pairs_per_step * world * K / (ms_e2e / 1e3)

    extra = not args.no_extra
    rates64 = per_level_rates(wl, xis) if extra else None
    levels64 = whole_level(wl, xis, hbm) if extra else None
    fp64_tflops = hb.probe_fp64(reps=40)
    roof = roofline(wl.ctx, flush_buf, peaks, fp64_tflops)
    wl.close()

    # ---- FP32 multigrid inside FP64 defect correction, same workload -------
    fp32 = None
    if not args.no_fp32:
        sched32, tune32_s = tune_schedules("fp32mg")
        wl32 = Workload(hb.PREC_FP32_MG, sched32, loop, args.pairs)
        ms32, _, launches32, _ = time_steps(wl32, xis, K, W, barrier, flush)
        fp32 = {"value": round(pairs_per_step * world * K / (ms32 / 1e3), 2),
                "ms_per_step": round(ms32 / K, 2), "per_level": per_level_rates(wl32, xis),
                "gpu_launches": launches32,
                "schedule": {f"L{l}": sched_str(s) for l, s in sched32.items()},
                "tuning_s": round(tune32_s, 1),
                "whole_level": whole_level(wl32, xis, hbm),
                "smoother_cold": kernel_line(wl32.ctx, 3, 0, 50, flush_buf, hbm, fp64_tflops,
                                             4, "k_smooth<float> red half-sweep, level 3 "
                                                "(256x128 x 16), cold")}
        wl32.close()

    stream = streaming(flush_buf, hbm, fp64_tflops) if extra else None
    adj = None if args.no_adjoint else adjoint_timing(rank, world)
    mlmc_res = None
    if not args.no_mlmc:
        mlmc_res = mlmc_wall_times() if world == 1 else {"skipped": "single-GPU measurement"}

    cpu = None
    if not args.no_cpu and rank == 0 and world == 1:
        cpu = cpu_baseline()

    line = {"metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world,
            "steps": K, "warmup": W, "ms_per_step": round(t_max / K, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded SplitMix64 xi ~ U[-1,1]^3)",
            "config": dict(CONFIG, parallelism=f"{world} GPU(s), samples sharded, 4 level streams"),
            "schedule": {f"L{l}": sched_str(s) for l, s in sched64.items()},
            "tuning_s": round(tune64_s, 1),
            "loop": args.loop, "pairs": args.pairs,
            "per_level": rates64, "whole_level": levels64, "failed_samples": bad,
            "roofline": roof, "streaming": stream, "clocks": clk, "gpu_launches": launches,
            "e2e": {"value": round(e2e_value, 2), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "fp32_mg": fp32, "mlmc": mlmc_res, "adjoint": adj, "cpu_baseline": cpu,
            "step_ms": [round(x, 2) for x in per_step]}
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
