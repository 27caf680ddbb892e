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


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-fp32", action="store_true", help="skip the FP32-multigrid variant")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the discrete-adjoint timing")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    return ap.parse_args()


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
# GPU arm
# ---------------------------------------------------------------------------
def make_inputs(rank, n_xi=3):
    import torch
    from paper_2403_17018_gb300.inputs import xi_batch
    xis = {}
    for l in LEVELS:
        B = BATCH[l]
        xis[l] = torch.from_numpy(xi_batch(l, rank * B, B, n_xi=n_xi)).cuda()
    return xis


class Workload:
    """One context per level (its schedule autotuned), one stream per level."""

    def __init__(self, precision, schedules):
        import torch
        from paper_2403_17018_gb300 import binding as hb
        self.hb = hb
        self.ctxs = {}
        for l in LEVELS:
            sc = schedules[l]
            cfg = hb.default_config(nlevels=4, precision=precision, vcycles=sc["vcycles"],
                                    nu1=sc["nu1"], nu2=sc["nu2"],
                                    mg_small_cells=sc.get("mg_small_cells", 512),
                                    jac_lag=sc.get("jac_lag", 0))
            self.ctxs[l] = hb.Context(cfg)
        self.cfg = self.ctxs[0].cfg
        self.streams = {l: torch.cuda.Stream() for l in LEVELS}
        self.out = {}

    def launch_count(self):
        return sum(c.launch_count() for c in self.ctxs.values())

    def step(self, xis, host=None):
        """Enqueue all level pairs; then merge level statistics (synchronous
        per level). With `host` = dict of pinned buffers, copy xi in from
        host memory and the QoIs back to host memory inside the step."""
        import torch
        main = torch.cuda.current_stream()
        ev = torch.cuda.Event()
        ev.record(main)
        for l in LEVELS:
            s = self.streams[l]
            s.wait_event(ev)
            with torch.cuda.stream(s):
                xi = xis[l]
                if host is not None:
                    xi.copy_(host["xi"][l], non_blocking=True)
                self.out[l] = self.ctxs[l].sample_pairs(l, xi, stream=s)
        stats = {}
        for l in LEVELS:
            s = self.streams[l]
            qf, qc, _, _, st = self.out[l]
            S = self.hb.LevelStats()
            self.ctxs[l].level_stats(l, qf, qc, st, S, stream=s)
            stats[l] = S
            if host is not None:
                with torch.cuda.stream(s):
                    host["qf"][l].copy_(qf, non_blocking=True)
                    if qc is not None:
                        host["qc"][l].copy_(qc, non_blocking=True)
                    host["st"][l].copy_(st, non_blocking=True)
        for l in LEVELS:
            e = torch.cuda.Event()
            e.record(self.streams[l])
            main.wait_event(e)
        return stats


def tune_schedules(precision_name):
    """Autotuned schedule per level: V-cycles per iteration x smoothing sweeps
    x shared-memory V-cycle threshold, then the operator reuse factor, each
    timed on one solve of the level over the whole horizon."""
    from paper_2403_17018_gb300 import autotune as A
    A.CANDIDATES = {"vcycles": (2, 3), "nu": ((2, 2), (3, 3)), "small_cells": (0, 128, 512),
                    "jac_lag": (0, 10, 30)}
    out = {}
    for l in LEVELS:
        best, _ = A.tune_level(l, BATCH[l], precision_name, steps=None, reps=1, splits=(1,))
        out[l] = best
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


def flush_l2(buf):
    buf.add_(1.0)


def time_steps(wl, xis, K, W, barrier, flush, host=None):
    import torch
    for _ in range(W):
        wl.step(xis, host)
    torch.cuda.synchronize()
    total_ms = 0.0
    per_step = []
    n0 = wl.launch_count()
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


def per_level_rates(wl, xis, reps=1):
    """Solves/s of each level's pair batch run alone (device time)."""
    import torch
    rates = {}
    for l in LEVELS:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            wl.ctxs[l].sample_pairs(l, xis[l])
        e1.record()
        torch.cuda.synchronize()
        rates[f"L{l}"] = round(BATCH[l] * reps / (e0.elapsed_time(e1) / 1e3), 2)
    return rates


FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12   # SMs x FP64 FMA/clk x 2 FLOP x max clock

# DRAM bytes (read + write) of one launch of the roofline kernels, from the
# ncu captures summarised in profiles/k_smooth_fp64_level3_256x128_b16.md and
# profiles/k_smooth_fp32_level5_1024x512_b16.md; valid while the kernels are
# unchanged since those captures.
NCU_TRAFFIC_BYTES = {"k_smooth<double> L3": 41820160 + 64512}


def roofline(wl, peaks):
    """Dominant kernel of the FP64 form (ncu launch list, level 3: the
    smoother is ~56% of device time): the FP64 red-black block Gauss-Seidel
    half-sweep on the finest grid of level 3, bound by the FP64 pipe on
    GB300 (FP64 is 1/64 of FP32), so reported against the FP64 peak derived
    from unit counts and clock. The FP64 residual/Jacobian kernel, next in
    the list, is reported beside it."""
    ms, by, fl = wl.ctxs[3].time_kernel(3, 0, 0, reps=50)
    ach = fl / (ms / 1e3) / 1e12
    ms2, by2, fl2 = wl.ctxs[3].time_kernel(3, 0, 1, reps=20)
    return {"bound": "alu", "achieved": round(ach, 4), "peak": round(FP64_PEAK_TFLOPS, 4),
            "unit": "TFLOP/s", "frac": round(ach / FP64_PEAK_TFLOPS, 4),
            "traffic": NCU_TRAFFIC_BYTES["k_smooth<double> L3"],
            "kernel": "k_smooth<double> red half-sweep (level 3: 256x128 cells x 16 samples)",
            "flops_per_launch": fl, "bytes_per_launch": by, "ms_per_launch": round(ms, 5),
            "achieved_gbs": round(by / (ms / 1e3) / 1e9, 1),
            "peak_note": "derived: 152 SMs x 2 FP64 FMA/clk x 2 FLOP x 2.07 GHz "
                         "(probe measured 1.19 TFLOP/s)",
            "second": {"kernel": "k_resjac<double> (FP64 residual + Jacobian, level 3)",
                       "bound": "alu", "ms_per_launch": round(ms2, 5),
                       "achieved_tflops": round(fl2 / (ms2 / 1e3) / 1e12, 4),
                       "frac": round(fl2 / (ms2 / 1e3) / 1e12 / FP64_PEAK_TFLOPS, 4)}}


def smoother_roofline(wl, peaks):
    ms, by, fl = wl.ctxs[3].time_kernel(3, 0, 0, reps=50)
    ach = by / (ms / 1e3) / 1e9
    return {"bound": "hbm", "achieved": round(ach, 1), "peak": peaks.get("hbm_gbs", 6800.0),
            "unit": "GB/s", "frac": round(ach / peaks.get("hbm_gbs", 6800.0), 4),
            "kernel": "k_smooth<float> red half-sweep (level 3, 256x128 cells x 16 samples)",
            "ms_per_launch": round(ms, 5), "bytes_per_launch": by}


def cpu_baseline(budget_s=20.0):
    """The FP64 oracle timed on this host on a bounded sample of the
    workload: whole level-0 solves and level-1 pairs, and a few time steps of
    one level-2 and one level-3 solve scaled to their full step counts."""
    import numpy as np
    from oracle import henry as H
    from paper_2403_17018_gb300.inputs import xi_batch
    ph = H.Physics()
    t_solve = {}
    t0 = time.perf_counter()
    # level 0: whole solves
    xi = xi_batch(0, 0, 4)
    t = time.perf_counter()
    n0 = 0
    for b in range(4):
        H.solve(H.level_grid(0), ph, xi[b])
        n0 += 1
        if time.perf_counter() - t0 > budget_s / 4:
            break
    t_solve[0] = (time.perf_counter() - t) / n0
    # level 1: one whole solve
    t = time.perf_counter()
    H.solve(H.level_grid(1), ph, xi_batch(1, 0, 1)[0])
    t_solve[1] = time.perf_counter() - t
    # levels 2, 3: two steps each, scaled by the step count
    for l, ns in ((2, 3), (3, 2)):
        g = H.level_grid(l)
        gs = H.Grid(g.nx, g.ny, ns, g.tau * ns)
        t = time.perf_counter()
        H.solve(gs, ph, xi_batch(l, 0, 1)[0])
        t_solve[l] = (time.perf_counter() - t) / ns * g.nt
    pair = {0: t_solve[0]}
    for l in (1, 2, 3):
        pair[l] = t_solve[l] + t_solve[l - 1]
    step_s = sum(BATCH[l] * pair[l] for l in LEVELS)
    total = sum(BATCH.values())
    return {"value": round(total / step_s, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": ("numpy/scipy FP64 oracle, 1 core: %d level-0 solves, 1 level-1 solve, 3 "
                       "level-2 and 2 level-3 time steps scaled to 96/192 steps; seconds per "
                       "pair L0..L3 = %s; wall %.1f s" % (n0, [round(pair[l], 3) for l in LEVELS],
                                                          time.perf_counter() - t0)),
            "pair_seconds": {f"L{l}": round(pair[l], 4) for l in LEVELS}}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    K, W = args.steps, args.warmup
    # each step: a bounded sample of the workload on the oracle (a few seconds)
    import numpy as np
    from oracle import henry as H
    from paper_2403_17018_gb300.inputs import xi_batch
    ph = H.Physics()
    for _ in range(W):
        H.solve(H.level_grid(0), ph, xi_batch(0, 0, 1)[0])
    t = time.perf_counter()
    for k in range(K):
        H.solve(H.level_grid(0), ph, xi_batch(0, k, 1)[0])
    t_l0 = (time.perf_counter() - t) / K
    base = cpu_baseline(budget_s=10.0)
    val = base["value"]
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": 0,
            "steps": K, "warmup": W, "ms_per_step": round(sum(BATCH.values()) / val * 1e3, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": base["sample"] + "; level-0 solve %.3f s" % t_l0},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
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
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except OSError:
        peaks = {"hbm_gbs": 6800.0, "note": "fallback"}
    flush_buf = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2
    flush = lambda: flush_l2(flush_buf)
    xis = make_inputs(rank)
    K, W = args.steps, max(args.warmup, 3)
    pairs_per_step = sum(BATCH.values())

    # ---- headline: FP64 multigrid ------------------------------------------
    sched64 = tune_schedules("fp64")
    wl = Workload(hb.PREC_FP64, sched64)
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
    rates64 = per_level_rates(wl, xis)
    roof = roofline(wl, peaks)
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

    # ---- FP32 multigrid inside FP64 defect correction, same workload -------
    fp32 = None
    if not args.no_fp32:
        sched32 = tune_schedules("fp32mg")
        wl32 = Workload(hb.PREC_FP32_MG, sched32)
        ms32, _, launches32, _ = time_steps(wl32, xis, K, W, barrier, flush)
        fp32 = {"value": round(pairs_per_step * world * K / (ms32 / 1e3), 2),
                "ms_per_step": round(ms32 / K, 2), "per_level": per_level_rates(wl32, xis),
                "gpu_launches": launches32,
                "schedule": {f"L{l}": f"V({s['nu1']},{s['nu2']}) x{s['vcycles']} "
                                      f"smem<={s['mg_small_cells']} lag={s['jac_lag']}"
                             for l, s in sched32.items()},
                "smoother_roofline": smoother_roofline(wl32, peaks)}

    adj = None
    if not args.no_adjoint:
        adj = adjoint_timing(rank, world)

    cpu = None
    if not args.no_cpu and rank == 0 and world == 1:
        cpu = cpu_baseline()

    line = {"metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world,
            "steps": K, "warmup": W, "ms_per_step": round(t_max / K, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded SplitMix64 xi ~ U[-1,1]^3)",
            "config": {"workload": WORKLOAD, "levels": list(LEVELS),
                       "batch": [BATCH[l] for l in LEVELS],
                       "multigrid": "FP64, autotuned per level: " + ", ".join(
                           f"L{l} V({s['nu1']},{s['nu2']}) x{s['vcycles']} smem<={s['mg_small_cells']} "
                           f"lag={s['jac_lag']}"
                           for l, s in sched64.items()),
                       "newton_rtol": wl.cfg.newton_rtol, "newton_atol": wl.cfg.newton_atol,
                       "l2": "flushed between timed steps (256 MB write)",
                       "parallelism": f"{world} GPU(s), samples sharded, 4 level streams"},
            "per_level": rates64, "failed_samples": bad,
            "roofline": roof, "clocks": clk, "gpu_launches": launches,
            "e2e": {"value": round(e2e_value, 2), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "fp32_mg": fp32, "adjoint": adj, "cpu_baseline": cpu,
            "step_ms": [round(x, 2) for x in per_step]}
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
