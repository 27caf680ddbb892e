"""Adaptive multilevel Monte Carlo driver (arxiv 2403.17018, section 3).

The estimator of E[g_L] is the telescoping sum Y = sum_l Y_l (Eqs. EgL, A),
Y_l the mean of g_l - g_{l-1} over m_l independent level pairs (g_{-1} = 0),
with Var Y = sum_l V_l / m_l (Eq. goal_variance). For a target root mean
square error eps the variance budget is eps^2 / 2 (Eq. var_error) and the
cost-optimal sample numbers are

    m_l = 2 eps^-2 sqrt(V_l / s_l) sum_i sqrt(V_i s_i)          (Eq. M_ell)

with V_l the variance of g_l - g_{l-1} and s_l the cost of one pair. Here
s_l is the measured GPU time per pair of the last batch of level l and
V_l the largest variance over the selected QoIs. The driver starts from a
pilot, recomputes m_l from the running statistics, draws the missing
samples, and stops when no level needs more. The bias is estimated from
the finest correction, |E Y_L| / (2^alpha - 1), with alpha fitted to
log2 |E Y_l| (the build refines by 2 per level; the paper fits in log_4).

Samples are drawn by a sampler object; GpuSampler runs level pairs through
the C ABI (henry_sample_pairs + mlmc_level_stats). Sample i of level l
always gets the same xi, so a run is reproducible and can be resumed from
its saved state. Under torch.distributed each rank draws a disjoint slice
of every batch and the per-level statistics are merged with Chan's formula.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import sys
import time
from dataclasses import dataclass, field

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

NQ = 22


@dataclass
class LevelState:
    """Running statistics of one level: count, means and M2 (sum of squared
    deviations) of g_l and of g_l - g_{l-1}, cost in seconds and pairs."""
    n: int = 0
    mean_f: np.ndarray = field(default_factory=lambda: np.zeros(NQ))
    m2_f: np.ndarray = field(default_factory=lambda: np.zeros(NQ))
    mean_d: np.ndarray = field(default_factory=lambda: np.zeros(NQ))
    m2_d: np.ndarray = field(default_factory=lambda: np.zeros(NQ))
    seconds: float = 0.0
    timed_pairs: int = 0
    failed: int = 0
    drawn: int = 0           # next sample index of this level's stream

    def var_d(self):
        return self.m2_d / (self.n - 1) if self.n > 1 else np.full(NQ, np.inf)

    def var_f(self):
        return self.m2_f / (self.n - 1) if self.n > 1 else np.full(NQ, np.inf)

    def to_json(self):
        return {k: (v.tolist() if isinstance(v, np.ndarray) else v) for k, v in self.__dict__.items()}

    @staticmethod
    def from_json(d):
        s = LevelState()
        for k, v in d.items():
            setattr(s, k, np.array(v) if isinstance(v, list) else v)
        return s


def chan_merge(a: LevelState, n_b: int, mean_f, m2_f, mean_d, m2_d) -> None:
    """Merge a batch's statistics into `a` (Chan, Golub and LeVeque)."""
    if n_b == 0:
        return
    n = a.n + n_b
    for mean, m2, mb, m2b in ((a.mean_f, a.m2_f, mean_f, m2_f), (a.mean_d, a.m2_d, mean_d, m2_d)):
        d = np.asarray(mb) - mean
        m2 += np.asarray(m2b) + d * d * (a.n * n_b / n)
        mean += d * (n_b / n)
    a.n = n


def allocate(V, s, eps, var_budget_fraction=0.5):
    """Eq. M_ell: m_l = eps^-2 / f sqrt(V_l/s_l) sum_i sqrt(V_i s_i), rounded up."""
    V = np.asarray(V, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    total = float(np.sum(np.sqrt(V * s)))
    m = np.sqrt(V / s) * total / (var_budget_fraction * eps * eps)
    return np.ceil(m * (1 - 1e-12)).astype(np.int64)


def fit_alpha(means):
    """Weak rate alpha from |E Y_l| ~ 2^(-alpha l), l >= 1 (least squares)."""
    l = np.arange(1, len(means))
    y = np.abs(np.asarray(means[1:], dtype=np.float64))
    ok = y > 0
    if ok.sum() < 2:
        return 1.0
    A = np.vstack([-l[ok], np.ones(ok.sum())]).T
    (alpha, _), *_ = np.linalg.lstsq(A, np.log2(y[ok]), rcond=None)
    return float(max(alpha, 0.5))


def levels_needed(means_d, eps):
    """Finest level from the weak-error model (Eq. weak_error_model, Eq.
    num_levels): fit log_4 |E Y_l| = -alpha l + zeta over l >= 1, read the
    bias of level L as the tail of the finer corrections, c1 4^(-alpha L)
    with c1 = 4^zeta / (4^alpha - 1), and return the smallest L with
    c1 4^(-alpha L) <= eps / sqrt(2) (eps absolute), with (alpha, c1)."""
    l = np.arange(1, len(means_d))
    y = np.abs(np.asarray(means_d[1:], dtype=np.float64))
    ok = y > 0
    if ok.sum() < 2:
        return None, None, None
    A = np.vstack([-l[ok], np.ones(ok.sum())]).T
    (alpha, zeta), *_ = np.linalg.lstsq(A, np.log(y[ok]) / math.log(4.0), rcond=None)
    alpha = max(float(alpha), 0.25)          # no slower than h^(1/2)
    c1 = 4.0 ** float(zeta) / (4.0 ** alpha - 1.0)
    L = -math.log(eps / (math.sqrt(2.0) * c1), 4.0) / alpha
    return max(0, int(math.ceil(L - 1e-12))), alpha, c1


class GpuSampler:
    """Level pairs on the GPU through the C ABI; statistics merged on device.

    `schedules` (level -> {vcycles, nu1, nu2, mg_small_cells, jac_lag}, e.g. from the
    autotuner) gives every level its own context and multigrid schedule.
    Each level has its own CUDA stream, so `batches` can run the pending
    pairs of all levels at the same time."""

    def __init__(self, cfg, rank=0, world=1, schedules=None):
        import torch
        from paper_2403_17018_gb300 import binding as hb
        self.torch = torch
        self.hb = hb
        self.n_xi = cfg.n_xi
        self.rank, self.world = rank, world
        self.ctxs = {}
        shared = None
        for l in range(cfg.nlevels):
            sc = (schedules or {}).get(l)
            if sc is None:
                shared = shared or hb.Context(cfg)
                self.ctxs[l] = shared
            else:
                kw = cfg.as_dict()
                kw.update({k: sc[k] for k in ("vcycles", "nu1", "nu2", "mg_small_cells", "jac_lag",
                                              "res_rows", "mg_tb_cells", "jac_keep") if k in sc})
                self.ctxs[l] = hb.Context(hb.default_config(**kw))
        # one stream per level; the finest levels' pairs are the long chains
        # (most steps, fewest samples), so their streams get the higher
        # scheduling priority and the coarser levels fill the SMs left idle
        least, greatest = torch.cuda.Stream.priority_range()
        self.streams = {l: torch.cuda.Stream(priority=min(least, greatest + cfg.nlevels - 1 - l))
                        for l in range(cfg.nlevels)}

    def _slice(self, first, count):
        lo = first + (count * self.rank) // self.world
        hi = first + (count * (self.rank + 1)) // self.world
        return lo, hi

    def batches(self, requests):
        """Run several (level, first, count) requests at once, one stream per
        level (at most one request per level). Returns, per request, (n,
        mean_f, m2_f, mean_d, m2_d, seconds, failed); seconds is the
        request's device time on its stream (CUDA events)."""
        from paper_2403_17018_gb300.inputs import xi_batch
        torch = self.torch
        assert len({r[0] for r in requests}) == len(requests), "one request per level"
        launched = []
        for level, first, count in requests:
            lo, hi = self._slice(first, count)
            if hi <= lo:
                launched.append(None)
                continue
            s = self.streams[level]
            xi = torch.from_numpy(xi_batch(level, lo, hi - lo, n_xi=self.n_xi)).pin_memory()
            with torch.cuda.stream(s):
                xi_d = xi.to("cuda", non_blocking=True)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(s)
                out = self.ctxs[level].sample_pairs(level, xi_d, stream=s)
                e1.record(s)
            launched.append((level, xi, xi_d, out, e0, e1))
        res = []
        for item in launched:
            if item is None:
                res.append((0, np.zeros(NQ), np.zeros(NQ), np.zeros(NQ), np.zeros(NQ), 0.0, 0))
                continue
            level, _, _, (qf, qc, _, _, st), e0, e1 = item
            S = self.hb.LevelStats()
            self.ctxs[level].level_stats(level, qf, qc, st, S, stream=self.streams[level])
            e1.synchronize()
            failed = int((st != 0).sum().item())
            res.append((S.n, np.array(S.mean_f[:]), np.array(S.m2_f[:]), np.array(S.mean_d[:]),
                        np.array(S.m2_d[:]), e0.elapsed_time(e1) / 1e3, failed))
        return res

    def batch(self, level, first, count):
        """Run pairs first..first+count-1 of `level` (this rank's slice);
        returns (n, mean_f, m2_f, mean_d, m2_d, seconds, failed)."""
        return self.batches([(level, first, count)])[0]


def _merge_ranks(levels, dist):
    """Chan-merge every rank's per-level statistics (a few hundred bytes)."""
    if dist is None:
        return levels
    gathered = [None] * dist.get_world_size()
    dist.all_gather_object(gathered, [s.to_json() for s in levels])
    merged = []
    for l in range(len(levels)):
        m = LevelState(drawn=levels[l].drawn)
        for r in gathered:
            s = LevelState.from_json(r[l])
            chan_merge(m, s.n, s.mean_f, s.m2_f, s.mean_d, s.m2_d)
            m.seconds = max(m.seconds, s.seconds)
            m.timed_pairs = max(m.timed_pairs, s.timed_pairs)
            m.failed += s.failed
        merged.append(m)
    return merged


def run(sampler, L, eps, qois=(3, 4, 5), pilot=None, max_batch=None, var_budget_fraction=0.5,
        max_rounds=20, log=None, dist=None, state=None, concurrent=True, adaptive_levels=False,
        L_start=2, relative=False):
    """Adaptive MLMC on levels 0..L to RMSE eps for the QoIs `qois`.
    With `concurrent` and a sampler that has `batches`, the pending pairs
    of all levels run at the same time (cost per pair then measured under
    sharing, which scales every level's cost alike to first order).

    adaptive_levels: start on levels 0..L_start and add a level whenever the
    weak-error model fitted to the level means (Eq. num_levels) asks for a
    finer one, up to L. relative: eps is relative to E0 = |E g_0| of each
    QoI (the paper's scaling, Eq. scaled_m_l_S), estimated from level 0.

    Returns a dict with the estimate per QoI, Var Y, the bias estimate, the
    RMSE estimate, samples and cost per level and the wall time. `state`
    (from a previous result's "state") resumes a run."""
    L_max = L
    if state is not None:
        L = len(state) - 1
    elif adaptive_levels:
        L = min(L_start, L_max)
    pilot = pilot or [max(16, 512 >> (2 * l)) for l in range(L_max + 1)]
    max_batch = max_batch or [max(32, 16384 >> (2 * l)) for l in range(L_max + 1)]
    local = [LevelState() for _ in range(L + 1)] if state is None else \
        [LevelState.from_json(d) for d in state]
    target = [max(pilot[l], local[l].n) for l in range(L + 1)]
    t_start = time.perf_counter()
    rounds = 0
    qs = list(qois)
    levels = _merge_ranks(local, dist)
    level_choice = []

    def record(l, cnt, out):
        n, mf, m2f, md, m2d, dt, failed = out
        chan_merge(local[l], n, mf, m2f, md, m2d)
        local[l].drawn += cnt
        local[l].seconds = dt
        local[l].timed_pairs = cnt
        local[l].failed += failed

    while True:
        need = [target[l] - levels[l].n for l in range(L + 1)]
        if concurrent and hasattr(sampler, "batches"):
            # waves: the next batch of every level that still needs pairs,
            # all levels at once (one stream per level)
            while any(k > 0 for k in need):
                wave = [(l, local[l].drawn, min(need[l], max_batch[l]))
                        for l in range(L + 1) if need[l] > 0]
                for (l, _, cnt), out in zip(wave, sampler.batches(wave)):
                    record(l, cnt, out)
                    need[l] -= cnt
        else:
            for l in range(L + 1):
                while need[l] > 0:
                    cnt = min(need[l], max_batch[l])
                    record(l, cnt, sampler.batch(l, local[l].drawn, cnt))
                    need[l] -= cnt
        levels = _merge_ranks(local, dist)
        V = np.array([[lv.var_d()[q] for q in qs] for lv in levels])          # [L+1, nq]
        bad = [l for l in range(L + 1) if not np.all(np.isfinite(V[l]))]
        if bad:
            raise RuntimeError(
                f"MLMC: no variance estimate on level(s) {bad} "
                f"(valid samples {[levels[l].n for l in bad]}, failed "
                f"{[levels[l].failed for l in bad]}); the solves of these levels did not converge")
        s = np.array([max(lv.seconds, 1e-9) / max(lv.timed_pairs, 1) for lv in levels])
        eps_q = [eps * abs(levels[0].mean_f[q]) if relative else eps for q in qs]
        m = np.max(np.stack([allocate(V[:, k], s, eps_q[k], var_budget_fraction)
                             for k in range(len(qs))]), axis=0)
        rounds += 1
        if log:
            log({"round": rounds, "n": [lv.n for lv in levels], "m": m.tolist(),
                 "V": V.max(axis=1).tolist(), "s": s.tolist()})
        if adaptive_levels and L < L_max and L >= 2:
            fits = [levels_needed([lv.mean_d[q] for lv in levels], eps_q[k])
                    for k, q in enumerate(qs)]
            chosen = [f[0] for f in fits if f[0] is not None]
            L_need = max(chosen) if chosen else L
            level_choice.append({"levels_fitted": L + 1, "L_needed": L_need,
                                 "alpha4": [f[1] for f in fits], "c1": [f[2] for f in fits]})
            if log:
                log({"round": rounds, "L": L, "L_needed": L_need})
            if L_need > L:
                # one finer level at a time, with its pilot; the next round
                # re-allocates every level with the new level's V and cost
                L += 1
                local.append(LevelState())
                levels = _merge_ranks(local, dist)
                target = [int(max(levels[l].n, m[l])) for l in range(L)] + [pilot[L]]
                continue
        if all(m[l] <= levels[l].n for l in range(L + 1)) or rounds >= max_rounds:
            break
        target = [int(max(levels[l].n, m[l])) for l in range(L + 1)]
    wall = time.perf_counter() - t_start
    n = np.array([lv.n for lv in levels], dtype=np.float64)
    Y = np.sum([lv.mean_d for lv in levels], axis=0)
    varY = np.sum([lv.var_d() / max(lv.n, 1) for lv in levels], axis=0)
    alphas = [fit_alpha([lv.mean_d[q] for lv in levels]) if L >= 2 else 1.0 for q in range(NQ)]
    bias = np.array([abs(levels[L].mean_d[q]) / (2.0 ** alphas[q] - 1.0) if L >= 1 else 0.0
                     for q in range(NQ)])
    rmse = np.sqrt(varY + bias ** 2)
    return {"levels": L + 1, "eps": eps, "relative": relative, "qois": qs,
            "level_choice": level_choice, "estimate": Y.tolist(),
            "var_Y": varY.tolist(), "bias": bias.tolist(), "alpha": alphas,
            "rmse": rmse.tolist(), "rmse_sampling": np.sqrt(varY).tolist(),
            "n": n.astype(int).tolist(), "V_l": [lv.var_d().tolist() for lv in levels],
            "mean_l": [lv.mean_d.tolist() for lv in levels],
            "seconds_per_pair": [max(lv.seconds, 1e-9) / max(lv.timed_pairs, 1) for lv in levels],
            "failed": int(sum(lv.failed for lv in levels)), "rounds": rounds, "wall_s": wall,
            "state": [lv.to_json() for lv in local]}


TUNE_CANDIDATES = {"vcycles": (2, 3, 4), "nu": ((2, 2), (3, 3)), "small_cells": (128, 512),
                   "jac_lag": (0, 10, 30), "tb_cells": (0, 2048), "keep_lags": (30, 100)}


def tuned_schedules(levels, precision, n_xi, nx0=32, ny0=16, world=1, extra=None,
                    paper_workload=False, candidates=None):
    """Autotuned multigrid schedule of every level (autotune.tune_level on at
    most 1024 pairs and about 24 steps of the level), cached by GPU, level,
    precision, batch and workload. Returns (schedules, seconds spent)."""
    import torch
    from paper_2403_17018_gb300 import autotune as A
    A.CANDIDATES = dict(candidates or TUNE_CANDIDATES)
    # the candidate set is part of the key: a schedule tuned over other
    # candidates is not reused
    tag = "|c" + hashlib.sha1(json.dumps(A.CANDIDATES, sort_keys=True).encode()).hexdigest()[:8]
    t0 = time.perf_counter()
    schedules = {}
    gpu = torch.cuda.get_device_name(0)
    cache = A.load_cache()
    for l in range(levels):
        B = min(1024, max(1, max(32, 16384 >> (2 * l)) // world))
        key = A._key(gpu, l, precision, B, nx0, ny0) + f"|xi{n_xi}|lag" + (
            "|paper" if paper_workload else "") + tag
        if key not in cache:
            cache[key], _ = A.tune_level(l, B, precision, steps=24, reps=1, splits=(1,),
                                         n_xi=n_xi, cfg_extra=extra or {})
        schedules[l] = cache[key]
    A.save_cache(cache)
    return schedules, time.perf_counter() - t0


def tuned_run(levels=6, eps=1e-3, n_xi=6, precision="fp32mg", vcycles=3, tune=True, qois=(3, 4, 5),
              adaptive_levels=False, relative=False, paper_workload=False, concurrent=True,
              candidates=None, log=None, rank=0, world=1, dist=None):
    """Adaptive MLMC to RMSE eps on levels 0..levels-1 (config 5 by default:
    6 levels 32x16 .. 1024x512, 6 random variables, RMSE 1e-3 on c at the
    three points), with the schedules autotuned first (the tuning time is
    reported apart from the MLMC wall time). Returns run()'s dict plus the
    precision, tuning time and schedules."""
    from paper_2403_17018_gb300 import binding as hb
    extra = {}
    if paper_workload:
        extra = {"field_model": 1, "T": 6016.0, "nt0": 94}
        n_xi = 3
    cfg = hb.default_config(nlevels=levels, n_xi=n_xi, vcycles=vcycles,
                            precision=hb.PREC_FP64 if precision == "fp64" else hb.PREC_FP32_MG,
                            **extra)
    schedules, tune_s = None, 0.0
    if tune:
        schedules, tune_s = tuned_schedules(levels, precision, n_xi, cfg.nx0, cfg.ny0, world, extra,
                                            paper_workload, candidates)
    sampler = GpuSampler(cfg, rank, world, schedules=schedules)
    res = run(sampler, levels - 1, eps, qois=tuple(qois), log=log, dist=dist,
              concurrent=concurrent, adaptive_levels=adaptive_levels, relative=relative)
    for ctx in {id(c): c for c in sampler.ctxs.values()}.values():
        ctx.close()
    res["paper_workload"] = paper_workload
    res.update({"precision": precision, "n_gpus": world, "tuning_s": tune_s,
                "concurrent_levels": concurrent,
                "schedules": {l: {k: v for k, v in sc.items() if k in ("vcycles", "nu1", "nu2",
                                                                      "mg_small_cells", "jac_lag",
                                                                      "res_rows", "mg_tb_cells", "jac_keep")}
                              for l, sc in (schedules or {}).items()}})
    return res


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--levels", type=int, default=6)
    ap.add_argument("--eps", type=float, default=1e-3)
    ap.add_argument("--n-xi", type=int, default=6)
    ap.add_argument("--precision", choices=["fp64", "fp32mg"], default="fp32mg")
    ap.add_argument("--vcycles", type=int, default=3)
    ap.add_argument("--tune", action="store_true",
                    help="autotune the multigrid schedule of every level on its largest batch "
                         "first (cached; the tuning time is reported apart from the MLMC wall time)")
    ap.add_argument("--adaptive-levels", action="store_true",
                    help="start on levels 0..2 and add levels while the fitted weak-error model "
                         "(Eq. num_levels) asks for them, up to --levels")
    ap.add_argument("--relative", action="store_true",
                    help="eps relative to |E g_0| of each QoI (the paper's scaling)")
    ap.add_argument("--sequential", action="store_true",
                    help="run the levels one after another instead of on concurrent streams")
    ap.add_argument("--paper-workload", action="store_true",
                    help="the paper's own setting: field_model 1 (two-layer multiscale porosity, "
                         "Kozeny-Carman permeability, periodic recharge), 3 variables, "
                         "T = 6016 s in 94 steps on level 0")
    ap.add_argument("--qois", type=int, nargs="*", default=None,
                    help="QoI indices (henry.h) that set the sample numbers; default: c at the "
                         "three points (3 4 5)")
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    import torch
    import __graft_entry__
    __graft_entry__.build()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    log = (lambda d: print(json.dumps(d), flush=True)) if rank == 0 else None
    res = tuned_run(a.levels, a.eps, a.n_xi, a.precision, a.vcycles, a.tune,
                    tuple(a.qois or (3, 4, 5)), a.adaptive_levels, a.relative, a.paper_workload,
                    not a.sequential, log=log, rank=rank, world=world, dist=dist)
    if rank == 0:
        out = {k: v for k, v in res.items() if k != "state"}
        print(json.dumps(out))
        if a.out:
            with open(a.out, "w") as fh:
                json.dump(res, fh)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
