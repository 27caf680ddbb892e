"""Quasi-Monte Carlo runs on one level (arxiv 2403.17018, section 4: the QMC
computations with Halton points, tests A1-A3).

Samples are Halton points mapped to xi = 2u - 1 (indices from 1, skipping
the corner point of index 0). With R > 1 replicates every replicate shifts
the same points by its own seeded uniform vector modulo 1 (randomised QMC),
so the R replicate means are independent unbiased estimates whose spread
gives a standard error; with R = 1 the points are the plain Halton sequence
as in the paper.

Per replicate and batch the solves run through the C ABI (henry_solve with
the c field), the QoI statistics through mlmc_level_stats, the per-cell
mean and variance of c through mlmc_field_stats and the per-cell exceedance
counts P(c > threshold) through mlmc_field_exceedance, all on the device.
The host gathers the B x NQ QoI values of every sample for the quantiles
(the sample quantile of Hyndman and Fan's definition 7).

  python -m paper_2403_17018_gb300.qmc --level 2 --samples 600
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

QUANTILES = (0.025, 0.25, 0.5, 0.75, 0.975)


def sample_quantiles(values, probs):
    """Quantiles of each column of values [n, k] at probabilities probs:
    linear interpolation between order statistics at h = (n - 1) p."""
    v = np.sort(np.asarray(values, dtype=np.float64), axis=0)
    n = v.shape[0]
    out = []
    for p in probs:
        h = (n - 1) * p
        lo = min(int(math.floor(h)), n - 1)
        hi = min(lo + 1, n - 1)
        out.append(v[lo] + (h - lo) * (v[hi] - v[lo]))
    return np.stack(out)                      # [len(probs), k]


def _chan(n_a, mean_a, m2_a, n_b, mean_b, m2_b):
    """Chan, Golub and LeVeque's merge of two (count, mean, M2) states."""
    n = n_a + n_b
    if n == 0:
        return 0, mean_a, m2_a
    d = mean_b - mean_a
    return n, mean_a + d * (n_b / n), m2_a + m2_b + d * d * (n_a * n_b / n)


def _chan_cells(n_a, mean_a, m2_a, n_b, mean_b, m2_b):
    """_chan per cell (arrays; cells with no samples stay at zero)."""
    n = n_a + n_b
    safe = np.maximum(n, 1.0)
    d = mean_b - mean_a
    return (n, mean_a + np.where(n > 0, d * (n_b / safe), 0.0),
            m2_a + m2_b + np.where(n > 0, d * d * (n_a * n_b / safe), 0.0))


def run(ctx, level, n_samples, n_xi=3, batch=256, replicates=1, thresholds=(0.5,),
        probs=QUANTILES, first=1, log=None, series_every=0, rank=0, world=1, dist=None,
        device="cuda"):
    """QMC on `level` with n_samples Halton points per replicate. Returns a
    dict: per-QoI mean (over replicates) and standard error (R > 1), the
    per-replicate means and variances, quantiles of every QoI over all
    valid samples, and per-cell mean, variance and exceedance probability
    fields of c (numpy), plus timing and failed samples. series_every = k > 0
    also solves through henry_solve_series (without the c field statistics)
    and returns the quantiles of every QoI after each k-th step (test A3:
    "series_quantiles" [steps/k, probs, NQ], "series_steps").

    Under torch.distributed (world > 1, `dist` the module) every rank solves
    a disjoint slice of each batch; the replicate statistics and the
    per-cell fields are merged with Chan's formula, the exceedance counts
    summed and the QoI values gathered for the quantiles, so every rank
    returns the result of the whole run."""
    import torch
    from paper_2403_17018_gb300 import binding as hb
    from paper_2403_17018_gb300.inputs import xi_halton
    li = ctx.level_info(level)
    ncell = li.ny * li.nx
    dev = torch.device(device)
    rep_means, rep_vars, all_q, all_series = [], [], [], []
    fstats = {k: torch.zeros(ncell, dtype=torch.float64, device=dev)
              for k in ("mean_f", "m2_f", "mean_d", "m2_d")}
    fstats["n"] = torch.zeros(ncell, dtype=torch.int64, device=dev)
    counts = [torch.zeros(ncell, dtype=torch.int64, device=dev) for _ in thresholds]
    failed = 0
    t0 = time.perf_counter()
    for r in range(replicates):
        shift = None if replicates == 1 else 2403017018 + 7919 * (r + 1)
        S = hb.LevelStats()
        for k in range(0, n_samples, batch):
            cnt_all = min(batch, n_samples - k)
            lo = (cnt_all * rank) // world
            cnt = (cnt_all * (rank + 1)) // world - lo
            if cnt == 0:
                continue
            xi = torch.from_numpy(xi_halton(first + k + lo, cnt, n_xi, shift)).to(dev)
            if series_every:
                out = ctx.solve_series(level, xi, series_every)
            else:
                out = ctx.solve(level, xi, want_c=True)
            st = out["status"]
            ctx.level_stats(level, out["q"], None, st, S)
            if not series_every:
                c = out["c"].reshape(cnt, ncell)
                ctx.field_stats(level, c, None, st, fstats)
                for th, cn in zip(thresholds, counts):
                    ctx.field_exceedance(level, c, st, th, cn)
            ok = (st == 0).cpu().numpy()
            failed += int((~ok).sum())
            all_q.append(out["q"].cpu().numpy()[ok])
            if series_every:
                all_series.append(out["series"].cpu().numpy()[ok])
        n, mf, m2 = int(S.n), np.array(S.mean_f[:]), np.array(S.m2_f[:])
        if dist is not None and world > 1:
            parts = [None] * world
            dist.all_gather_object(parts, (n, mf, m2))
            n, mf, m2 = 0, np.zeros(hb.NQ), np.zeros(hb.NQ)
            for nb, mb, m2b in parts:
                n, mf, m2 = _chan(n, mf, m2, nb, mb, m2b)
        rep_means.append(mf)
        rep_vars.append(m2 / (n - 1) if n > 1 else np.full(hb.NQ, np.nan))
        if log:
            log({"replicate": r, "n": n, "mean": rep_means[-1].tolist()})
    if dev.type == "cuda":
        torch.cuda.synchronize()
    fs = {k: v.cpu().numpy() for k, v in fstats.items()}
    cnts = [cn.cpu().numpy().reshape(li.ny, li.nx) for cn in counts]
    if dist is not None and world > 1:
        parts = [None] * world
        dist.all_gather_object(parts, (fs, cnts, all_q, all_series, failed))
        fs = {k: np.zeros_like(v) for k, v in fs.items()}
        n_c = np.zeros(ncell)
        for f, _, _, _, _ in parts:
            n_c, fs["mean_f"], fs["m2_f"] = _chan_cells(n_c, fs["mean_f"], fs["m2_f"],
                                                       f["n"].astype(np.float64), f["mean_f"],
                                                       f["m2_f"])
        fs["n"] = n_c.astype(np.int64)
        cnts = [sum(p[1][i] for p in parts) for i in range(len(thresholds))]
        all_q = [a for p in parts for a in p[2]]
        all_series = [a for p in parts for a in p[3]]
        failed = sum(p[4] for p in parts)
    wall = time.perf_counter() - t0
    rm = np.array(rep_means)
    mean = rm.sum(axis=0) / replicates
    se = (np.sqrt(((rm - mean) ** 2).sum(axis=0) / (replicates - 1) / replicates)
          if replicates > 1 else np.full(mean.shape, np.nan))
    q = np.concatenate(all_q, axis=0)
    nf = int(fs["n"][0])
    return {"level": level, "samples": n_samples, "replicates": replicates,
            "mean": mean, "std_error": se, "replicate_means": rm,
            "replicate_vars": np.array(rep_vars),
            "quantile_probs": list(probs), "quantiles": sample_quantiles(q, probs), "q": q,
            "mean_field": fs["mean_f"].reshape(li.ny, li.nx),
            "var_field": (fs["m2_f"] / max(nf - 1, 1)).reshape(li.ny, li.nx),
            "thresholds": list(thresholds), "counts": cnts, "n_field": nf,
            # exact counts divided on the host (a device division by a scalar
            # may go through its reciprocal and differ in the last bit)
            "exceedance": [k / max(nf, 1) for k in cnts],
            "failed": failed, "wall_s": wall,
            "series_steps": (list(range(series_every, li.nt + 1, series_every))
                             if series_every else []),
            "series_quantiles": (np.stack([sample_quantiles(v, probs)
                                           for v in np.concatenate(all_series, axis=0)
                                           .transpose(1, 0, 2)])
                                 if series_every else None)}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--level", type=int, default=2)
    ap.add_argument("--samples", type=int, default=600)
    ap.add_argument("--replicates", type=int, default=1)
    ap.add_argument("--n-xi", type=int, default=3)
    ap.add_argument("--batch", type=int, default=600)
    ap.add_argument("--precision", choices=["fp64", "fp32mg"], default="fp32mg")
    ap.add_argument("--threshold", type=float, nargs="*", default=[0.5])
    ap.add_argument("--series-every", type=int, default=0,
                    help="also record the QoIs after every k-th step and report their "
                         "quantiles over time (test A3)")
    ap.add_argument("--paper-workload", action="store_true",
                    help="field_model 1, T = 6016 s in 94 steps on level 0 (the paper's setting)")
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2403_17018_gb300 import binding as hb
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    extra = {"field_model": 1, "T": 6016.0, "nt0": 94} if a.paper_workload else {}
    if a.paper_workload:
        a.n_xi = 3
    cfg = hb.default_config(nlevels=a.level + 1, n_xi=a.n_xi,
                            precision=hb.PREC_FP64 if a.precision == "fp64" else hb.PREC_FP32_MG,
                            **extra)
    ctx = hb.Context(cfg)
    res = run(ctx, a.level, a.samples, n_xi=a.n_xi, batch=a.batch, replicates=a.replicates,
              thresholds=a.threshold,
              log=(lambda d: print(json.dumps(d), flush=True)) if rank == 0 else None,
              series_every=a.series_every, rank=rank, world=world, dist=dist)
    summary = {"level": a.level, "samples": a.samples, "replicates": a.replicates,
               "paper_workload": a.paper_workload,
               "precision": a.precision, "mean": res["mean"].tolist(),
               "std_error": res["std_error"].tolist(), "quantile_probs": res["quantile_probs"],
               "quantiles": res["quantiles"].tolist(),
               "exceedance_area_fraction": [float(e.mean()) for e in res["exceedance"]],
               "max_var_c": float(res["var_field"].max()), "failed": res["failed"],
               "series_steps": res["series_steps"],
               "series_quantiles_Q_FW_Q_S": (res["series_quantiles"][:, :, [6, 0]].tolist()
                                             if a.series_every else None),
               "wall_s": res["wall_s"]}
    summary["n_gpus"] = world
    if rank == 0:
        print(json.dumps(summary))
        if a.out:
            np.savez(a.out, **{k: v for k, v in res.items() if isinstance(v, np.ndarray)})
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
