"""Autotuner of the per-level solver schedule.

For each MLMC level it times short batched solves (a few implicit Euler
steps at the level's own time step) for every candidate cycle shape —
V-cycles per defect-correction iteration, pre/post smoothing sweeps, the
largest grid handed to the shared-memory V-cycle kernel and, for the level's
batch size, several batch splits — under a reference operator reuse (the
largest factor of keep_lags with the operators kept across time steps,
jac_keep); then, for the winner, the other reuse variants (the factors of
jac_lag, and of keep_lags with kept operators), the residual kernel's tile
height (res_rows) and the temporally blocked legs (mg_tb_cells), and keeps
the schedule with the highest solves per second. Results are cached in a
JSON file keyed by GPU name, level grid, precision and batch so that later
runs reuse them.

  python -m paper_2403_17018_gb300.autotune --levels 4 --precision fp32mg
"""
from __future__ import annotations

import argparse
import itertools
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_tuning", "schedules.json")
CANDIDATES = {"vcycles": (1, 2, 3), "nu": ((1, 1), (2, 2), (3, 3)), "small_cells": (0, 128, 512),
              "jac_lag": (0, 10, 30), "res_rows": (0, 2, 4, 16), "tb_cells": (0, 2048),
              "keep_lags": (30, 100)}


def _key(gpu, level, precision, batch, nx0, ny0):
    return f"{gpu}|L{level}|{nx0 << level}x{ny0 << level}|{precision}|B{batch}"


def load_cache(path=CACHE):
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def save_cache(cache, path=CACHE):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(cache, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def best_schedule(level, precision, batch, gpu=None, nx0=32, ny0=16, path=CACHE):
    """Cached schedule for a level, or None if it was never tuned."""
    import torch
    gpu = gpu or torch.cuda.get_device_name(0)
    return load_cache(path).get(_key(gpu, level, precision, batch, nx0, ny0))


def tune_level(level, batch, precision="fp32mg", steps=4, reps=2, splits=(1, 2), log=None, n_xi=3,
               cfg_extra=None):
    """Time every candidate cycle shape (V-cycles per iteration, sweeps,
    shared-memory threshold, batch split) under the reference operator reuse
    (the largest factor of keep_lags with kept operators, else the largest
    jac_lag), then the other reuse variants, residual tile heights and
    blocked legs on the best one, each on about `steps` steps of level `level` at
    the level's own time step (steps=None: the whole 43200 s horizon, whose
    early steps need more iterations than the later ones); returns the best
    {vcycles, nu1, nu2, mg_small_cells, jac_lag, res_rows, mg_tb_cells,
    split, solves_per_s} and the table."""
    import torch
    from paper_2403_17018_gb300 import binding as hb
    from paper_2403_17018_gb300.inputs import xi_batch
    prec = hb.PREC_FP64 if precision == "fp64" else hb.PREC_FP32_MG
    f = 1 << level
    extra = dict(cfg_extra or {})
    nt_full = extra.pop("nt0", 24)
    T_full = extra.pop("T", 43200.0)
    tau0 = T_full / nt_full                  # level-0 step of the workload
    k = nt_full if steps is None else min(nt_full, max(1, steps // f))
    xi = torch.from_numpy(xi_batch(level, 0, batch, n_xi=n_xi)).cuda()
    table = []

    def timed(vc, n1, n2, sc, lag, split, rr=0, tb=0, keep=0):
        cfg = hb.default_config(nlevels=level + 1, precision=prec, vcycles=vc, nu1=n1, nu2=n2,
                                mg_small_cells=sc, jac_lag=lag, res_rows=rr, mg_tb_cells=tb,
                                jac_keep=keep, nt0=k, T=tau0 * k, n_xi=n_xi, **extra)
        ctx = hb.Context(cfg)
        sub = batch // split
        parts = [xi[i * sub:(i + 1) * sub].contiguous() for i in range(split)]
        for p in parts:                      # warm-up: allocation and graph capture
            ctx.solve(level, p)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        bad = 0
        for _ in range(reps):
            for p in parts:
                bad += int((ctx.solve(level, p)["status"] != 0).sum().item())
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / reps
        row = {"vcycles": vc, "nu1": n1, "nu2": n2, "mg_small_cells": sc, "jac_lag": lag,
               "res_rows": rr, "mg_tb_cells": tb, "jac_keep": keep, "split": split,
               "solves_per_s": batch / dt, "failed": bad}
        table.append(row)
        if log:
            log(row)
        ctx.close()
        return row

    def best_of(rows):
        ok = [r for r in rows if r["failed"] == 0] or rows
        return max(ok, key=lambda r: r["solves_per_s"])

    # the cycle shapes are compared under the reuse that usually wins: the
    # largest factor of keep_lags with the operators kept across steps, or,
    # without keep_lags, the largest jac_lag (reuse changes which shape
    # wins: with a rebuild at every iteration more V-cycles per iteration
    # amortise it, with reuse fewer are faster); the other reuse variants,
    # tile heights and blocked legs are then timed on the best shape
    lags = tuple(CANDIDATES.get("jac_lag", (0,)))
    keep_lags = tuple(CANDIDATES.get("keep_lags", ()))
    ref = (max(keep_lags), 1) if keep_lags else (max(lags), 0)
    for vc, (n1, n2), sc, split in itertools.product(
            CANDIDATES["vcycles"], CANDIDATES["nu"], CANDIDATES.get("small_cells", (512,)), splits):
        if batch % split:
            continue
        timed(vc, n1, n2, sc, ref[0], split, keep=ref[1])
    best = best_of(table)
    for lag, keep in [(l, 0) for l in lags] + [(l, 1) for l in keep_lags]:
        if (lag, keep) != ref:
            timed(best["vcycles"], best["nu1"], best["nu2"], best["mg_small_cells"], lag,
                  best["split"], keep=keep)
    best = best_of(table)
    for rr in CANDIDATES.get("res_rows", (0,)):
        if rr:
            timed(best["vcycles"], best["nu1"], best["nu2"], best["mg_small_cells"],
                  best["jac_lag"], best["split"], rr, keep=best["jac_keep"])
    best = best_of(table)
    for tb in CANDIDATES.get("tb_cells", (0,)):
        if tb:
            timed(best["vcycles"], best["nu1"], best["nu2"], best["mg_small_cells"],
                  best["jac_lag"], best["split"], best["res_rows"], tb, best["jac_keep"])
    return best_of(table), table


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--levels", type=int, default=4)
    ap.add_argument("--precision", choices=["fp64", "fp32mg"], default="fp32mg")
    ap.add_argument("--batch", type=int, nargs="*", default=None,
                    help="batch per level (default 1024/256/64/16...)")
    ap.add_argument("--steps", type=int, default=4)
    a = ap.parse_args(argv)
    import torch
    import __graft_entry__
    __graft_entry__.build()
    gpu = torch.cuda.get_device_name(0)
    cache = load_cache()
    for level in range(a.levels):
        B = a.batch[level] if a.batch else max(16, 1024 >> (2 * level))
        best, table = tune_level(level, B, a.precision, steps=a.steps,
                                 log=lambda r: print(json.dumps(r), flush=True))
        cache[_key(gpu, level, a.precision, B, 32, 16)] = best
        print(json.dumps({"level": level, "batch": B, "best": best}), flush=True)
    save_cache(cache)


if __name__ == "__main__":
    main()
