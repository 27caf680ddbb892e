"""Small, self-contained case for ncu captures of the hot kernels.

Runs one batched solve of one MLMC level for a few implicit Euler steps,
then replays the finest-level smoother half-sweep, the residual +
Jacobian kernel and the residual-only evaluation a few times
(henry_time_kernel) and prints their timings.

  python -m paper_2403_17018_gb300.profile_case --level 3 --batch 16 --steps 2
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--level", type=int, default=3)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--steps", type=int, default=8,
                    help="implicit Euler steps of the level (rounded to a multiple of 2^level)")
    ap.add_argument("--precision", choices=["fp64", "fp32mg"], default="fp64")
    ap.add_argument("--vcycles", type=int, default=2)
    ap.add_argument("--nu", type=int, nargs=2, default=(2, 2), metavar=("NU1", "NU2"),
                    help="pre- and post-smoothing sweeps")
    ap.add_argument("--jac-lag", type=int, default=0,
                    help="operator reuse factor (0: operators rebuilt every iteration)")
    ap.add_argument("--small-cells", type=int, default=512,
                    help="largest multigrid level (cells per sample) run by the shared-memory "
                         "V-cycle kernel; 0 disables it")
    ap.add_argument("--jac-keep", type=int, default=0, choices=(0, 1),
                    help="keep the operators across time steps (with --jac-lag > 0)")
    ap.add_argument("--res-rows", type=int, default=0, help="residual kernel tile height")
    ap.add_argument("--tb-cells", type=int, default=0,
                    help="largest batched multigrid level run with temporally blocked legs")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--loop", choices=["graph", "host"], default="graph",
                    help="host: plain launches with a host convergence check (visible to ncu "
                         "kernel by kernel); graph: the production CUDA-graph loop")
    a = ap.parse_args(argv)
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2403_17018_gb300 import binding as hb
    from paper_2403_17018_gb300.inputs import xi_batch
    prec = hb.PREC_FP64 if a.precision == "fp64" else hb.PREC_FP32_MG
    f = 1 << a.level
    nt_full = 24 * f
    # same time step as the full workload (tau_l = 1800 s / 2^l), fewer steps:
    # level l runs k 2^l steps with k = max(1, steps // 2^l)
    k = max(1, a.steps // f)
    cfg = hb.default_config(nlevels=a.level + 1, precision=prec, vcycles=a.vcycles,
                            nu1=a.nu[0], nu2=a.nu[1], mg_small_cells=a.small_cells,
                            jac_lag=a.jac_lag, jac_keep=a.jac_keep, res_rows=a.res_rows,
                            mg_tb_cells=a.tb_cells, nt0=k, T=1800.0 * k,
                            loop_mode=hb.LOOP_HOST if a.loop == "host" else hb.LOOP_GRAPH)
    ctx = hb.Context(cfg)
    xi = torch.from_numpy(xi_batch(a.level, 0, a.batch)).cuda()
    out = ctx.solve(a.level, xi, want_iters=True)
    torch.cuda.synchronize()
    # the whole solve once more, timed on the device (the first one built
    # the workspaces and graphs)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record()
    ctx.solve(a.level, xi)
    ev[1].record()
    torch.cuda.synchronize()
    res = {"level": a.level, "batch": a.batch, "steps": ctx.level_info(a.level).nt,
           "full_steps": nt_full, "precision": a.precision, "tb_cells": a.tb_cells,
           "solve_ms": ev[0].elapsed_time(ev[1]),
           "iters": out["iters"].float().mean().item(),
           "status_bad": int((out["status"] != 0).sum().item())}
    # replays of the finest-level kernels, each inside an NVTX range named
    # after it so that ncu can select exactly these launches
    # (--nvtx --nvtx-include "smooth_half_sweep/", "resjac/", "resid/")
    for which, name in ((0, "smooth_half_sweep"), (1, "resjac"), (2, "resid")):
        torch.cuda.nvtx.range_push(name)
        ms, by, fl = ctx.time_kernel(a.level, 0, which, reps=a.reps)
        torch.cuda.nvtx.range_pop()
        res[name] = {"ms": ms, "bytes": by, "flops": fl, "GB/s": by / ms / 1e6,
                     "TFLOP/s": fl / ms / 1e9}
    print(json.dumps(res))


if __name__ == "__main__":
    main()
