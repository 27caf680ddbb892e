"""Operators kept across time steps (jac_keep with operator reuse): the
Jacobian and multigrid operators are rebuilt before a solve's first
iteration and after any iteration that reduced the residual by less than
jac_lag, no longer at every step. Each iteration is still a defect
correction with the current FP64 residual, so the converged solutions meet
the parity bar; the decisions are per sample (batch independence, graph
loop = host loop bitwise); the adjoint's forward rebuilds per step whatever
jac_keep says (gradients bitwise those without it). Also the orders of the
extrapolated Newton guess, which likewise change iterations only."""
import numpy as np
import pytest

from paper_2403_17018_gb300 import binding as hb

from gpu_helpers import oracle_solve, tight_config, xi_cuda

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    hb.load()


@pytest.mark.parametrize("precision", [hb.PREC_FP64, hb.PREC_FP32_MG])
def test_kept_operators_at_full_size_match_the_oracle(precision):
    """Level 3 at full size (256x128, 16 samples, 8 steps of 225 s), reuse
    factor 100 with operators kept across steps, shipped tolerances."""
    cfg = hb.default_config(nlevels=4, nt0=1, T=1800.0, precision=precision, vcycles=3,
                            mg_small_cells=512, jac_lag=100, jac_keep=1)
    ctx = hb.Context(cfg)
    xi = xi_cuda(3, 0, 16)
    out = ctx.solve(3, xi, want_c=True, want_p=True)
    assert out["status"].cpu().numpy().tolist() == [0] * 16
    p_o, c_o, _ = oracle_solve(cfg, 3, xi[11].cpu().numpy())
    assert np.max(np.abs(out["c"][11].cpu().numpy() - c_o)) <= 1e-9
    assert np.max(np.abs(out["p"][11].cpu().numpy() - p_o)) <= 1e-9 * np.max(np.abs(p_o))


def test_kept_operators_graph_equals_host_loop_and_batch():
    res = {}
    for loop in (hb.LOOP_GRAPH, hb.LOOP_HOST):
        cfg = tight_config(nlevels=3, nt0=2, T=3600.0, jac_lag=30, jac_keep=1, loop_mode=loop)
        ctx = hb.Context(cfg)
        res[loop] = ctx.solve(2, xi_cuda(2, 0, 4), want_c=True, want_p=True, want_iters=True)
        assert res[loop]["status"].cpu().numpy().tolist() == [0] * 4
    for k in ("c", "p", "q", "iters"):
        assert torch.equal(res[hb.LOOP_GRAPH][k], res[hb.LOOP_HOST][k]), k
    # the second sample alone: the same as in the batch of four
    cfg = tight_config(nlevels=3, nt0=2, T=3600.0, jac_lag=30, jac_keep=1)
    one = hb.Context(cfg).solve(2, xi_cuda(2, 1, 1), want_c=True, want_iters=True)
    assert torch.equal(one["c"][0], res[hb.LOOP_GRAPH]["c"][1])
    assert torch.equal(one["iters"][0], res[hb.LOOP_GRAPH]["iters"][1])


def test_kept_operators_reach_the_same_solution():
    """Against per-step rebuilds with the same reuse factor the solutions
    agree far inside the parity bar (only the path of the iteration
    changes)."""
    out = {}
    for keep in (0, 1):
        cfg = tight_config(nlevels=3, nt0=2, T=3600.0, jac_lag=100, jac_keep=keep)
        ctx = hb.Context(cfg)
        out[keep] = ctx.solve(2, xi_cuda(2, 2, 4), want_c=True, want_p=True)
        assert out[keep]["status"].cpu().numpy().tolist() == [0] * 4
    assert torch.max(torch.abs(out[0]["c"] - out[1]["c"])).item() <= 1e-10
    dp = torch.max(torch.abs(out[0]["p"] - out[1]["p"])).item()
    assert dp <= 1e-10 * torch.max(torch.abs(out[0]["p"])).item()


def test_adjoint_ignores_kept_operators():
    grads = []
    for keep in (0, 1):
        cfg = tight_config(nlevels=3, nt0=1, T=1800.0, jac_lag=30, jac_keep=keep)
        q, g, gl, st = hb.Context(cfg).adjoint(2, xi_cuda(2, 1, 2))
        assert st.cpu().numpy().tolist() == [0, 0]
        grads.append((q, g, gl))
    for a, b in zip(*grads):
        assert torch.equal(a, b)


def test_schedule_carries_kept_operators():
    """henry_set_schedule passes jac_keep: sample_levels with it equals the
    per-level pairs with the same schedules."""
    ctxs = [hb.Context(tight_config(nlevels=3, nt0=1, T=1800.0)) for _ in range(2)]
    for ctx in ctxs:
        for l in range(3):
            ctx.set_schedule(l, vcycles=3, nu1=2, nu2=2, mg_small_cells=512, jac_lag=100,
                             res_rows=0, mg_tb_cells=0, jac_keep=1)
    xis = {1: xi_cuda(1, 0, 3), 2: xi_cuda(2, 0, 2)}
    got = ctxs[0].sample_levels(xis, want_c=True)
    for l, xi in xis.items():
        want = ctxs[1].sample_pairs(l, xi, want_c=True)
        for a, b in zip(got[l], want):
            if b is None:
                continue
            assert torch.equal(a, b), l


def test_guess_orders_reach_the_same_solution():
    """The extrapolated Newton guess (guess_extrapolation 0..6) changes the
    iterations, not the converged solution; order 4 takes fewer iterations
    than the previous state or the linear guess on this level."""
    out = {}
    for order in (0, 1, 2, 4, 6):
        cfg = tight_config(nlevels=3, nt0=4, T=7200.0, jac_lag=30, guess_extrapolation=order)
        out[order] = hb.Context(cfg).solve(2, xi_cuda(2, 0, 3), want_c=True, want_p=True,
                                           want_iters=True)
        assert out[order]["status"].cpu().numpy().tolist() == [0, 0, 0]
    for order in (0, 1, 2, 6):
        assert torch.max(torch.abs(out[order]["c"] - out[4]["c"])).item() <= 1e-10
        dp = torch.max(torch.abs(out[order]["p"] - out[4]["p"])).item()
        assert dp <= 1e-10 * torch.max(torch.abs(out[4]["p"])).item()
    its = {k: int(v["iters"].sum().item()) for k, v in out.items()}
    assert its[4] < its[1] < its[0], its
