"""henry_sample_levels (all level pairs of an MLMC round, one CUDA graph
launch per coarse time step) and per-level schedules (henry_set_schedule):
the results are bitwise those of henry_sample_pairs run level by level with
the same schedules; the graph is reused while the batches stay, rebuilt
when they change; the residual kernel's tile height (res_rows) is a pure
schedule knob (solutions within the parity bar of the oracle)."""
import numpy as np
import pytest

from paper_2403_17018_gb300 import binding as hb

from gpu_helpers import oracle_solve, tight_config, xi_cuda

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SCHED = {0: dict(vcycles=3, nu1=2, nu2=2, mg_small_cells=0, jac_lag=0, res_rows=0),
         1: dict(vcycles=2, nu1=2, nu2=2, mg_small_cells=128, jac_lag=30, res_rows=2),
         2: dict(vcycles=3, nu1=3, nu2=3, mg_small_cells=512, jac_lag=10, res_rows=0),
         3: dict(vcycles=2, nu1=2, nu2=2, mg_small_cells=512, jac_lag=30, res_rows=16)}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    hb.load()


def _ctx(precision, **kw):
    # level 3 with 2 coarse steps keeps the test short (16 steps of 225 s)
    ctx = hb.Context(tight_config(nlevels=4, precision=precision, nt0=2, T=3600.0, **kw))
    for l, sc in SCHED.items():
        ctx.set_schedule(l, **sc)
    return ctx


@pytest.mark.parametrize("precision", [hb.PREC_FP64, hb.PREC_FP32_MG])
def test_sample_levels_is_bitwise_the_per_level_pairs(precision):
    xis = {0: xi_cuda(0, 0, 9), 1: xi_cuda(1, 0, 5), 2: xi_cuda(2, 0, 3), 3: xi_cuda(3, 0, 2)}
    multi = _ctx(precision)
    got = multi.sample_levels(xis, want_c=True)
    again = multi.sample_levels(xis, want_c=True)        # the kept graph, relaunched
    single = _ctx(precision)
    for l, xi in xis.items():
        ref = single.sample_pairs(l, xi, want_c=True)
        for a, b, c in zip(got[l], ref, again[l]):
            if b is None:
                assert a is None and c is None
                continue
            assert torch.equal(a, b) and torch.equal(c, b), l
        assert got[l][4].cpu().numpy().tolist() == [0] * xi.shape[0]


def test_sample_levels_rebuilds_for_new_batches_and_subsets():
    ctx = _ctx(hb.PREC_FP32_MG)
    ref = _ctx(hb.PREC_FP32_MG)
    for xis in ({1: xi_cuda(1, 3, 4), 3: xi_cuda(3, 3, 2)},          # two levels
                {0: xi_cuda(0, 7, 6), 1: xi_cuda(1, 3, 7), 2: xi_cuda(2, 1, 2)},   # new set
                {1: xi_cuda(1, 3, 4), 3: xi_cuda(3, 3, 2)}):         # the first again
        got = ctx.sample_levels(xis)
        for l, xi in xis.items():
            want = ref.sample_pairs(l, xi)
            assert torch.equal(got[l][0], want[0]) and torch.equal(got[l][4], want[4])
            if l > 0:
                assert torch.equal(got[l][1], want[1])


def test_sample_levels_matches_the_oracle_and_rejects_bad_batches():
    ctx = _ctx(hb.PREC_FP64)
    xi1 = xi_cuda(1, 0, 2)
    out = ctx.sample_levels({0: xi_cuda(0, 0, 3), 1: xi1}, want_c=True)
    cfg = ctx.cfg
    _, c1, q1 = oracle_solve(cfg, 1, xi1[0].cpu().numpy())
    _, c0, q0 = oracle_solve(cfg, 0, xi1[0].cpu().numpy())
    assert np.max(np.abs(out[1][2][0].cpu().numpy() - c1)) <= 1e-9
    assert np.max(np.abs(out[1][3][0].cpu().numpy() - c0)) <= 1e-9
    assert np.allclose(out[1][0][0].cpu().numpy(), q1, rtol=1e-9, atol=1e-9)
    with pytest.raises(hb.HenryError):
        ctx.sample_levels({5: xi_cuda(0, 0, 2)})
    with pytest.raises(hb.HenryError):
        ctx.set_schedule(1, vcycles=0, nu1=2, nu2=2)


@pytest.mark.parametrize("res_rows", [1, 3, 16])
def test_residual_tile_height_keeps_parity(res_rows):
    cfg = tight_config(nlevels=2, res_rows=res_rows)
    ctx = hb.Context(cfg)
    xi = xi_cuda(1, 4, 2)
    out = ctx.solve(1, xi, want_c=True, want_p=True)
    assert out["status"].cpu().numpy().tolist() == [0, 0]
    p_o, c_o, _ = oracle_solve(cfg, 1, xi[0].cpu().numpy())
    assert np.max(np.abs(out["c"][0].cpu().numpy() - c_o)) <= 1e-9
    assert np.max(np.abs(out["p"][0].cpu().numpy() - p_o)) <= 1e-9 * np.max(np.abs(p_o))


@pytest.mark.parametrize("precision", [hb.PREC_FP64, hb.PREC_FP32_MG])
def test_bench_schedule_at_full_size_matches_the_oracle(precision):
    """Level 3 at full size (256x128, 16 samples) with the schedule the
    benchmark tunes for it (V(2,2) x3, shared-memory V-cycle up to 512 cells,
    operator reuse 30: the residual-only kernel decides convergence) and the
    shipped tolerances: 8 steps of 225 s, one sample against the oracle."""
    cfg = hb.default_config(nlevels=4, nt0=1, T=1800.0, precision=precision, vcycles=3,
                            mg_small_cells=512, jac_lag=30)
    ctx = hb.Context(cfg)
    xi = xi_cuda(3, 0, 16)
    out = ctx.solve(3, xi, want_c=True, want_p=True)
    assert out["status"].cpu().numpy().tolist() == [0] * 16
    p_o, c_o, _ = oracle_solve(cfg, 3, xi[11].cpu().numpy())
    assert np.max(np.abs(out["c"][11].cpu().numpy() - c_o)) <= 1e-9
    assert np.max(np.abs(out["p"][11].cpu().numpy() - p_o)) <= 1e-9 * np.max(np.abs(p_o))
