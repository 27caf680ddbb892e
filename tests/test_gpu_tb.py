"""Temporally blocked multigrid legs (mg_tb_cells): one launch per leg and
level (pre-sweeps + residual restriction, prolongation + post-sweeps) on
tiles with a halo. Every cell gets the operations of one launch per
operation in the same order, so solutions, QoIs, iteration counts and
adjoint gradients are bitwise those of the per-operation path; a stale halo
value (a tile reading a neighbour's updated unknowns, a halo one cell too
narrow) breaks that. Parity with the oracle at full size with the blocked
legs on."""
import numpy as np
import pytest

from paper_2403_17018_gb300 import binding as hb

from gpu_helpers import oracle_solve, tight_config, xi_cuda

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ALL = 1 << 30


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    hb.load()


def _solve(level, tb, B=3, seed=0, **kw):
    cfg = tight_config(nlevels=level + 1, nt0=1, T=1800.0, mg_tb_cells=tb, **kw)
    ctx = hb.Context(cfg)
    out = ctx.solve(level, xi_cuda(level, seed, B), want_c=True, want_p=True, want_iters=True)
    assert out["status"].cpu().numpy().tolist() == [0] * B
    return out


def _same(a, b):
    for k in ("c", "p", "q", "iters"):
        assert torch.equal(a[k], b[k]), k


@pytest.mark.parametrize("precision", [hb.PREC_FP64, hb.PREC_FP32_MG])
@pytest.mark.parametrize("level,nu", [(2, (2, 2)), (3, (2, 2)), (3, (1, 1)), (3, (3, 2))])
def test_blocked_legs_equal_per_operation_launches_bitwise(precision, level, nu):
    """Level 3 (256x128: 16 tiles of 64x32 per sample on the finest grid,
    4 on 128x64, one whole-grid tile on 64x32) and level 2, several
    (nu1, nu2): halos 2 nu1 + 1 and 2 nu2."""
    kw = dict(precision=precision, nu1=nu[0], nu2=nu[1], vcycles=2)
    _same(_solve(level, 0, **kw), _solve(level, ALL, **kw))


@pytest.mark.parametrize("small", [0, 512])
def test_blocked_legs_on_a_ragged_hierarchy(small):
    """160x48 cells (tiles of 64, 64, 32 columns and 32, 16 rows; coarser
    grids 80x24, 40x12, 20x6 down to 10x3): partial tiles and halos clipped by
    the domain; with no shared-memory V-cycle every level down to 20x6 is
    blocked."""
    kw = dict(nx0=40, ny0=12, precision=hb.PREC_FP32_MG, mg_small_cells=small, vcycles=2)
    _same(_solve(2, 0, **kw), _solve(2, ALL, **kw))


def test_threshold_selects_levels():
    """mg_tb_cells between two grid sizes blocks only the coarser batched
    levels; the result stays the same."""
    kw = dict(precision=hb.PREC_FP64, vcycles=2)
    ref = _solve(3, 0, **kw)
    for tb in (2048, 8192):
        _same(ref, _solve(3, tb, **kw))


@pytest.mark.parametrize("precision", [hb.PREC_FP64, hb.PREC_FP32_MG])
def test_blocked_legs_as_bicgstab_preconditioner(precision):
    kw = dict(precision=precision, krylov_iters=2)
    _same(_solve(2, 0, **kw), _solve(2, ALL, **kw))


def test_blocked_legs_in_the_adjoint():
    """The transposed solves of henry_adjoint run the same V-cycles on the
    transposed operators."""
    grads = []
    for tb in (0, ALL):
        cfg = tight_config(nlevels=3, nt0=1, T=1800.0, mg_tb_cells=tb)
        ctx = hb.Context(cfg)
        q, g, gl, st = ctx.adjoint(2, xi_cuda(2, 1, 2))
        assert st.cpu().numpy().tolist() == [0, 0]
        grads.append((q, g, gl))
    for a, b in zip(*grads):
        assert torch.equal(a, b)


def test_per_level_schedule_carries_the_threshold():
    """henry_set_schedule takes mg_tb_cells per level; sample_levels with it
    equals sample_levels without."""
    res = []
    for tb in (0, ALL):
        ctx = hb.Context(tight_config(nlevels=4, nt0=1, T=1800.0, precision=hb.PREC_FP32_MG))
        for l in range(4):
            ctx.set_schedule(l, vcycles=2, nu1=2, nu2=2, mg_small_cells=512, jac_lag=10,
                             res_rows=0, mg_tb_cells=tb)
        res.append(ctx.sample_levels({2: xi_cuda(2, 3, 3), 3: xi_cuda(3, 3, 2)}, want_c=True))
    for l in (2, 3):
        for a, b in zip(res[0][l], res[1][l]):
            assert torch.equal(a, b), l


@pytest.mark.parametrize("precision", [hb.PREC_FP64, hb.PREC_FP32_MG])
def test_blocked_full_size_level3_matches_the_oracle(precision):
    """Level 3 at full size (256x128, 16 samples, 8 steps of 225 s) with the
    blocked legs on every batched level and operator reuse: one sample
    against the oracle at the parity bar."""
    cfg = hb.default_config(nlevels=4, nt0=1, T=1800.0, precision=precision, vcycles=3,
                            mg_small_cells=512, jac_lag=30, mg_tb_cells=ALL)
    ctx = hb.Context(cfg)
    xi = xi_cuda(3, 0, 16)
    out = ctx.solve(3, xi, want_c=True, want_p=True)
    assert out["status"].cpu().numpy().tolist() == [0] * 16
    p_o, c_o, _ = oracle_solve(cfg, 3, xi[11].cpu().numpy())
    assert np.max(np.abs(out["c"][11].cpu().numpy() - c_o)) <= 1e-9
    assert np.max(np.abs(out["p"][11].cpu().numpy() - p_o)) <= 1e-9 * np.max(np.abs(p_o))
