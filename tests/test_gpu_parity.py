"""Parity of the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances: residual and Jacobian entries to 1e-12 (relative to the flux
scale of the grid); solutions to max|dc| <= 1e-9 and max|dp|/max|p| <= 1e-9
(the parity bar for FP64 and for FP32 multigrid inside FP64 defect
correction, whose converged solution is fixed by the FP64 residual).
"""
import numpy as np
import pytest

from oracle import henry as H
from oracle import mlmc as M
from paper_2403_17018_gb300 import binding as hb
from paper_2403_17018_gb300.inputs import logk_perturbation, xi_batch

from gpu_helpers import oracle_grid, oracle_physics, oracle_solve, tight_config, xi_cuda

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

C_TOL = 1e-9
P_TOL = 1e-9


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    hb.load()


def _oracle_jacobian_blocks(J, nx, ny):
    """Oracle sparse Jacobian -> [20, ny, nx] in the C ABI's block layout."""
    J = J.tocsr()
    out = np.zeros((20, ny, nx))
    for j in range(ny):
        for i in range(nx):
            P = j * nx + i
            nbs = [P, P - 1 if i > 0 else -1, P + 1 if i < nx - 1 else -1,
                   P - nx if j > 0 else -1, P + nx if j < ny - 1 else -1]
            for q, Q in enumerate(nbs):
                if Q < 0:
                    continue
                for e in range(2):
                    for v in range(2):
                        out[4 * q + 2 * e + v, j, i] = J[2 * P + e, 2 * Q + v]
    return out


@pytest.mark.parametrize("nx,ny", [(32, 16), (24, 6), (10, 4)])
def test_residual_and_jacobian_match_oracle(nx, ny):
    cfg = hb.default_config()
    ph = oracle_physics(cfg)
    g = H.Grid(nx=nx, ny=ny, nt=1, T=1800.0)
    B = 3
    rng = np.random.default_rng(nx * 100 + ny)
    xis = xi_batch(0, 40, B)
    lk = logk_perturbation(ny, nx, B)
    phi, K, qin, p, c, c_old = [], [], [], [], [], []
    for b in range(B):
        f = H.fields(g, ph, xis[b], lk[b])
        phi.append(f.phi); K.append(f.K); qin.append(f.qin)
        c.append(np.clip(rng.random((ny, nx)), 0, 1))
        c_old.append(np.clip(c[-1] + 0.1 * rng.standard_normal((ny, nx)), 0, 1))
        p.append(H.hydrostatic_guess(g, ph) + 40 * rng.standard_normal((ny, nx)))
    cuda = lambda a: torch.from_numpy(np.ascontiguousarray(np.array(a))).cuda()
    R, J = hb.residual_jacobian(cfg, g.tau, cuda(phi), cuda(K), cuda(qin), cuda(p), cuda(c),
                                cuda(c_old))
    R, J = R.cpu().numpy(), J.cpu().numpy()
    for b in range(B):
        f = H.Fields(phi=phi[b], K=K[b], qin=qin[b])
        Rp, Rc = H.residual(g, ph, f, p[b], c[b], c_old[b])
        Fx = H.face_fluxes(g, ph, f, p[b], c[b])
        scale = max(np.max(np.abs(Fx["mass_y"])), np.max(np.abs(Fx["mass_x"])), np.max(np.abs(Rp)))
        assert np.max(np.abs(R[b, 0] - Rp)) <= 1e-12 * scale
        assert np.max(np.abs(R[b, 1] - Rc)) <= 1e-12 * scale
        Jo = _oracle_jacobian_blocks(H.jacobian(g, ph, f, p[b], c[b], c_old[b]), nx, ny)
        for m in range(20):
            sc = max(np.max(np.abs(Jo[m])), 1e-300)
            assert np.max(np.abs(J[b, m] - Jo[m])) <= 1e-11 * sc, (b, m)


@pytest.mark.parametrize("n_xi", [3, 6])
def test_fields_match_oracle(n_xi):
    cfg = hb.default_config(n_xi=n_xi, nlevels=2)
    ctx = hb.Context(cfg)
    ph = oracle_physics(cfg)
    for level in (0, 1):
        B = 4
        xi = xi_cuda(level, 0, B, n_xi)
        g = oracle_grid(cfg, level)
        lk = torch.from_numpy(logk_perturbation(g.ny, g.nx, B)).cuda()
        phi, K, qin = ctx.fields(level, xi, lk)
        for b in range(B):
            f = H.fields(g, ph, xi[b].cpu().numpy(), lk[b].cpu().numpy())
            assert np.allclose(phi[b].cpu().numpy(), f.phi, rtol=1e-14, atol=0)
            assert np.allclose(K[b].cpu().numpy(), f.K, rtol=1e-13, atol=0)
            assert np.allclose(qin[b].cpu().numpy(), f.qin, rtol=1e-14, atol=0)


@pytest.mark.parametrize("precision,loop", [(hb.PREC_FP64, hb.LOOP_HOST),
                                            (hb.PREC_FP64, hb.LOOP_GRAPH),
                                            (hb.PREC_FP32_MG, hb.LOOP_GRAPH)])
def test_level0_solve_matches_oracle(precision, loop):
    cfg = tight_config(precision=precision, loop_mode=loop)
    ctx = hb.Context(cfg)
    B = 3
    xi = xi_cuda(0, 0, B)
    out = ctx.solve(0, xi, want_c=True, want_p=True, want_iters=True)
    assert out["status"].cpu().numpy().tolist() == [0] * B
    for b in range(B):
        p_o, c_o, q_o = oracle_solve(cfg, 0, xi[b].cpu().numpy())
        c_g = out["c"][b].cpu().numpy()
        p_g = out["p"][b].cpu().numpy()
        assert np.max(np.abs(c_g - c_o)) <= C_TOL
        assert np.max(np.abs(p_g - p_o)) <= P_TOL * np.max(np.abs(p_o))
        q_g = out["q"][b].cpu().numpy()
        assert np.allclose(q_g, q_o, rtol=1e-9, atol=1e-9)


def test_graph_loop_is_bitwise_equal_to_host_loop():
    res = []
    for loop in (hb.LOOP_HOST, hb.LOOP_GRAPH):
        ctx = hb.Context(tight_config(loop_mode=loop))
        out = ctx.solve(0, xi_cuda(0, 3, 4), want_c=True, want_iters=True)
        res.append(out)
    assert torch.equal(res[0]["c"], res[1]["c"])
    assert torch.equal(res[0]["q"], res[1]["q"])
    assert torch.equal(res[0]["iters"], res[1]["iters"])


def test_sample_result_does_not_depend_on_batch():
    ctx = hb.Context(tight_config())
    xi = xi_cuda(0, 0, 7)
    full = ctx.solve(0, xi, want_c=True)
    part = ctx.solve(0, xi[2:5].contiguous(), want_c=True)
    assert torch.equal(full["c"][2:5], part["c"])
    assert torch.equal(full["q"][2:5], part["q"])


def test_pair_coarse_is_bitwise_the_level_below():
    ctx = hb.Context(tight_config(nlevels=2))
    xi = xi_cuda(1, 0, 3)
    qf, qc, cf, cc, st = ctx.sample_pairs(1, xi, want_c=True)
    below = ctx.solve(0, xi, want_c=True)
    fine = ctx.solve(1, xi, want_c=True)
    assert st.cpu().numpy().tolist() == [0, 0, 0]
    assert torch.equal(qc, below["q"]) and torch.equal(cc, below["c"])
    assert torch.equal(qf, fine["q"]) and torch.equal(cf, fine["c"])


@pytest.mark.parametrize("precision", [hb.PREC_FP64, hb.PREC_FP32_MG])
def test_level1_pairs_match_oracle(precision):
    cfg = tight_config(nlevels=2, precision=precision)
    ctx = hb.Context(cfg)
    xi = xi_cuda(1, 0, 2)
    qf, qc, cf, cc, st = ctx.sample_pairs(1, xi, want_c=True)
    assert st.cpu().numpy().tolist() == [0, 0]
    for b in range(2):
        _, c1, q1 = oracle_solve(cfg, 1, xi[b].cpu().numpy())
        _, c0, q0 = oracle_solve(cfg, 0, xi[b].cpu().numpy())
        assert np.max(np.abs(cf[b].cpu().numpy() - c1)) <= C_TOL
        assert np.max(np.abs(cc[b].cpu().numpy() - c0)) <= C_TOL
        assert np.allclose(qf[b].cpu().numpy(), q1, rtol=1e-9, atol=1e-9)
        assert np.allclose(qc[b].cpu().numpy(), q0, rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("jac_lag,res_rows", [(0, 0), (10, 0), (10, 3)])
def test_ragged_grid_matches_oracle(jac_lag, res_rows):
    """24x12 cells (coarsest multigrid grid 6x3, odd ny), 5 steps: blocks of
    256 threads end mid-sample and mid-row; with operator reuse the
    residual-only kernel runs, whose warps here span two row groups of 24
    columns (its west faces come from the neighbouring lane only inside a
    row group)."""
    cfg = tight_config(nx0=24, ny0=12, nt0=5, T=5 * 1800.0, nlevels=1, jac_lag=jac_lag,
                       res_rows=res_rows)
    ctx = hb.Context(cfg)
    assert ctx.level_info(0).n_mg == 3
    xi = xi_cuda(0, 9, 5)
    out = ctx.solve(0, xi, want_c=True, want_p=True)
    for b in range(5):
        p_o, c_o, q_o = oracle_solve(cfg, 0, xi[b].cpu().numpy())
        assert np.max(np.abs(out["c"][b].cpu().numpy() - c_o)) <= C_TOL
        assert np.max(np.abs(out["p"][b].cpu().numpy() - p_o)) <= P_TOL * np.max(np.abs(p_o))


def test_level_stats_match_two_pass():
    ctx = hb.Context(hb.default_config(nlevels=2))
    rng = np.random.default_rng(5)
    qf = rng.standard_normal((300, hb.NQ)) * 3 + 10
    qc = qf + 0.01 * rng.standard_normal(qf.shape)
    st = np.zeros(300, dtype=np.int32)
    st[[4, 77]] = 1
    S = hb.LevelStats()
    for a, b in ((0, 129), (129, 300)):
        ctx.level_stats(1, torch.from_numpy(qf[a:b]).cuda(), torch.from_numpy(qc[a:b]).cuda(),
                        torch.from_numpy(st[a:b]).cuda(), S)
    keep = st == 0
    ref = M.level_stats(qf[keep], qc[keep])
    got = S.numpy()
    assert got["n"] == keep.sum()
    for k in ("mean_f", "var_f", "mean_d", "var_d"):
        assert np.allclose(got[k], ref[k], rtol=1e-12, atol=0), k


def test_field_stats_match_two_pass():
    ctx = hb.Context(hb.default_config(nlevels=2))
    li1, li0 = ctx.level_info(1), ctx.level_info(0)
    rng = np.random.default_rng(6)
    cf = rng.random((40, li1.ny, li1.nx))
    cc = rng.random((40, li0.ny, li0.nx))
    st = np.zeros(40, dtype=np.int32)
    acc = hb.new_field_accumulator(li1.ny, li1.nx)
    for a, b in ((0, 17), (17, 40)):
        ctx.field_stats(1, torch.from_numpy(cf[a:b]).cuda(), torch.from_numpy(cc[a:b]).cuda(),
                        torch.from_numpy(st[a:b]).cuda(), acc)
    d = cf - H.prolong_constant(cc.transpose(1, 2, 0)).transpose(2, 0, 1)
    assert int(acc["n"][0, 0]) == 40
    assert np.allclose(acc["mean_f"].cpu().numpy(), cf.mean(0), rtol=1e-13, atol=1e-15)
    assert np.allclose(acc["m2_f"].cpu().numpy() / 39, cf.var(0, ddof=1), rtol=1e-11, atol=1e-15)
    assert np.allclose(acc["mean_d"].cpu().numpy(), d.mean(0), rtol=1e-12, atol=1e-15)
    assert np.allclose(acc["m2_d"].cpu().numpy() / 39, d.var(0, ddof=1), rtol=1e-11, atol=1e-15)


def test_bad_input_and_iteration_cap_are_reported_per_sample():
    ctx = hb.Context(hb.default_config(nlevels=1, newton_maxit=30))
    xi = xi_cuda(0, 0, 3)
    xi[1, 0] = float("nan")
    out = ctx.solve(0, xi)
    st = out["status"].cpu().numpy()
    assert st[1] & hb.S_BADINPUT and st[0] == 0 and st[2] == 0
    ref = hb.Context(hb.default_config(nlevels=1)).solve(0, xi[[0, 2]].contiguous())
    assert torch.equal(out["q"][[0, 2]], ref["q"])
    capped = hb.Context(hb.default_config(nlevels=1, newton_maxit=1)).solve(0, xi_cuda(0, 0, 2))
    assert np.all(capped["status"].cpu().numpy() & hb.S_MAXIT)


def test_invalid_arguments_are_rejected():
    ctx = hb.Context(hb.default_config(nlevels=2))
    with pytest.raises(hb.HenryError) as e:
        ctx.solve(5, xi_cuda(0, 0, 2))
    assert e.value.code == -1
    with pytest.raises(ValueError):
        ctx.solve(0, xi_cuda(0, 0, 2).float())
    with pytest.raises(hb.HenryError):
        hb.Context(hb.default_config(nx0=30, ny0=15))   # 15 rows cannot be coarsened
    empty = ctx.solve(0, xi_cuda(0, 0, 0))
    assert empty["q"].shape == (0, hb.NQ)


def test_fp32_multigrid_matches_fp64_multigrid_on_identical_xi():
    """Config-3 pattern (FP32 V-cycles inside FP64 defect correction vs FP64
    multigrid) on level 2 (128x64 cells, 96 steps): both converge to the same
    FP64 discrete solution, far inside the 1e-7 bound on c."""
    xi = xi_cuda(2, 0, 4)
    out = {}
    for prec in (hb.PREC_FP64, hb.PREC_FP32_MG):
        ctx = hb.Context(tight_config(nlevels=3, precision=prec))
        out[prec] = ctx.solve(2, xi, want_c=True)
        assert out[prec]["status"].cpu().numpy().tolist() == [0] * 4
    dc = (out[hb.PREC_FP64]["c"] - out[hb.PREC_FP32_MG]["c"]).abs().max().item()
    assert dc <= 1e-9
    dq = (out[hb.PREC_FP64]["q"][:, 3:6] - out[hb.PREC_FP32_MG]["q"][:, 3:6]).abs().max().item()
    assert dq <= 1e-9


def test_full_size_level3_step_residual_under_the_oracle():
    """Level 3 at full size (256x128 cells) in the launch configuration of the
    benchmark (16 samples): after 2 steps at the level's time step, the GPU
    state satisfies the oracle's discrete equations (its FP64 residual, in
    units of c per step) and matches the oracle's state (one sample checked,
    the oracle needs ~25 s for it)."""
    cfg = tight_config(nlevels=4, nt0=1, T=1800.0)   # level 3: 8 steps of 225 s
    ctx = hb.Context(cfg)
    xi = xi_cuda(3, 0, 16)
    out = ctx.solve(3, xi, want_c=True, want_p=True)
    assert out["status"].cpu().numpy().tolist() == [0] * 16
    for b in (11,):
        p_o, c_o, _ = oracle_solve(cfg, 3, xi[b].cpu().numpy())
        assert np.max(np.abs(out["c"][b].cpu().numpy() - c_o)) <= C_TOL
        assert np.max(np.abs(out["p"][b].cpu().numpy() - p_o)) <= P_TOL * np.max(np.abs(p_o))


@pytest.mark.parametrize("precision", [hb.PREC_FP64, hb.PREC_FP32_MG])
def test_default_tolerances_meet_the_parity_bar(precision):
    """The shipped Newton tolerances (rtol 1e-10, atol 1e-11 in units of c
    per step, stagnation at the rounding floor), not only the tight ones of
    the other tests, give solutions within 1e-9 of the oracle: level-1 pairs
    over the full 43200 s and the full-size level-3 grid in the benchmark's
    launch configuration (16 samples, 8 steps)."""
    cfg = hb.default_config(nlevels=2, precision=precision)
    ctx = hb.Context(cfg)
    xi = xi_cuda(1, 0, 2)
    qf, qc, cf, cc, st = ctx.sample_pairs(1, xi, want_c=True)
    assert st.cpu().numpy().tolist() == [0, 0]
    for b in range(2):
        _, c1, q1 = oracle_solve(cfg, 1, xi[b].cpu().numpy())
        _, c0, q0 = oracle_solve(cfg, 0, xi[b].cpu().numpy())
        assert np.max(np.abs(cf[b].cpu().numpy() - c1)) <= C_TOL
        assert np.max(np.abs(cc[b].cpu().numpy() - c0)) <= C_TOL
        assert np.allclose(qf[b].cpu().numpy(), q1, rtol=1e-9, atol=1e-9)
    cfg = hb.default_config(nlevels=4, nt0=1, T=1800.0, precision=precision)
    ctx = hb.Context(cfg)
    xi = xi_cuda(3, 0, 16)
    out = ctx.solve(3, xi, want_c=True, want_p=True)
    assert out["status"].cpu().numpy().tolist() == [0] * 16
    p_o, c_o, _ = oracle_solve(cfg, 3, xi[11].cpu().numpy())
    assert np.max(np.abs(out["c"][11].cpu().numpy() - c_o)) <= C_TOL
    assert np.max(np.abs(out["p"][11].cpu().numpy() - p_o)) <= P_TOL * np.max(np.abs(p_o))


@pytest.mark.parametrize("precision", [hb.PREC_FP64, hb.PREC_FP32_MG])
@pytest.mark.parametrize("level", [0, 2, 3, 4])
def test_fused_multigrid_kernels_equal_plain_launches_bitwise(precision, level):
    """The shared-memory V-cycle (level 0), the thread-block-cluster V-cycle
    (levels 2, 3: 4 and 8 blocks per sample) and cluster + per-level launches
    (level 4) perform the same per-cell operations in the same order as one
    launch per operation, so the solutions agree bit for bit; a stale read
    across the cluster's blocks would break this."""
    res = []
    for fusion in (0, 1):
        cfg = tight_config(nlevels=level + 1, nt0=1, T=1800.0, precision=precision,
                           mg_fusion=fusion, vcycles=2, mg_cluster_cells=32768)
        ctx = hb.Context(cfg)
        out = ctx.solve(level, xi_cuda(level, 0, 3), want_c=True, want_p=True, want_iters=True)
        assert out["status"].cpu().numpy().tolist() == [0, 0, 0]
        res.append(out)
    for k in ("c", "p", "q", "iters"):
        assert torch.equal(res[0][k], res[1][k]), k


@pytest.mark.parametrize("precision", [hb.PREC_FP64, hb.PREC_FP32_MG])
def test_shared_memory_vcycle_threshold_does_not_change_the_result(precision):
    """Moving the boundary between per-level launches and the shared-memory
    V-cycle kernel (no grid, the 32-cell grid, the 512-cell grid of level 2's
    hierarchy) changes only which kernel runs each level's operations, so the
    solutions agree bit for bit."""
    res = []
    for sc in (0, 32, 128, 512):
        cfg = tight_config(nlevels=3, nt0=1, T=1800.0, precision=precision,
                           mg_small_cells=sc, vcycles=2)
        ctx = hb.Context(cfg)
        out = ctx.solve(2, xi_cuda(2, 5, 3), want_c=True, want_p=True, want_iters=True)
        assert out["status"].cpu().numpy().tolist() == [0, 0, 0]
        res.append(out)
    for r in res[1:]:
        for k in ("c", "p", "q", "iters"):
            assert torch.equal(res[0][k], r[k]), k
    with pytest.raises(hb.HenryError):
        hb.Context(hb.default_config(mg_small_cells=513))


@pytest.mark.parametrize("precision", [hb.PREC_FP64, hb.PREC_FP32_MG])
def test_operator_reuse_keeps_parity_and_determinism(precision):
    """Reusing the Jacobian and the multigrid operators across defect-
    correction iterations (jac_lag) changes the iteration path, not the
    equations: level-1 pairs still match the oracle, the graph loop equals
    the host loop bit for bit, and a sample's result does not depend on its
    batch (the reuse decision is per sample)."""
    cfg = tight_config(nlevels=2, precision=precision, jac_lag=10)
    ctx = hb.Context(cfg)
    xi = xi_cuda(1, 0, 4)
    qf, qc, cf, cc, st = ctx.sample_pairs(1, xi, want_c=True)
    assert st.cpu().numpy().tolist() == [0] * 4
    for b in range(2):
        _, c1, q1 = oracle_solve(cfg, 1, xi[b].cpu().numpy())
        _, c0, _ = oracle_solve(cfg, 0, xi[b].cpu().numpy())
        assert np.max(np.abs(cf[b].cpu().numpy() - c1)) <= C_TOL
        assert np.max(np.abs(cc[b].cpu().numpy() - c0)) <= C_TOL
        assert np.allclose(qf[b].cpu().numpy(), q1, rtol=1e-9, atol=1e-9)
    part = ctx.solve(1, xi[1:3].contiguous(), want_c=True, want_iters=True)
    full = ctx.solve(1, xi, want_c=True, want_iters=True)
    assert torch.equal(full["c"][1:3], part["c"]) and torch.equal(full["iters"][1:3], part["iters"])
    host = hb.Context(tight_config(nlevels=2, precision=precision, jac_lag=10,
                                   loop_mode=hb.LOOP_HOST)).solve(1, xi, want_c=True,
                                                                  want_iters=True)
    assert torch.equal(full["c"], host["c"]) and torch.equal(full["iters"], host["iters"])


def test_contexts_with_different_shared_memory_kernels_interleave():
    """The shared-memory V-cycle's dynamic shared-memory limit belongs to the
    kernel, not to a context: a context that captures a new step graph (a
    larger batch) after another context with a smaller shared-memory
    hierarchy has run must still launch it."""
    big = hb.Context(hb.default_config(nlevels=2, precision=hb.PREC_FP32_MG, mg_small_cells=512,
                                       nt0=1, T=1800.0))
    small = hb.Context(hb.default_config(nlevels=2, precision=hb.PREC_FP32_MG,
                                         mg_small_cells=128, nt0=1, T=1800.0))
    a = big.solve(1, xi_cuda(1, 0, 2))
    small.solve(1, xi_cuda(1, 0, 2))
    b = big.solve(1, xi_cuda(1, 0, 3))        # new batch size: graph captured again
    small.solve(1, xi_cuda(1, 0, 5))
    assert b["status"].cpu().numpy().tolist() == [0, 0, 0]
    assert torch.equal(a["q"], b["q"][:2])


@pytest.mark.parametrize("precision", [hb.PREC_FP64, hb.PREC_FP32_MG])
@pytest.mark.parametrize("kry", [2, 3])
def test_bicgstab_preconditioned_by_multigrid_keeps_parity(precision, kry):
    """krylov_iters > 0: each defect correction solves the finest-level
    system with BiCGStab right-preconditioned by V-cycles instead of plain
    V-cycles. The FP64 residual still decides convergence, so level-1 pairs
    match the oracle; graph and host loops agree bit for bit, and a sample's
    result does not depend on its batch (every scalar is per sample)."""
    cfg = tight_config(nlevels=2, precision=precision, krylov_iters=kry)
    ctx = hb.Context(cfg)
    xi = xi_cuda(1, 2, 3)
    qf, qc, cf, cc, st = ctx.sample_pairs(1, xi, want_c=True)
    assert st.cpu().numpy().tolist() == [0, 0, 0]
    for b in range(2):
        _, c1, q1 = oracle_solve(cfg, 1, xi[b].cpu().numpy())
        _, c0, _ = oracle_solve(cfg, 0, xi[b].cpu().numpy())
        assert np.max(np.abs(cf[b].cpu().numpy() - c1)) <= C_TOL
        assert np.max(np.abs(cc[b].cpu().numpy() - c0)) <= C_TOL
        assert np.allclose(qf[b].cpu().numpy(), q1, rtol=1e-9, atol=1e-9)
    full = ctx.solve(1, xi, want_c=True, want_iters=True)
    part = ctx.solve(1, xi[1:].contiguous(), want_c=True, want_iters=True)
    assert torch.equal(full["c"][1:], part["c"]) and torch.equal(full["iters"][1:], part["iters"])
    host = hb.Context(tight_config(nlevels=2, precision=precision, krylov_iters=kry,
                                   loop_mode=hb.LOOP_HOST)).solve(1, xi, want_c=True,
                                                                  want_iters=True)
    assert torch.equal(full["c"], host["c"]) and torch.equal(full["iters"], host["iters"])
