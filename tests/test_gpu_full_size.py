"""Full-size levels that the other parity tests do not reach: level 4
(512x256 cells) and level 5 (1024x512 cells) with 16 samples, the batch the
MLMC driver gives these levels, and the FP32-multigrid check of the
five-level configuration.

A level-l solver depends only on its grid, time step and batch, so a
context whose level 0 is the 512x256 (1024x512) grid with the time step of
level 4 (5) runs exactly the kernels and launch shapes of level 4 (5) of
the standard hierarchy, for as many steps as the test asks.

* Level 4, first two steps: sample 0 against the oracle's own solve (no GPU
  data enters the oracle).
* Levels 4 and 5, well into the horizon (step 48 of level 4, step 24 of
  level 5): the oracle's residual, evaluated at the GPU's states, is the
  check that the discrete equations hold for every sample (scaled to units
  of c per step like the solver's own stopping test, bounded by the
  oracle's own rounding floor for these grids), and the salt-mass balance
  (change of stored salt = boundary outflow) holds.
* Five levels (32x16 .. 512x256, 4096/1024/256/64/16 pairs): per-level mean
  and variance of c at the three points, FP32 multigrid vs FP64 multigrid
  on identical xi, at the default tolerances.
"""
import numpy as np
import pytest

from oracle import henry as H
from paper_2403_17018_gb300 import binding as hb

from gpu_helpers import oracle_physics, tight_config, xi_cuda

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

C_TOL = 1e-9
P_TOL = 1e-9


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    hb.load()


def _level_as_level0(level, steps, **kw):
    """Config whose level 0 is MLMC level `level` (grid and time step) and
    runs `steps` steps of it."""
    tau = 43200.0 / (24 << level)
    return tight_config(nx0=32 << level, ny0=16 << level, nt0=steps, T=steps * tau, nlevels=1,
                        **kw)


def test_level4_first_steps_match_the_oracle_solve():
    cfg = _level_as_level0(4, 2)
    ctx = hb.Context(cfg)
    xi = xi_cuda(4, 0, 16)
    out = ctx.solve(0, xi, want_c=True, want_p=True)
    assert out["status"].cpu().numpy().tolist() == [0] * 16
    ph = oracle_physics(cfg)
    g = H.Grid(nx=cfg.nx0, ny=cfg.ny0, nt=cfg.nt0, T=cfg.T)
    r = H.solve(g, ph, xi[0].cpu().numpy())
    assert np.max(np.abs(out["c"][0].cpu().numpy() - r["c"])) <= C_TOL
    assert np.max(np.abs(out["p"][0].cpu().numpy() - r["p"])) <= P_TOL * np.max(np.abs(r["p"]))


@pytest.mark.parametrize("level,step", [(4, 48), (5, 24)])
@pytest.mark.parametrize("precision", [hb.PREC_FP64, hb.PREC_FP32_MG])
def test_full_size_states_satisfy_the_oracle_equations(level, step, precision):
    B = 16
    xi = xi_cuda(level, 0, B)
    st = {}
    for k in (step - 1, step):
        # solving to step k-1 and to step k: the k-th step starts from the
        # (k-1)-th state, whatever the horizon, because every step converges
        ctx = hb.Context(_level_as_level0(level, k, precision=precision))
        st[k] = ctx.solve(0, xi, want_c=True, want_p=True)
        assert st[k]["status"].cpu().numpy().tolist() == [0] * B
        ctx.close()
    cfg = _level_as_level0(level, step)
    ph = oracle_physics(cfg)
    g = H.Grid(nx=cfg.nx0, ny=cfg.ny0, nt=cfg.nt0, T=cfg.T)
    hx, hy = g.lengths(ph)
    V = hx * hy
    scale = g.tau / (V * ph.phi0 * ph.rho0)          # residual -> units of c per step
    # rounding floor of the oracle's residual in these units: it forms each
    # vertical flux from the full pressure, (p_U - p_L)/hy + rho g, two terms
    # of size rho1 g that cancel to the small driving difference, so the
    # flux carries an absolute error of about eps rho1 g Ly (K/mu)/hy, which
    # scaled by tau/(hx hy phi0 rho0) x (hx rho) gives the floor below
    # (1.7e-10 on the 1024x512 grid with the largest K, half that on
    # 512x256; measured 6.8e-11 on 1024x512; the solver's
    # own residual removes the fresh-water hydrostatic part first and sits
    # ~40x lower)
    Kmax = ph.K0 * np.exp(0.55)
    floor = (Kmax / ph.mu) * np.finfo(float).eps * ph.rho1 * ph.g * ph.Ly * g.tau / (hy * hy * ph.phi0)
    c_prev = st[step - 1]["c"].cpu().numpy()
    c_now = st[step]["c"].cpu().numpy()
    p_now = st[step]["p"].cpu().numpy()
    assert np.all((c_now > -1e-6) & (c_now < 1 + 1e-6))
    assert np.max(np.abs(c_now - c_prev)) > 1e-6       # the step did change the state
    for b in range(B):
        f = H.fields(g, ph, xi[b].cpu().numpy())
        Rp, Rc = H.residual(g, ph, f, p_now[b], c_now[b], c_prev[b])
        rms = np.sqrt(np.sum(Rp * Rp + Rc * Rc) / (g.nx * g.ny)) * scale
        assert rms <= 1e-11 + 2 * floor, (b, rms, floor)
        assert max(np.max(np.abs(Rc)), np.max(np.abs(Rp))) * scale <= 1e-11 + 10 * floor
        # salt balance: stored-salt change = -tau x boundary outflow
        F = H.face_fluxes(g, ph, f, p_now[b], c_now[b])
        rho = ph.rho0 + (ph.rho1 - ph.rho0) * c_now[b]
        rho_o = ph.rho0 + (ph.rho1 - ph.rho0) * c_prev[b]
        dsalt = V * np.sum(f.phi * (rho * c_now[b] - rho_o * c_prev[b]))
        out_salt = F["salt_left"].sum() + F["salt_right"].sum()
        flux_scale = g.tau * hy * ph.rho1 * ph.q0 * g.ny
        assert abs(dsalt + g.tau * out_salt) <= 1e-9 * flux_scale


def test_five_level_statistics_fp32_multigrid_vs_fp64():
    """Per-level MLMC statistics of c at the three points (mean and variance
    of g_l and of g_l - g_(l-1)) over levels 0..4 with 4096/1024/256/64/16
    pairs on identical xi: FP32 V-cycles inside FP64 defect correction
    against FP64 multigrid, default tolerances (relative 1e-10). Both
    converge to the same FP64 discrete solutions; the bound is 1e-7 on c,
    far above the solver tolerance and far below the MLMC target RMSE of
    1e-3; the measured difference is printed."""
    batch = (4096, 1024, 256, 64, 16)
    stats = {}
    for prec in (hb.PREC_FP64, hb.PREC_FP32_MG):
        ctx = hb.Context(hb.default_config(nlevels=5, precision=prec))
        stats[prec] = []
        for level, B in enumerate(batch):
            qf, qc, _, _, st = ctx.sample_pairs(level, xi_cuda(level, 0, B))
            assert int((st != 0).sum().item()) == 0
            S = ctx.level_stats(level, qf, qc, st, hb.LevelStats()).numpy()
            stats[prec].append(S)
        ctx.close()
    worst = 0.0
    for level in range(5):
        a, b = stats[hb.PREC_FP64][level], stats[hb.PREC_FP32_MG][level]
        assert a["n"] == b["n"] == batch[level]
        for k in ("mean_f", "var_f", "mean_d", "var_d"):
            worst = max(worst, float(np.max(np.abs(a[k][3:6] - b[k][3:6]))))
    print(f"max |FP32 MG - FP64 MG| over levels 0..4, c at 3 points: {worst:.2e}")
    assert worst <= 1e-7
