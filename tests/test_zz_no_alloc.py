"""henry_residual_jacobian_noalloc: the residual/Jacobian entry point for
callers that cannot allocate device memory during a call (processes whose
device memory belongs to another allocator or a fixed budget,
latency-critical loops where an allocation could synchronise or fail). It
must give the same R and J as the allocating henry_residual_jacobian, call
after call, although every call shares one file-scope scratch array; it
must refuse batches larger than that array.

Kept in a file of its own, collected last, so that a run stopping at the
first failure has already run every other test.
"""
import numpy as np
import pytest

from oracle import henry as H
from paper_2403_17018_gb300 import binding as hb
from paper_2403_17018_gb300.inputs import logk_perturbation, xi_batch

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _case(nx, ny, B, seed):
    """Oracle fields and random states of B samples, as CUDA tensors."""
    cfg = hb.default_config()
    ph = H.Physics(rho0=cfg.rho0, rho1=cfg.rho1, mu=cfg.mu, g=cfg.g, D=cfg.D, K0=cfg.K0,
                   phi0=cfg.phi0, q0=cfg.q0, Lx=cfg.Lx, Ly=cfg.Ly)
    g = H.Grid(nx=nx, ny=ny, nt=1, T=1800.0)
    rng = np.random.default_rng(seed)
    xis = xi_batch(0, seed, B)
    lk = logk_perturbation(ny, nx, B, seed=seed)
    arrs = {k: [] for k in ("phi", "K", "qin", "p", "c", "c_old")}
    for b in range(B):
        f = H.fields(g, ph, xis[b], lk[b])
        arrs["phi"].append(f.phi)
        arrs["K"].append(f.K)
        arrs["qin"].append(f.qin)
        c = np.clip(rng.random((ny, nx)), 0, 1)
        arrs["c"].append(c)
        arrs["c_old"].append(np.clip(c + 0.1 * rng.standard_normal((ny, nx)), 0, 1))
        arrs["p"].append(H.hydrostatic_guess(g, ph) + 40 * rng.standard_normal((ny, nx)))
    t = {k: torch.from_numpy(np.ascontiguousarray(np.array(v))).cuda() for k, v in arrs.items()}
    return cfg, g.tau, t


def _both(cfg, tau, t):
    args = (cfg, tau, t["phi"], t["K"], t["qin"], t["p"], t["c"], t["c_old"])
    R0, J0 = hb.residual_jacobian(*args)
    R1, J1 = hb.residual_jacobian(*args, noalloc=True)
    torch.cuda.synchronize()
    return R0.cpu().numpy(), J0.cpu().numpy(), R1.cpu().numpy(), J1.cpu().numpy()


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    hb.load()


def test_noalloc_matches_allocating_entry_point_on_two_calls():
    # two calls in a row with different sizes and states: the second call
    # reuses the scratch the first left behind
    for nx, ny, B, seed in ((32, 16, 3, 1), (64, 32, 5, 2)):
        cfg, tau, t = _case(nx, ny, B, seed)
        R0, J0, R1, J1 = _both(cfg, tau, t)
        rscale = np.max(np.abs(R0))
        assert np.max(np.abs(R1 - R0)) <= 1e-12 * rscale
        for m in range(20):
            jscale = max(np.max(np.abs(J0[:, m])), 1e-300)
            assert np.max(np.abs(J1[:, m] - J0[:, m])) <= 1e-11 * jscale


def test_noalloc_residual_only_call_matches():
    """J = NULL: only R is written, equal to the allocating entry point's."""
    cfg, tau, t = _case(24, 12, 4, 5)
    args = (cfg, tau, t["phi"], t["K"], t["qin"], t["p"], t["c"], t["c_old"])
    R0, _ = hb.residual_jacobian(*args, want_J=False)
    R1, J1 = hb.residual_jacobian(*args, want_J=False, noalloc=True)
    torch.cuda.synchronize()
    assert J1 is None
    R0, R1 = R0.cpu().numpy(), R1.cpu().numpy()
    assert np.max(np.abs(R1 - R0)) <= 1e-12 * np.max(np.abs(R0))


def test_noalloc_rejects_batches_beyond_its_scratch():
    cfg, tau, t = _case(32, 16, 1, 3)
    B = 26 * 16   # 26*16*512 cells > 2^20 / 5
    big = {k: v.expand((B,) + tuple(v.shape[1:])).contiguous() for k, v in t.items()}
    with pytest.raises(hb.HenryError) as e:
        hb.residual_jacobian(cfg, tau, big["phi"], big["K"], big["qin"], big["p"], big["c"],
                             big["c_old"], noalloc=True)
    assert e.value.code == -1
    assert "exceeds the maximum" in str(e.value)
