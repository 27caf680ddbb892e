"""The vertex-centred variant on the GPU (discretisation = HENRY_DISC_VERTEX)
against the vertex-centred oracle (oracle/henry_vc.py): residual and exact
Jacobian through henry_residual_jacobian_vc at 1e-12 / 1e-11 of the flux and
plane scales; whole solves (levels 0 and 1, both field models) within the
parity bar, c <= 1e-9 and p <= 1e-9 relative, and the QoIs; level pairs
bitwise the solves below."""
import numpy as np
import pytest

from oracle import henry as H
from oracle import henry_vc as V
from paper_2403_17018_gb300 import binding as hb
from paper_2403_17018_gb300.inputs import xi_batch

from gpu_helpers import oracle_physics, tight_config, xi_cuda

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    hb.load()


def _oracle_blocks(J, nx, ny1):
    J = J.tocsr()
    out = np.zeros((20, ny1, nx))
    for j in range(ny1):
        for i in range(nx):
            P = j * nx + i
            nbs = [P, P - 1 if i > 0 else -1, P + 1 if i < nx - 1 else -1,
                   P - nx if j > 0 else -1, P + nx if j < ny1 - 1 else -1]
            for q, Q in enumerate(nbs):
                if Q < 0:
                    continue
                for e in range(2):
                    for v in range(2):
                        out[4 * q + 2 * e + v, j, i] = J[2 * P + e, 2 * Q + v]
    return out


@pytest.mark.parametrize("nx,ny,n_xi,model", [(16, 8, 3, 0), (10, 4, 6, 0), (24, 6, 3, 1)])
def test_vc_residual_and_jacobian_match_oracle(nx, ny, n_xi, model):
    cfg = hb.default_config(n_xi=n_xi, field_model=model)
    ph = oracle_physics(cfg)
    g = H.Grid(nx=nx, ny=ny, nt=1, T=900.0)
    B = 3
    rng = np.random.default_rng(nx * 7 + ny)
    xis = xi_batch(0, 60, B, n_xi=n_xi)
    p0, _ = V.initial_state(g, ph)
    P, C, CO = [], [], []
    for b in range(B):
        C.append(np.clip(rng.random(p0.shape), 0, 1))
        CO.append(np.clip(C[-1] + 0.1 * rng.standard_normal(p0.shape), 0, 1))
        P.append(p0 + 40 * rng.standard_normal(p0.shape))
    cuda = lambda a: torch.from_numpy(np.ascontiguousarray(np.array(a))).cuda()
    R, J = hb.residual_jacobian_vc(cfg, g.tau, cuda(xis), cuda(P), cuda(C), cuda(CO))
    R, J = R.cpu().numpy(), J.cpu().numpy()
    for b in range(B):
        vf = V.vfields(g, ph, xis[b])
        Rp, Rc = V.residual(g, ph, vf, P[b], C[b], CO[b])
        F = V.face_fluxes(g, ph, vf, P[b], C[b])
        scale = max(np.max(np.abs(F["mass_y"])), np.max(np.abs(F["mass_x"])), np.max(np.abs(Rp)))
        assert np.max(np.abs(R[b, 0] - Rp)) <= 1e-12 * scale
        assert np.max(np.abs(R[b, 1] - Rc)) <= 1e-12 * scale
        Jo = _oracle_blocks(V.jacobian(g, ph, vf, P[b], C[b], CO[b]), nx, ny + 1)
        for m in range(20):
            sc = max(np.max(np.abs(Jo[m])), 1e-300)
            assert np.max(np.abs(J[b, m] - Jo[m])) <= 1e-11 * sc, (b, m)


@pytest.mark.parametrize("level,model", [(0, 0), (1, 0), (0, 1)])
def test_vc_solve_matches_the_oracle(level, model):
    kw = dict(nlevels=2, discretisation=hb.DISC_VERTEX, field_model=model)
    if model == 1:
        kw.update(nt0=8, T=8 * 64.0)     # the paper's tau = 64 s, 8 steps
    cfg = tight_config(**kw)
    ctx = hb.Context(cfg)
    B = 3
    xi = xi_cuda(level, 0, B)
    out = ctx.solve(level, xi, want_c=True, want_p=True)
    assert out["status"].cpu().numpy().tolist() == [0] * B
    ph = oracle_physics(cfg)
    g = H.Grid(nx=cfg.nx0 << level, ny=cfg.ny0 << level, nt=cfg.nt0 << level, T=cfg.T)
    for b in range(2):
        r = V.solve(g, ph, xi[b].cpu().numpy())
        assert np.max(np.abs(out["c"][b].cpu().numpy() - r["c"])) <= 1e-9
        assert np.max(np.abs(out["p"][b].cpu().numpy() - r["p"])) <= 1e-9 * np.max(np.abs(r["p"]))
        qo = V.qoi(g, ph, r["vfields"], r["c"])
        qg = out["q"][b].cpu().numpy()
        keep = np.arange(hb.NQ) != 6          # Q_FW counts boxes at a c threshold
        assert np.allclose(qg[keep], qo[keep], rtol=1e-9, atol=1e-9)


def test_vc_pairs_are_bitwise_the_solves_and_other_entry_points_refuse():
    ctx = hb.Context(tight_config(nlevels=2, discretisation=hb.DISC_VERTEX))
    xi = xi_cuda(1, 3, 4)
    qf, qc, cf, cc, st = ctx.sample_pairs(1, xi, want_c=True)
    fine = ctx.solve(1, xi, want_c=True)
    below = ctx.solve(0, xi, want_c=True)
    assert st.cpu().numpy().tolist() == [0] * 4
    assert torch.equal(qf, fine["q"]) and torch.equal(cf, fine["c"])
    assert torch.equal(qc, below["q"]) and torch.equal(cc, below["c"])
    lv = ctx.sample_levels({0: xi_cuda(0, 1, 2), 1: xi})
    assert torch.equal(lv[1][0], qf) and torch.equal(lv[1][1], qc)
    with pytest.raises(hb.HenryError) as e:
        ctx.adjoint(0, xi_cuda(0, 0, 2))
    assert e.value.code == -5
