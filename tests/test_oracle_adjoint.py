"""Pins of the oracle's discrete adjoint: central finite differences of the
oracle's forward solve (h = 1e-4 in xi and log K; the Newton solve is
converged to 1e-12, so truncation and rounding both stay below 1e-7
relative), and the transpose identity of the linearised step."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import adjoint as A
from oracle import henry as H
from paper_2403_17018_gb300.inputs import logk_perturbation, xi_batch


def _grid():
    return H.Grid(nx=16, ny=8, nt=5, T=5 * 3600.0)


@pytest.mark.parametrize("qoi", ["Q_S", "toe"])
def test_adjoint_gradient_matches_central_differences_in_xi(qoi):
    ph = H.Physics()
    g = _grid()
    xi = xi_batch(0, 3, 1)[0]
    adj = A.adjoint(g, ph, xi, qoi)
    h = 1e-4
    for j in range(3):
        e = np.zeros(3)
        e[j] = h
        fd = (A.forward_qoi(g, ph, xi + e, qoi) - A.forward_qoi(g, ph, xi - e, qoi)) / (2 * h)
        assert abs(adj["dq_dxi"][j] - fd) <= 1e-5 * max(abs(fd), 1e-3 * abs(adj["q"])), (j, fd)


def test_adjoint_gradient_matches_central_differences_in_logk():
    ph = H.Physics()
    g = _grid()
    xi = xi_batch(0, 4, 1)[0]
    lk = logk_perturbation(g.ny, g.nx, 1)[0]
    adj = A.adjoint(g, ph, xi, "toe", lk)
    h = 1e-4
    scale = np.max(np.abs(adj["dq_dlogk"]))
    for (j, i) in ((0, 0), (3, 7), (7, 15), (5, 1), (2, 12)):
        e = np.zeros_like(lk)
        e[j, i] = h
        fd = (A.forward_qoi(g, ph, xi, "toe", lk + e) - A.forward_qoi(g, ph, xi, "toe", lk - e)) / (2 * h)
        assert abs(adj["dq_dlogk"][j, i] - fd) <= 1e-5 * scale, ((j, i), fd)


def test_transposed_solve_dot_product_identity():
    """<J v, w> = <v, J^T w> for the step Jacobian the adjoint inverts."""
    ph = H.Physics()
    g = _grid()
    f = H.fields(g, ph, xi_batch(0, 5, 1)[0])
    rng = np.random.default_rng(2)
    p = H.hydrostatic_guess(g, ph) + rng.standard_normal((g.ny, g.nx))
    c = rng.random((g.ny, g.nx))
    J = H.jacobian(g, ph, f, p, c, c)
    v, w = rng.standard_normal(J.shape[0]), rng.standard_normal(J.shape[0])
    assert abs(np.dot(J @ v, w) - np.dot(v, J.T @ w)) <= 1e-12 * np.linalg.norm(J @ v) * np.linalg.norm(w)
    lam = spla.spsolve(J.T.tocsc(), w)
    assert np.linalg.norm(J.T @ lam - w) <= 1e-10 * np.linalg.norm(w)


def test_adjoint_of_the_paper_model_matches_central_differences():
    """The paper's field model (two-layer multiscale porosity, Kozeny-Carman
    permeability, recharge with its time factor at each step's end): the
    adjoint gradient in xi_1..xi_3 and in log K against central differences
    of the forward solve (steps of 13 s so that the recharge factor varies)."""
    ph = H.Physics(field_model=1)
    g = H.Grid(nx=16, ny=8, nt=6, T=6 * 13.0)
    xi = xi_batch(0, 6, 1)[0]
    lk = logk_perturbation(g.ny, g.nx, 1)[0]
    adj = A.adjoint(g, ph, xi, "Q_S", lk)
    h = 1e-4
    for j in range(3):
        e = np.zeros(3)
        e[j] = h
        fd = (A.forward_qoi(g, ph, xi + e, "Q_S", lk) - A.forward_qoi(g, ph, xi - e, "Q_S", lk)) / (2 * h)
        assert abs(adj["dq_dxi"][j] - fd) <= 1e-5 * max(abs(fd), 1e-3 * abs(adj["q"])), (j, fd)
    scale = np.max(np.abs(adj["dq_dlogk"]))
    for (j, i) in ((0, 0), (3, 7), (7, 15)):
        e = np.zeros_like(lk)
        e[j, i] = h
        fd = (A.forward_qoi(g, ph, xi, "Q_S", lk + e) - A.forward_qoi(g, ph, xi, "Q_S", lk - e)) / (2 * h)
        assert abs(adj["dq_dlogk"][j, i] - fd) <= 1e-5 * scale, ((j, i), fd)
