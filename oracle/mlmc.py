"""MLMC estimator pieces of the paper's section 3 (test infrastructure only).

Plain two-pass statistics, the closed-form sample allocation and the number
of levels from the weak-error model.
"""
from __future__ import annotations

import math

import numpy as np


def level_stats(g_fine, g_coarse=None):
    """Two-pass per-QoI statistics of one level's samples (Def. of Y_l, V_l).

    g_fine, g_coarse: [m, nq]; g_coarse is None on level 0 (g_{-1} = 0).
    Returns dict: n, mean_f, var_f (of g_l), mean_d, var_d (of g_l - g_{l-1}),
    variances with the 1/(n-1) normalisation."""
    gf = np.asarray(g_fine, dtype=np.float64)
    d = gf if g_coarse is None else gf - np.asarray(g_coarse, dtype=np.float64)
    n = gf.shape[0]

    def two_pass(a):
        m = a.sum(axis=0) / n
        v = ((a - m) ** 2).sum(axis=0) / (n - 1) if n > 1 else np.zeros_like(m)
        return m, v

    mf, vf = two_pass(gf)
    md, vd = two_pass(d)
    return {"n": n, "mean_f": mf, "var_f": vf, "mean_d": md, "var_d": vd}


def estimator(means_d, vars_d, m):
    """Multilevel estimator Y = sum_l Y_l (Eq. A) and Var Y = sum V_l / m_l
    (Eq. goal_variance)."""
    means_d = np.asarray(means_d, dtype=np.float64)
    vars_d = np.asarray(vars_d, dtype=np.float64)
    m = np.asarray(m, dtype=np.float64)
    return means_d.sum(axis=0), (vars_d / m.reshape((-1,) + (1,) * (vars_d.ndim - 1))).sum(axis=0)


def allocation(V, s, eps, var_budget_fraction=0.5):
    """Optimal samples per level, Eq. M_ell: with Var Y fixed to
    f * eps^2 the cost sum m_l s_l is minimal for
      m_l = eps^-2 / f * sqrt(V_l / s_l) * sum_i sqrt(V_i s_i),
    rounded up. f = 1/2 is the paper's split of the MSE (Eq. var_error)."""
    V = np.asarray(V, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    tot = np.sum(np.sqrt(V * s))
    m = np.sqrt(V / s) * tot / (var_budget_fraction * eps * eps)
    return np.array([int(math.ceil(x - 1e-9 * x)) for x in m])


def optimal_cost(V, s, eps, var_budget_fraction=0.5):
    """Eq. total_cost_MLMC: S = eps^-2 / f * (sum_l sqrt(V_l s_l))^2."""
    V = np.asarray(V, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    return np.sum(np.sqrt(V * s)) ** 2 / (var_budget_fraction * eps * eps)


def mc_cost(var_g, s_L, eps):
    """Plain Monte Carlo cost at level L for MSE eps^2 (Test B4):
    S_MC = 2 eps^-2 s_L Var g."""
    return 2.0 * s_L * var_g / (eps * eps)


def cost_exponent(alpha, beta, gamma=1.0, d_hat=3.0):
    """Exponent of eps^-1 in the MLMC cost theorem (Theorem 1): 2 for
    beta > d_hat gamma, else 2 + (d_hat gamma - beta) / alpha (the log^2 case
    at equality is reported as 2)."""
    if beta >= d_hat * gamma:
        return 2.0
    return 2.0 + (d_hat * gamma - beta) / alpha


def fit_rate(levels, values, base=2.0):
    """Least-squares fit log_base|values| = -rate * l + zeta (Test B3 fits in
    log_4 because its levels refine by 4; this build's refine by 2).
    Returns (rate, zeta)."""
    l = np.asarray(levels, dtype=np.float64)
    y = np.log(np.abs(np.asarray(values, dtype=np.float64))) / math.log(base)
    A = np.vstack([-l, np.ones_like(l)]).T
    (rate, zeta), *_ = np.linalg.lstsq(A, y, rcond=None)
    return float(rate), float(zeta)


def weak_error_constants(levels, means_d):
    """Weak-error model of Eq. weak_error_model, |E(g_l - g)| <= c1 4^(-alpha l),
    from the level corrections E Y_l = E(g_l - g_(l-1)), l >= 1: least-squares
    fit log_4 |E Y_l| = -alpha l + zeta (the paper's log_4 convention, one
    level = h halved = cells x 4), c_Y = 4^zeta, and the bias of level L read
    as the tail of the finer corrections, sum_(k > L) c_Y 4^(-alpha k) =
    c_Y 4^(-alpha L) / (4^alpha - 1), so c1 = c_Y / (4^alpha - 1).
    Returns (alpha, c1)."""
    alpha, zeta = fit_rate(levels, means_d, base=4.0)
    c_y = 4.0 ** zeta
    return alpha, c_y / (4.0 ** alpha - 1.0)


def num_levels(eps, E0, c1, alpha):
    """Eq. num_levels: the finest level L with c1 4^(-alpha L) = eps E0 / sqrt(2),
    L = -(1/alpha) log_4(eps E0 / (sqrt(2) c1)), taken as the smallest integer
    level that meets the bias bound (never below 0). E0 = 1 for an absolute
    eps, E0 = |E g_0| for the paper's relative error."""
    L = -math.log(eps * E0 / (math.sqrt(2.0) * c1), 4.0) / alpha
    return max(0, int(math.ceil(L - 1e-12)))
