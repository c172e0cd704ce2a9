"""Quadrature rules that define the Nystrom discretisation (Section 5).

Panels carry p = 16 Gauss-Legendre nodes in a panel-local parameter tau in
[-1, 1].  A source panel that is neither the target's own panel nor one of
its two neighbours is integrated with the plain scaled Gauss-Legendre
weights (eq. disequ).  The target's own panel and its neighbours are
integrated with support nodes and the Legendre transform U (eqs. eq_nyslike,
eq_nyslike2); since sum_j U_jk P_j(y) is the Lagrange basis polynomial L_k(y),
the quadrature kernel is Q(x, y_k) = sum_s W_s g(x, y_s) L_k(y_s).

The paper's generalized Gaussian tables come from external code and are not
reproduced.  These rules are written out from their definition instead; they
integrate p(y) log|x-y| + q(y) (the form in the Remark of Section 5) to about
machine precision:

* self rule, target at tau_i: split [-1, 1] at tau_i; on each side of length
  L map u in [0, 1] to distance L*u from tau_i and use the reference rule
  R_self on [0, 1]: for j = 0..9 the interval [4^-(j+1), 4^-j] with 16 Gauss
  points, plus [0, 4^-10] with 4 nodes at the 4 Gauss points whose weights
  make the rule exact for {1, u, log u, u log u}.  164 nodes per side.
* adjacent rule: graded toward the shared endpoint: u in [0, 1] -> tau =
  -1 + 2u (or 1 - 2u); intervals [4^-(j+1), 4^-j], j = 0..4, and [0, 4^-5],
  each with 16 Gauss points.  96 nodes, target independent.
"""
from __future__ import annotations

import numpy as np

P = 16
SELF_LEVELS = 10
SELF_GAUSS = 16
ADJ_LEVELS = 5
ADJ_GAUSS = 16


def gauss_legendre(n: int, a: float = -1.0, b: float = 1.0):
    """n-point Gauss-Legendre nodes and weights on [a, b]."""
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (a + b) + 0.5 * (b - a) * x, 0.5 * (b - a) * w


def lagrange_basis(nodes: np.ndarray, t: np.ndarray) -> np.ndarray:
    """L[s, k] = prod_{l != k} (t_s - x_l) / (x_k - x_l)  (plain product form)."""
    t = np.atleast_1d(np.asarray(t, float))
    n = len(nodes)
    L = np.ones((len(t), n))
    for k in range(n):
        for l in range(n):
            if l != k:
                L[:, k] *= (t - nodes[l]) / (nodes[k] - nodes[l])
    return L


def log_end_rule():
    """4-node rule on [0, 1] at the Gauss points, exact for 1, u, log u, u log u."""
    x, _ = gauss_legendre(4, 0.0, 1.0)
    V = np.vstack([np.ones(4), x, np.log(x), x * np.log(x)])
    mom = np.array([1.0, 0.5, -1.0, -0.25])
    return x, np.linalg.solve(V, mom)


def graded_rule(levels: int, n_gauss: int, inner: str):
    """Reference rule on [0, 1] graded toward 0 with ratio 4.

    inner = 'log': innermost [0, 4^-levels] uses the 4-node log rule;
    inner = 'gauss': innermost interval uses n_gauss Gauss points."""
    us, ws = [], []
    for j in range(levels):
        a, b = 4.0 ** -(j + 1), 4.0 ** -j
        x, w = gauss_legendre(n_gauss, a, b)
        us.append(x); ws.append(w)
    h = 4.0 ** -levels
    if inner == "log":
        x, w = log_end_rule()
        us.append(h * x); ws.append(h * w)
    else:
        x, w = gauss_legendre(n_gauss, 0.0, h)
        us.append(x); ws.append(w)
    u = np.concatenate(us); w = np.concatenate(ws)
    order = np.argsort(u)
    return u[order], w[order]


def self_rule(i: int):
    """Support nodes tau_s and tau-weights for a target at node i of its own panel."""
    x, _ = gauss_legendre(P)
    u, w = graded_rule(SELF_LEVELS, SELF_GAUSS, "log")
    ti = x[i]
    Lm, Lp = ti + 1.0, 1.0 - ti
    tau = np.concatenate([ti - Lm * u, ti + Lp * u])
    wt = np.concatenate([Lm * w, Lp * w])
    return tau, wt


def adjacent_rule(shared_end: int):
    """Support nodes for a neighbouring panel whose endpoint tau = shared_end
    (-1 or +1) touches the target's panel."""
    u, w = graded_rule(ADJ_LEVELS, ADJ_GAUSS, "gauss")
    if shared_end < 0:
        return -1.0 + 2.0 * u, 2.0 * w
    return 1.0 - 2.0 * u, 2.0 * w
