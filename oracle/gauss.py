"""Quadrature rules that define the Nystrom discretisation (Section 5).

Panels carry p = 16 Gauss-Legendre nodes in a panel-local parameter tau in
[-1, 1].  A source panel that is neither the target's own panel nor one of
its two neighbours is integrated with the plain scaled Gauss-Legendre
weights (eq. disequ).  The target's own panel and its neighbours are
integrated with support nodes and the Legendre transform U (eqs. eq_nyslike,
eq_nyslike2); since sum_j U_jk P_j(y) is the Lagrange basis polynomial L_k(y),
the quadrature kernel is Q(x, y_k) = sum_s W_s g(x, y_s) L_k(y_s).

The paper's generalized Gaussian tables come from external code and are not
reproduced.  The rules used instead integrate p(y) log|x-y| + q(y) (the form
in the Remark of Section 5):

* self rule, target at tau_i: split [-1, 1] at tau_i; on each side of length
  L map u in [0, 1] to distance L*u from tau_i and use the reference rule on
  [0, 1]: the 16-node generalized Gaussian rule that integrates P_j(2u-1)
  and P_j(2u-1) log u, j < 16, exactly.  Its nodes and weights are data of
  the discretisation, read from include/mueller_near_rules.h (the table the
  CUDA library compiles in); tests/test_oracle_pins.py checks them against
  the closed-form moments.  32 nodes per target.
* adjacent rules, target independent, in u in [0, 1] -> tau = -1 + 2u (or
  1 - 2u), u the distance from the shared endpoint: where the curve is
  smooth across the junction, the 26-node rule of the near-rule data, exact
  (to 3e-14) for P_j(2u-1) and P_j(2u-1) log|u - s| with the singular point
  s off the panel near the extension of the curve (the table's comment gives
  the family); at a corner (the end tangents of the two panels differ by more
  than 10 degrees) a rule graded toward the shared endpoint, intervals
  [4^-(j+1), 4^-j], j = 0..4, and [0, 4^-5], each with 16 Gauss points (96
  nodes), which also covers singular points off the real axis.
"""
from __future__ import annotations

import os
import re

import numpy as np

P = 16
ADJ_LEVELS = 5
ADJ_GAUSS = 16
RULES_HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                            "mueller_near_rules.h")


def near_rule_table(name: str) -> np.ndarray:
    """The array MUELLER_<name> of the near-rule data file, as float64."""
    text = open(RULES_HEADER).read()
    m = re.search(r"MUELLER_" + name + r"\[[^\]]*\]\s*=\s*\{([^}]*)\}", text)
    if m is None:
        raise KeyError(name)
    return np.array([float(v) for v in m.group(1).replace("\n", " ").split(",") if v.strip()])


def self_side_rule():
    """Generalized Gaussian reference rule (u, w) on [0, 1] for one side of the self panel."""
    return near_rule_table("SELF_U"), near_rule_table("SELF_W")


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


def graded_rule(levels: int, n_gauss: int):
    """Reference rule on [0, 1] graded toward 0 with ratio 4: intervals
    [4^-(j+1), 4^-j] (j < levels) and [0, 4^-levels], n_gauss Gauss points each."""
    us, ws = [], []
    for j in range(levels + 1):
        a, b = (4.0 ** -(j + 1) if j < levels else 0.0), 4.0 ** -j
        x, w = gauss_legendre(n_gauss, a, b)
        us.append(x); ws.append(w)
    u = np.concatenate(us); w = np.concatenate(ws)
    order = np.argsort(u)
    return u[order], w[order]


def self_rule(i: int):
    """Support nodes tau_s and tau-weights for a target at node i of its own panel."""
    x, _ = gauss_legendre(P)
    u, w = self_side_rule()
    ti = x[i]
    Lm, Lp = ti + 1.0, 1.0 - ti
    tau = np.concatenate([ti - Lm * u, ti + Lp * u])
    wt = np.concatenate([Lm * w, Lp * w])
    return tau, wt


def adjacent_rule(shared_end: int, corner: bool = True):
    """Support nodes for a neighbouring panel whose endpoint tau = shared_end
    (-1 or +1) touches the target's panel: the graded composite rule at a
    corner, the tabulated rule for smooth junctions otherwise."""
    if corner:
        u, w = graded_rule(ADJ_LEVELS, ADJ_GAUSS)
    else:
        u, w = near_rule_table("ADJ_U"), near_rule_table("ADJ_W")
    if shared_end < 0:
        return -1.0 + 2.0 * u, 2.0 * w
    return 1.0 - 2.0 * u, 2.0 * w
