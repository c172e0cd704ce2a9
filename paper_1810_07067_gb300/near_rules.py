"""Generate the near-panel quadrature table include/mueller_near_rules.h.

Section 5 integrates the target's own panel with a rule that is exact for
p(t) log|t - t_i| + q(t), p and q polynomials of degree < 16 (Remark after
eq. eq_nyslike); the paper's generalized Gaussian tables come from external
code and are not printed.  This script computes the rule from its definition
and writes it as a C table that the library compiles in.

Self panel.  Split at the target, each side maps onto u in [0, 1] (distance
from the target over the side's length), where the class is the span of
Pt_j(u) and Pt_j(u) log u, j < n (Pt_j(u) = P_j(2u - 1); log of a scaled
distance differs from log u by a constant).  The n-node rule with positive
weights that integrates these 2n functions exactly is unique (they form a
Chebyshev system on (0, 1]).  It is found by the node-elimination procedure
of Bremer, Gimbutas and Rokhlin (SIAM J. Sci. Comput. 32, 2010) in 60-digit
arithmetic: start from 2n nodes graded toward u = 0 with the interpolatory
weights of the exact moments, then remove one node at a time, each time
re-solving the 2n moment equations for the remaining nodes and weights by
minimum-norm Gauss-Newton steps, until n nodes remain.  The moments are

    int_0^1 Pt_j(u) du = delta_j0,   int_0^1 log u du = -1,
    int_0^1 Pt_j(u) log u du = (-1)^(j+1) / (j (j+1))   (j >= 1).

Usage: python -m paper_1810_07067_gb300.near_rules   (about a minute)
"""
from __future__ import annotations

import os

import mpmath as mp

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(os.path.dirname(HERE), "include", "mueller_near_rules.h")
SELF_N = 16


def _legendre(x, n):
    """Pt_j(x) and d/dx Pt_j(x) for j < n at x in [0, 1]."""
    y = 2 * x - 1
    P, D = [mp.mpf(1), y], [mp.mpf(0), mp.mpf(1)]
    for j in range(1, n - 1):
        P.append(((2 * j + 1) * y * P[j] - j * P[j - 1]) / (j + 1))
        D.append(D[j - 1] + (2 * j + 1) * P[j])
    return P[:n], [2 * d for d in D[:n]]


def _moments(n):
    mu = [mp.mpf(1)] + [mp.mpf(0)] * (n - 1) + [mp.mpf(-1)]
    mu += [mp.mpf((-1) ** (j + 1)) / (j * (j + 1)) for j in range(1, n)]
    return mu


def _family(x, n):
    """Values and x-derivatives of the 2n functions at x."""
    P, D = _legendre(x, n)
    lx = mp.log(x)
    return P + [p * lx for p in P], D + [d * lx + p / x for p, d in zip(P, D)]


def _gauss_newton(u, w, n, mu, iters=40):
    """Minimum-norm Gauss-Newton steps on sum_s w_s f_i(u_s) = mu_i with the
    nodes kept in (0, 1); the solution (u, w), or None."""
    k = len(u)
    tol = mp.mpf(10) ** -(mp.mp.dps - 15)
    for _ in range(iters):
        cols = [_family(x, n) for x in u]
        R = mp.matrix([sum(cols[s][0][i] * w[s] for s in range(k)) - mu[i] for i in range(2 * n)])
        if mp.norm(R, mp.inf) < tol:
            return u, w
        J = mp.matrix(2 * n, 2 * k)
        for s in range(k):
            for i in range(2 * n):
                J[i, s] = cols[s][1][i] * w[s]
                J[i, k + s] = cols[s][0][i]
        Jt = J.T
        d = Jt * mp.lu_solve(J * Jt, -R)
        t = mp.mpf(1)
        while any(not (0 < u[s] + t * d[s] < 1) for s in range(k)):
            t /= 2
            if t < mp.mpf(2) ** -40:
                return None
        u = [u[s] + t * d[s] for s in range(k)]
        w = [w[s] + t * d[k + s] for s in range(k)]
    return None


def self_side_rule(n=SELF_N, dps=60):
    """Nodes and weights (mpf lists, increasing nodes) of the n-node rule."""
    mp.mp.dps = dps
    mu = _moments(n)
    x, _ = _gl(2 * n)
    u = [((1 + v) / 2) ** 3 for v in x]              # 2n nodes graded toward u = 0
    V = mp.matrix(2 * n, 2 * n)
    for s, xs in enumerate(u):
        f = _family(xs, n)[0]
        for i in range(2 * n):
            V[i, s] = f[i]
    w = list(mp.lu_solve(V, mp.matrix(mu)))
    while len(u) > n:
        sig = []
        for s in range(len(u)):
            f = _family(u[s], n)[0]
            sig.append(abs(w[s]) * sum(v * v for v in f))
        for k in sorted(range(len(u)), key=lambda s: sig[s]):
            res = _gauss_newton(u[:k] + u[k + 1:], w[:k] + w[k + 1:], n, mu)
            if res is not None and all(v > 0 for v in res[1]):
                u, w = res
                break
        else:
            raise RuntimeError(f"node elimination stalled at {len(u)} nodes")
    order = sorted(range(n), key=lambda s: u[s])
    return [u[s] for s in order], [w[s] for s in order]


def _gl(n):
    """Gauss-Legendre nodes and weights on [-1, 1] (Newton on P_n)."""
    x, w = [], []
    for i in range(n):
        t = mp.cos(mp.pi * (i + mp.mpf(3) / 4) / (n + mp.mpf(1) / 2))
        for _ in range(100):
            p0, p1 = mp.mpf(1), t
            for k in range(2, n + 1):
                p0, p1 = p1, ((2 * k - 1) * t * p1 - (k - 1) * p0) / k
            dp = n * (t * p1 - p0) / (t * t - 1)
            dt = p1 / dp
            t -= dt
            if abs(dt) < mp.mpf(10) ** -(mp.mp.dps - 5):
                break
        x.append(t)
        w.append(2 / ((1 - t * t) * dp * dp))
    order = sorted(range(n), key=lambda s: x[s])
    return [x[s] for s in order], [w[s] for s in order]


def write_header(path=HEADER):
    u, w = self_side_rule()
    lines = [
        "/*",
        " * mueller_near_rules.h -- near-panel quadrature data of the Nystrom",
        " * discretisation (Section 5), written by paper_1810_07067_gb300/near_rules.py.",
        " *",
        " * MUELLER_SELF_U / MUELLER_SELF_W: the generalized Gaussian rule on [0, 1]",
        " * with MUELLER_SELF_SIDE nodes that integrates Pt_j(u) and Pt_j(u) log u,",
        " * j < MUELLER_SELF_SIDE (Pt_j the Legendre polynomials shifted to [0, 1]),",
        " * exactly.  The target's own panel is split at the target and each side",
        " * mapped onto [0, 1] (u = distance from the target / side length), so the",
        " * pair of sides integrates p(t) log|t - t_i| + q(t), deg p, q < 16, exactly",
        " * (Remark after eq. eq_nyslike).  Values are the 60-digit solution rounded",
        " * to double.",
        " */",
        "#ifndef MUELLER_NEAR_RULES_H",
        "#define MUELLER_NEAR_RULES_H",
        f"#define MUELLER_SELF_SIDE {len(u)}",
        "static const double MUELLER_SELF_U[MUELLER_SELF_SIDE] = {",
    ]
    lines += [f"  {repr(float(v))}," for v in u]
    lines += ["};", "static const double MUELLER_SELF_W[MUELLER_SELF_SIDE] = {"]
    lines += [f"  {repr(float(v))}," for v in w]
    lines += ["};", "#endif", ""]
    with open(path, "w") as f:
        f.write("\n".join(lines))
    return path


if __name__ == "__main__":
    print(write_header())
