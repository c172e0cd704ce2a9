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

Neighbouring panels.  A panel that shares an endpoint with the target's
panel is integrated with a target-independent rule in u in [0, 1], the
distance from the shared endpoint over the panel's parameter length.  Where
the curve is smooth across the junction, the integrand's singular part sits
at u = s* just outside the panel: s* = delta e^{i a} with delta the target's
distance from the junction in the panel's units (at least half the first
Gauss node's offset, 0.0026, up to 2 under dyadic grading) and a near 180
degrees (a = 180 for a straight continuation; curvature and parametrisation
move it slightly off the real axis).  The rule is built for the span of
Pt_j(u) and Pt_j(u) log|u - s*|, j < 16, delta in [0.002, 2.5] (40
log-spaced values) and a in [135, 180] degrees (4 values): the sampled
functions (unit L2 norm on a composite rule graded toward u = 0, 17 pieces
of 40 Gauss points) are compressed by an SVD to the singular values above
3e-14 (50 directions), an interpolatory rule on 50 of the composite nodes
(column-pivoted QR) is reduced by node elimination with minimum-norm
Gauss-Newton steps (nodes kept in (0, 1), weights positive), in double
precision: the orthonormal directions are well conditioned.  The result
integrates every member of the family, and members between the sampled
(delta, a), to 3e-14 of its L1 norm.  At a corner (the two panels' end
tangents differ by more than 10 degrees) the singular point leaves the real
axis (a down to 30 degrees for the wedges of cones); that family does not
compress below the graded composite rule the library keeps for corners.

Usage: python -m paper_1810_07067_gb300.near_rules   (about five minutes)
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


ADJ_DELTA = (0.002, 2.5, 40)     # log-spaced distances of the singular point
ADJ_ANGLE = (135.0, 180.0, 4)    # its angles, degrees
ADJ_EPS = 3e-14                  # singular values kept (unit-norm functions)


def _composite(levels=16, npts=40):
    """Gauss-Legendre pieces [2^-(l+1), 2^-l] and [0, 2^-levels] of [0, 1]."""
    import numpy as np
    xs, ws, iv = [], [], []
    xg, wg = np.polynomial.legendre.leggauss(npts)
    for l in range(levels + 1):
        a = 2.0 ** -(l + 1) if l < levels else 0.0
        b = 2.0 ** -l
        xs.append(0.5 * (a + b) + 0.5 * (b - a) * xg)
        ws.append(0.5 * (b - a) * wg)
        iv.append((a, b))
    return np.concatenate(xs), np.concatenate(ws), iv


def _adjacent_family(u, J=16):
    import numpy as np
    u = np.asarray(u, float)
    y = 2.0 * u - 1.0
    P = np.zeros((J,) + u.shape)
    P[0] = 1.0
    P[1] = y
    for j in range(1, J - 1):
        P[j + 1] = ((2 * j + 1) * y * P[j] - j * P[j - 1]) / (j + 1)
    rows = [P]
    deltas = np.logspace(np.log10(ADJ_DELTA[0]), np.log10(ADJ_DELTA[1]), ADJ_DELTA[2])
    angles = np.deg2rad(np.linspace(ADJ_ANGLE[0], ADJ_ANGLE[1], ADJ_ANGLE[2]))
    for d in deltas:
        for a in angles:
            sr, si = d * np.cos(a), d * np.sin(a)
            rows.append(P * (0.5 * np.log((u - sr) ** 2 + si ** 2)))
    return np.concatenate(rows)


def adjacent_smooth_rule(levels=16, npts=40):
    """Nodes and weights (increasing nodes) of the neighbouring-panel rule for
    smooth junctions (see the module docstring)."""
    import numpy as np
    import scipy.linalg
    x0, w0, iv = _composite(levels, npts)
    F = _adjacent_family(x0)
    F /= np.sqrt((F ** 2 * w0).sum(1, keepdims=True))
    U, S, _ = np.linalg.svd((F * np.sqrt(w0)[None, :]).T, full_matrices=False)
    r = int((S > ADJ_EPS).sum())
    Psi = U[:, :r] / np.sqrt(w0)[:, None]        # orthonormal directions at the composite nodes
    mu = (w0[:, None] * Psi).sum(0)
    xg, _ = np.polynomial.legendre.leggauss(npts)
    bw = np.array([1.0 / np.prod([xg[k] - xg[l] for l in range(npts) if l != k]) for k in range(npts)])

    def basis(x):  # values and derivatives: barycentric interpolation on the composite pieces
        V = np.zeros((len(x), r))
        D = np.zeros((len(x), r))
        for q, xv in enumerate(x):
            l = next(l for l, (a, b) in enumerate(iv) if a <= xv <= b)
            a, b = iv[l]
            t = (2.0 * xv - a - b) / (b - a)
            vals = Psi[l * npts:(l + 1) * npts]
            dif = t - xg
            k = int(np.argmin(np.abs(dif)))
            if abs(dif[k]) < 1e-15:
                dk = np.array([(bw[j] / bw[k]) / (xg[k] - xg[j]) if j != k else 0.0 for j in range(npts)])
                dk[k] = -dk.sum()
                V[q], D[q] = vals[k], (dk @ vals) * 2.0 / (b - a)
                continue
            c = bw / dif
            p = c @ vals / c.sum()
            V[q] = p
            D[q] = ((c / dif) @ (p[None, :] - vals)) / c.sum() * 2.0 / (b - a)
        return V, D

    def gauss_newton(u, w, iters=60):
        for _ in range(iters):
            V, D = basis(u)
            R = V.T @ w - mu
            if np.abs(R).max() < 1e-15:
                return u, w
            J = np.concatenate([D.T * w[None, :], V.T], axis=1)
            st = np.linalg.lstsq(J, -R, rcond=None)[0]
            du, dw = st[:len(u)], st[len(u):]
            t = 1.0
            while not (np.all(u + t * du > 0.0) and np.all(u + t * du < 1.0)):
                t *= 0.5
                if t < 1e-8:
                    return None
            u, w = u + t * du, w + t * dw
        V, _ = basis(u)
        return (u, w) if np.abs(V.T @ w - mu).max() < 1e-14 else None

    _, _, piv = scipy.linalg.qr(Psi.T * np.sqrt(w0)[None, :], pivoting=True, mode="economic")
    u = np.sort(x0[piv[:r]])
    w = np.linalg.solve(basis(u)[0].T, mu)
    while True:
        V, _ = basis(u)
        sig = np.abs(w) * (V ** 2).sum(1)
        for k in np.argsort(sig)[:8]:
            res = gauss_newton(np.delete(u, k), np.delete(w, k))
            if res is not None and np.all(res[1] > 0):
                u, w = res
                break
        else:
            break
    o = np.argsort(u)
    return u[o], w[o]


def write_header(path=HEADER):
    u, w = self_side_rule()
    ua, wa = adjacent_smooth_rule()
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
    lines += ["};",
              "/* MUELLER_ADJ_U / MUELLER_ADJ_W: the neighbouring-panel rule on [0, 1] (u = distance",
              " * from the shared endpoint over the panel's parameter length) for smooth junctions:",
              " * exact to 3e-14 for Pt_j(u) and Pt_j(u) log|u - s*|, j < 16, with s* = delta e^{ia},",
              " * delta in [0.002, 2.5], a in [135, 180] degrees (compressed generalized Gaussian rule). */",
              f"#define MUELLER_ADJ_SMOOTH {len(ua)}",
              "static const double MUELLER_ADJ_U[MUELLER_ADJ_SMOOTH] = {"]
    lines += [f"  {repr(float(v))}," for v in ua]
    lines += ["};", "static const double MUELLER_ADJ_W[MUELLER_ADJ_SMOOTH] = {"]
    lines += [f"  {repr(float(v))}," for v in wa]
    lines += ["};", "#endif", ""]
    with open(path, "w") as f:
        f.write("\n".join(lines))
    return path


if __name__ == "__main__":
    print(write_header())
