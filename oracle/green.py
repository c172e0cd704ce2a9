"""Modal Green's functions by direct azimuthal quadrature (no FFT, no splitting).

For a target (r_t, z_t) and a source (r_s, z_s) on the generating curve,
with rho(phi) the 3D distance of eq. (rho) and G^k = exp(i k rho)/(4 pi rho)
(eq. greenfun), this module returns for m = 0..M+1 the nine spectra

  F0 = g^{k0}_m,  F1 = g^{k1}_m                       (eq. green11)
  F2 = d/dr_t g^{k0}_m,  F3 = d/dz_t g^{k0}_m          (eq. firstder)
  F4 = d/dr_t g^{k1}_m,  F5 = d/dz_t g^{k1}_m
  F6, F7, F8 = d2/dr_t2, d2/dr_t dz_t, d2/dz_t2 of (g^{k0} - g^{k1})_m
                                                         (Section 4.3; only
                                                          the k0-k1 difference
                                                          enters eq. mullerrep)

with g_m = int_0^{2pi} (.) e^{-i m phi} dphi = 2 int_0^pi (.) cos(m phi) dphi
(the integrands are even in phi).  Negative m follow from g_{-m} = g_m.

Quadrature: composite Gauss-Legendre on [0, pi] with dyadic breakpoints
graded toward phi = 0 down to an eighth of the peak width
s = d / sqrt(r_t r_s) (d the distance in the (r, z) plane), and intervals no
longer than ``seg_max`` above phi = 1/4.  Every pair is integrated with 24
and with 32 points per interval; the two must agree to ``check_tol`` relative
to the family's largest coefficient or the call raises.

The difference of the k0 and k1 kernels is formed inside the integrand with
its Taylor series in rho when max|k| rho < 1/2, so no cancellation of the two
hypersingular kernels occurs.
"""
from __future__ import annotations

import math

import numpy as np

FOUR_PI = 4.0 * math.pi
N_LO, N_HI = 24, 32


def _segments(s: float, M: int, seg_max: float | None = None):
    if seg_max is None:
        seg_max = min(math.pi / 8, 24.0 / (M + 2))
    pts = [0.0]
    if s < 2.0:
        J = min(64, max(1, math.ceil(math.log2(2.0 / s))))
        pts += [2.0 ** (-2 - j) for j in range(J - 1, -1, -1)]
    else:
        pts.append(0.25)
    n_up = max(1, math.ceil((math.pi - 0.25) / seg_max))
    pts += list(np.linspace(0.25, math.pi, n_up + 1)[1:])
    return np.array(pts)


def _nodes(breaks: np.ndarray, n: int):
    x, w = np.polynomial.legendre.leggauss(n)
    a, b = breaks[:-1, None], breaks[1:, None]
    phi = (0.5 * (a + b) + 0.5 * (b - a) * x[None, :]).ravel()
    wt = (0.5 * (b - a) * w[None, :]).ravel()
    return phi, wt


def _series_diff(k0, k1, rho, order, nterms=28):
    """(1/4pi) d^order/drho^order of (e^{ik0 rho} - e^{ik1 rho})/rho by its
    Taylor series sum_{n>=1} i^n (k0^n - k1^n) rho^(n-1)/n!."""
    out = np.zeros_like(rho, dtype=complex)
    for n in range(1, nterms):
        p = n - 1 - order
        if p < 0:
            continue
        c = (1j ** n) * (k0 ** n - k1 ** n) / math.factorial(n)
        fac = 1.0
        for q in range(order):
            fac *= (n - 1 - q)
        out += c * fac * rho ** p
    return out / FOUR_PI


def integrands(rt, zt, dr, dz, k0, k1, phi):
    """The nine integrands at azimuths phi; rows F0..F8 (see module doc).

    The pair is given by the target (rt, zt) and the displacement
    (dr, dz) = (r_t - r_s, z_t - z_s), so that near pairs keep the relative
    accuracy of their separation; arrays broadcast against phi."""
    rs = rt - dr
    s2 = np.sin(0.5 * phi) ** 2
    u = dr ** 2 + dz ** 2 + 4.0 * rt * rs * s2
    rho = np.sqrt(u)
    rd = dr + 2.0 * rs * s2
    zd = dz + 0.0 * rho
    out = np.empty((9,) + rho.shape, dtype=complex)
    d1, d2 = {}, {}
    for idx, k in ((0, k0), (1, k1)):
        e = np.exp(1j * k * rho)
        out[idx] = e / (FOUR_PI * rho)
        d1[idx] = e * (1j * k * rho - 1.0) / (FOUR_PI * rho ** 2)
        d2[idx] = e * (2.0 - 2j * k * rho - (k * rho) ** 2) / (FOUR_PI * rho ** 3)
        out[2 + 2 * idx] = d1[idx] * rd / rho
        out[3 + 2 * idx] = d1[idx] * zd / rho
    kmax = max(abs(k0), abs(k1))
    small = kmax * rho < 0.5
    D1 = d1[0] - d1[1]
    D2 = d2[0] - d2[1]
    if np.any(small):
        D1 = np.where(small, _series_diff(k0, k1, rho, 1), D1)
        D2 = np.where(small, _series_diff(k0, k1, rho, 2), D2)
    out[6] = D2 * (rd / rho) ** 2 + D1 * (1.0 / rho - rd ** 2 / rho ** 3)
    out[7] = D2 * rd * zd / rho ** 2 - D1 * rd * zd / rho ** 3
    out[8] = D2 * (zd / rho) ** 2 + D1 * (1.0 / rho - zd ** 2 / rho ** 3)
    return out


def _levels(s: float) -> int:
    return 0 if s >= 2.0 else min(64, max(1, math.ceil(math.log2(2.0 / s))))


def _segments_J(J: int, M: int):
    seg_max = min(math.pi / 8, 24.0 / (M + 2))
    pts = [0.0] + ([2.0 ** (-2 - j) for j in range(J - 1, -1, -1)] if J > 0 else [0.25])
    n_up = max(1, math.ceil((math.pi - 0.25) / seg_max))
    pts += list(np.linspace(0.25, math.pi, n_up + 1)[1:])
    return np.array(pts)


def modal_families_batch(rt, zt, rs, zs, k0, k1, M, check_tol=1e-12, chunk=64, disp=None, return_lo=False):
    """Spectra F[pair, f, m] (f = 0..8, m = 0..M+1) for arrays of pairs.

    ``disp = (dr, dz)`` optionally gives the displacements r_t - r_s, z_t - z_s
    directly (used for support points next to the target, where they are
    known more accurately than the difference of absolute coordinates).
    Pairs sharing the same number of graded levels are integrated together
    on the same composite rule.  With ``return_lo`` the 24-point results are
    returned too (their difference from the 32-point ones is the oracle's own
    noise level)."""
    rt, zt, rs, zs = (np.atleast_1d(np.asarray(a, float)) for a in (rt, zt, rs, zs))
    rt, zt, rs, zs = np.broadcast_arrays(rt, zt, rs, zs)
    if disp is None:
        dr, dz = rt - rs, zt - zs
    else:
        dr, dz = np.broadcast_arrays(*(np.atleast_1d(np.asarray(a, float)) for a in disp))
    n = rt.size
    out = np.empty((n, 9, M + 2), dtype=complex)
    out_lo = np.empty((n, 9, M + 2), dtype=complex) if return_lo else None
    s = np.sqrt((dr ** 2 + dz ** 2) / (rt * (rt - dr)))
    J = np.array([_levels(max(v, 1e-300)) for v in s])
    m = np.arange(M + 2)
    for Jv in np.unique(J):
        idx = np.nonzero(J == Jv)[0]
        breaks = _segments_J(int(Jv), M)
        rules = []
        for nq in (N_LO, N_HI):
            phi, wt = _nodes(breaks, nq)
            rules.append((phi, 2.0 * wt[:, None] * np.cos(np.outer(phi, m))))
        for c0 in range(0, len(idx), chunk):
            sel = idx[c0:c0 + chunk]
            res = []
            for phi, Wc in rules:
                F = integrands(rt[sel, None], zt[sel, None], dr[sel, None], dz[sel, None], k0, k1, phi[None, :])
                res.append(F @ Wc)                       # [9, pairs, M+2]
            lo, hi = res
            scale = np.max(np.abs(hi), axis=2, keepdims=True) + 1e-300
            err = np.max(np.abs(hi - lo) / scale)
            if err > check_tol:
                raise RuntimeError(f"azimuthal quadrature not converged: {err:.2e}")
            out[sel] = hi.transpose(1, 0, 2)
            if return_lo:
                out_lo[sel] = lo.transpose(1, 0, 2)
    return (out, out_lo) if return_lo else out


def modal_families(rt, zt, rs, zs, k0, k1, M, check_tol=1e-12):
    """Spectra F[f, m] of a single pair."""
    return modal_families_batch(rt, zt, rs, zs, k0, k1, M, check_tol)[0]
