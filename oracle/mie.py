"""Mie series for a homogeneous dielectric sphere (textbook closed form,
e.g. Bohren & Huffman ch. 4), used to pin the whole solver.

Incident field E = e exp(i k0 d.x) with e orthogonal to d (time factor
exp(-i omega t)).  Far field E_oo(xh) with E_sc ~ exp(i k0 |x|)/|x| E_oo:
in the frame where d = z and e = x,
  E_oo = (1/(-i k0)) [ cos(Phi) S2(Theta) e_Theta - sin(Phi) S1(Theta) e_Phi ].
"""
from __future__ import annotations

import numpy as np
from scipy.special import spherical_jn, spherical_yn


def _coefficients(k0, k1, a, nmax):
    """a_n, b_n for a non-magnetic sphere (mu1 = mu0), relative index m = k1/k0."""
    x = k0 * a
    m = k1 / k0
    mx = m * x
    n = np.arange(1, nmax + 1)
    psi = lambda z: z * spherical_jn(n, z)
    dpsi = lambda z: spherical_jn(n, z) + z * spherical_jn(n, z, derivative=True)
    xi = lambda z: z * (spherical_jn(n, z) + 1j * spherical_yn(n, z))
    dxi = lambda z: (spherical_jn(n, z) + 1j * spherical_yn(n, z)) + z * (
        spherical_jn(n, z, derivative=True) + 1j * spherical_yn(n, z, derivative=True))
    an = (m * psi(mx) * dpsi(x) - psi(x) * dpsi(mx)) / (m * psi(mx) * dxi(x) - xi(x) * dpsi(mx))
    bn = (psi(mx) * dpsi(x) - m * psi(x) * dpsi(mx)) / (psi(mx) * dxi(x) - m * xi(x) * dpsi(mx))
    return n, an, bn


def amplitudes(k0, k1, a, cos_theta, nmax=None):
    """S1, S2 at scattering angles with cosine cos_theta."""
    if nmax is None:
        nmax = int(abs(k0 * a) + 4 * abs(k0 * a) ** (1 / 3) + 20)
    n, an, bn = _coefficients(k0, k1, a, nmax)
    mu = np.atleast_1d(cos_theta)
    pi_prev = np.zeros_like(mu); pi_cur = np.ones_like(mu)
    S1 = np.zeros(mu.shape, complex); S2 = np.zeros(mu.shape, complex)
    for idx, nn in enumerate(n):
        tau = nn * mu * pi_cur - (nn + 1) * pi_prev
        f = (2 * nn + 1) / (nn * (nn + 1))
        S1 += f * (an[idx] * pi_cur + bn[idx] * tau)
        S2 += f * (an[idx] * tau + bn[idx] * pi_cur)
        pi_next = ((2 * nn + 1) * mu * pi_cur - (nn + 1) * pi_prev) / nn
        pi_prev, pi_cur = pi_cur, pi_next
    return S1, S2


def far_field(k0, k1, a, d, e, directions):
    """E_oo for unit directions [nd, 3] (Cartesian components)."""
    d = np.asarray(d, float); e = np.asarray(e, float)
    y = np.cross(d, e)
    X = np.asarray(directions, float)
    ct = X @ d
    px, py = X @ e, X @ y
    Phi = np.arctan2(py, px)
    Theta = np.arccos(np.clip(ct, -1, 1))
    S1, S2 = amplitudes(k0, k1, a, ct)
    eT = (np.cos(Theta) * np.cos(Phi))[:, None] * e + (np.cos(Theta) * np.sin(Phi))[:, None] * y \
        - np.sin(Theta)[:, None] * d
    eP = -np.sin(Phi)[:, None] * e + np.cos(Phi)[:, None] * y
    return (np.cos(Phi) * S2)[:, None] * eT / (-1j * k0) - (np.sin(Phi) * S1)[:, None] * eP / (-1j * k0)
