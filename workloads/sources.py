"""Known exact fields for accuracy tests (inputs and expected values only).

The current loop of the numerical examples (Section 6, eq. loop): a circle
of radius a in the plane z = z0 around (x0, y0, z0) carrying the vector
potential A(x) = int_loop G^k(x, y) dl(y), G^k = e^{ik|x-y|}/(4 pi |x-y|), and

    E = curl A,    H = (1/(i omega mu)) curl curl A,

a Maxwell field with wavenumber k everywhere off the loop.  The line integral
is periodic and smooth away from the loop, so the trapezoid rule in the loop
angle converges geometrically; 256 points are far beyond double precision at
the distances used here.
"""
from __future__ import annotations

import numpy as np

LOOP_CENTER = (0.4, 0.5, 5.0)
LOOP_RADIUS = 0.42


def current_loop_field(points, k, omega, mu, center=LOOP_CENTER, radius=LOOP_RADIUS, n_seg=256, chunk=2048):
    """E and H [npts, 3] of the loop at the given points [npts, 3]."""
    x = np.atleast_2d(np.asarray(points, float))
    if len(x) > chunk:
        parts = [current_loop_field(x[i:i + chunk], k, omega, mu, center, radius, n_seg, chunk)
                 for i in range(0, len(x), chunk)]
        return np.concatenate([p[0] for p in parts]), np.concatenate([p[1] for p in parts])
    c = np.asarray(center, float)
    s = 2 * np.pi * np.arange(n_seg) / n_seg
    y = c[None, :] + radius * np.stack([np.cos(s), np.sin(s), np.zeros_like(s)], -1)      # [S, 3]
    dl = (2 * np.pi / n_seg) * radius * np.stack([-np.sin(s), np.cos(s), np.zeros_like(s)], -1)
    Rv = x[:, None, :] - y[None, :, :]                                                    # [P, S, 3]
    R = np.linalg.norm(Rv, axis=-1)
    Rh = Rv / R[..., None]
    g = np.exp(1j * k * R) / (4 * np.pi * R)
    # curl (G dl) = grad G x dl, grad G = G (ik - 1/R) Rh
    E = np.einsum("ps,psk->pk", g * (1j * k - 1 / R), np.cross(Rh, dl[None, :, :]))
    # curl curl (G dl) = G [(k^2 + ik/R - 1/R^2) dl + (-k^2 - 3ik/R + 3/R^2)(Rh.dl) Rh]
    a = g * (k * k + 1j * k / R - 1 / R ** 2)
    b = g * (-k * k - 3j * k / R + 3 / R ** 2) * np.einsum("psk,sk->ps", Rh, dl)
    CC = np.einsum("ps,sk->pk", a, dl) + np.einsum("ps,psk->pk", b, Rh)
    H = CC / (1j * omega * mu)
    return E, H


def ring_points(r, z, n_theta):
    """Ring points [N, n_theta, 3] of nodes (r_i, z_i) at theta_t = 2 pi t / n_theta."""
    th = 2 * np.pi * np.arange(n_theta) / n_theta
    r = np.asarray(r, float)[:, None]
    z = np.asarray(z, float)[:, None]
    return np.stack([r * np.cos(th)[None, :], r * np.sin(th)[None, :], np.broadcast_to(z, (len(r), n_theta))], -1)
