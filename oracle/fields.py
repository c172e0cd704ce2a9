"""Modal incident data and far fields.

* Incident plane wave (eq. pw): E = e exp(i k0 d.x), H = (k0/(omega mu0)) d x e
  exp(i k0 d.x), e the unit polarisation (the printed (d x p) x d is not a
  unit vector unless p is orthogonal to d; it is normalised).
* Modal data: the tangential traces n x E, n x H at each node ring, split into
  (t, theta) components with n x v = v_theta t - v_t e_theta, and their
  Fourier coefficients f_m = (1/2pi) int f(theta) e^{-i m theta} dtheta by the
  trapezoid rule in theta.  Rows are scaled as in eq. mullerrep (i omega eps0
  for the E rows, i omega mu0 for the H rows) or eq. dualmullrep.
* Far field: letting |x| -> oo in eq. exteriorfield,
  E_oo(xh) = (1/4pi) [ -(k0^2/(i omega eps0)) (Jh - (xh.Jh) xh) + i k0 xh x Mh ],
  Jh = int_Gamma exp(-i k0 xh.y) J(y) da(y); the last term of the printed
  eq. farfieldform integrates J where eq. exteriorfield has M.  The surface
  integral uses the nodes' ds-weights along the curve and the trapezoid rule
  in theta.
* Fields at points off the surface: eq. exteriorfield (exterior, k0) and
  eq. interiorfield (direct form) or eq. interior_dual (indirect form) in the
  body (k1), with
    curl S J (x)      = int grad_x G x J da = int G (ik - 1/R) Rh x J da,
    curl curl S J (x) = int G [(k^2 + ik/R - 1/R^2) J + (-k^2 - 3ik/R + 3/R^2)(Rh.J) Rh] da,
  R = x - y, Rh = R/|R| (the second from curl curl = grad div + k^2 off the
  surface).  The surface rule is refined for points near the surface: each
  panel split into sub-panels (geometry and currents from the panel's
  interpolants), and more azimuths the closer the nearest point.
* Modal data from sampled fields: the same traces and scaling as for the
  plane wave, from E and H given at the ring points.
"""
from __future__ import annotations

import numpy as np

from .system import node_geometry, wavenumbers, coefficients


def _frame(theta):
    c, s = np.cos(theta), np.sin(theta)
    er = np.stack([c, s, np.zeros_like(c)], -1)
    et = np.stack([-s, c, np.zeros_like(c)], -1)
    return er, et


def modal_rhs(curve, media, M, waves, formulation=0, n_theta=None):
    """b[q, 4N, nrhs] for modes q = m + M and the given plane waves."""
    geo = node_geometry(curve)
    k0, _ = wavenumbers(media)
    co = coefficients(media, formulation)
    if n_theta is None:
        n_theta = 2 * M + 2 * int(np.ceil(abs(k0) * np.max(geo.r))) + 64
    th = 2 * np.pi * np.arange(n_theta) / n_theta
    er, et = _frame(th)
    ez = np.array([0.0, 0.0, 1.0])
    N = curve.N
    ms = np.arange(-M, M + 1)
    E_ph = np.exp(-1j * np.outer(th, ms)) / n_theta      # [theta, modes]
    b = np.zeros((2 * M + 1, 4 * N, len(waves)), dtype=complex)
    for w_i, wv in enumerate(waves):
        hvec = (k0 / (media.omega * complex(media.mu0))) * np.cross(wv.d, wv.e)
        for i in range(N):
            x = geo.r[i] * er + geo.z[i] * ez            # [theta, 3]
            ph = np.exp(1j * k0 * (x @ wv.d))
            for fvec, rows, sc in ((wv.e, (0, 1), co["sE"]), (hvec, (2, 3), co["sH"])):
                v = ph[:, None] * fvec[None, :]
                vr = (v * er).sum(1); vth = (v * et).sum(1); vz = v[:, 2]
                vt = geo.rp[i] * vr + geo.zp[i] * vz
                b[:, 4 * i + rows[0], w_i] = sc * (vth @ E_ph)
                b[:, 4 * i + rows[1], w_i] = sc * (-vt @ E_ph)
    return b


def far_field(curve, media, M, x, directions, n_theta=None):
    """E_oo at unit directions [nd, 3] for modal currents x[q, 4N, nrhs];
    returns [nrhs, nd, 3]."""
    geo = node_geometry(curve)
    k0, _ = wavenumbers(media)
    if n_theta is None:
        n_theta = 2 * M + 2 * int(np.ceil(abs(k0) * np.max(geo.r))) + 64
    th = 2 * np.pi * np.arange(n_theta) / n_theta
    er, et = _frame(th)
    ez = np.array([0.0, 0.0, 1.0])
    ms = np.arange(-M, M + 1)
    E_ph = np.exp(1j * np.outer(th, ms))                 # [theta, modes]
    N = curve.N
    nrhs = x.shape[2]
    dirs = np.asarray(directions, float)
    out = np.zeros((nrhs, len(dirs), 3), dtype=complex)
    for i in range(N):
        y = geo.r[i] * er + geo.z[i] * ez                 # [theta, 3]
        t = geo.rp[i] * er + geo.zp[i] * ez
        da = geo.w[i] * geo.r[i] * (2 * np.pi / n_theta)
        ph = np.exp(-1j * k0 * (y @ dirs.T)) * da         # [theta, nd]
        for comp in range(nrhs):
            J1 = E_ph @ x[:, 4 * i + 0, comp]; J2 = E_ph @ x[:, 4 * i + 1, comp]
            M1 = E_ph @ x[:, 4 * i + 2, comp]; M2 = E_ph @ x[:, 4 * i + 3, comp]
            Jv = J1[:, None] * t + J2[:, None] * et       # [theta, 3]
            Mv = M1[:, None] * t + M2[:, None] * et
            Jh = ph.T @ Jv; Mh = ph.T @ Mv                 # [nd, 3]
            out[comp] += _combine(Jh, Mh, dirs, k0, media)
    return out


def _combine(Jh, Mh, dirs, k0, media):
    xJ = (dirs * Jh).sum(1, keepdims=True)
    pre = -(k0 ** 2) / (1j * media.omega * complex(media.eps0))
    return (pre * (Jh - xJ * dirs) + 1j * k0 * np.cross(dirs, Mh)) / (4 * np.pi)


def modal_rhs_samples(curve, media, M, EH, formulation=0):
    """b[q, 4N, nrhs] from incident fields sampled at the ring points:
    EH[nrhs, N, n_theta, 6] holds (E, H) in Cartesian components at
    (r_i cos th_t, r_i sin th_t, z_i), th_t = 2 pi t / n_theta."""
    geo = node_geometry(curve)
    co = coefficients(media, formulation)
    EH = np.asarray(EH, complex)
    nrhs, N, n_theta, _ = EH.shape
    th = 2 * np.pi * np.arange(n_theta) / n_theta
    er, et = _frame(th)
    ms = np.arange(-M, M + 1)
    E_ph = np.exp(-1j * np.outer(th, ms)) / n_theta
    b = np.zeros((2 * M + 1, 4 * N, nrhs), dtype=complex)
    for w_i in range(nrhs):
        for i in range(N):
            for sl, rows, sc in ((slice(0, 3), (0, 1), co["sE"]), (slice(3, 6), (2, 3), co["sH"])):
                v = EH[w_i, i, :, sl]
                vr = (v * er).sum(1); vth = (v * et).sum(1); vz = v[:, 2]
                vt = geo.rp[i] * vr + geo.zp[i] * vz
                b[:, 4 * i + rows[0], w_i] = sc * (vth @ E_ph)
                b[:, 4 * i + rows[1], w_i] = sc * (-vt @ E_ph)
    return b


def field_coefficients(media, region, formulation=0):
    """(k, cJ, cM, dM, dJ) with E = cJ curl curl S J + cM curl S M and
    H = dM curl curl S M + dJ curl S J in the region (0 exterior, 1 body)."""
    k0, k1 = wavenumbers(media)
    om = media.omega
    e0, e1, u0, u1 = (complex(media.eps0), complex(media.eps1), complex(media.mu0), complex(media.mu1))
    if region == 0:                      # eq. exteriorfield
        return k0, -1 / (1j * om * e0), 1.0, 1 / (1j * om * u0), 1.0
    if formulation == 0:                 # eq. interiorfield
        return k1, 1 / (1j * om * e1), -1.0, -1 / (1j * om * u1), -1.0
    return k1, -1 / (1j * om * e0), u1 / u0, 1 / (1j * om * u0), e1 / e0   # eq. interior_dual


def near_field(curve, media, M, x, targets, region, formulation=0, n_theta=None, upsample=8):
    """E, H [nrhs, nt, 3] at points targets [nt, 3] off the surface, from modal
    currents x[q, 4N, nrhs]; region 0 = exterior, 1 = inside the body.  Each
    panel is split into `upsample` sub-panels of 16 Gauss points, geometry
    and currents from the panel's degree-15 interpolants of the node values;
    the azimuthal rule has max(2M + 2 ceil(|k| r_max) + 64, 40 r_max / d)
    points, d the smallest target-to-node distance in the meridian plane."""
    from .gauss import gauss_legendre, lagrange_basis
    geo = node_geometry(curve)
    k, cJ, cM, dM, dJ = field_coefficients(media, region, formulation)
    X = np.atleast_2d(np.asarray(targets, float))
    rt, zt = np.hypot(X[:, 0], X[:, 1]), X[:, 2]
    dmin = np.min(np.hypot(rt[:, None] - geo.r[None, :], zt[:, None] - geo.z[None, :]))
    if n_theta is None:
        n_theta = 2 * M + 2 * int(np.ceil(abs(k) * np.max(geo.r))) + 64
        n_theta = max(n_theta, int(np.ceil(40 * np.max(geo.r) / dmin)))
    xg, wg = gauss_legendre(16)
    U = int(upsample)
    tsub = np.concatenate([-1 + (2 * u + 1 + xg) / U for u in range(U)])      # [16U] in the panel parameter
    wsub = np.concatenate([wg / U] * U)
    Lr = lagrange_basis(xg, tsub)                                             # [16U, 16]
    th = 2 * np.pi * np.arange(n_theta) / n_theta
    er, et = _frame(th)
    ez = np.array([0.0, 0.0, 1.0])
    ms = np.arange(-M, M + 1)
    E_ph = np.exp(1j * np.outer(th, ms))                  # [theta, modes]
    nrhs = x.shape[2]
    E = np.zeros((nrhs, len(X), 3), dtype=complex)
    H = np.zeros_like(E)
    for P in range(curve.n_panels):
        sl = slice(16 * P, 16 * P + 16)
        r_s, z_s = Lr @ curve.r[sl], Lr @ curve.z[sl]
        dr_s, dz_s = Lr @ curve.dr[sl], Lr @ curve.dz[sl]
        sp = np.hypot(dr_s, dz_s)
        xs = np.einsum("sk,qkaw->qsaw", Lr, x[:, 64 * P:64 * (P + 1), :].reshape(len(ms), 16, 4, nrhs))
        for i in range(len(tsub)):
            y = r_s[i] * er + z_s[i] * ez                  # [T, 3]
            t = (dr_s[i] / sp[i]) * er + (dz_s[i] / sp[i]) * ez
            da = wsub[i] * sp[i] * r_s[i] * (2 * np.pi / n_theta)
            cur = [E_ph @ xs[:, i, a, :] for a in range(4)]                   # 4 x [T, nrhs]
            Jv = cur[0][..., None] * t[:, None, :] + cur[1][..., None] * et[:, None, :]   # [T, nrhs, 3]
            Mv = cur[2][..., None] * t[:, None, :] + cur[3][..., None] * et[:, None, :]
            Rv = X[None, :, :] - y[:, None, :]             # [T, nt, 3]
            R = np.linalg.norm(Rv, axis=-1)
            Rh = Rv / R[..., None]
            g = da * np.exp(1j * k * R) / (4 * np.pi * R)
            c1 = g * (1j * k - 1 / R)
            a = g * (k * k + 1j * k / R - 1 / R ** 2)
            b = g * (-k * k - 3j * k / R + 3 / R ** 2)

            def curl(V):      # [nrhs, nt, 3]
                return np.einsum("tp,twpk->wpk", c1, np.cross(Rh[:, None, :, :], V[:, :, None, :]))

            def curlcurl(V):
                proj = np.einsum("tpk,twk->twp", Rh, V)
                return (np.einsum("tp,twk->wpk", a, V) + np.einsum("tp,twp,tpk->wpk", b, proj, Rh))

            E += cJ * curlcurl(Jv) + cM * curl(Mv)
            H += dM * curlcurl(Mv) + dJ * curl(Jv)
    return E, H
