"""Per-mode Mueller systems (Sections 2-3 and 5), assembled the plain way.

Unknowns at node j (index 4j + b): b = 0 J^1, 1 J^2, 2 M^1, 3 M^2 with
J = J^1 t + J^2 e_theta (Section 3).  Equations at node i (row 4i + a):
a = 0 E_t, 1 E_theta, 2 H_t, 3 H_theta (tangential components of the two
vector equations of eq. mullerrep, or eq. dualmullrep for the indirect form).

Readings of the paper applied here:
* g^2_m = (g_{m+1} + g_{m-1})/2 and g^3_m = (g_{m-1} - g_{m+1})/2, which is
  what the definitions of eqs. green21/green31 give (the printed relation
  after eq. equrelation carries a spurious factor 1/i).
* Cylindrical components follow Lemma 1 (eqs. equc1-equc3).  The tangential
  part of n x v is v_theta t - v_t e_theta with v_t = r' v_r + z' v_z (a
  direct evaluation of the cross product with n = z' e_r - r' e_z in the
  right-handed frame (e_r, e_theta, e_z)); the theta components printed for
  N and K in Section 3 carry the opposite sign and are not used.
* K J = n x (k^2 S J + grad div S J), with div and grad in cylindrical
  coordinates; only K^{k0} - K^{k1} is formed, from the k0-k1 difference
  kernels (Section 4.3).
* L2 weighting (Section 6 remark): rows are scaled by sqrt(w_i) and columns
  by 1/sqrt(w_j), w the ds-weights of the nodes; the weighting is a
  similarity transform and does not change the solution.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import gauss
from .green import modal_families_batch

P = gauss.P


@dataclass
class Geometry:
    r: np.ndarray
    z: np.ndarray
    rp: np.ndarray   # unit tangent r'
    zp: np.ndarray   # unit tangent z'
    w: np.ndarray    # ds weights
    speed: np.ndarray


def node_geometry(curve) -> Geometry:
    _, wg = gauss.gauss_legendre(P)
    speed = np.hypot(curve.dr, curve.dz)
    w = np.tile(wg, curve.n_panels) * speed
    return Geometry(curve.r.copy(), curve.z.copy(), curve.dr / speed, curve.dz / speed, w, speed)


def wavenumbers(media):
    k0 = media.omega * np.sqrt(complex(media.eps0) * complex(media.mu0))
    k1 = media.omega * np.sqrt(complex(media.eps1) * complex(media.mu1))
    return complex(k0), complex(k1)


def junction_is_corner(curve, A: int, B: int) -> bool:
    """Whether the curve turns by more than 10 degrees where panel A's end
    (tau = +1) meets panel B's start (tau = -1): the end tangents are the
    panels' degree-15 Lagrange interpolants of (dr, dz) at tau = +1 and -1."""
    x, _ = gauss.gauss_legendre(P)
    Lp = gauss.lagrange_basis(x, np.array([1.0]))[0]
    Lm = gauss.lagrange_basis(x, np.array([-1.0]))[0]
    sa, sb = slice(A * P, (A + 1) * P), slice(B * P, (B + 1) * P)
    ta = np.array([Lp @ curve.dr[sa], Lp @ curve.dz[sa]])
    tb = np.array([Lm @ curve.dr[sb], Lm @ curve.dz[sb]])
    return float(ta @ tb / (np.linalg.norm(ta) * np.linalg.norm(tb))) < np.cos(np.deg2rad(10.0))


def panel_support(curve, target_panel: int, target_local: int, Q: int):
    """Support points on source panel Q for a target node, as
    (r, z, r', z', W, L, disp) with W the ds-weights, L[s, k] the Lagrange
    basis and disp = (r_t - r_s, z_t - z_s) for the target's own panel (None
    otherwise); None for a far panel (plain Gauss-Legendre).

    On the own panel the displacement is formed as
    x_t - x_s = -sum_{k != a} L_k(tau_s) (x_k - x_a), which equals the
    difference of interpolated and node positions but keeps its relative
    accuracy when the support point is very close to the target."""
    nP = curve.n_panels
    if Q == target_panel:
        tau, wt = gauss.self_rule(target_local)
    else:
        # panels sharing an endpoint with the target's panel take the near
        # rule (Section 5); a closed curve also wraps around, which needs at
        # least 3 panels for the two neighbours to be distinct
        wrap = curve.closed and nP > 2
        nxt = target_panel + 1 if target_panel + 1 < nP else (0 if wrap else None)
        prv = target_panel - 1 if target_panel - 1 >= 0 else (nP - 1 if wrap else None)
        if Q == nxt:
            tau, wt = gauss.adjacent_rule(-1, junction_is_corner(curve, target_panel, Q))
        elif Q == prv:
            tau, wt = gauss.adjacent_rule(+1, junction_is_corner(curve, Q, target_panel))
        else:
            return None
    x, _ = gauss.gauss_legendre(P)
    L = gauss.lagrange_basis(x, tau)
    sl = slice(Q * P, (Q + 1) * P)
    r, z = L @ curve.r[sl], L @ curve.z[sl]
    dr, dz = L @ curve.dr[sl], L @ curve.dz[sl]
    sp = np.hypot(dr, dz)
    disp = None
    if Q == target_panel:
        a = target_local
        ra, za = curve.r[sl][a], curve.z[sl][a]
        others = [k for k in range(P) if k != a]
        disp = (-(L[:, others] @ (curve.r[sl][others] - ra)), -(L[:, others] @ (curve.z[sl][others] - za)))
    return r, z, dr / sp, dz / sp, wt * sp, L, disp


def _gfam(F, fam, m):
    """G1, G2, G3 of one spectrum family for signed modes m (arrays [S, nm])."""
    f = F[:, fam, :] if isinstance(fam, int) else fam
    am, ap, a1 = np.abs(m - 1), np.abs(m + 1), np.abs(m)
    return f[:, a1], 0.5 * (f[:, ap] + f[:, am]), 0.5 * (f[:, am] - f[:, ap])


def operator_blocks(F, rs, rps, zps, rt, rpt, zpt, k0, k1, m):
    """Source-point contributions of N^{k0}, N^{k1} and K^{k0}-K^{k1}.

    F: [S, 9, M+2] spectra; source arrays [S]; returns three arrays
    [S, nm, 2, 2] (rows t, theta; columns J^1, J^2), without weights."""
    S = F.shape[0]
    fams = {
        "g0": F[:, 0], "g1": F[:, 1], "dr0": F[:, 2], "dz0": F[:, 3],
        "dr1": F[:, 4], "dz1": F[:, 5], "drr": F[:, 6], "drz": F[:, 7], "dzz": F[:, 8],
    }
    fams["W"] = k0 ** 2 * F[:, 0] - k1 ** 2 * F[:, 1]
    fams["D"] = F[:, 0] - F[:, 1]
    fams["drD"] = F[:, 2] - F[:, 4]
    fams["dzD"] = F[:, 3] - F[:, 5]
    mm = m[None, :]
    rsv, rpv, zpv = rs[:, None], rps[:, None], zps[:, None]

    def c(name):
        G1, G2, G3 = _gfam(None, fams[name], m)
        c1 = np.stack([rsv * rpv * G2, -1j * rsv * G3], -1)
        c2 = np.stack([1j * rsv * rpv * G3, rsv * G2], -1)
        c3 = np.stack([rsv * zpv * G1, np.zeros_like(G1)], -1)
        return c1, c2, c3

    cache = {}

    def C(name):
        if name not in cache:
            cache[name] = c(name)
        return cache[name]

    im = (1j * mm)[..., None]
    out = []
    for g, dr, dz in (("g0", "dr0", "dz0"), ("g1", "dr1", "dz1")):
        c1g, c2g, c3g = C(g)
        c1r, c2r, c3r = C(dr)
        c1z, c2z, c3z = C(dz)
        Nt = c1z - c3r
        Nth = -((zpt / rt) * (c2g + rt * c2r - im * c1g) + rpt * ((im / rt) * c3g - c2z))
        out.append(np.stack([Nt, Nth], -2))
    c1W, c2W, c3W = C("W")
    c1D, c2D, c3D = C("D")
    c1rD, c2rD, _ = C("drD")
    c1zD, c2zD, c3zD = C("dzD")
    c1rr, _, _ = C("drr")
    c1rz, _, c3rz = C("drz")
    _, _, c3zz = C("dzz")
    Kt = c2W + (im / rt ** 2) * c1D + (im / rt) * c1rD - (mm[..., None] ** 2 / rt ** 2) * c2D + (im / rt) * c3zD
    dPr = -c1D / rt ** 2 + c1rD / rt + c1rr - (im / rt ** 2) * c2D + (im / rt) * c2rD + c3rz
    dPz = c1zD / rt + c1rz + (im / rt) * c2zD + c3zz
    Kth = -(rpt * (c1W + dPr) + zpt * (c3W + dPz))
    out.append(np.stack([Kt, Kth], -2))
    return out


def coefficients(media, formulation: int):
    """Block coefficients of eq. mullerrep (0) or eq. dualmullrep (1)."""
    om = media.omega
    e0, e1, u0, u1 = (complex(media.eps0), complex(media.eps1), complex(media.mu0), complex(media.mu1))
    if formulation == 0:
        return dict(aEJ=1.0, x=(e0, e1), dEM=0.5j * om * (e0 + e1), y=(u0, u1),
                    dHJ=0.5j * om * (u0 + u1), aHM=-1.0, sE=1j * om * e0, sH=1j * om * u0)
    return dict(aEJ=u0 / e0, x=(u0, u1), dEM=-0.5j * om * (u0 + u1), y=(e0, e1),
                dHJ=-0.5j * om * (e0 + e1), aHM=-e0 / u0, sE=1j * om * u0, sH=1j * om * e0)


def assemble_row(curve, media, M: int, i: int, formulation: int = 0, modes=None, geo=None, lo_modes=None):
    """Rows 4i..4i+3 of the per-mode matrices (unweighted) for target node i:
    an array [len(modes), 4, 4N] (default all signed modes -M..M).  With
    ``lo_modes`` (a list of signed modes) also those modes' rows from the
    24-point azimuthal rule (see green.modal_families_batch), returned second:
    their difference from the same rows of the first is the oracle's own noise."""
    R = _assemble_row(curve, media, M, i, formulation, modes, geo, lo_modes)
    return R if lo_modes is not None else R[0]


def _assemble_row(curve, media, M, i, formulation, modes, geo, lo_modes):
    geo = node_geometry(curve) if geo is None else geo
    k0, k1 = wavenumbers(media)
    co = coefficients(media, formulation)
    N = curve.N
    ms = np.arange(-M, M + 1) if modes is None else np.asarray(modes)
    with_lo = lo_modes is not None
    mss = [ms] + ([np.asarray(lo_modes)] if with_lo else [])
    Rs = [np.zeros((len(m_), 4, 4 * N), dtype=complex) for m_ in mss]
    om = media.omega
    Pt, a = divmod(i, P)
    rt, zt, rpt, zpt = geo.r[i], geo.z[i], geo.rp[i], geo.zp[i]
    for Q in range(curve.n_panels):
        sup = panel_support(curve, Pt, a, Q)
        disp = None
        if sup is None:
            sl = slice(Q * P, (Q + 1) * P)
            rs, zs, rps, zps, W = geo.r[sl], geo.z[sl], geo.rp[sl], geo.zp[sl], geo.w[sl]
            L = np.eye(P)
        else:
            rs, zs, rps, zps, W, L, disp = sup
        Fs = modal_families_batch(rt, zt, rs, zs, k0, k1, M, disp=disp, return_lo=with_lo)
        for R, F, m_ in zip(Rs, Fs if with_lo else (Fs,), mss):
            N0, N1, KD = operator_blocks(F, rs, rps, zps, rt, rpt, zpt, k0, k1, m_)
            x0, x1 = co["x"]; y0, y1 = co["y"]
            EM = -1j * om * (x0 * N0 - x1 * N1)
            HJ = -1j * om * (y0 * N0 - y1 * N1)
            blk = np.zeros(N0.shape[:2] + (4, 4), dtype=complex)
            blk[..., 0:2, 0:2] = co["aEJ"] * KD
            blk[..., 0:2, 2:4] = EM
            blk[..., 2:4, 0:2] = HJ
            blk[..., 2:4, 2:4] = co["aHM"] * KD
            # contract support points into the panel's 16 columns
            contrib = np.einsum("s,sk,sqab->qkab", W, L, blk)
            for k in range(P):
                j = Q * P + k
                R[:, :, 4 * j:4 * j + 4] += contrib[:, k]
    for R in Rs:
        R[:, 0, 4 * i + 2] += co["dEM"]
        R[:, 1, 4 * i + 3] += co["dEM"]
        R[:, 2, 4 * i + 0] += co["dHJ"]
        R[:, 3, 4 * i + 1] += co["dHJ"]
    return Rs


def assemble(curve, media, M: int, formulation: int = 0, modes=None, rows=None, progress=None):
    """Dense per-mode matrices A[q] (q = m + M), unweighted, n = 4N.

    ``modes``: optional list of signed modes to return (default all);
    ``rows``: optional list of target nodes to fill (other rows stay 0)."""
    geo = node_geometry(curve)
    N = curve.N
    ms = np.arange(-M, M + 1) if modes is None else np.asarray(modes)
    A = np.zeros((len(ms), 4 * N, 4 * N), dtype=complex)
    rows = range(N) if rows is None else rows
    for i in rows:
        A[:, 4 * i:4 * i + 4, :] = assemble_row(curve, media, M, i, formulation, ms, geo)
        if progress:
            progress(i)
    return A


def l2_weights(curve):
    """sqrt of the ds-weights, repeated for the 4 unknowns of each node."""
    return np.repeat(np.sqrt(node_geometry(curve).w), 4)


def weight_matrix(A, sw):
    """L2 weighting: A' = diag(sw) A diag(1/sw)."""
    return A * sw[None, :, None] / sw[None, None, :]


def block(curve, media, M: int, i: int, j: int, formulation: int = 0, modes=None, noise=False):
    """The 4x4 blocks A_m[4i:4i+4, 4j:4j+4] (unweighted) for the given modes,
    computed for this one (target node, column node) pair: the source panel's
    support points if it is near the target's panel, else the single node.

    With ``noise`` also returns |block(32-point spectra) - block(24-point
    spectra)|, the oracle's own noise level for each entry."""
    geo = node_geometry(curve)
    k0, k1 = wavenumbers(media)
    co = coefficients(media, formulation)
    ms = np.arange(-M, M + 1) if modes is None else np.asarray(modes)
    Pt, a = divmod(i, P)
    Q, kloc = divmod(j, P)
    rt, zt, rpt, zpt = geo.r[i], geo.z[i], geo.rp[i], geo.zp[i]
    sup = panel_support(curve, Pt, a, Q)
    disp = None
    if sup is None:
        rs, zs, rps, zps, W = (np.array([v[j]]) for v in (geo.r, geo.z, geo.rp, geo.zp, geo.w))
        Lk = np.ones(1)
    else:
        rs, zs, rps, zps, W, L, disp = sup
        Lk = L[:, kloc]
    F, F_lo = modal_families_batch(rt, zt, rs, zs, k0, k1, M, disp=disp, return_lo=True)
    om = media.omega
    x0, x1 = co["x"]; y0, y1 = co["y"]

    def contract(Fv):
        N0, N1, KD = operator_blocks(Fv, rs, rps, zps, rt, rpt, zpt, k0, k1, ms)
        blk = np.zeros(N0.shape[:2] + (4, 4), dtype=complex)
        blk[..., 0:2, 0:2] = co["aEJ"] * KD
        blk[..., 0:2, 2:4] = -1j * om * (x0 * N0 - x1 * N1)
        blk[..., 2:4, 0:2] = -1j * om * (y0 * N0 - y1 * N1)
        blk[..., 2:4, 2:4] = co["aHM"] * KD
        return np.einsum("s,s,sqab->qab", W, Lk, blk)

    out = contract(F)
    if i == j:
        out[:, 0, 2] += co["dEM"]; out[:, 1, 3] += co["dEM"]
        out[:, 2, 0] += co["dHJ"]; out[:, 3, 1] += co["dHJ"]
    if noise:
        lo = contract(F_lo)
        if i == j:
            lo[:, 0, 2] += co["dEM"]; lo[:, 1, 3] += co["dEM"]
            lo[:, 2, 0] += co["dHJ"]; lo[:, 3, 1] += co["dHJ"]
        return out, np.abs(out - lo)
    return out
