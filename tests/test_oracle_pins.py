"""Pins of the oracle against facts that do not come from the oracle itself:
closed forms, an independent extended-precision integrator, finite
differences, the Jacobi-Anger expansion, library LU, exact moments, the
reflection symmetry and the Mie series."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import gauss, green, linalg, fields, mie, system

mp = pytest.importorskip("mpmath")


# ---------------------------------------------------------------- rules
@pytest.mark.parametrize("j", [0, 1, 2, 7, 9, 15])
def test_self_rule_exact_log_moments(j):
    """The self-panel reference rule (16-node generalized Gaussian rule of the
    near-rule data) integrates P_j(2u-1) and P_j(2u-1) log u on [0, 1]
    exactly: moments delta_j0 and -1 (j = 0) or (-1)^(j+1)/(j(j+1)), the
    closed forms of the shifted Legendre polynomials (Remark of Section 5)."""
    u, w = gauss.self_side_rule()
    assert len(u) == 16 and (w > 0).all() and (np.diff(u) > 0).all() and 0 < u[0] and u[-1] < 1
    Pj = np.polynomial.legendre.Legendre.basis(j)(2 * u - 1)
    assert abs((w * Pj).sum() - (1.0 if j == 0 else 0.0)) < 2e-15
    ref = -1.0 if j == 0 else (-1.0) ** (j + 1) / (j * (j + 1))
    assert abs((w * Pj * np.log(u)).sum() - ref) < 2e-15


def test_self_rule_beyond_its_class():
    """Integrands outside the rule's exact class (analytic factors of higher
    degree) still come out to about 1e-13 on a side, against mpmath."""
    u, w = gauss.self_side_rule()
    f = lambda v: np.exp(2 * v) * np.log(v) + np.sin(4 * v) + np.cos(5 * v) * np.log(v)
    ex = mp.quad(lambda v: mp.exp(2 * v) * mp.log(v) + mp.sin(4 * v) + mp.cos(5 * v) * mp.log(v), [0, 1])
    assert abs((w * f(u)).sum() - float(ex)) < 1e-14


@pytest.mark.parametrize("i", [0, 5, 15])
def test_self_rule_on_panel(i):
    """Full self rule at target tau_i: int_{-1}^{1} P(t) log|t - tau_i| dt for a
    degree-15 polynomial, against mpmath."""
    tau, wt = gauss.self_rule(i)
    x, _ = gauss.gauss_legendre(16)
    ti = x[i]
    coef = np.cos(np.arange(16) * 0.7)
    f = lambda t: np.polynomial.legendre.legval(t, coef)
    num = (wt * f(tau) * np.log(np.abs(tau - ti))).sum()
    ex = mp.quad(lambda t: mp.mpf(float(f(float(t)))) * mp.log(abs(t - ti)), [-1, ti, 1])
    assert abs(num - float(ex)) < 1e-14


@pytest.mark.parametrize("delta", [0.0053, 0.02, 0.3])
def test_adjacent_rule(delta):
    """Adjacent rule: smooth x log|t + 1 + delta| over the panel."""
    tau, wt = gauss.adjacent_rule(-1)
    f = lambda t: np.cos(2 * t) * np.log(np.abs(t + 1 + delta)) + t ** 9
    num = (wt * f(tau)).sum()
    ex = mp.quad(lambda t: mp.cos(2 * t) * mp.log(t + 1 + delta) + t ** 9, [-1, 1])
    assert abs(num - float(ex)) < 2e-15


@pytest.mark.parametrize("delta,angle,j", [(0.0026, 180.0, 0), (0.0026, 180.0, 15), (0.02, 150.0, 7),
                                           (0.3, 135.0, 15), (1.9, 170.0, 3), (0.0041, 140.0, 11)])
def test_adjacent_smooth_rule(delta, angle, j):
    """Neighbouring-panel rule for smooth junctions: P_j(2u-1) log|u - s| with
    the singular point s = delta e^{i angle} beside the shared endpoint
    (including values between the ones the rule was built on), against mpmath."""
    u, w = gauss.near_rule_table("ADJ_U"), gauss.near_rule_table("ADJ_W")
    assert (w > 0).all() and 0 < u.min() and u.max() < 1
    sr, si = delta * math.cos(math.radians(angle)), delta * math.sin(math.radians(angle))
    Pj = np.polynomial.legendre.Legendre.basis(j)
    f = lambda v: Pj(2 * v - 1) * 0.5 * np.log((v - sr) ** 2 + si ** 2)
    g = lambda v: mp.legendre(j, 2 * v - 1) * 0.5 * mp.log((v - sr) ** 2 + si ** 2)
    ex = mp.quad(g, [0, min(1.0, 4 * delta), 1]) if 4 * delta < 1 else mp.quad(g, [0, 1])
    l1 = mp.quad(lambda v: abs(g(v)), [0, min(1.0, 4 * delta), 1]) if 4 * delta < 1 else mp.quad(lambda v: abs(g(v)), [0, 1])
    assert abs((w * f(u)).sum() - float(ex)) < 1e-13 * float(l1)


def test_junction_corners():
    """Junctions where the curve turns by more than 10 degrees take the corner
    rule: the cylinder's two edges, the cone's rim; none on smooth curves."""
    cyl = W.cylinder(3)
    corners = [j for j in range(cyl.n_panels - 1) if system.junction_is_corner(cyl, j, j + 1)]
    assert len(corners) == 2
    for j in corners:                      # at r = 1, z = +-1
        assert abs(cyl.r[16 * j + 15] - 1.0) < 0.05 and abs(abs(cyl.z[16 * j + 15]) - 1.0) < 0.05
    cone = W.cone(3, 1.0, 0.7)
    assert sum(system.junction_is_corner(cone, j, j + 1) for j in range(cone.n_panels - 1)) == 1
    for smooth in (W.sphere(6), W.random_body(12, seed=3)):
        assert not any(system.junction_is_corner(smooth, j, j + 1) for j in range(smooth.n_panels - 1))
    tor = W.torus(8)
    assert not any(system.junction_is_corner(tor, j, (j + 1) % 8) for j in range(8))


def test_lagrange_basis_interpolates():
    x, _ = gauss.gauss_legendre(16)
    L = gauss.lagrange_basis(x, x)
    assert np.allclose(L, np.eye(16), atol=1e-14)
    t = np.linspace(-1, 1, 7)
    assert np.allclose(gauss.lagrange_basis(x, t) @ x ** 11, t ** 11, atol=1e-13)


# ---------------------------------------------------------------- modal kernels
def _chi(rt, zt, rs, zs):
    rt, zt, rs, zs = (mp.mpf(v) for v in (rt, zt, rs, zs))
    return (rt ** 2 + rs ** 2 + (zt - zs) ** 2) / (2 * rt * rs)


PAIRS = [(1.0, 0.0, 0.9, 0.1), (0.5, 0.2, 0.5, 0.2 + 1e-7), (0.5, 0.2, 0.5 + 3e-9, 0.2 + 1e-9),
         (1.0, 0.0, 0.3, 2.0), (0.02, -0.99, 0.01, -0.995)]


@pytest.mark.parametrize("pair", PAIRS)
def test_green_k0_closed_form(pair):
    """k = 0: g_m = Q_{m-1/2}(chi) / (2 pi sqrt(r_t r_s)) (eq. lm)."""
    rt, zt, rs, zs = pair
    F = green.modal_families(rt, zt, rs, zs, 0.0, 0.0, 8)
    with mp.workdps(40):
        chi = _chi(*pair)
        for m in (0, 1, 4, 9):
            ex = mp.legenq(m - 0.5, 0, chi, type=3) / (2 * mp.pi * mp.sqrt(mp.mpf(rt) * rs))
            assert abs(F[0, m] - complex(ex)) <= 2e-15 * abs(F[0, 0]) + 1e-300


@pytest.mark.parametrize("pair", [(1.0, 0.0, 0.95, 0.02), (0.7, 0.3, 0.7001, 0.3002)])
def test_green_against_mpmath_quadrature(pair):
    """All nine families against mpmath's tanh-sinh quadrature of the same
    definitions (an independent integrator, 30 digits)."""
    rt, zt, rs, zs = pair
    k0, k1 = 2.0, 3.0 + 0.05j
    M = 5
    F = green.modal_families(rt, zt, rs, zs, k0, k1, M)
    s = math.sqrt(((rt - rs) ** 2 + (zt - zs) ** 2) / (rt * rs))
    pts = [0, s / 4, s, 4 * s, mp.pi]
    for f in (0, 3, 4, 6, 7, 8):
        for m in (0, 3, 6):
            def integrand(phi, f=f, m=m):
                val = green.integrands(rt, zt, rt - rs, zt - zs, k0, k1, np.array([float(phi)]))[f, 0]
                return mp.mpc(val.real, val.imag) * mp.cos(m * phi)
            with mp.workdps(30):
                ex = 2 * mp.quad(integrand, pts)
            scale = np.max(np.abs(F[f]))
            assert abs(F[f, m] - complex(ex)) < 1e-13 * scale, (f, m)


def test_green_derivatives_by_finite_differences():
    """F2..F5 are d/dr_t, d/dz_t of F0, F1 and F6..F8 the second derivatives
    of F0 - F1: five-point central differences."""
    rt, zt, rs, zs = 0.8, 0.1, 0.6, -0.2
    k0, k1, M = 3.0, 4.5 + 0.1j, 6
    h = 1e-3
    f = lambda a, b: green.modal_families(a, b, rs, zs, k0, k1, M)
    F = f(rt, zt)
    d_r = lambda g: (-g(rt + 2 * h, zt) + 8 * g(rt + h, zt) - 8 * g(rt - h, zt) + g(rt - 2 * h, zt)) / (12 * h)
    d_z = lambda g: (-g(rt, zt + 2 * h) + 8 * g(rt, zt + h) - 8 * g(rt, zt - h) + g(rt, zt - 2 * h)) / (12 * h)
    Fr, Fz = d_r(f), d_z(f)
    tol = 1e-9 * np.abs(F).max()
    assert np.abs(Fr[0] - F[2]).max() < tol and np.abs(Fz[0] - F[3]).max() < tol
    assert np.abs(Fr[1] - F[4]).max() < tol and np.abs(Fz[1] - F[5]).max() < tol
    # second derivatives: 5-point differences of the first-derivative families
    Dr = lambda a, b: f(a, b)[2] - f(a, b)[4]
    Dz = lambda a, b: f(a, b)[3] - f(a, b)[5]
    tol2 = 1e-8 * np.abs(F[6:]).max()
    assert np.abs(d_r(Dr) - F[6]).max() < tol2
    assert np.abs(d_z(Dr) - F[7]).max() < tol2
    assert np.abs(d_r(Dz) - F[7]).max() < tol2
    assert np.abs(d_z(Dz) - F[8]).max() < tol2


def test_difference_kernel_series_branch_continuous():
    """The Taylor branch of the k0-k1 difference agrees with the direct
    difference where both are accurate (max|k| rho = 1/2)."""
    k0, k1 = 2.0, 3.0 + 0.2j
    rho = np.array([0.5 / abs(k1)])
    for order, idx in ((1, 0), (2, 1)):
        ser = green._series_diff(k0, k1, rho, order)
        e0, e1 = np.exp(1j * k0 * rho), np.exp(1j * k1 * rho)
        if order == 1:
            ref = (e0 * (1j * k0 * rho - 1) - e1 * (1j * k1 * rho - 1)) / (4 * np.pi * rho ** 2)
        else:
            ref = (e0 * (2 - 2j * k0 * rho - (k0 * rho) ** 2) - e1 * (2 - 2j * k1 * rho - (k1 * rho) ** 2)) / (4 * np.pi * rho ** 3)
        assert abs(ser[0] - ref[0]) < 1e-12 * abs(ref[0])


# ---------------------------------------------------------------- linear algebra
def test_lu_against_scipy():
    sla = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(3)
    n = 40
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    b = rng.standard_normal((n, 3)) + 1j * rng.standard_normal((n, 3))
    LU, piv = linalg.lu_factor(A)
    x = linalg.lu_solve(LU, piv, b)
    xr = sla.lu_solve(sla.lu_factor(A), b)
    assert np.abs(x - xr).max() < 1e-12 * np.abs(xr).max()
    P = np.eye(n)[piv]
    L = np.tril(LU, -1) + np.eye(n); U = np.triu(LU)
    assert np.abs(P @ A - L @ U).max() < 1e-13 * np.abs(A).max()


def test_lu_pivot_ties_lowest_row():
    A = np.array([[1.0, 2.0], [1.0, 3.0]], dtype=complex)
    _, piv = linalg.lu_factor(A)
    assert list(piv) == [0, 1]
    with pytest.raises(ZeroDivisionError):
        linalg.lu_factor(np.zeros((2, 2)))


# ---------------------------------------------------------------- incident data
def test_rhs_jacobi_anger():
    """Modal plane-wave data against the Jacobi-Anger expansion
    exp(i a cos(t - t_d)) = sum_n i^n J_n(a) exp(i n (t - t_d))."""
    from scipy.special import jv
    cur = W.sphere(2)
    med = W.Media.from_k(2.0, 3.0)
    M = 7
    wv = W.paper_default_wave()
    b = fields.modal_rhs(cur, med, M, [wv])
    geo = system.node_geometry(cur)
    k0 = 2.0
    dperp = math.hypot(wv.d[0], wv.d[1]); thd = math.atan2(wv.d[1], wv.d[0])
    sE = 1j * med.omega
    for i in (0, 9, 20):
        r, z = geo.r[i], geo.z[i]
        c = lambda n: (1j ** n) * jv(n, k0 * r * dperp) * np.exp(-1j * n * thd) * np.exp(1j * k0 * wv.d[2] * z)
        ex, ey, ez = wv.e
        for m in range(-M, M + 1):
            Er = 0.5 * (ex - 1j * ey) * c(m - 1) + 0.5 * (ex + 1j * ey) * c(m + 1)
            Et = 0.5 * (ey + 1j * ex) * c(m - 1) + 0.5 * (ey - 1j * ex) * c(m + 1)
            Ez = ez * c(m)
            assert abs(b[m + M, 4 * i + 0, 0] - sE * Et) < 1e-14
            assert abs(b[m + M, 4 * i + 1, 0] + sE * (geo.rp[i] * Er + geo.zp[i] * Ez)) < 1e-14


# ---------------------------------------------------------------- whole solver
@pytest.mark.slow
def test_reflection_symmetry(sphere_oracle):
    """A_{-m} = D_r A_m D_c: under theta -> -theta the polar traces (E, n x H = J)
    keep their t part and flip their theta part; the axial ones (H, n x E = M)
    do the opposite."""
    A, M = sphere_oracle["A"], sphere_oracle["cfg"].M
    n = A.shape[1]
    Dr = np.tile([-1.0, 1.0, 1.0, -1.0], n // 4)
    Dc = np.tile([1.0, -1.0, -1.0, 1.0], n // 4)
    for m in (1, 4, M):
        assert np.abs(Dr[:, None] * A[M + m] * Dc[None, :] - A[M - m]).max() == 0.0


@pytest.mark.slow
def test_mie_far_field(sphere_oracle):
    """Whole oracle (Lemma 1, N, K, eq. mullerrep, LU, far field) against the
    Mie series for the dielectric unit sphere, both polarisations."""
    cfg, x = sphere_oracle["cfg"], sphere_oracle["x"]
    th = np.linspace(0.0, np.pi, 13)
    ph = np.array([0.0, 1.1, 2.5])
    dirs = np.array([[math.sin(t) * math.cos(p), math.sin(t) * math.sin(p), math.cos(t)] for t in th for p in ph])
    Ef = fields.far_field(cfg.curve, cfg.media, cfg.M, x, dirs)
    for w_i, wv in enumerate(cfg.waves):
        Em = mie.far_field(1.0, 1.5, 1.0, wv.d, wv.e, dirs)
        assert np.linalg.norm(Ef[w_i] - Em) / np.linalg.norm(Em) < 1e-12


def test_mie_far_field_two_panels():
    """Two panels meeting at the equator share an endpoint, so each is the
    other's adjacent panel and takes the near-singular rule (Section 5): the
    whole oracle on this 2 x 16-node sphere still matches the Mie series.
    With plain Gauss-Legendre on the neighbour instead, the far field is off
    by about 2e-6; with the near rule it agrees to about 3e-15."""
    cur = W.sphere(2)
    med = W.Media.from_k(1.0, 1.5)
    M = 8
    wv = W.PlaneWave(np.array([0.6, 0.0, 0.8]), np.array([0.8, 0.0, -0.6]))
    A = system.assemble(cur, med, M)
    b = fields.modal_rhs(cur, med, M, [wv])
    sw = system.l2_weights(cur)
    Aw = system.weight_matrix(A, sw)
    x = np.zeros_like(b)
    for q in range(2 * M + 1):
        LU, piv = linalg.lu_factor(Aw[q])
        x[q] = linalg.lu_solve(LU, piv, b[q] * sw[:, None]) / sw[:, None]
    th = np.linspace(0.1, np.pi - 0.1, 7)
    dirs = np.array([[math.sin(t), 0.0, math.cos(t)] for t in th])
    Ef = fields.far_field(cur, med, M, x, dirs)[0]
    Em = mie.far_field(1.0, 1.5, 1.0, wv.d, wv.e, dirs)
    assert np.linalg.norm(Ef - Em) / np.linalg.norm(Em) < 1e-8


def test_mie_against_rayleigh_limit():
    """Mie amplitudes for a small sphere reduce to the Rayleigh dipole:
    S1 = -i x^3 (m^2-1)/(m^2+2), S2 = S1 cos(Theta) to leading order."""
    x, m = 1e-3, 1.5
    S1, S2 = mie.amplitudes(x, m * x, 1.0, np.array([0.3]))
    ray = -1j * x ** 3 * (m * m - 1) / (m * m + 2)
    assert abs(S1[0] - ray) < 1e-5 * abs(ray)
    assert abs(S2[0] - ray * 0.3) < 1e-5 * abs(ray)


def test_extinction_current_loop_indirect(loop_oracle):
    """Section 6's accuracy test: with the current loop's k1 field as the
    interior field and zero outside, the indirect formulation's currents must
    reproduce both through eqs. interior_dual and exteriorfield (uniqueness of
    the transmission problem).  Measured 4e-15 inside and 1e-16 outside."""
    from oracle import fields
    from workloads.sources import current_loop_field
    L = loop_oracle
    cfg = L["cfg"]
    Er, Hr = current_loop_field(L["inner"], L["k1"], cfg.media.omega, complex(cfg.media.mu1))
    Ei, Hi = fields.near_field(cfg.curve, cfg.media, L["M"], L["x"], L["inner"], 1, formulation=1)
    Eo, Ho = fields.near_field(cfg.curve, cfg.media, L["M"], L["x"], L["outer"], 0, formulation=1)
    se, sh = np.abs(Er).max(), np.abs(Hr).max()
    assert np.abs(Ei[0] - Er).max() <= 1e-12 * se
    assert np.abs(Hi[0] - Hr).max() <= 1e-12 * sh
    assert np.abs(Eo[0]).max() <= 1e-13 * se and np.abs(Ho[0]).max() <= 1e-13 * sh


def test_extinction_direct_plane_wave(sphere_oracle):
    """Direct form (eq. mullerrep) with a plane wave: the exterior
    representation (eq. exteriorfield) evaluated inside the body cancels the
    incident field, and the interior one (eq. interiorfield) vanishes outside
    (the extinction theorem of Section 3).  Measured 1e-14 and 2e-16."""
    from oracle import fields, system
    cfg = sphere_oracle["cfg"]
    M, x = cfg.M, sphere_oracle["x"]
    k0, _ = system.wavenumbers(cfg.media)
    rng = np.random.default_rng(5)
    d = rng.standard_normal((6, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    inner = d * rng.uniform(0.1, 0.6, (6, 1))
    outer = d * rng.uniform(1.8, 2.6, (6, 1))
    Eo, Ho = fields.near_field(cfg.curve, cfg.media, M, x, inner, 0, formulation=0)
    Ei, Hi = fields.near_field(cfg.curve, cfg.media, M, x, outer, 1, formulation=0)
    for w, wv in enumerate(cfg.waves):
        ph = np.exp(1j * k0 * inner @ wv.d)[:, None]
        Einc = wv.e[None, :] * ph
        Hinc = (k0 / (cfg.media.omega * complex(cfg.media.mu0))) * np.cross(wv.d, wv.e)[None, :] * ph
        assert np.abs(Eo[w] + Einc).max() <= 1e-12
        assert np.abs(Ho[w] + Hinc).max() <= 1e-12
        assert np.abs(Ei[w]).max() <= 1e-13 and np.abs(Hi[w]).max() <= 1e-13
