"""CUDA path against the CPU oracle, element by element (all through the C ABI)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import workloads as W
from oracle import green, system, linalg, fields, mie


@pytest.fixture(scope="module")
def mb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1810_07067_gb300 as m
    return m


DEV = "cuda:0"


def _pairs():
    base = [(1.0, 0.0, 0.3, 1.5), (0.5, -0.5, 0.9, 0.4), (1.0, 0.0, 0.95, 0.05), (0.7, 0.3, 0.72, 0.33),
            (0.5, 0.2, 0.5, 0.2 + 1e-7), (0.5, 0.2, 0.5 + 3e-9, 0.2 + 1e-9), (1.0, 0.0, 1.0 + 1e-5, 2e-5),
            (0.02, -0.99, 0.01, -0.995), (0.004, -1.0, 0.002, -1.0), (0.9, 0.1, 0.89, 0.12),
            (0.6, 0.0, 0.55, 0.02), (1.0, 0.5, 0.999, 0.503)]
    cur = W.sphere(4)
    for (P, a, Q) in ((1, 5, 1), (1, 0, 0), (2, 15, 3)):
        r, z, *_ = system.panel_support(cur, P, a, Q)
        i = 16 * P + a
        for s in range(0, len(r), 23):
            base.append((cur.r[i], cur.z[i], r[s], z[s]))
    return np.array(base)


@pytest.mark.parametrize("k0,k1,M,nphi", [(1.0, 1.5, 10, 64), (5.0, 7.5 + 0.01j, 64, 256),
                                           (10.0, 15.0, 20, 128)])
def test_modal_kernels_vs_oracle(mb, k0, k1, M, nphi):
    """Split (Legendre/Miller + convolution) and plain-trapezoid spectra of all
    nine families against direct quadrature of the unsplit integrands."""
    pairs = _pairs()
    out = torch.zeros((len(pairs), 9, M + 2), dtype=torch.complex128, device=DEV)
    mb.modal_kernels(pairs, k0, k1, M, nphi, out)
    got = out.cpu().numpy()
    ref = green.modal_families_batch(pairs[:, 0], pairs[:, 1], pairs[:, 2], pairs[:, 3], k0, k1, M)
    # per pair and family, relative to the family's largest coefficient
    # (families that vanish identically, e.g. d/dz_t at z_t = z_s, must vanish)
    scale = np.maximum(np.abs(ref).max(axis=2, keepdims=True), 1e-300)
    err = (np.abs(got - ref) / scale).max(axis=2)
    worst = np.unravel_index(err.argmax(), err.shape)
    assert err.max() < 1e-12, (err.max(), worst, pairs[worst[0]])


def test_lu_batched_vs_reconstruction(mb):
    """Sizes up to 400 rows factor each panel in one CTA; 900 spreads the
    panel over a cluster of four CTAs (row slices in distributed shared
    memory, pivots crossing slice boundaries) with a ragged last panel."""
    rng = np.random.default_rng(7)
    for n, batch in ((5, 2), (77, 3), (200, 2), (900, 2)):
        A = rng.standard_normal((batch, n, n)) + 1j * rng.standard_normal((batch, n, n))
        At = torch.tensor(np.ascontiguousarray(A.transpose(0, 2, 1)), device=DEV)  # column-major per matrix
        piv = torch.zeros((batch, n), dtype=torch.int32, device=DEV)
        info = torch.zeros(batch, dtype=torch.int32, device=DEV)
        mb.lu_batched(At, piv, info)
        LU = At.cpu().numpy().transpose(0, 2, 1)
        pv = piv.cpu().numpy()
        assert (info.cpu().numpy() == 0).all()
        for b in range(batch):
            L = np.tril(LU[b], -1) + np.eye(n); U = np.triu(LU[b])
            PA = A[b].copy()
            for k in range(n):
                p = pv[b, k]
                PA[[k, p]] = PA[[p, k]]
            assert np.abs(PA - L @ U).max() < 1e-13 * n * np.abs(A[b]).max()


def test_lu_detects_zero_pivot(mb):
    A = np.zeros((1, 40, 40), complex)
    A[0, :, :] = np.eye(40)
    A[0, 7, 7] = 0.0
    At = torch.tensor(A, device=DEV)
    piv = torch.zeros((1, 40), dtype=torch.int32, device=DEV)
    info = torch.zeros(1, dtype=torch.int32, device=DEV)
    mb.lu_batched(At, piv, info)
    assert info.item() == 8


def test_sphere_matrices_vs_oracle(mb, sphere_oracle):
    """All entries of modes 0..M: 1e-12 of the largest entry, except where the
    oracle's own noise (32- vs 24-point azimuthal rule) is larger: rows of
    nodes next to the axis carry 1/r_t^2 and m^2/r_t^2 factors that amplify
    rounding of the spectra.  Those entries are checked against a multiple of
    the oracle's noise there, sampled block by block."""
    cfg = sphere_oracle["cfg"]
    M, n = cfg.M, 4 * cfg.N
    A = torch.zeros((M + 1, n, n), dtype=torch.complex128, device=DEV)
    mb.assemble(cfg.curve, cfg.media, M, A, mb.Options(n_phi=cfg.n_phi))
    G = A.cpu().numpy().transpose(0, 2, 1)
    Aw = sphere_oracle["Aw"]
    sw = sphere_oracle["sw"]
    bad = set()
    for m in range(M + 1):
        ref = Aw[M + m]
        d = np.abs(G[m] - ref) > 1e-12 * np.abs(ref).max()
        for r, c in zip(*np.nonzero(d)):
            bad.add((r // 4, c // 4))
    # entries above the plain bar may only sit in rows of nodes next to the axis
    r = cfg.curve.r
    assert all(r[i] < 0.05 * r.max() for (i, _) in bad), sorted({i for (i, _) in bad})
    modes = np.arange(M + 1)
    for (i, j) in sorted(bad):
        ref, noise = system.block(cfg.curve, cfg.media, M, i, j, modes=modes, noise=True)
        s = sw[4 * i] / sw[4 * j]
        got = G[:, 4 * i:4 * i + 4, 4 * j:4 * j + 4]
        floor = 20 * noise.max() * s   # noise level of this (target, column) pair, all modes
        assert (np.abs(got - ref * s) <= 1e-12 * np.abs(Aw).max() + floor).all(), (i, j)


def test_sphere_rhs_vs_oracle(mb, sphere_oracle):
    cfg = sphere_oracle["cfg"]
    M, n = cfg.M, 4 * cfg.N
    ctx = mb.build(cfg.curve, cfg.media, M, mb.Options(n_phi=cfg.n_phi))
    rhs = torch.zeros((2 * M + 1, len(cfg.waves), n), dtype=torch.complex128, device=DEV)
    ctx.rhs_planewave([w.d for w in cfg.waves], [w.e for w in cfg.waves], rhs)
    got = rhs.cpu().numpy().transpose(0, 2, 1)
    ref = sphere_oracle["b"]
    assert np.abs(got - ref).max() < 1e-13 * np.abs(ref).max()


def test_sphere_currents_and_far_field(mb, sphere_oracle):
    """Modal currents and far fields against the oracle (1e-10) and Mie."""
    cfg = sphere_oracle["cfg"]
    M, n = cfg.M, 4 * cfg.N
    ctx = mb.build(cfg.curve, cfg.media, M, mb.Options(n_phi=cfg.n_phi))
    b = torch.tensor(np.ascontiguousarray(sphere_oracle["b"].transpose(0, 2, 1)), device=DEV)
    x = torch.zeros_like(b)
    ctx.solve(b, x)
    xg = x.cpu().numpy().transpose(0, 2, 1)
    xo = sphere_oracle["x"]
    num = max(np.linalg.norm(xg[q] - xo[q]) for q in range(2 * M + 1))
    den = max(np.linalg.norm(xo[q]) for q in range(2 * M + 1))
    assert num / den < 1e-10, num / den
    th = np.linspace(0.0, np.pi, 13)
    dirs = np.array([[math.sin(t) * math.cos(p), math.sin(t) * math.sin(p), math.cos(t)] for t in th for p in (0.0, 2.2)])
    E = torch.zeros((len(cfg.waves), len(dirs), 3), dtype=torch.complex128, device=DEV)
    ctx.far_field(x, torch.tensor(dirs, device=DEV), E)
    Eg = E.cpu().numpy()
    Eo = fields.far_field(cfg.curve, cfg.media, M, xo, dirs)
    assert np.linalg.norm(Eg - Eo) / np.linalg.norm(Eo) < 1e-10
    for w_i, wv in enumerate(cfg.waves):
        Em = mie.far_field(1.0, 1.5, 1.0, wv.d, wv.e, dirs)
        assert np.linalg.norm(Eg[w_i] - Em) / np.linalg.norm(Em) < 1e-11


def test_indirect_form_matrices(mb):
    """Indirect formulation (eq. dualmullrep) blocks on a small body."""
    cur = W.sphere(3)
    med = W.Media.from_k(2.0, 3.0 + 0.1j)
    M = 4
    n = 4 * cur.N
    A = torch.zeros((M + 1, n, n), dtype=torch.complex128, device=DEV)
    mb.assemble(cur, med, M, A, mb.Options(n_phi=64, formulation=1))
    G = A.cpu().numpy().transpose(0, 2, 1)
    sw = system.l2_weights(cur)
    for (i, j) in ((3, 3), (3, 20), (40, 10), (47, 47)):
        ref = system.block(cur, med, M, i, j, formulation=1, modes=np.arange(M + 1))
        ref = ref * sw[4 * i] / sw[4 * j]
        got = G[:, 4 * i:4 * i + 4, 4 * j:4 * j + 4]
        assert np.abs(got - ref).max() < 1e-12 * np.abs(G).max(), (i, j)


@pytest.fixture(scope="module")
def cylinder_full(mb):
    cfg = W.config_cylinder(7)
    M, n = cfg.M, 4 * cfg.N
    A = torch.zeros((M + 1, n, n), dtype=torch.complex128, device=DEV)
    mb.assemble(cfg.curve, cfg.media, M, A, mb.Options(n_phi=cfg.n_phi))
    return cfg, A


def test_cylinder_full_size_sampled_blocks(mb, cylinder_full):
    """Cylinder with edge-graded panels, N = 576, modes 0..64, 256 samples:
    sampled 4x4 blocks (far, self, adjacent, across the edge) against the
    oracle computed block by block."""
    cfg, A = cylinder_full
    M = cfg.M
    sw = system.l2_weights(cfg.curve)
    modes = np.array([0, 1, 17, 64])
    N = cfg.N
    samples = [(0, 300), (5, 5), (100, 117), (130, 112), (200, 480), (287, 289), (288, 272), (575, 560)]
    scale = max(float(A[q].abs().max()) for q in modes)
    for (i, j) in samples:
        ref, noise = system.block(cfg.curve, cfg.media, M, i, j, modes=modes, noise=True)
        s = sw[4 * i] / sw[4 * j]
        got = np.stack([A[q, 4 * j:4 * j + 4, 4 * i:4 * i + 4].cpu().numpy().T for q in modes])
        ok = np.abs(got - ref * s) <= 1e-12 * scale + 20 * noise.max() * s
        assert ok.all(), (i, j, (np.abs(got - ref * s) / scale).max())


def test_cylinder_full_size_backward_error(mb, cylinder_full):
    """Full-size build + solve: componentwise residual of every mode against the
    assembled (unfactored) matrices is at rounding level."""
    cfg, A = cylinder_full
    M, n = cfg.M, 4 * cfg.N
    ctx = mb.build(cfg.curve, cfg.media, M, mb.Options(n_phi=cfg.n_phi))
    nrhs = len(cfg.waves)
    b = torch.zeros((2 * M + 1, nrhs, n), dtype=torch.complex128, device=DEV)
    ctx.rhs_planewave([w.d for w in cfg.waves], [w.e for w in cfg.waves], b)
    x = torch.zeros_like(b)
    ctx.solve(b, x)
    sw = torch.tensor(system.l2_weights(cfg.curve), device=DEV, dtype=torch.float64)
    Dr = torch.tensor(np.tile([-1.0, 1.0, 1.0, -1.0], n // 4), device=DEV, dtype=torch.float64)
    Dc = torch.tensor(np.tile([1.0, -1.0, -1.0, 1.0], n // 4), device=DEV, dtype=torch.float64)
    worst = 0.0
    for m in (0, 1, 30, 64, -1, -64):
        Am = A[abs(m)].transpose(0, 1)  # weighted matrix, row-major view
        if m < 0:
            Am = Dr[:, None] * Am * Dc[None, :]
        xs = (x[M + m] * sw[None, :]).transpose(0, 1)
        bs = (b[M + m] * sw[None, :]).transpose(0, 1)
        r = Am @ xs - bs
        normA = Am.abs().sum(1).max()
        be = (r.abs().max(0).values / (normA * xs.abs().max(0).values + bs.abs().max(0).values)).max().item()
        worst = max(worst, be)
        # the same mode solved by a library solver from the same matrix
        ref = torch.linalg.solve(Am, bs)
        assert ((xs - ref).abs().max() / ref.abs().max()).item() < 1e-11
    assert worst < 1e-14, worst


def test_random_body_full_size(mb):
    """Smooth random body at full size (N = 1024, system 4096, modes 0..128,
    512 azimuthal samples, k0 = 10, k1 = 15): sampled blocks against the
    oracle, FP64 and mixed paths against each other and against the assembled
    matrices (normwise backward error)."""
    cfg = W.config_random()
    M, n = cfg.M, 4 * cfg.N
    sw = system.l2_weights(cfg.curve)
    A = torch.zeros((M + 1, n, n), dtype=torch.complex128, device=DEV)
    mb.assemble(cfg.curve, cfg.media, M, A, mb.Options(n_phi=cfg.n_phi))
    modes = np.array([0, 3, 64, 128])
    scale = max(float(A[q].abs().max()) for q in modes)
    for (i, j) in [(0, 700), (400, 400), (401, 391), (512, 530), (1023, 1000), (700, 100)]:
        ref, noise = system.block(cfg.curve, cfg.media, M, i, j, modes=modes, noise=True)
        s = sw[4 * i] / sw[4 * j]
        got = np.stack([A[q, 4 * j:4 * j + 4, 4 * i:4 * i + 4].cpu().numpy().T for q in modes])
        ok = np.abs(got - ref * s) <= 1e-12 * scale + 20 * noise.max() * s
        assert ok.all(), (i, j, (np.abs(got - ref * s) / scale).max())
    dirs = [w.d for w in cfg.waves]; pols = [w.e for w in cfg.waves]
    nrhs = len(cfg.waves)
    b = torch.zeros((2 * M + 1, nrhs, n), dtype=torch.complex128, device=DEV)
    xs = {}
    for prec in (0, 1):
        ctx = mb.build(cfg.curve, cfg.media, M, mb.Options(n_phi=cfg.n_phi, precision=prec, refine_tol=1e-14))
        if prec == 0:
            ctx.rhs_planewave(dirs, pols, b)
        x = torch.zeros_like(b)
        ctx.solve(b, x)
        xs[prec] = x
        ctx.close()
    swt = torch.tensor(sw, device=DEV, dtype=torch.float64)
    for prec in (0, 1):
        for m in (0, 1, 128):
            Am = A[m].transpose(0, 1)
            ys = (xs[prec][M + m] * swt[None, :]).transpose(0, 1)
            bs = (b[M + m] * swt[None, :]).transpose(0, 1)
            r = Am @ ys - bs
            be = (r.abs().max(0).values / (Am.abs().sum(1).max() * ys.abs().max(0).values +
                                          bs.abs().max(0).values)).max().item()
            assert be < 1e-14, (prec, m, be)
    num = max(float((xs[1][q] - xs[0][q]).norm()) for q in range(2 * M + 1))
    den = max(float(xs[0][q].norm()) for q in range(2 * M + 1))
    assert num / den < 1e-10


@pytest.mark.parametrize("precision", [0, 1])
def test_condition_estimate_vs_exact(mb, precision):
    """mueller_cond_estimate (Hager's estimate of ||A'^{-1}||_inf from the LU
    factors, times ||A'||_inf) against the exact kappa_inf of the same
    weighted matrices (numpy, from the matrices mueller_assemble gives): a
    lower bound, within a factor 3 (the estimator's usual accuracy; on small
    well-behaved matrices it is typically exact)."""
    cfg = W.config_sphere()
    M, n = cfg.M, 4 * cfg.N
    A = torch.zeros((M + 1, n, n), dtype=torch.complex128, device=DEV)
    mb.assemble(cfg.curve, cfg.media, M, A, mb.Options(n_phi=cfg.n_phi))
    ctx = mb.build(cfg.curve, cfg.media, M, mb.Options(n_phi=cfg.n_phi, precision=precision))
    est = ctx.cond_estimate()
    st = ctx.stats()
    ctx.close()
    Ah = A.cpu().numpy()
    exact = np.array([np.linalg.cond(Ah[m].T, np.inf) for m in range(M + 1)])
    assert (est <= exact * (1 + 1e-5)).all() and (est >= exact / 3).all(), (est / exact)
    assert st["kappa_max_mode"] == int(np.argmax(est)) and abs(st["kappa_max"] - est.max()) <= 1e-12 * est.max()
    assert abs(st["kappa_mode0"] - est[0]) <= 1e-12 * est[0]
