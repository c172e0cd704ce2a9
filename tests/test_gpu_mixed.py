"""Mixed-precision path: complex64 factors + FP64 iterative refinement."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import workloads as W

DEV = "cuda:0"


@pytest.fixture(scope="module")
def mb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1810_07067_gb300 as m
    return m


def _rel(xa, xb, M):
    num = max(np.linalg.norm(xa[q] - xb[q]) for q in range(2 * M + 1))
    den = max(np.linalg.norm(xb[q]) for q in range(2 * M + 1))
    return num / den


@pytest.mark.parametrize("precision", [1, 2])
def test_mixed_sphere_vs_oracle(mb, sphere_oracle, precision):
    """precision 1: residuals on BF16 tensor cores (exact digit slicing);
    precision 2: residuals on the FP64 pipe."""
    cfg = sphere_oracle["cfg"]
    M = cfg.M
    ctx = mb.build(cfg.curve, cfg.media, M, mb.Options(n_phi=cfg.n_phi, precision=precision, refine_tol=1e-14))
    b = torch.tensor(np.ascontiguousarray(sphere_oracle["b"].transpose(0, 2, 1)), device=DEV)
    x = torch.zeros_like(b)
    be = np.zeros((2 * M + 1) * b.shape[1])
    ctx.solve(b, x, backward_err=be)
    st = ctx.stats()
    assert st["refine_iters"] >= 1 and be.max() <= 1e-14
    xg = x.cpu().numpy().transpose(0, 2, 1)
    assert _rel(xg, sphere_oracle["x"], M) < 1e-10


def test_mixed_cylinder_full_size_vs_fp64(mb):
    """Cylinder workload at full size: mixed-path currents against the FP64
    path's (the FP64 path is itself checked against the oracle block by block)."""
    cfg = W.config_cylinder(7)
    M, n = cfg.M, 4 * cfg.N
    nrhs = len(cfg.waves)
    dirs = [w.d for w in cfg.waves]; pols = [w.e for w in cfg.waves]
    c64 = mb.build(cfg.curve, cfg.media, M, mb.Options(n_phi=cfg.n_phi))
    b = torch.zeros((2 * M + 1, nrhs, n), dtype=torch.complex128, device=DEV)
    c64.rhs_planewave(dirs, pols, b)
    x64 = torch.zeros_like(b)
    c64.solve(b, x64)
    c64.close()
    cmx = mb.build(cfg.curve, cfg.media, M, mb.Options(n_phi=cfg.n_phi, precision=1, refine_tol=1e-14))
    xmx = torch.zeros_like(b)
    be = np.zeros((2 * M + 1) * nrhs)
    cmx.solve(b, xmx, backward_err=be)
    assert be.max() <= 1e-14
    a, r = xmx.cpu().numpy(), x64.cpu().numpy()
    assert _rel(a, r, M) < 1e-11


@pytest.mark.parametrize("tile", [32, 64, 128])
def test_mixed_lu_tiles(mb, tile):
    """Each column tile of the tensor-core LU update (32, 64, 128 columns per
    CTA) gives FP32-grade factors: refinement reaches 1e-14 in a few steps and
    the currents agree with the FP64 path.  The body (N = 448, system 1792,
    modes 0..12) spans 14 row tiles of 128 and a ragged last tile per step;
    the factorization updates the trailing matrix once per 128 columns."""
    body = W.random_body(28, seed=7)
    media = W.Media.from_k(4.0, 6.0)
    M, n = 12, 4 * body.N
    waves = [W.paper_default_wave(), W.plane_wave([0.0, 0.0, 1.0], [1.0, 0.0, 0.0])]
    c64 = mb.build(body, media, M, mb.Options(n_phi=64))
    b = torch.zeros((2 * M + 1, len(waves), n), dtype=torch.complex128, device=DEV)
    c64.rhs_planewave([w.d for w in waves], [w.e for w in waves], b)
    x64 = torch.zeros_like(b)
    c64.solve(b, x64)
    c64.close()
    cmx = mb.build(body, media, M, mb.Options(n_phi=64, precision=1, refine_tol=1e-14, lu_tile=tile))
    st = cmx.stats()
    q = {32: 0, 64: 1, 128: 2}[tile]
    # one tensor-core update per 128-column block with a trailing matrix
    assert st["lu_tile_steps"][q] == sum(st["lu_tile_steps"]) == (n - 1) // 128
    x = torch.zeros_like(b)
    be = np.zeros((2 * M + 1) * len(waves))
    cmx.solve(b, x, backward_err=be)
    assert be.max() <= 1e-14 and cmx.stats()["refine_iters"] <= 3
    assert _rel(x.cpu().numpy(), x64.cpu().numpy(), M) < 1e-11


def test_tile_autotuner_table(mb):
    """With lu_tile = 0 the update tile comes from the autotuner: every entry
    holds measured times for the three tiles and keeps 64 unless another tile
    was at least 3 % faster."""
    body = W.random_body(28, seed=8)
    ctx = mb.build(body, W.Media.from_k(4.0, 6.0), 12, mb.Options(n_phi=64, precision=1))
    st = ctx.stats()
    assert sum(st["lu_tile_steps"]) == (4 * body.N - 1) // 128
    ctx.close()
    table = mb.lu_tile_table()
    assert table
    for e in table:
        t32, t64, t128 = e["ms_per_matrix"]
        assert e["tile"] in (32, 64, 128)
        if min(t32, t64, t128) > 0:
            best = {32: t32, 64: t64, 128: t128}[e["tile"]]
            if e["tile"] == 64:
                assert t32 >= 0.97 * t64 and t128 >= 0.97 * t64
            else:
                assert best < 0.97 * t64


def test_mixed_reports_no_convergence(mb):
    cur = W.sphere(2)
    med = W.Media.from_k(1.0, 1.5)
    M = 2
    ctx = mb.build(cur, med, M, mb.Options(n_phi=64, precision=1, refine_tol=1e-300, refine_max_iter=1))
    n = 4 * cur.N
    b = torch.ones((2 * M + 1, 1, n), dtype=torch.complex128, device=DEV)
    x = torch.zeros_like(b)
    with pytest.raises(mb.MuellerError) as e:
        ctx.solve(b, x)
    assert e.value.status == 4
    assert torch.isfinite(x.abs()).all()


def _reconstruction_err(A, LU, pv):
    n = A.shape[0]
    L = np.tril(LU, -1) + np.eye(n, dtype=LU.dtype)
    U = np.triu(LU)
    PA = A.astype(np.complex128).copy()
    for k in range(n):
        p = pv[k]
        PA[[k, p]] = PA[[p, k]]
    return np.abs(PA - L.astype(np.complex128) @ U.astype(np.complex128)).max()


def test_lu_c64_tensor_core_vs_lapack(mb):
    """The complex64 factorisation with split-BF16 tensor-core updates must be
    as accurate as LAPACK's complex64 LU on the same matrices (same pivoting
    rule): a split that dropped a piece product would be two or more orders
    of magnitude worse.  Sizes span one partial tile, several 128-row tiles
    with a ragged tail, a batch, and panels spread over clusters of two
    (1000 rows) and four (1700) CTAs."""
    sl = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(11)
    for n, batch in ((77, 2), (300, 3), (517, 1), (1000, 1), (1700, 1)):
        A = (rng.standard_normal((batch, n, n)) + 1j * rng.standard_normal((batch, n, n))).astype(np.complex64)
        At = torch.tensor(np.ascontiguousarray(A.transpose(0, 2, 1)), device=DEV)
        piv = torch.zeros((batch, n), dtype=torch.int32, device=DEV)
        info = torch.zeros(batch, dtype=torch.int32, device=DEV)
        mb.lu_batched_c64(At, piv, info)
        assert (info.cpu().numpy() == 0).all()
        LU = At.cpu().numpy().transpose(0, 2, 1)
        pv = piv.cpu().numpy()
        for b in range(batch):
            lu, pl = sl.lu_factor(A[b])
            ref = _reconstruction_err(A[b], lu, pl)
            got = _reconstruction_err(A[b], LU[b], pv[b])
            assert got <= 4 * ref + 1e-7 * np.abs(A[b]).max(), (n, b, got, ref)


def test_lu_c64_detects_zero_pivot(mb):
    A = np.eye(300, dtype=np.complex64)[None].copy()
    A[0, 150, 150] = 0.0
    At = torch.tensor(A, device=DEV)
    piv = torch.zeros((1, 300), dtype=torch.int32, device=DEV)
    info = torch.zeros(1, dtype=torch.int32, device=DEV)
    mb.lu_batched_c64(At, piv, info)
    assert info.item() == 151


def test_lu_c64_zero_pivot_in_cluster_panel(mb):
    """A zero pivot in the second CTA's row slice of a two-CTA panel."""
    n = 1000
    A = np.eye(n, dtype=np.complex64)[None].copy()
    A[0, 700, 700] = 0.0
    At = torch.tensor(A, device=DEV)
    piv = torch.zeros((1, n), dtype=torch.int32, device=DEV)
    info = torch.zeros(1, dtype=torch.int32, device=DEV)
    mb.lu_batched_c64(At, piv, info)
    assert info.item() == 701


@pytest.mark.parametrize("word,where", [("lu_timeout", "build"), ("residual_timeout", "solve")])
def test_timeout_status_reaches_the_api(mb, monkeypatch, word, where):
    """A device-side wait that gives up leaves 1 in a status word; the host
    must turn it into MUELLER_ETIMEOUT.  The word is set from the host
    (MUELLER_FAULT_INJECT), so no device wait is shortened and nothing faults."""
    cfg = W.config_sphere()
    M = 4
    opts = mb.Options(n_phi=cfg.n_phi, precision=1, refine_tol=1e-14)
    if where == "build":
        monkeypatch.setenv("MUELLER_FAULT_INJECT", word)
        with pytest.raises(mb.MuellerError, match="timed out") as ei:
            mb.build(cfg.curve, cfg.media, M, opts)
        assert ei.value.status == 5
        monkeypatch.delenv("MUELLER_FAULT_INJECT")
        mb.build(cfg.curve, cfg.media, M, opts).close()     # the context stays usable
        return
    ctx = mb.build(cfg.curve, cfg.media, M, opts)
    n = 4 * cfg.N
    rhs = torch.zeros((2 * M + 1, 1, n), dtype=torch.complex128, device=DEV)
    ctx.rhs_planewave(cfg.waves[0].d[None], cfg.waves[0].e[None], rhs)
    x = torch.zeros_like(rhs)
    monkeypatch.setenv("MUELLER_FAULT_INJECT", word)
    with pytest.raises(mb.MuellerError, match="timed out") as ei:
        ctx.solve(rhs, x)
    assert ei.value.status == 5
    monkeypatch.delenv("MUELLER_FAULT_INJECT")
    ctx.solve(rhs, x)
    ctx.close()
