"""Many bodies under a memory budget on several CUDA streams: each body's
currents must be bitwise those of the same body solved alone (no state is
shared between concurrent builds and every reduction is order-independent),
with backward errors at the refinement tolerance."""
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


def _bodies():
    waves = [W.paper_default_wave(), W.plane_wave([0.0, 0.0, 1.0], [1.0, 0.0, 0.0])]
    out = []
    for s, (npan, M, k0) in enumerate([(20, 40, 3.0), (10, 16, 1.5), (14, 24, 2.5), (12, 32, 4.0)]):
        out.append(W.Config(f"r{s}", W.random_body(npan, seed=100 + s), W.Media.from_k(k0, 1.5 * k0), M, 16,
                            list(waves)))
    out.append(W.Config("cyl", W.cylinder(2, 0.8, 1.1), W.Media.from_k(2.0, 3.0), 20, 16, list(waves)))
    out.append(W.Config("cone", W.cone(3, 1.0, 0.7), W.Media.from_k(2.0, 3.0), 24, 16, list(waves)))
    return out


def _solve_alone(mb, body):
    ctx = mb.build(body.curve, body.media, body.M, mb.Options(n_phi=body.n_phi, precision=1))
    n, nrhs = 4 * body.curve.N, len(body.waves)
    rhs = torch.zeros((2 * body.M + 1, nrhs, n), dtype=torch.complex128, device=DEV)
    ctx.rhs_planewave([w.d for w in body.waves], [w.e for w in body.waves], rhs)
    x = torch.zeros_like(rhs)
    ctx.solve(rhs, x)
    out = x.cpu().numpy()
    ctx.close()
    return out


def test_batch_matches_bodies_alone(mb):
    from paper_1810_07067_gb300 import batch
    bodies = _bodies()
    alone = [_solve_alone(mb, b) for b in bodies]
    got = {}

    def check(i, body, ctx, x, stream):
        stream.synchronize()
        got[i] = x.cpu().numpy()
        return {}

    peaks = [mb.build_bytes(b.curve.N, b.M, 1)[0] for b in bodies]
    budget = int(1.5 * max(peaks))                  # forces waves
    res, wall, adm = batch.run_batch(bodies, budget, n_streams=3, process=batch.make_process(1, check))
    assert adm.high_water <= budget and adm.in_use == 0
    assert len({r.worker for r in res}) >= 2
    for i, r in enumerate(res):
        assert np.array_equal(got[i], alone[i]), bodies[i].name
        assert r.backward_err <= 1e-14 and r.refine_iters >= 1
        assert r.resident_bytes <= r.peak_bytes


@pytest.mark.parametrize("precision", [0, 1])
def test_wave_matches_bodies_alone(mb, precision):
    """mueller_build_many factors all modes of several bodies of different
    sizes in one graph-launched LU over a ragged table of matrices; with the
    same LU tile each body's currents are bitwise those of its own build."""
    bodies = _bodies()[:3] + _bodies()[4:5]          # N = 320, 160, 224 and a cylinder; M = 40, 16, 24, 20
    opts = mb.Options(n_phi=16, precision=precision, lu_tile=64)

    def solve(body, ctx):
        n, nrhs = 4 * body.curve.N, len(body.waves)
        rhs = torch.zeros((2 * body.M + 1, nrhs, n), dtype=torch.complex128, device=DEV)
        ctx.rhs_planewave([w.d for w in body.waves], [w.e for w in body.waves], rhs)
        x = torch.zeros_like(rhs)
        be = np.zeros((2 * body.M + 1) * nrhs)
        ctx.solve(rhs, x, backward_err=be)
        return x.cpu().numpy(), be

    alone = []
    for b in bodies:
        ctx = mb.build(b.curve, b.media, b.M, opts)
        alone.append(solve(b, ctx))
        assert ctx.stats()["lu_graph"] == 0
        ctx.close()
    ctxs = mb.build_many([(b.curve, b.media, b.M) for b in bodies], opts)
    assert len(ctxs) == len(bodies)
    for b, ctx, (xa, bea) in zip(bodies, ctxs, alone):
        st = ctx.stats()
        assert st["lu_graph"] == 1 and st["lu_wave_bodies"] == len(bodies)
        if precision:
            assert st["lu_tile_steps"][1] > 0 and st["lu_tile_steps"][0] == st["lu_tile_steps"][2] == 0
        x, be = solve(b, ctx)
        assert np.array_equal(x, xa), b.name
        if precision:
            assert be.max() <= 1e-14
        ctx.close()


def test_wave_bytes_bound_the_device_use(mb):
    """The wave estimate covers what the contexts hold afterwards and at least
    the largest single build's peak."""
    bodies = _bodies()[:3]
    est = mb.build_many_bytes([b.curve.N for b in bodies], [b.M for b in bodies], 1)
    assert est >= max(mb.build_bytes(b.curve.N, b.M, 1)[0] for b in bodies)
    ctxs = mb.build_many([(b.curve, b.media, b.M) for b in bodies], mb.Options(n_phi=16, precision=1))
    held = sum(c.stats()["device_bytes"] for c in ctxs)
    assert held <= est
    for c in ctxs:
        c.close()


def test_waves_on_two_streams_match_bodies_alone(mb):
    """run_waves: waves planned under half the budget each, two worker
    streams admitted against the whole budget; with a fixed LU tile each
    body's currents are bitwise those of its own build."""
    from paper_1810_07067_gb300 import batch
    bodies = _bodies()
    alone = []
    for body in bodies:
        ctx = mb.build(body.curve, body.media, body.M, mb.Options(n_phi=body.n_phi, precision=1, lu_tile=64))
        n, nrhs = 4 * body.curve.N, len(body.waves)
        rhs = torch.zeros((2 * body.M + 1, nrhs, n), dtype=torch.complex128, device=DEV)
        ctx.rhs_planewave([w.d for w in body.waves], [w.e for w in body.waves], rhs)
        x = torch.zeros_like(rhs)
        ctx.solve(rhs, x)
        alone.append(x.cpu().numpy())
        ctx.close()
    got = {}

    def check(i, body, ctx, x, stream):
        stream.synchronize()
        got[i] = x.cpu().numpy()
        return {}

    budget = 2 * mb.build_many_bytes([b.curve.N for b in bodies[:3]], [b.M for b in bodies[:3]], 1)
    res, wall, plan, adm = batch.run_waves(bodies, budget, check=check, n_streams=2, lu_tile=64)
    assert adm.high_water <= budget and adm.in_use == 0
    assert len(plan) >= 2 and max(len(w) for w, _ in plan) >= 2
    for i, r in enumerate(res):
        assert np.array_equal(got[i], alone[i]), bodies[i].name
        assert r.backward_err <= 1e-14 and r.extra["lu_graph"] == 1


def test_batch_sample_vs_oracle(mb):
    """The seeded 8-body sample of the batched workload (6 random bodies, a
    5-level and an 11-level cylinder; oracle solutions in
    tests/golden/fullsize_batch<index>.npz, written by
    tests/golden/make_fullsize.py batch): all eight built together by one
    mueller_build_many (mixed path, one graph-launched LU over every mode of
    every body), then modes -1, 0 and M of each compared with the oracle --
    plane-wave currents to 1e-9 of the body's largest mode, the far field of
    those modes to 1e-9, and the solutions of two seeded random right-hand
    sides per mode to max(1e-9, 10 kappa_1 noise_1) (kappa_1 the mode's
    condition number and noise_1 the relative difference of the oracle's 32-
    and 24-point matrices, both from the oracle's file)."""
    import glob
    import os
    files = sorted(glob.glob(os.path.join(os.path.dirname(__file__), "golden", "fullsize_batch*.npz")))
    if len(files) < 8:
        pytest.skip("batch oracle files not generated")
    gs = [np.load(f) for f in files]
    bodies = []
    for g in gs:
        curve = W.Curve(int(g["n_panels"]), g["r"].copy(), g["z"].copy(), g["dr"].copy(), g["dz"].copy(),
                        bool(int(g["closed"])))
        media = W.Media(float(g["omega"]), complex(g["eps0"]), complex(g["mu0"]), complex(g["eps1"]),
                        complex(g["mu1"]))
        bodies.append((curve, media, int(g["M"])))
    ctxs = mb.build_many(bodies, mb.Options(n_phi=int(gs[0]["n_phi"]), precision=1, refine_tol=1e-14))
    tol = 1e-9
    for g, (curve, media, M), ctx in zip(gs, bodies, ctxs):
        n = 4 * curve.N
        nrhs = len(g["wave_d"])
        b = torch.zeros((2 * M + 1, nrhs, n), dtype=torch.complex128, device=DEV)
        ctx.rhs_planewave(g["wave_d"], g["wave_e"], b)
        x = torch.zeros_like(b)
        ctx.solve(b, x)
        xg = x.cpu().numpy()
        modes, waves = [int(m) for m in g["modes"]], [int(w) for w in g["waves"]]
        top = max(np.linalg.norm(g["x"][qi, wi]) for qi in range(len(modes)) for wi in range(len(waves)))
        for qi, m in enumerate(modes):
            for wi, w in enumerate(waves):
                assert np.linalg.norm(xg[m + M, w] - g["x"][qi, wi]) < tol * top, (g["workload"], m, w)
        keep = torch.zeros_like(x)
        for m in modes:
            keep[m + M] = x[m + M]
        dirs = torch.tensor(g["ff_dirs"], device=DEV)
        E = torch.zeros((nrhs, len(dirs), 3), dtype=torch.complex128, device=DEV)
        ctx.far_field(keep, dirs, E)
        assert np.linalg.norm(E.cpu().numpy() - g["ff"]) < tol * np.linalg.norm(g["ff"]), g["workload"]
        br = torch.zeros((2 * M + 1, 2, n), dtype=torch.complex128, device=DEV)
        for qi, m in enumerate(modes):
            br[m + M] = torch.tensor(g["b_rand"][qi], device=DEV)
        xr = torch.zeros_like(br)
        ctx.solve(br, xr)
        xr = xr.cpu().numpy()
        for qi, m in enumerate(modes):
            err = max(np.linalg.norm(xr[m + M, c] - g["x_rand"][qi, c]) / np.linalg.norm(g["x_rand"][qi, c])
                      for c in range(2))
            bound = max(tol, 10.0 * float(g["kappa1"][qi]) * max(float(g["noise1"][qi]), 1e-15))
            assert err < bound, (str(g["workload"]), m, err)
        ctx.close()
