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
