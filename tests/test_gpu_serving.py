"""Serving loop on the GPU: every request's far field must equal that of the
same request solved alone (fresh factors, its own right-hand sides only),
whether it was batched with other requests of its body or not, with the
factor cache holding all keys or evicting between them."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import workloads as W

DEV = "cuda:0"
GRID = (8, 16)


@pytest.fixture(scope="module")
def mb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1810_07067_gb300 as m
    return m


def _pool():
    out = []
    for s, (npan, M, k0) in enumerate([(10, 14, 2.0), (12, 18, 2.5), (14, 12, 3.0)]):
        out.append(W.Config(f"p{s}", W.random_body(npan, seed=200 + s), W.Media.from_k(k0, 1.5 * k0), M, 16, []))
    return out


def _requests(serving):
    rng = np.random.default_rng(9)
    reqs = []
    for i, key in enumerate([0, 0, 1, 0, 2, 1, 1, 0, 2, 2, 0]):
        k = int(rng.integers(1, 7))
        d = rng.standard_normal((k, 3)); d /= np.linalg.norm(d, axis=1, keepdims=True)
        p = np.cross(d, rng.standard_normal((k, 3))); p /= np.linalg.norm(p, axis=1, keepdims=True)
        reqs.append(serving.Request(i, key, 0.005 * i, d, p))
    return reqs


def _second_round(serving):
    """One request per key, all at once: after a first round that left one
    key resident, the other two are misses whatever the timing was."""
    d = np.array([[0.0, 0.0, 1.0]])
    p = np.array([[1.0, 0.0, 0.0]])
    return [serving.Request(100 + k, k, 0.0, d, p) for k in range(3)]


def _alone(mb, body, r):
    ctx = mb.build(body.curve, body.media, body.M, mb.Options(n_phi=body.n_phi, precision=1))
    n = 4 * body.curve.N
    rhs = torch.zeros((2 * body.M + 1, r.nrhs, n), dtype=torch.complex128, device=DEV)
    ctx.rhs_planewave(r.dirs, r.pols, rhs)
    x = torch.zeros_like(rhs)
    ctx.solve(rhs, x)
    E = torch.zeros((r.nrhs, GRID[0], GRID[1], 3), dtype=torch.complex128, device=DEV)
    ctx.far_field_grid(x, E)
    out = E.cpu().numpy()
    ctx.close()
    return out


@pytest.mark.parametrize("tight", [False, True])
def test_served_equals_alone(mb, tight):
    from paper_1810_07067_gb300 import serving
    pool = _pool()
    reqs = _requests(serving)
    peaks = [mb.build_bytes(b.curve.N, b.M, 1)[0] for b in pool]
    probe = serving.Server(pool, 10 ** 13, max_rhs=16, grid=GRID)
    head = probe.headroom
    probe.close()
    # tight: room for one key's build at a time, so keys are evicted and rebuilt
    budget = head + (max(peaks) + 1 if tight else 4 * sum(peaks))
    srv = serving.Server(pool, budget, max_rhs=16, grid=GRID)
    st, res = srv.run(reqs, keep_results=True)
    resident = len(srv.cache)
    st2 = srv.run(_second_round(serving))
    srv.close()
    assert len(st.done) == len(reqs) and st.unfinished == 0
    assert len(st2.done) == 3 and st2.unfinished == 0
    if tight:  # not all keys fit: the first round evicts, the second rebuilds every key it does not find
        assert st.evictions >= 1 and st.builds >= 3 and resident < 3
        assert st2.builds == 3 - resident
    else:
        assert st.builds == 3 and st.evictions == 0 and resident == 3
        assert st2.builds == 0
    assert st.batches < len(reqs)                      # some requests shared a batch
    for r in reqs:
        ref = _alone(mb, pool[r.key], r)
        got = res[r.id].numpy()
        assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max(), r.id


@pytest.mark.parametrize("precision", [0, 1])
def test_spill_restore_and_checkpoint_roundtrip(mb, tmp_path, precision):
    """Factors parked in host memory and brought back, or written to a
    checkpoint and loaded in a new context, give bit-identical solves; a
    spilled context refuses to solve until restored."""
    body = _pool()[1]
    ctx = mb.build(body.curve, body.media, body.M, mb.Options(n_phi=body.n_phi, precision=precision))
    n = 4 * body.curve.N
    rhs = torch.zeros((2 * body.M + 1, 3, n), dtype=torch.complex128, device=DEV)
    d = np.array([[0.0, 0.0, 1.0], [0.6, 0.0, 0.8], [0.0, 1.0, 0.0]])
    p = np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [1.0, 0.0, 0.0]])
    ctx.rhs_planewave(d, p, rhs)
    x0 = torch.zeros_like(rhs)
    ctx.solve(rhs, x0)
    dev_bytes = ctx.stats()["device_bytes"]
    ctx.spill()
    st = ctx.stats()
    assert st["spilled"] == 1 and st["device_bytes"] == 0 and st["host_bytes"] >= dev_bytes
    with pytest.raises(mb.MuellerError, match="restore"):
        ctx.solve(rhs, torch.zeros_like(rhs))
    path = str(tmp_path / "body.ctx")
    ctx.save(path)                                      # from the host copies
    ctx.restore()
    assert ctx.stats()["spilled"] == 0
    x1 = torch.zeros_like(rhs)
    ctx.solve(rhs, x1)
    assert torch.equal(x0, x1)
    ctx.close()
    loaded = mb.Context.load(path)
    x2 = torch.zeros_like(rhs)
    loaded.solve(rhs, x2)
    assert torch.equal(x0, x2)
    assert loaded.stats()["device_bytes"] == dev_bytes
    loaded.close()


def test_served_with_host_cache_and_checkpoints(mb, tmp_path):
    """A device budget for one key at a time: with a host cache every key is
    built once and evicted keys come back from host memory; with a checkpoint
    directory a second server loads every key instead of building it.  Every
    request's far field still equals the same request solved alone."""
    from paper_1810_07067_gb300 import serving
    pool = _pool()
    reqs = _requests(serving)
    peaks = [mb.build_bytes(b.curve.N, b.M, 1)[0] for b in pool]
    probe = serving.Server(pool, 10 ** 13, max_rhs=16, grid=GRID)
    head = probe.headroom
    probe.close()
    budget = head + max(peaks) + 1
    srv = serving.Server(pool, budget, max_rhs=16, grid=GRID, host_budget_bytes=4 * sum(peaks))
    st, res = srv.run(reqs, keep_results=True)
    resident = len(srv.cache)
    st2 = srv.run(_second_round(serving))
    srv.close()
    assert len(st.done) == len(reqs) and st.unfinished == 0
    assert st.builds == 3 and st.spills >= 1 and resident < 3
    # the second round brings every key it does not find on the device back from host memory
    assert st2.builds == 0 and st2.restores == 3 - resident and len(st2.done) == 3
    refs = {r.id: _alone(mb, pool[r.key], r) for r in reqs}
    for r in reqs:
        got = res[r.id].numpy()
        assert np.abs(got - refs[r.id]).max() <= 1e-11 * np.abs(refs[r.id]).max(), r.id
    ck = str(tmp_path / "ckpt")
    first = serving.Server(pool, head + 4 * sum(peaks), max_rhs=16, grid=GRID, checkpoint_dir=ck)
    st1 = first.run(reqs)
    first.close()
    assert st1.builds == 3 and st1.loads == 0
    second = serving.Server(pool, head + 4 * sum(peaks), max_rhs=16, grid=GRID, checkpoint_dir=ck)
    st2, res2 = second.run(reqs, keep_results=True)
    second.close()
    assert st2.builds == 0 and st2.loads == 3
    for r in reqs:
        got = res2[r.id].numpy()
        assert np.abs(got - refs[r.id]).max() <= 1e-11 * np.abs(refs[r.id]).max(), r.id
