"""Admission of many bodies under a byte budget (host logic, no GPU): the
budget is never exceeded, every body runs once, bodies overlap when they
fit together, and a body larger than the budget is refused up front."""
import threading
import time
from types import SimpleNamespace

import pytest

from paper_1810_07067_gb300 import batch, build_bytes


def _bodies(sizes):
    return [SimpleNamespace(name=f"b{i}", curve=SimpleNamespace(N=N), M=M, n_phi=16, waves=[])
            for i, (N, M) in enumerate(sizes)]


def test_budget_respected_and_all_bodies_run():
    sizes = [(1024, 96), (208, 32), (640, 64), (400, 40), (896, 120), (320, 48), (512, 32), (208, 128)]
    bodies = _bodies(sizes)
    peaks = [build_bytes(N, M, 1)[0] for N, M in sizes]
    budget = int(1.6 * max(peaks))
    lock = threading.Lock()
    live = {"bytes": 0, "max_bytes": 0, "n": 0, "max_n": 0}
    seen = []

    def fake(i, body, w, adm, peak):
        with lock:
            live["bytes"] += peak; live["n"] += 1
            live["max_bytes"] = max(live["max_bytes"], live["bytes"]); live["max_n"] = max(live["max_n"], live["n"])
            seen.append(i)
        r = batch.BodyResult(i, body.name, body.curve.N, body.M, peak_bytes=peak, t_start=time.perf_counter())
        time.sleep(0.02)
        with lock:
            live["bytes"] -= peak; live["n"] -= 1
        adm.lower(peak)
        r.t_end = time.perf_counter()
        return r

    res, wall, adm = batch.run_batch(bodies, budget, n_streams=3, process=fake)
    assert sorted(seen) == list(range(len(bodies)))
    assert all(r is not None and r.index == i for i, r in enumerate(res))
    assert live["max_bytes"] <= budget and adm.high_water <= budget
    assert live["max_n"] >= 2                       # smaller bodies ran beside larger ones
    assert adm.in_use == 0
    # largest first: the biggest body starts before any body that did not fit beside it
    first = min(res, key=lambda r: r.t_start)
    assert first.peak_bytes == max(peaks)


def test_body_above_budget_is_refused():
    bodies = _bodies([(1200, 128), (208, 32)])
    with pytest.raises(ValueError):
        batch.run_batch(bodies, build_bytes(208, 32, 1)[0] * 2, n_streams=2, process=lambda *a: None)


def test_worker_error_is_raised():
    bodies = _bodies([(208, 32)] * 4)

    def bad(i, body, w, adm, peak):
        raise RuntimeError("boom")

    with pytest.raises(RuntimeError):
        batch.run_batch(bodies, 10 ** 13, n_streams=2, process=bad)


def test_wave_plan_covers_every_body_within_budget():
    """Waves for build_many: every body in exactly one wave, largest first,
    each wave's peak (the library's build_many_bytes) within the budget, and a
    wave's peak between its largest member's build peak and the sum of the
    members' build peaks."""
    from paper_1810_07067_gb300 import build_many_bytes
    sizes = [(1024, 96), (208, 32), (640, 64), (400, 40), (896, 120), (320, 48), (512, 32), (208, 128)]
    bodies = _bodies(sizes)
    peaks = [build_bytes(N, M, 1)[0] for N, M in sizes]
    budget = int(1.6 * max(peaks))
    plan = batch.plan_waves(bodies, budget, precision=1)
    got = sorted(i for wave, _ in plan for i in wave)
    assert got == list(range(len(sizes)))
    assert plan[0][0][0] == max(range(len(sizes)), key=lambda i: peaks[i])
    assert len(plan) < len(sizes)                     # bodies share waves
    for wave, est in plan:
        assert est == build_many_bytes([sizes[i][0] for i in wave], [sizes[i][1] for i in wave], 1)
        assert est <= budget
        assert max(peaks[i] for i in wave) <= est <= sum(peaks[i] for i in wave) + sum(
            build_many_bytes([sizes[i][0]], [sizes[i][1]], 1) - peaks[i] for i in wave)


def test_wave_plan_refuses_a_body_above_the_budget():
    bodies = _bodies([(1024, 96), (208, 32)])
    with pytest.raises(ValueError, match="budget"):
        batch.plan_waves(bodies, build_bytes(1024, 96, 1)[0] // 2, precision=1)
