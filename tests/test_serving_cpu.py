"""Host logic of the serving workload: request generation and the device
factor cache's eviction into the host cache (no GPU)."""
import numpy as np

from paper_1810_07067_gb300 import serving


def test_poisson_stream_statistics():
    reqs = serving.poisson_requests(32, rate=200.0, duration=20.0, seed=5, zipf=1.1, max_rhs=256)
    n = len(reqs)
    assert abs(n - 4000) < 4 * np.sqrt(4000)                     # Poisson count, mean rate * duration
    gaps = np.diff([0.0] + [r.arrival for r in reqs])
    assert abs(gaps.mean() - 1 / 200) < 0.1 / 200
    keys = np.bincount([r.key for r in reqs], minlength=32) / n
    w = 1 / np.arange(1, 33) ** 1.1
    assert np.abs(keys - w / w.sum()).max() < 0.02                # Zipf(1.1) over the pool
    k = np.array([r.nrhs for r in reqs])
    assert k.min() >= 1 and k.max() <= 256 and abs(k.mean() - 128.5) < 5
    r = reqs[0]
    assert np.allclose(np.linalg.norm(r.dirs, axis=1), 1) and np.allclose(np.linalg.norm(r.pols, axis=1), 1)
    assert np.abs((r.dirs * r.pols).sum(1)).max() < 1e-12


def test_uniform_choice():
    reqs = serving.poisson_requests(8, rate=100.0, duration=20.0, seed=1, zipf=0.0, max_rhs=4)
    keys = np.bincount([r.key for r in reqs], minlength=8) / len(reqs)
    assert np.abs(keys - 1 / 8).max() < 0.03


class _FakeCtx:
    """Stands in for a Context in the cache bookkeeping: records spills and closes."""

    def __init__(self, key, log):
        self.key, self.log = key, log

    def spill(self, stream=None):
        self.log.append(("spill", self.key))

    def close(self):
        self.log.append(("close", self.key))


def _server(budget, host_budget, resident):
    """A Server's cache state without its CUDA resources (host logic only)."""
    from collections import OrderedDict
    s = object.__new__(serving.Server)
    s.cache, s.host_cache = OrderedDict(), OrderedDict()
    s.budget, s.host_budget = budget, host_budget
    s.charged, s.host_charged = 0, 0
    s.serve_stream = None
    log = []
    for key, nbytes in resident:                  # least recently used first
        s.cache[key] = serving._Entry(_FakeCtx(key, log), nbytes)
        s.charged += nbytes
    return s, log


def test_eviction_is_lru_and_spares_keys_with_waiting_requests():
    s, log = _server(100, 0, [(0, 40), (1, 30), (2, 20)])
    st = serving.ServeStats()
    assert s._evict_for(50, st, keep={0})
    assert log == [("close", 1), ("close", 2)]      # key 0 waits: kept although least recently used
    assert list(s.cache) == [0] and s.charged == 40 and st.evictions == 2 and st.spills == 0


def test_eviction_stops_as_soon_as_the_request_fits():
    s, log = _server(100, 0, [(0, 40), (1, 30), (2, 20)])
    st = serving.ServeStats()
    assert s._evict_for(40, st)
    assert log == [("close", 0)] and list(s.cache) == [1, 2] and s.charged == 50


def test_eviction_refuses_when_only_kept_keys_remain():
    s, log = _server(100, 0, [(0, 60), (1, 30)])
    st = serving.ServeStats()
    assert not s._evict_for(50, st, keep={0, 1})
    assert log == [] and s.charged == 90 and st.evictions == 0


def test_evicted_keys_park_in_the_host_cache_within_its_budget():
    s, log = _server(100, 35, [(0, 40), (1, 30), (2, 20)])
    st = serving.ServeStats()
    assert s._evict_for(60, st, keep={0})
    # key 1 (30 bytes) is spilled; key 2 (20) needs room: the host cache drops key 1, its oldest entry
    assert log == [("spill", 1), ("close", 1), ("spill", 2)]
    assert list(s.host_cache) == [2] and s.host_charged == 20
    assert st.spills == 2 and st.evictions == 2 and list(s.cache) == [0]


def test_keys_larger_than_the_host_budget_are_closed():
    s, log = _server(100, 25, [(0, 40), (1, 30)])
    st = serving.ServeStats()
    assert s._evict_for(80, st)
    assert log == [("close", 0), ("close", 1)] and not s.host_cache and st.spills == 0
