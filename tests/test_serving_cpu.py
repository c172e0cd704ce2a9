"""Request generation of the serving workload (host only)."""
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
