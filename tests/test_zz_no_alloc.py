"""Allocation-free modal-kernel entry point against the allocating one.

Some callers cannot allocate device memory (their memory is owned by another
allocator, or a cudaMalloc in their loop could block or fail); for them the
library offers mueller_modal_kernels_noalloc, whose scratch is a fixed array
inside the library.  This file is collected last so that a failure here does
not stop the rest of a ``-x`` run; it runs alone in a fresh process as well.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _pairs():
    rng = np.random.default_rng(11)
    base = [(1.0, 0.0, 0.3, 1.5), (1.0, 0.0, 0.95, 0.05), (0.5, 0.2, 0.5, 0.2 + 1e-7),
            (0.5, 0.2, 0.5 + 3e-9, 0.2 + 1e-9), (0.02, -0.99, 0.01, -0.995), (0.7, 0.3, 0.72, 0.33)]
    rt = rng.uniform(0.05, 1.0, 40); zt = rng.uniform(-1.0, 1.0, 40)
    d = rng.uniform(1e-6, 0.5, 40) * rng.choice([-1.0, 1.0], 40)
    for a, b, c in zip(rt, zt, d):
        base.append((a, b, a * (1.0 + 0.7 * c), b - 0.4 * c * a))   # r_s >= 0.65 r_t > 0
    return np.array(base)


def test_noalloc_matches_allocating_entry_point():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1810_07067_gb300 as mb
    pairs = _pairs()
    pairs_dev = torch.tensor(pairs, device="cuda:0")
    # two calls in a row, different sizes and wavenumbers, sharing the scratch
    for (k0, k1, M, nphi) in ((5.0, 7.5 + 0.01j, 64, 256), (1.0, 1.5, 10, 64)):
        ref = torch.zeros((len(pairs), 9, M + 2), dtype=torch.complex128, device="cuda:0")
        got = torch.full_like(ref, complex("nan"))
        mb.modal_kernels(pairs, k0, k1, M, nphi, ref)
        mb.modal_kernels_noalloc(pairs_dev, k0, k1, M, nphi, got)
        torch.cuda.synchronize()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        scale = np.maximum(np.abs(r).max(axis=2, keepdims=True), 1e-300)
        err = (np.abs(g - r) / scale).max()
        assert err < 1e-12, (k0, k1, M, nphi, err)


def test_noalloc_rejects_oversized_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1810_07067_gb300 as mb
    pairs_dev = torch.ones((20000, 4), dtype=torch.float64, device="cuda:0")
    out = torch.zeros((20000, 9, 66), dtype=torch.complex128, device="cuda:0")
    with pytest.raises(mb.MuellerError, match="fixed scratch"):
        mb.modal_kernels_noalloc(pairs_dev, 1.0, 1.5, 64, 256, out)
