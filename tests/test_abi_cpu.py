"""Host-side checks of the C ABI (no GPU work): the library loads and exports
every function that include/mueller.h declares; host logic of the binding."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mueller.h")
LIB = os.path.join(ROOT, "paper_1810_07067_gb300", "libmueller.so")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mueller_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        import __graft_entry__
        __graft_entry__.build()
    import ctypes
    return ctypes.CDLL(LIB)


def test_header_declares_entry_points():
    names = _declared()
    for n in ("mueller_build", "mueller_solve", "mueller_far_field", "mueller_modal_kernels"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_lists_every_export(lib):
    import paper_1810_07067_gb300 as mb
    assert sorted(mb.EXPORTS) == _declared()


def test_footprint_and_strerror(lib):
    import paper_1810_07067_gb300 as mb
    assert mb.footprint_bytes(64, 10) == 16 * 256 * 256 * 21
    assert mb._lib.mueller_strerror(0) == b"ok"
    assert mb._lib.mueller_strerror(3) == b"exact zero pivot"


def test_build_rejects_bad_inputs_before_device_work(lib):
    """Argument checks run on the host before any CUDA call."""
    import numpy as np
    import paper_1810_07067_gb300 as mb
    import workloads as W
    cur = W.sphere(2)
    with pytest.raises(mb.MuellerError, match="omega"):
        mb.build(cur, W.Media(omega=0.0), 2, stream=0)
    with pytest.raises(mb.MuellerError, match="eps1"):
        mb.build(cur, W.Media(omega=1.0, eps1=-1.0 + 0j), 2, stream=0)
    bad = W.Curve(cur.n_panels, cur.r.copy(), -cur.z.copy(), cur.dr.copy(), -cur.dz.copy())
    with pytest.raises(mb.MuellerError, match="counterclockwise"):
        mb.build(bad, W.Media.from_k(1.0, 1.5), 2, stream=0)
    with pytest.raises(mb.MuellerError, match="FP64"):
        mb.build(cur, W.Media.from_k(1.0, 1.5), 2, mb.Options(precision=7), stream=0)
    with pytest.raises(mb.MuellerError, match="lu_tile"):
        mb.build(cur, W.Media.from_k(1.0, 1.5), 2, mb.Options(precision=1, lu_tile=48), stream=0)


def test_build_many_rejects_bad_inputs_before_device_work(lib):
    """Wave builds check the count and every body on the host first."""
    import paper_1810_07067_gb300 as mb
    import workloads as W
    cur = W.sphere(2)
    with pytest.raises(mb.MuellerError, match="count"):
        mb.build_many([], stream=0)
    with pytest.raises(mb.MuellerError, match="omega"):
        mb.build_many([(cur, W.Media(omega=0.0), 2), (cur, W.Media.from_k(1.0, 1.5), 2)], stream=0)
    assert mb.build_many_bytes([64, 32], [10, 4], 1) >= max(mb.build_bytes(64, 10, 1)[0], mb.build_bytes(32, 4, 1)[0])
    assert mb.build_many_bytes([], [], 1) == 0


def test_modal_kernel_wrappers_check_buffers_before_the_call(lib):
    """A wrongly typed or too small buffer is refused on the host: the kernels
    would otherwise read or write past it."""
    torch = pytest.importorskip("torch")
    import numpy as np
    import paper_1810_07067_gb300 as mb
    M, n = 4, 3
    good_pairs = torch.ones((n, 4), dtype=torch.float64)
    good_out = torch.zeros((n, 9, M + 2), dtype=torch.complex128)
    with pytest.raises(ValueError, match="float64"):
        mb.modal_kernels_noalloc(good_pairs.float(), 1.0, 1.5, M, 64, good_out)
    with pytest.raises(ValueError, match="shape"):
        mb.modal_kernels_noalloc(torch.ones((n, 3), dtype=torch.float64), 1.0, 1.5, M, 64, good_out)
    with pytest.raises(ValueError, match="complex128"):
        mb.modal_kernels_noalloc(good_pairs, 1.0, 1.5, M, 64, good_out.to(torch.complex64))
    with pytest.raises(ValueError, match="need"):
        mb.modal_kernels_noalloc(good_pairs, 1.0, 1.5, M + 1, 64, good_out)
    with pytest.raises(ValueError, match="need"):
        mb.modal_kernels(np.ones((n, 4)), 1.0, 1.5, M, 64, good_out[:2])
    with pytest.raises(ValueError, match="complex128"):
        mb.modal_kernels(np.ones((n, 4)), 1.0, 1.5, M, 64, good_out.real.contiguous())
    if not torch.cuda.is_available():  # CPU tensors of the right type and size: refused as off-device
        with pytest.raises((ValueError, RuntimeError, AssertionError)):
            mb.modal_kernels_noalloc(good_pairs, 1.0, 1.5, M, 64, good_out)
