"""Python binding of libmueller (ctypes; argument marshalling only).

Every computation runs in the CUDA library built from ``csrc/``; there is no
CPU fallback: importing this package raises if ``libmueller.so`` is missing.
Device buffers are torch tensors (complex128 / float64 / int32 on CUDA,
contiguous); streams default to torch's current stream.
"""
from __future__ import annotations

import ctypes as ct
import os
from dataclasses import dataclass

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libmueller.so")
if not os.path.exists(_LIB_PATH):
    raise ImportError(f"{_LIB_PATH} is missing: build it with paper_1810_07067_gb300.build.build() "
                      "(or __graft_entry__.build()); there is no CPU fallback")
_lib = ct.CDLL(_LIB_PATH)


class c128(ct.Structure):
    _fields_ = [("re", ct.c_double), ("im", ct.c_double)]


def _c(z) -> c128:
    z = complex(z)
    return c128(z.real, z.imag)


class _Curve(ct.Structure):
    _fields_ = [("n_panels", ct.c_int), ("closed", ct.c_int), ("r", ct.POINTER(ct.c_double)),
                ("z", ct.POINTER(ct.c_double)), ("dr", ct.POINTER(ct.c_double)), ("dz", ct.POINTER(ct.c_double))]


class _Media(ct.Structure):
    _fields_ = [("omega", ct.c_double), ("eps0", c128), ("mu0", c128), ("eps1", c128), ("mu1", c128)]


class _Options(ct.Structure):
    _fields_ = [("n_phi", ct.c_int), ("formulation", ct.c_int), ("precision", ct.c_int),
                ("refine_tol", ct.c_double), ("refine_max_iter", ct.c_int), ("split_eps", ct.c_double),
                ("lu_tile", ct.c_int)]


class Stats(ct.Structure):
    _fields_ = [("ms_legendre", ct.c_double), ("ms_far", ct.c_double), ("ms_support", ct.c_double),
                ("ms_near", ct.c_double), ("ms_lu", ct.c_double), ("ms_build", ct.c_double),
                ("ms_solve", ct.c_double), ("n_phi_used", ct.c_int), ("n_split_pairs", ct.c_longlong),
                ("n_far_pairs", ct.c_longlong), ("n_support_pairs", ct.c_longlong), ("singular_mode", ct.c_int),
                ("singular_column", ct.c_int), ("device_bytes", ct.c_size_t), ("ms_lu_gemm", ct.c_double),
                ("lu_gemm_flops", ct.c_double), ("lu_gemm_launches", ct.c_int), ("launches", ct.c_int),
                ("solve_launches", ct.c_int), ("refine_iters", ct.c_int), ("backward_err_max", ct.c_double),
                ("ms_residual", ct.c_double), ("residual_launches", ct.c_int), ("residual_tc_flops", ct.c_double),
                ("lu_graph", ct.c_int), ("lu_tile_steps", ct.c_int * 3), ("lu_wave_bodies", ct.c_int),
                ("lu_launches", ct.c_int), ("lu_gemm_bytes", ct.c_double), ("spilled", ct.c_int),
                ("host_bytes", ct.c_size_t), ("kappa_mode0", ct.c_double), ("kappa_max", ct.c_double),
                ("kappa_max_mode", ct.c_int), ("ms_cond", ct.c_double), ("ms_far_sample", ct.c_double),
                ("ms_far_product", ct.c_double), ("ms_far_assemble", ct.c_double), ("far_blocks", ct.c_double)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["lu_tile_steps"] = list(d["lu_tile_steps"])
        return d


_vp = ct.c_void_p
_lib.mueller_build.argtypes = [ct.POINTER(_Curve), ct.POINTER(_Media), ct.c_int, ct.POINTER(_Options), _vp,
                               ct.POINTER(_vp)]
_lib.mueller_build_many.argtypes = [ct.c_int, ct.POINTER(_Curve), ct.POINTER(_Media), ct.POINTER(ct.c_int),
                                    ct.POINTER(_Options), _vp, ct.POINTER(_vp)]
_lib.mueller_build_many_bytes.argtypes = [ct.c_int, ct.POINTER(ct.c_int), ct.POINTER(ct.c_int), ct.c_int]
_lib.mueller_build_many_bytes.restype = ct.c_size_t
_lib.mueller_lu_tile_table.argtypes = [ct.POINTER(ct.c_int), ct.POINTER(ct.c_int), ct.POINTER(ct.c_int),
                                       ct.POINTER(ct.c_float), ct.c_int]
_lib.mueller_cache_trim.argtypes = []
_lib.mueller_cache_trim.restype = None
_lib.mueller_cache_limit.argtypes = [ct.c_size_t]
_lib.mueller_cache_limit.restype = ct.c_size_t
_lib.mueller_cache_bytes.argtypes = []
_lib.mueller_cache_bytes.restype = ct.c_size_t
_lib.mueller_assemble.argtypes = [ct.POINTER(_Curve), ct.POINTER(_Media), ct.c_int, ct.POINTER(_Options), _vp, _vp]
_lib.mueller_solve.argtypes = [_vp, _vp, ct.c_int, _vp, ct.POINTER(ct.c_double), _vp]
_lib.mueller_rhs_planewave.argtypes = [_vp, ct.POINTER(ct.c_double), ct.POINTER(ct.c_double), ct.c_int, _vp, _vp]
_lib.mueller_far_field.argtypes = [_vp, _vp, ct.c_int, _vp, ct.c_int, _vp, _vp]
_lib.mueller_modal_kernels.argtypes = [ct.POINTER(ct.c_double), ct.c_longlong, c128, c128, ct.c_int, ct.c_int,
                                       ct.c_double, _vp, _vp]
_lib.mueller_lu_batched.argtypes = [_vp, ct.c_int, ct.c_int, _vp, _vp, _vp]
_lib.mueller_rhs_fields.argtypes = [_vp, _vp, ct.c_int, ct.c_int, _vp, _vp]
_lib.mueller_eval.argtypes = [_vp, _vp, ct.c_int, _vp, ct.c_int, ct.c_int, _vp, _vp]
_lib.mueller_far_field_grid.argtypes = [_vp, _vp, ct.c_int, ct.c_int, ct.c_int, _vp, _vp]
_lib.mueller_lu_batched_c64.argtypes = [_vp, ct.c_int, ct.c_int, _vp, _vp, _vp]
_lib.mueller_modal_kernels_noalloc.argtypes = [_vp, ct.c_longlong, c128, c128, ct.c_int, ct.c_int, ct.c_double,
                                               _vp, _vp]
_lib.mueller_footprint_bytes.argtypes = [ct.c_int, ct.c_int]
_lib.mueller_build_bytes.argtypes = [ct.c_int, ct.c_int, ct.c_int, ct.POINTER(ct.c_size_t)]
_lib.mueller_build_bytes.restype = ct.c_size_t
_lib.mueller_footprint_bytes.restype = ct.c_size_t
_lib.mueller_fp64_peak.argtypes = [ct.POINTER(ct.c_double), _vp]
_lib.mueller_cond_estimate.argtypes = [_vp, ct.POINTER(ct.c_double), _vp]
_lib.mueller_ctx_spill.argtypes = [_vp, _vp]
_lib.mueller_ctx_restore.argtypes = [_vp, _vp]
_lib.mueller_ctx_save.argtypes = [_vp, ct.c_char_p]
_lib.mueller_ctx_load.argtypes = [ct.c_char_p, _vp, ct.POINTER(_vp)]
_lib.mueller_stats_get.argtypes = [_vp, ct.POINTER(Stats)]
_lib.mueller_destroy.argtypes = [_vp]
_lib.mueller_strerror.restype = ct.c_char_p
_lib.mueller_strerror.argtypes = [ct.c_int]
_lib.mueller_last_error.restype = ct.c_char_p

EXPORTS = ["mueller_build", "mueller_assemble", "mueller_solve", "mueller_rhs_planewave", "mueller_rhs_fields",
           "mueller_far_field", "mueller_far_field_grid", "mueller_eval",
           "mueller_modal_kernels", "mueller_modal_kernels_noalloc", "mueller_lu_batched", "mueller_lu_batched_c64", "mueller_footprint_bytes", "mueller_build_bytes", "mueller_stats_get",
           "mueller_build_many", "mueller_build_many_bytes", "mueller_lu_tile_table",
           "mueller_cache_trim", "mueller_cache_limit", "mueller_cache_bytes",
           "mueller_fp64_peak", "mueller_cond_estimate", "mueller_ctx_spill", "mueller_ctx_restore", "mueller_ctx_save", "mueller_ctx_load",
           "mueller_destroy", "mueller_strerror", "mueller_last_error"]


class MuellerError(RuntimeError):
    def __init__(self, status: int):
        msg = _lib.mueller_strerror(status).decode()
        detail = _lib.mueller_last_error().decode()
        super().__init__(f"{msg}: {detail}" if detail else msg)
        self.status = status


def _check(rc: int):
    if rc != 0:
        raise MuellerError(rc)


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("device buffers must be contiguous CUDA tensors")
    return ct.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is not None:
        return ct.c_void_p(getattr(stream, "cuda_stream", stream))
    import torch
    return ct.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ct.POINTER(ct.c_double))


@dataclass
class Options:
    n_phi: int = 64
    formulation: int = 0
    precision: int = 0
    refine_tol: float = 1e-14
    refine_max_iter: int = 10
    split_eps: float = 1e-17
    lu_tile: int = 0          # mixed path: LU update column tile 32 / 64 / 128, 0 = autotuned

    def _c(self):
        return _Options(self.n_phi, self.formulation, self.precision, self.refine_tol, self.refine_max_iter,
                        self.split_eps, self.lu_tile)


def _curve_struct(curve):
    arrs = [np.ascontiguousarray(np.asarray(a, dtype=np.float64)) for a in (curve.r, curve.z, curve.dr, curve.dz)]
    s = _Curve(int(curve.n_panels), int(bool(getattr(curve, "closed", False))), *[_dptr(a) for a in arrs])
    return s, arrs


def _media_struct(m):
    return _Media(float(m.omega), _c(m.eps0), _c(m.mu0), _c(m.eps1), _c(m.mu1))


class Context:
    """Per-body factors of modes 0..M resident on the device."""

    def __init__(self, curve, media, M: int, options: Options | None = None, stream=None, _handle=None):
        if _handle is not None:  # a context made by build_many
            self._h, self.M, self.N, self._keep = _handle, int(M), int(curve.n_panels) * 16, None
            return
        options = options or Options()
        cs, self._keep = _curve_struct(curve)
        ms = _media_struct(media)
        h = ct.c_void_p()
        self.M = int(M)
        self.N = int(curve.n_panels) * 16
        rc = _lib.mueller_build(ct.byref(cs), ct.byref(ms), self.M, ct.byref(options._c()), _stream(stream),
                                ct.byref(h))
        self._h = h
        _check(rc)

    def solve(self, rhs, x, backward_err: np.ndarray | None = None, stream=None):
        nrhs = rhs.shape[1]
        be = None if backward_err is None else backward_err.ctypes.data_as(ct.POINTER(ct.c_double))
        _check(_lib.mueller_solve(self._h, _ptr(rhs), nrhs, _ptr(x), be, _stream(stream)))
        return x

    def rhs_planewave(self, dirs, pols, rhs, stream=None):
        d = np.ascontiguousarray(np.asarray(dirs, np.float64).reshape(-1, 3))
        p = np.ascontiguousarray(np.asarray(pols, np.float64).reshape(-1, 3))
        _check(_lib.mueller_rhs_planewave(self._h, _dptr(d), _dptr(p), len(d), _ptr(rhs), _stream(stream)))
        return rhs

    def rhs_fields(self, EH, rhs, stream=None):
        """Modal data from sampled fields EH [nrhs, N, n_theta, 6] (device, complex128)."""
        _check(_lib.mueller_rhs_fields(self._h, _ptr(EH), EH.shape[0], EH.shape[2], _ptr(rhs), _stream(stream)))
        return rhs

    def eval(self, x, targets, region, out, stream=None):
        """E, H at host points targets [nt, 3] into out [nrhs, nt, 6] (device); region 0 exterior, 1 body."""
        t = np.ascontiguousarray(np.asarray(targets, np.float64).reshape(-1, 3))
        _check(_lib.mueller_eval(self._h, _ptr(x), x.shape[1], _dptr(t), len(t), int(region), _ptr(out),
                                 _stream(stream)))
        return out

    def far_field_grid(self, x, E, stream=None):
        """E [nrhs, n_polar, n_azim, 3] (device) on the grid theta_p = (p + 1/2) pi / n_polar, phi_s = 2 pi s / n_azim."""
        _check(_lib.mueller_far_field_grid(self._h, _ptr(x), x.shape[1], E.shape[1], E.shape[2], _ptr(E),
                                           _stream(stream)))
        return E

    def far_field(self, x, dirs, E, stream=None):
        _check(_lib.mueller_far_field(self._h, _ptr(x), x.shape[1], _ptr(dirs), dirs.shape[0], _ptr(E),
                                      _stream(stream)))
        return E

    def cond_estimate(self, stream=None) -> np.ndarray:
        """kappa_inf of the weighted system of every mode 0..M (Hager's estimate from the factors)."""
        k = np.zeros(self.M + 1)
        _check(_lib.mueller_cond_estimate(self._h, k.ctypes.data_as(ct.POINTER(ct.c_double)), _stream(stream)))
        return k

    def spill(self, stream=None):
        """Move the factors to pinned host memory and free their device memory."""
        _check(_lib.mueller_ctx_spill(self._h, _stream(stream)))

    def restore(self, stream=None):
        """Bring spilled factors back to the device."""
        _check(_lib.mueller_ctx_restore(self._h, _stream(stream)))

    def save(self, path: str):
        """Write a checkpoint (build inputs + factors) to path."""
        _check(_lib.mueller_ctx_save(self._h, os.fsencode(path)))

    @classmethod
    def load(cls, path: str, stream=None) -> "Context":
        """A context from a checkpoint written by save (no assembly or factorization)."""
        h = _vp()
        _check(_lib.mueller_ctx_load(os.fsencode(path), _stream(stream), ct.byref(h)))
        ctx = cls.__new__(cls)
        ctx._h, ctx._keep = h, None
        with open(path, "rb") as f:                      # header: magic, version, panels, closed, M, N
            head = np.frombuffer(f.read(28)[8:], dtype="<i4")
        ctx.M, ctx.N = int(head[3]), int(head[4])
        return ctx

    def stats(self) -> dict:
        st = Stats()
        _check(_lib.mueller_stats_get(self._h, ct.byref(st)))
        return st.as_dict()

    def close(self):
        if getattr(self, "_h", None):
            _lib.mueller_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def build(curve, media, M: int, options: Options | None = None, stream=None) -> Context:
    return Context(curve, media, M, options, stream)


def build_many(bodies, options: Options | None = None, stream=None) -> list[Context]:
    """Build a wave of bodies, given as (curve, media, M) triples: each is
    assembled in turn, then all modes of all bodies are factored together in
    one graph-launched LU (mueller_build_many)."""
    options = options or Options()
    count = len(bodies)
    curves = (_Curve * count)()
    medias = (_Media * count)()
    Ms = (ct.c_int * count)()
    keep = []
    for i, (curve, media, M) in enumerate(bodies):
        cs, arrs = _curve_struct(curve)
        keep.append(arrs)
        curves[i] = cs
        medias[i] = _media_struct(media)
        Ms[i] = int(M)
    hs = (_vp * count)()
    rc = _lib.mueller_build_many(count, curves, medias, Ms, ct.byref(options._c()), _stream(stream), hs)
    ctxs = [Context(b[0], b[1], b[2], _handle=ct.c_void_p(hs[i])) for i, b in enumerate(bodies) if hs[i]]
    if rc != 0:
        for c in ctxs:
            c.close()
        raise MuellerError(rc)
    return ctxs


def build_many_bytes(N, M, precision: int) -> int:
    """Peak device bytes of build_many for bodies of N[i] nodes and modes 0..M[i]."""
    count = len(N)
    n_arr = (ct.c_int * count)(*[int(v) for v in N])
    m_arr = (ct.c_int * count)(*[int(v) for v in M])
    return int(_lib.mueller_build_many_bytes(count, n_arr, m_arr, int(precision)))


def lu_tile_table(cap: int = 256) -> list[dict]:
    """The LU tile autotuner's decisions in this process (see mueller.h)."""
    rh = (ct.c_int * cap)()
    ch = (ct.c_int * cap)()
    tl = (ct.c_int * cap)()
    ms = (ct.c_float * (3 * cap))()
    k = _lib.mueller_lu_tile_table(rh, ch, tl, ms, cap)
    return [{"rest_hi": rh[i], "count_hi": ch[i], "tile": tl[i], "ms_per_matrix": list(ms[3 * i:3 * i + 3])}
            for i in range(max(k, 0))]


def assemble(curve, media, M: int, A, options: Options | None = None, stream=None):
    """Weighted per-mode matrices for modes 0..M into A [M+1, 4N, 4N] (column-major per mode:
    A[m] holds the transpose of the matrix in row-major view)."""
    options = options or Options()
    cs, keep = _curve_struct(curve)
    ms = _media_struct(media)
    _check(_lib.mueller_assemble(ct.byref(cs), ct.byref(ms), int(M), ct.byref(options._c()), _ptr(A),
                                 _stream(stream)))
    return A


def _check_spectra_out(out, npairs: int, M: int):
    """out must hold npairs x 9 x (M + 2) complex128 values (the kernels write all of them)."""
    import torch
    if out.dtype != torch.complex128:
        raise ValueError(f"out must be complex128, got {out.dtype}")
    if M < 0 or out.numel() < npairs * 9 * (M + 2):
        raise ValueError(f"out holds {out.numel()} values; {npairs} pairs x 9 families x (M + 2) need "
                         f"{npairs * 9 * (M + 2)}")


def _check_current_device(*tensors):
    import torch
    cur = torch.cuda.current_device()
    for t in tensors:
        if not t.is_cuda or t.device.index != cur:
            raise ValueError(f"tensors must be on the current CUDA device (cuda:{cur}), got {t.device}")


def modal_kernels(pairs: np.ndarray, k0, k1, M: int, n_phi: int, out, split_eps: float = 1e-17, stream=None):
    p = np.ascontiguousarray(np.asarray(pairs, np.float64).reshape(-1, 4))
    _check_spectra_out(out, len(p), int(M))
    _check_current_device(out)
    _check(_lib.mueller_modal_kernels(_dptr(p), len(p), _c(k0), _c(k1), int(M), int(n_phi), float(split_eps),
                                      _ptr(out), _stream(stream)))
    return out


def modal_kernels_noalloc(pairs_dev, k0, k1, M: int, n_phi: int, out, split_eps: float = 1e-17, stream=None):
    """Same spectra as ``modal_kernels`` for pairs already on the device, using
    the library's fixed scratch array instead of allocating (see mueller.h)."""
    import torch
    if pairs_dev.dtype != torch.float64 or pairs_dev.dim() != 2 or pairs_dev.shape[1] != 4:
        raise ValueError(f"pairs_dev must be float64 of shape (npairs, 4), got {pairs_dev.dtype} "
                         f"{tuple(pairs_dev.shape)}")
    _check_spectra_out(out, pairs_dev.shape[0], int(M))
    _check_current_device(pairs_dev, out)
    _check(_lib.mueller_modal_kernels_noalloc(_ptr(pairs_dev), pairs_dev.shape[0], _c(k0), _c(k1), int(M),
                                              int(n_phi), float(split_eps), _ptr(out), _stream(stream)))
    return out


def lu_batched(A, piv, info, stream=None):
    n = A.shape[-1]
    batch = A.shape[0]
    _check(_lib.mueller_lu_batched(_ptr(A), n, batch, _ptr(piv), _ptr(info), _stream(stream)))


def lu_batched_c64(A, piv, info, stream=None):
    """Complex64 batched LU with tensor-core trailing updates (in place)."""
    import torch
    if A.dtype != torch.complex64:
        raise ValueError("lu_batched_c64 takes complex64 matrices")
    n = A.shape[-1]
    batch = A.shape[0]
    _check(_lib.mueller_lu_batched_c64(_ptr(A), n, batch, _ptr(piv), _ptr(info), _stream(stream)))


def build_bytes(N: int, M: int, precision: int) -> tuple[int, int]:
    """(peak bytes during mueller_build, bytes resident afterwards)."""
    res = ct.c_size_t(0)
    peak = int(_lib.mueller_build_bytes(int(N), int(M), int(precision), ct.byref(res)))
    return peak, int(res.value)


def cache_trim() -> None:
    """Return every cached device block to the driver (see mueller_cache_limit)."""
    _lib.mueller_cache_trim()


def cache_limit(nbytes: int) -> int:
    """Cap on the library's cache of freed device blocks; returns the previous cap."""
    return int(_lib.mueller_cache_limit(int(nbytes)))


def cache_bytes() -> int:
    return int(_lib.mueller_cache_bytes())


def fp64_peak(stream=None) -> float:
    """Measured FP64 peak of the current device, TFLOP/s (DFMA register loop)."""
    v = ct.c_double(0.0)
    _check(_lib.mueller_fp64_peak(ct.byref(v), _stream(stream)))
    return float(v.value)


def footprint_bytes(N: int, M: int) -> int:
    return int(_lib.mueller_footprint_bytes(N, M))


def library_path() -> str:
    return _LIB_PATH
