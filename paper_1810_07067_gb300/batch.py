"""Many bodies on one GPU under a device-memory budget.

Every body is an independent problem (its own curve, wavenumbers and modes).
A body is admitted when the peak bytes of its build (mueller_build_bytes)
fit beside what the bodies in flight hold; the first waiting body that fits
is taken, so smaller bodies fill the room a large one leaves.  Each admitted
body is built, solved and released by one of n_streams worker threads, each
with its own CUDA stream, so the latency-bound phases of one body (LU panels,
small modes) overlap the arithmetic of another.  After a build the admission
drops the body's charge from the build peak to its resident bytes; after the
solve (and the caller's check, if any) the body's factors are freed.  The
factors of 1.7 TB of bodies therefore pass through the device in waves.
"""
from __future__ import annotations

import threading
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class BodyResult:
    index: int
    name: str
    N: int
    M: int
    n_phi: int = 0
    worker: int = -1
    t_start: float = 0.0          # seconds since the batch started
    t_end: float = 0.0
    build_ms: float = 0.0         # library stage times (CUDA events)
    lu_ms: float = 0.0
    solve_ms: float = 0.0
    peak_bytes: int = 0
    resident_bytes: int = 0
    refine_iters: int = 0
    backward_err: float = 0.0
    launches: int = 0             # kernel launches of the build, RHS and solve
    extra: dict = field(default_factory=dict)


class Admission:
    """Byte budget shared by the worker threads; hands out waiting bodies."""

    def __init__(self, items, budget: int):
        # items: list of (key, peak_bytes); taken in the given order when they fit
        self._cv = threading.Condition()
        self._wait = list(items)
        self.budget = int(budget)
        self.in_use = 0
        self.high_water = 0
        for key, peak in self._wait:
            if peak > self.budget:
                raise ValueError(f"body {key} needs {peak} bytes, above the budget of {self.budget}")

    def next(self):
        """Block until a waiting body fits (or none is left: returns None);
        charges its peak bytes."""
        with self._cv:
            while True:
                if not self._wait:
                    return None
                for i, (key, peak) in enumerate(self._wait):
                    if self.in_use + peak <= self.budget:
                        del self._wait[i]
                        self.in_use += peak
                        self.high_water = max(self.high_water, self.in_use)
                        return key, peak
                self._cv.wait()

    def lower(self, nbytes: int):
        """Return nbytes of a body's charge (build scratch freed, or the body done)."""
        with self._cv:
            self.in_use -= int(nbytes)
            self._cv.notify_all()


def run_batch(bodies, budget_bytes: int, n_streams: int = 2, precision: int = 1, process=None,
              order: str = "largest_first"):
    """Build and solve every body (workloads.Config-like: curve, media, M,
    n_phi, waves) under budget_bytes of device memory with n_streams
    concurrent workers.  process(index, body, worker, admission, peak)
    overrides the per-body work and must lower the admission by the body's
    whole peak when done; the default builds, solves the body's plane waves
    and records the library's stage times and backward errors.  Returns (results in body
    order, wall seconds, admission)."""
    from . import build_bytes
    peaks = [build_bytes(b.curve.N, b.M, precision)[0] for b in bodies]
    idx = list(range(len(bodies)))
    if order == "largest_first":
        idx.sort(key=lambda i: -peaks[i])
    adm = Admission([(i, peaks[i]) for i in idx], budget_bytes)
    results = [None] * len(bodies)
    errors = []
    t0 = time.perf_counter()
    work = process or _default_process(precision)

    def worker(w):
        try:
            while True:
                item = adm.next()
                if item is None:
                    return
                i, peak = item
                r = work(i, bodies[i], w, adm, peak)
                r.worker = w
                r.t_start -= t0
                r.t_end -= t0
                results[i] = r
        except BaseException as e:  # surfaced to the caller below
            errors.append(e)
            with adm._cv:
                adm._wait.clear()
                adm._cv.notify_all()

    threads = [threading.Thread(target=worker, args=(w,), daemon=True) for w in range(n_streams)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    wall = time.perf_counter() - t0
    if errors:
        raise errors[0]
    return results, wall, adm


def _default_process(precision: int, check=None):
    def process(i, body, w, adm, peak):
        import torch
        from . import Options, build
        stream = torch.cuda.Stream()
        r = BodyResult(i, body.name, body.curve.N, body.M, peak_bytes=peak)
        r.t_start = time.perf_counter()
        with torch.cuda.stream(stream):
            ctx = build(body.curve, body.media, body.M, Options(n_phi=body.n_phi, precision=precision),
                        stream=stream)
            st = ctx.stats()
            r.resident_bytes = int(st["device_bytes"])
            adm.lower(peak - r.resident_bytes)           # build scratch and matrices freed
            n, nrhs = 4 * body.curve.N, len(body.waves)
            rhs = torch.zeros((2 * body.M + 1, nrhs, n), dtype=torch.complex128, device=stream.device)
            x = torch.zeros_like(rhs)
            be = np.zeros((2 * body.M + 1) * nrhs)
            ctx.rhs_planewave([wv.d for wv in body.waves], [wv.e for wv in body.waves], rhs, stream=stream)
            ctx.solve(rhs, x, backward_err=be, stream=stream)
            st = ctx.stats()
            if check is not None:
                r.extra = check(i, body, ctx, x, stream)
            stream.synchronize()
            ctx.close()
            del rhs, x
        adm.lower(r.resident_bytes)
        r.t_end = time.perf_counter()
        r.n_phi = int(st["n_phi_used"])
        r.build_ms, r.lu_ms, r.solve_ms = st["ms_build"], st["ms_lu"], st["ms_solve"]
        r.refine_iters, r.backward_err = int(st["refine_iters"]), float(be.max())
        r.launches = int(st["launches"]) + int(st["solve_launches"]) + 1
        return r
    return process


def make_process(precision: int = 1, check=None):
    """The default per-body work with an optional check(i, body, ctx, x,
    stream) -> dict run while the factors are resident."""
    return _default_process(precision, check)
