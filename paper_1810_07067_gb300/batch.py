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

run_waves is the other schedule: bodies grouped into waves that fit the
budget, each wave built by one build_many call, so that all modes of all its
bodies are factored together in one graph-launched LU over a ragged table of
matrices (tile shapes from the library's autotuner).
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


def plan_waves(bodies, budget_bytes: int, precision: int = 1, max_bodies: int = 16):
    """Group the bodies into waves for build_many: largest first, each wave
    taking every later body (same n_phi request) whose addition keeps the
    wave's peak (build_many_bytes) within budget_bytes, up to max_bodies
    bodies and 65535 mode matrices.  Returns [(body indices, peak bytes)]."""
    from . import build_bytes, build_many_bytes
    peaks = [build_bytes(b.curve.N, b.M, precision)[0] for b in bodies]
    todo = sorted(range(len(bodies)), key=lambda i: -peaks[i])
    waves = []
    while todo:
        wave = [todo[0]]
        est = build_many_bytes([bodies[todo[0]].curve.N], [bodies[todo[0]].M], precision)
        if est > budget_bytes:
            raise ValueError(f"body {todo[0]} needs {est} bytes, above the budget of {budget_bytes}")
        for i in todo[1:]:
            if len(wave) >= max_bodies:
                break
            if bodies[i].n_phi != bodies[wave[0]].n_phi:
                continue
            cand = wave + [i]
            if sum(bodies[j].M + 1 for j in cand) > 65535:
                continue
            e = build_many_bytes([bodies[j].curve.N for j in cand], [bodies[j].M for j in cand], precision)
            if e <= budget_bytes:
                wave, est = cand, e
        todo = [i for i in todo if i not in wave]
        waves.append((wave, est))
    return waves


def run_waves(bodies, budget_bytes: int, precision: int = 1, check=None, max_bodies: int = 16, n_streams: int = 2,
              lu_tile: int = 0):
    """Build and solve every body in waves: plan_waves with budget_bytes /
    n_streams per wave (at least what the largest body needs alone), then
    n_streams worker threads, each on its own CUDA stream, take waves as
    their peaks fit the whole budget (Admission).  A wave is assembled body by
    body and all modes of all its bodies are factored in one graph-launched
    LU (build_many: one launch per kernel and step over the ragged set of
    matrices, column tiles from the autotuner unless lu_tile is set); its
    bodies are then solved in turn and released, so one wave's assembly
    overlaps another's factorization and solves.  Returns (results in body
    order, wall seconds, [(wave indices, peak bytes)], admission)."""
    from . import build_many_bytes
    single = max(build_many_bytes([b.curve.N], [b.M], precision) for b in bodies)
    plan = plan_waves(bodies, max(budget_bytes // max(n_streams, 1), single), precision, max_bodies)
    adm = Admission([(w, est) for w, (_, est) in enumerate(plan)], budget_bytes)
    results = [None] * len(bodies)
    errors = []
    t0 = time.perf_counter()

    def run_wave(w, wave, est):
        import torch
        from . import Options, build_many
        stream = torch.cuda.Stream()
        ts = time.perf_counter()
        with torch.cuda.stream(stream):
            ctxs = build_many([(bodies[i].curve, bodies[i].media, bodies[i].M) for i in wave],
                              Options(n_phi=bodies[wave[0]].n_phi, precision=precision, lu_tile=lu_tile),
                              stream=stream)
            for k, (i, ctx) in enumerate(zip(wave, ctxs)):
                body = bodies[i]
                r = BodyResult(i, body.name, body.curve.N, body.M, peak_bytes=est)
                r.t_start = ts - t0
                st = ctx.stats()
                r.resident_bytes = int(st["device_bytes"])
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
                r.t_end = time.perf_counter() - t0
                r.n_phi = int(st["n_phi_used"])
                r.build_ms, r.lu_ms, r.solve_ms = st["ms_build"] - st["ms_lu"], st["ms_lu"], st["ms_solve"]
                r.refine_iters, r.backward_err = int(st["refine_iters"]), float(be.max())
                # the wave's LU launches are counted once, with its first body
                r.launches = int(st["launches"]) - (0 if k == 0 else int(st["lu_launches"])) + \
                    int(st["solve_launches"]) + 1
                r.extra = dict(r.extra or {}, wave=w, wave_bodies=len(wave), lu_graph=int(st["lu_graph"]),
                               lu_tile_steps=st["lu_tile_steps"])
                results[i] = r

    def worker(wid):
        try:
            while True:
                item = adm.next()
                if item is None:
                    return
                w, est = item
                run_wave(w, plan[w][0], est)
                for i in plan[w][0]:
                    results[i].worker = wid
                adm.lower(est)
        except BaseException as e:  # surfaced to the caller below
            errors.append(e)
            with adm._cv:
                adm._wait.clear()
                adm._cv.notify_all()

    threads = [threading.Thread(target=worker, args=(k,), daemon=True) for k in range(max(n_streams, 1))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    wall = time.perf_counter() - t0
    if errors:
        raise errors[0]
    return results, wall, plan, adm


def make_process(precision: int = 1, check=None):
    """The default per-body work with an optional check(i, body, ctx, x,
    stream) -> dict run while the factors are resident."""
    return _default_process(precision, check)
