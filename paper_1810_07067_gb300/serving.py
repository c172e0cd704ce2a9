"""Serving: a request loop over a pool of bodies with device-resident factors.

Requests (a body of the pool, plane waves, an arrival time) come as a stream.
The factors of a body (its key) are built once and kept on the device in a
least-recently-used cache whose resident bytes stay within a budget (the
budget is charged with a build's peak while it runs, mueller_build_bytes).
A request for a key that is not resident starts its build on a separate CUDA
stream in a builder thread, while the serving thread keeps solving requests
of resident keys on its own stream.  With a host budget, an evicted key's
factors are moved to pinned host memory (mueller_ctx_spill) instead of being
destroyed, and a later miss on it copies them back (mueller_ctx_restore)
instead of building; with a checkpoint directory, every build is saved there
(mueller_ctx_save) and a miss on a key with a saved checkpoint loads it
(mueller_ctx_load), so a restarted server resumes without rebuilding.  Requests of one key that are waiting
together are solved as one batch of right-hand sides (continuous batching, up
to max_rhs columns); each request's far field is then evaluated on its grid
and copied to pinned host memory.  Latency is completion minus arrival.
"""
from __future__ import annotations

import threading
import time
from collections import OrderedDict, deque
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    id: int
    key: int                 # body index in the pool
    arrival: float           # seconds from the start of the run
    dirs: np.ndarray         # [nrhs, 3] unit propagation directions
    pols: np.ndarray         # [nrhs, 3] unit polarisations, orthogonal to dirs

    @property
    def nrhs(self) -> int:
        return len(self.dirs)


@dataclass
class Done:
    id: int
    key: int
    nrhs: int
    arrival: float
    start: float             # batch start
    end: float               # far field on the host
    hit: bool                # factors were resident at arrival
    batch: int
    batch_rhs: int

    @property
    def latency(self) -> float:
        return self.end - self.arrival


def poisson_requests(n_bodies, rate, duration, seed=5, zipf=1.1, max_rhs=256):
    """Poisson arrivals of the given mean rate for `duration` seconds; body
    index Zipf(zipf) over the pool (zipf = 0: uniform); nrhs ~ U{1..max_rhs};
    directions uniform on the sphere with a random orthogonal polarisation."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    if zipf > 0:
        w = 1.0 / np.arange(1, n_bodies + 1) ** zipf
        w /= w.sum()
    else:
        w = np.full(n_bodies, 1.0 / n_bodies)
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            return out
        key = int(rng.choice(n_bodies, p=w))
        k = int(rng.integers(1, max_rhs + 1))
        d = rng.standard_normal((k, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        p = np.cross(d, rng.standard_normal((k, 3)))
        p /= np.linalg.norm(p, axis=1, keepdims=True)
        out.append(Request(len(out), key, t, d, p))


@dataclass
class _Entry:
    ctx: object
    resident: int
    last_use: float = 0.0


@dataclass
class ServeStats:
    done: list = field(default_factory=list)
    unfinished: int = 0
    builds: int = 0
    restores: int = 0            # misses served from the host cache
    loads: int = 0               # misses served from a checkpoint file
    spills: int = 0              # evictions parked in host memory
    evictions: int = 0
    build_s: float = 0.0
    batches: int = 0
    budget: int = 0
    high_water: int = 0
    wall: float = 0.0


class Server:
    """pool: list of workloads.Config-like bodies (curve, media, M, n_phi)."""

    def __init__(self, pool, budget_bytes: int, precision: int = 1, max_rhs: int = 256,
                 grid=(180, 360), refine_tol: float = 1e-14, host_budget_bytes: int = 0,
                 checkpoint_dir: str | None = None):
        import torch
        from . import build_bytes
        self.pool = pool
        self.host_budget = int(host_budget_bytes)
        self.host_cache: OrderedDict[int, _Entry] = OrderedDict()   # spilled keys, least recently used first
        self.host_charged = 0
        self.checkpoint_dir = checkpoint_dir
        if checkpoint_dir:
            import os
            os.makedirs(checkpoint_dir, exist_ok=True)
        self.precision = precision
        self.max_rhs = max_rhs
        self.grid = grid
        self.refine_tol = refine_tol
        self.dev = torch.device("cuda", torch.cuda.current_device())
        self.serve_stream = torch.cuda.Stream()
        self.build_stream = torch.cuda.Stream()
        self.peaks = [build_bytes(b.curve.N, b.M, precision)[0] for b in pool]
        # serving buffers for the largest body: rhs, currents, far field, solve scratch
        nmax = max(4 * b.curve.N * (2 * b.M + 1) for b in pool)
        self.headroom = 16 * nmax * max_rhs * 8 + 48 * grid[0] * grid[1] * max_rhs
        self.budget = int(budget_bytes) - self.headroom
        if max(self.peaks) > self.budget:
            raise ValueError("the budget cannot hold the largest body's build beside the serving buffers")
        self.cache: OrderedDict[int, _Entry] = OrderedDict()
        self.charged = 0                  # resident factors + a running build's peak
        self.E_host = torch.empty((max_rhs, grid[0], grid[1], 3), dtype=torch.complex128, pin_memory=True)
        self._lock = threading.Lock()
        self._built = deque()             # (key, ctx or exception, seconds)
        self._building = None             # key being built
        self._charged_now = 0             # bytes charged for the running build / restore / load

    # ---------------------------------------------------------------- builds
    def _evict_for(self, nbytes, st, keep=()):
        """Evict least recently used keys (none with waiting requests) until
        nbytes fit; False if they cannot fit yet."""
        for key in list(self.cache.keys()):
            if self.charged + nbytes <= self.budget:
                break
            if key in keep:
                continue
            e = self.cache.pop(key)
            self.charged -= e.resident
            st.evictions += 1
            if self.host_budget > 0 and e.resident <= self.host_budget:
                while self.host_cache and self.host_charged + e.resident > self.host_budget:
                    _, old = self.host_cache.popitem(last=False)
                    old.ctx.close()
                    self.host_charged -= old.resident
                e.ctx.spill(stream=self.serve_stream)
                self.host_cache[key] = e
                self.host_charged += e.resident
                st.spills += 1
            else:
                e.ctx.close()
        return self.charged + nbytes <= self.budget

    def _checkpoint_path(self, key):
        """File of a key's checkpoint: named by a hash of everything the build depends on."""
        import hashlib
        import os
        b = self.pool[key]
        h = hashlib.sha1()
        for a in (b.curve.r, b.curve.z, b.curve.dr, b.curve.dz):
            h.update(np.ascontiguousarray(a, dtype=np.float64).tobytes())
        m = b.media
        h.update(repr((int(b.curve.n_panels), bool(getattr(b.curve, "closed", False)), float(m.omega),
                       complex(m.eps0), complex(m.mu0), complex(m.eps1), complex(m.mu1), int(b.M),
                       int(b.n_phi), self.precision, self.refine_tol)).encode())
        return os.path.join(self.checkpoint_dir, f"key{key}_{h.hexdigest()[:16]}.ctx")

    def _start_build(self, key, st, keep=()):
        """Make a key resident: restore it from the host cache, load its
        checkpoint, or build it; runs in a builder thread."""
        import os
        from . import Context, Options, build
        spilled = self.host_cache.pop(key, None)
        ckpt = self._checkpoint_path(key) if self.checkpoint_dir else None
        from_file = spilled is None and ckpt is not None and os.path.exists(ckpt)
        # a restore or a load needs the context's resident bytes; a build its peak
        need = spilled.resident if spilled is not None else self.peaks[key]
        if spilled is not None:
            self.host_charged -= spilled.resident
        if not self._evict_for(need, st, keep):
            if spilled is not None:                      # back to the host cache; retry later
                self.host_cache[key] = spilled
                self.host_charged += spilled.resident
            return False
        self.charged += need
        self._charged_now = need
        st.high_water = max(st.high_water, self.charged)
        self._building = key
        body = self.pool[key]

        def run():
            t = time.perf_counter()
            kind = "build"
            try:
                with self._torch().cuda.stream(self.build_stream):
                    if spilled is not None:
                        spilled.ctx.restore(stream=self.build_stream)
                        ctx, kind = spilled.ctx, "restore"
                    elif from_file:
                        ctx, kind = Context.load(ckpt, stream=self.build_stream), "load"
                    else:
                        ctx = build(body.curve, body.media, body.M,
                                    Options(n_phi=body.n_phi, precision=self.precision, refine_tol=self.refine_tol),
                                    stream=self.build_stream)
                        if ckpt is not None:
                            ctx.save(ckpt)
                res = ctx
            except BaseException as e:  # handed to the serving thread
                res = e
            with self._lock:
                self._built.append((key, res, time.perf_counter() - t, kind))

        threading.Thread(target=run, daemon=True).start()
        return True

    @staticmethod
    def _torch():
        import torch
        return torch

    def _collect_builds(self, now, st):
        with self._lock:
            items = list(self._built)
            self._built.clear()
        for key, res, secs, kind in items:
            self._building = None
            self.charged -= self._charged_now
            if isinstance(res, BaseException):
                raise res
            resident = int(res.stats()["device_bytes"])
            self.cache[key] = _Entry(res, resident, now)
            self.charged += resident
            if kind == "restore":
                st.restores += 1
            elif kind == "load":
                st.loads += 1
            else:
                st.builds += 1
            st.build_s += secs

    # ---------------------------------------------------------------- serving
    def _serve(self, key, reqs, t0, st):
        torch = self._torch()
        body = self.pool[key]
        e = self.cache[key]
        self.cache.move_to_end(key)
        start = time.perf_counter() - t0
        n, M = 4 * body.curve.N, body.M
        dirs = np.concatenate([r.dirs for r in reqs])
        pols = np.concatenate([r.pols for r in reqs])
        k = len(dirs)
        s = self.serve_stream
        with torch.cuda.stream(s):
            rhs = torch.zeros((2 * M + 1, k, n), dtype=torch.complex128, device=self.dev)
            x = torch.zeros_like(rhs)
            e.ctx.rhs_planewave(dirs, pols, rhs, stream=s)
            e.ctx.solve(rhs, x, stream=s)
            E = torch.empty((k, self.grid[0], self.grid[1], 3), dtype=torch.complex128, device=self.dev)
            e.ctx.far_field_grid(x, E, stream=s)           # one far-field pass for the whole batch
            self.E_host[:k].copy_(E, non_blocking=True)
            s.synchronize()
            end = time.perf_counter() - t0
            out, c0 = [], 0
            for r in reqs:
                out.append(self.E_host[c0:c0 + r.nrhs].clone() if self.keep_results else None)
                c0 += r.nrhs
                st.done.append(Done(r.id, key, r.nrhs, r.arrival, start, end, r.hit, st.batches, k))
        e.last_use = time.perf_counter() - t0
        st.batches += 1
        return out

    def run(self, requests, drain_limit: float = 120.0, keep_results: bool = False):
        """Serve the requests in real time (arrivals relative to the start);
        returns ServeStats (and the far fields by request id when keep_results)."""
        self.keep_results = keep_results
        reqs = sorted(requests, key=lambda r: r.arrival)
        st = ServeStats(budget=self.budget)
        pending: dict[int, deque] = {}
        results = {}
        i = 0
        t0 = time.perf_counter()
        t_last = reqs[-1].arrival if reqs else 0.0
        while True:
            now = time.perf_counter() - t0
            while i < len(reqs) and reqs[i].arrival <= now:
                r = reqs[i]
                r.hit = r.key in self.cache
                pending.setdefault(r.key, deque()).append(r)
                i += 1
            self._collect_builds(now, st)
            waiting = {k: q for k, q in pending.items() if q}
            if not waiting and i >= len(reqs):
                break
            if now > t_last + drain_limit:
                st.unfinished = sum(len(q) for q in waiting.values()) + (len(reqs) - i)
                break
            # a miss: start building the key whose oldest request waits longest
            if self._building is None:
                missing = [k for k in waiting if k not in self.cache]
                if missing:
                    k = min(missing, key=lambda k: waiting[k][0].arrival)
                    self._start_build(k, st, keep=set(waiting))
            # serve the resident key whose oldest request waits longest
            ready = [k for k in waiting if k in self.cache]
            if ready:
                k = min(ready, key=lambda k: waiting[k][0].arrival)
                q = waiting[k]
                batch, nr = [], 0
                while q and (not batch or nr + q[0].nrhs <= self.max_rhs):
                    nr += q[0].nrhs
                    batch.append(q.popleft())
                out = self._serve(k, batch, t0, st)
                if keep_results:
                    for r, E in zip(batch, out):
                        results[r.id] = E
                continue
            nxt = reqs[i].arrival - now if i < len(reqs) else 0.002
            time.sleep(min(max(nxt, 0.0), 0.002))
        if self._building is not None:           # let a build still running finish before returning
            while self._building is not None:
                time.sleep(0.01)
                self._collect_builds(time.perf_counter() - t0, st)
        st.wall = time.perf_counter() - t0
        st.high_water = max(st.high_water, self.charged)
        return (st, results) if keep_results else st

    def close(self):
        for e in list(self.cache.values()) + list(self.host_cache.values()):
            e.ctx.close()
        self.cache.clear()
        self.host_cache.clear()
        self.charged = 0
        self.host_charged = 0


def summarize(st: ServeStats, n_offered: int, duration: float) -> dict:
    lat = np.array([d.latency for d in st.done]) if st.done else np.zeros(1)
    nrhs = sum(d.nrhs for d in st.done)
    return {"requests_offered": n_offered, "requests_done": len(st.done), "unfinished": st.unfinished,
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "solves_per_s": nrhs / st.wall if st.wall else 0.0,
            "hit_rate": float(np.mean([d.hit for d in st.done])) if st.done else 0.0,
            "builds": st.builds, "restores_from_host": st.restores, "loads_from_checkpoint": st.loads,
            "spills_to_host": st.spills, "evictions": st.evictions, "batches": st.batches,
            "mean_batch_rhs": float(np.mean([d.batch_rhs for d in st.done])) if st.done else 0.0,
            "build_s_total": st.build_s, "wall_s": st.wall, "arrival_window_s": duration,
            "budget_gb": st.budget / 1e9, "high_water_gb": st.high_water / 1e9}
