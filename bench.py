"""Benchmark: modal assemble + solve on one body of revolution per GPU.

One step = mueller_build (modal Green's functions, assembly and LU of modes
0..M) + mueller_rhs_planewave (modal incident data) + mueller_solve for all
plane waves of the workload.  Default workload: the smooth random body
r = sin t (1 + sum_{j<=6} a_j cos jt), z = -cos t, a_j ~ U(-0.08, 0.08) from
default_rng(1810), 64 panels (N = 1024 nodes, system 4096 x 4096 complex128
per mode), modes -128..128, 512 azimuthal samples, k0 = 10, k1 = 15, two
plane waves.  The headline value is the mixed path (complex64 LU + FP64
refinement); the FP64 path is timed beside it, and both are compared with
the oracle's stored solution of the same body (per-mode current errors and
the far field).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
       [--workload random|cylinder|sphere|small|batched|serving|tables]
Under torchrun each rank solves its own copy of the body (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)


def _log_dir() -> str:
    """Directory for the clock-sample CSV files (BENCH_LOG_DIR, else the temp dir)."""
    import tempfile
    d = os.environ.get("BENCH_LOG_DIR") or tempfile.gettempdir()
    os.makedirs(d, exist_ok=True)
    return d


import numpy as np  # noqa: E402

def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max(values, dist=None, device="cpu"):
    """Per-rank timings -> their maximum over all ranks (the job's time);
    identity on a single rank."""
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def job_throughput(n_ranks, step_s):
    """Bodies per second of the whole job: every rank solves its own body per
    step (weak scaling), the step lasting the slowest rank's time."""
    return n_ranks / step_s


def _clock_sampler(path):
    cmd = ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
           "--format=csv,noheader,nounits", "-lms", "200"]
    try:
        return subprocess.Popen(cmd, stdout=open(path, "w"), stderr=subprocess.DEVNULL)
    except Exception:
        return None


def _clock_summary(path, gpu_index):
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    try:
        for line in open(path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9 or f[0] != str(gpu_index):
                continue
            sm.append(float(f[1])); mx.append(float(f[2]))
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
    except Exception:
        pass
    if not sm:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons)}


def _workload(name):
    import workloads as W
    if name == "random":
        return W.config_random()
    if name == "cylinder":
        return W.config_cylinder(7)
    if name == "sphere":
        return W.config_sphere()
    if name == "small":
        return W.config_random(16, 1810, 32, 128)
    raise SystemExit(f"unknown workload {name}")


_ONE_THREAD = {"OMP_NUM_THREADS": "1", "OPENBLAS_NUM_THREADS": "1", "MKL_NUM_THREADS": "1"}


def _oracle_rows(args):
    """Worker: the oracle assembles the given target rows (all 2M+1 modes)."""
    name, rows = args
    from oracle import system
    cfg = _workload(name)
    geo = system.node_geometry(cfg.curve)
    t0 = time.perf_counter()
    for i in rows:
        system.assemble_row(cfg.curve, cfg.media, cfg.M, int(i), 0, None, geo)
    return time.perf_counter() - t0


def _oracle_lu_steps(args):
    """Worker: the first k elimination steps of the oracle's naive LU on a
    full-size matrix (the oracle's LU restarted on the leading steps only)."""
    n, k, seed = args
    from oracle import linalg
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) + n * np.eye(n)
    t0 = time.perf_counter()
    linalg.lu_factor(A, steps=k)
    return time.perf_counter() - t0


def _lu_fraction(n, k):
    """Share of the naive LU's work (sum over steps j of (n - j - 1)^2) in its first k steps."""
    j = np.arange(n, dtype=np.float64)
    w = (n - j - 1) ** 2
    return float(w[:k].sum() / w.sum())


class OracleBaseline:
    """The oracle (as it stands) on the host cores, on a bounded sample of the
    workload, projected to one step: every worker assembles `rows` target rows
    (all 2M+1 modes) and runs the first `lu_steps` steps of one full-size
    naive LU, all workers at once; the step is N rows and 2M+1 LUs spread over
    the same workers."""

    def __init__(self, name, cores=None):
        import multiprocessing as mp
        self.name = name
        self.cfg = _workload(name)
        self.cores = cores or os.cpu_count() or 1
        # one BLAS thread per process: the spawned workers import numpy before any
        # initializer runs, so the environment is set before they start
        saved = {k: os.environ.get(k) for k in _ONE_THREAD}
        os.environ.update(_ONE_THREAD)
        try:
            self.pool = mp.get_context("spawn").Pool(self.cores)
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        self.pool.map(_oracle_rows, [(name, []) for _ in range(self.cores)])   # imports done before timing

    def sample(self, budget_s):
        cfg, P = self.cfg, self.cores
        N, M, n = cfg.N, cfg.M, 4 * cfg.N
        rows = np.linspace(0, N - 1, P).astype(int)
        # workers run at once; the slowest one's compute time is the sample's wall time
        t_row = max(self.pool.map(_oracle_rows, [(self.name, [int(r)]) for r in rows]))
        if getattr(self, "k", None) is None:            # elimination steps that fill about half the budget
            t8 = max(self.pool.map(_oracle_lu_steps, [(n, 8, s) for s in range(P)]))
            self.k = int(max(8, min(n, 8 * 0.5 * budget_s / max(t8, 1e-3))))
        k = self.k
        t_lu = max(self.pool.map(_oracle_lu_steps, [(n, k, s) for s in range(P)]))
        frac = _lu_fraction(n, k)
        value = t_row * N / P + (t_lu / frac) * (2 * M + 1) / P
        sample = (f"projection from a sample: {P} host processes each assembled 1 of {N} target rows (all "
                  f"{2 * M + 1} modes; {t_row:.2f} s wall) and ran the first {k} of {n} steps of the naive LU of "
                  f"a {n}x{n} matrix ({t_lu:.2f} s wall, {100 * frac:.2f}% of its work); step = {N} rows + "
                  f"{2 * M + 1} LUs over {P} processes")
        return value, sample

    def close(self):
        self.pool.terminate()
        self.pool.join()


def run_reference(args, cfg):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    ob = OracleBaseline(args.workload)
    budget = max(2.0, min(25.0, 150.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        ob.sample(budget)
    vals = []
    sample = ""
    for _ in range(max(1, args.steps)):
        v, sample = ob.sample(budget)
        vals.append(v)
    ob.close()
    value = statistics.mean(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "s", "n_gpus": args.gpus,
            "steps": len(vals), "warmup": args.warmup, "ms_per_step": value * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "config": _config(cfg),
            "cpu_baseline": {"value": value, "unit": "s", "cores": ob.cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


METRIC = ("modal assemble+solve time (mueller_build + mueller_solve) at backward error <= 1e-14: "
          "mixed path (complex64 LU + FP64 refinement); FP64 GPU path beside it")


def _config(cfg):
    if cfg.name.startswith("cylinder"):
        body = "finite cylinder R=1 H=2, edge-graded panels"
    elif cfg.name.startswith("sphere"):
        body = "dielectric unit sphere"
    else:
        body = "smooth random body r = sin t (1 + sum_{j<=6} a_j cos jt), a_j ~ U(-0.08, 0.08)"
    k0 = cfg.media.omega
    k1 = k0 * complex(cfg.media.eps1) ** 0.5
    fb = 16 * (4 * cfg.N) ** 2 * (cfg.M + 1) / 1e9
    return {"workload": f"{cfg.name}: {body}, N={cfg.N} nodes (system {4 * cfg.N}x{4 * cfg.N} c128 per mode), "
                        f"modes -{cfg.M}..{cfg.M}, n_phi={cfg.n_phi}, k0={k0:g}, k1={k1:.4g}, "
                        f"{len(cfg.waves)} plane waves",
            "precision": "mixed", "l2_flush": f"inputs larger than L2 ({fb:.2g} GB of matrices per step)"}


def _golden(cfg, name):
    """The oracle's stored full-size solution of this workload (written by
    tests/golden/make_fullsize.py), if it exists and describes the same body."""
    path = os.path.join(ROOT, "tests", "golden", f"fullsize_{name}.npz")
    if not os.path.exists(path):
        return None
    g = np.load(path)
    if g["r"].shape != cfg.curve.r.shape or int(g["M"]) != cfg.M:
        return None
    if max(np.abs(g["r"] - cfg.curve.r).max(), np.abs(g["z"] - cfg.curve.z).max()) > 1e-13:
        return None
    return g


def _errors_vs_oracle(ctx, x, g, M, dev):
    """Against the oracle's stored solution: per stored mode, the relative l2
    error of the solutions of two seeded random right-hand sides (full-size
    solutions in every mode) and of the plane-wave currents normalised by the
    largest mode's currents; the relative l2 error of the far field of the
    stored modes' plane-wave currents at the stored directions."""
    import torch
    modes, waves = [int(m) for m in g["modes"]], [int(w) for w in g["waves"]]
    xg = x.cpu().numpy()
    top = max(np.linalg.norm(g["x"][qi, wi]) for qi in range(len(modes)) for wi in range(len(waves)))
    pw = {str(m): float(max(np.linalg.norm(xg[m + M, w] - g["x"][qi, wi]) / top for wi, w in enumerate(waves)))
          for qi, m in enumerate(modes)}
    n = x.shape[2]
    per_mode = {}
    if "b_rand" in g.files:
        br = torch.zeros((2 * M + 1, 2, n), dtype=torch.complex128, device=dev)
        for qi, m in enumerate(modes):
            br[m + M] = torch.tensor(g["b_rand"][qi], device=dev)
        xr = torch.zeros_like(br)
        ctx.solve(br, xr)
        xr = xr.cpu().numpy()
        per_mode = {str(m): float(max(np.linalg.norm(xr[m + M, c] - g["x_rand"][qi, c]) /
                                      np.linalg.norm(g["x_rand"][qi, c]) for c in range(2)))
                    for qi, m in enumerate(modes)}
    keep = torch.zeros_like(x)
    for m in [int(v) for v in g["solved_modes"]]:
        keep[m + M] = x[m + M]
    dirs = torch.tensor(g["ff_dirs"], device=dev)
    E = torch.zeros((x.shape[1], len(dirs), 3), dtype=torch.complex128, device=dev)
    ctx.far_field(keep, dirs, E)
    Eg = E.cpu().numpy()
    ff = float(np.linalg.norm(Eg - g["ff"]) / np.linalg.norm(g["ff"]))
    return {"currents_rel_l2_per_mode": per_mode, "currents_rel_l2_max": max(per_mode.values(), default=None),
            "currents_rel_l2_per_mode_kind": "solutions of 2 seeded random right-hand sides per mode",
            "planewave_currents_err_per_mode_over_largest_mode": pw,
            "far_field_rel_l2": ff,
            "far_field_modes": "all" if len(g["solved_modes"]) == 2 * M + 1 else
            [int(v) for v in g["solved_modes"]]}


def _kernel_rooflines(st, M, N, fp64_peak, hbm_peak):
    """Per kernel: device time (ms) from the build's CUDA events and the
    algorithmic work it stands for.

    FP64 stages (kernel evaluation and assembly), per pair:
      far_kernel      9 FFT-class transforms 9 * 2.5 n log2 n, sampling
                      (n/2 + 1) * 140 flops (both wavenumbers), assembly
                      256 flops per mode, n = n_phi;
      support_stage   the same without assembly, plus 6 convolution
                      transforms 6 * 2.5 n log2 n for split pairs (the
                      stage samples on the FP64 pipe and runs the transform
                      as digit products on the tensor cores: the count is
                      the paper's method over the stage's time);
      near_kernel     the rule contraction, 4 flops per (support point,
                      column, family x weight, mode), and 16 x 3 blocks of
                      256 flops per mode for every target;
      legendre_kernel 10 flops per recurrence step, n/2 steps per split pair.
    LU trailing update (mixed path): read + write of the trailing complex64
    matrix per step, 16 bytes per entry (HBM bound)."""
    nphi = st["n_phi_used"]
    fft = 2.5 * nphi * math.log2(nphi)
    samp = (nphi // 2 + 1) * 140
    out = {}
    far = st["n_far_pairs"] * (9 * fft + samp + 256 * (M + 1))
    # the far pairs: one fused kernel, or (tensor-core transform) sampling,
    # digit products and assembly kernels, timed apart
    far_split = st.get("ms_far_assemble", 0) > 0
    out["far_stage" if far_split else "far_kernel"] = (st["ms_far"], far, "alu")
    n_split = st["n_split_pairs"]
    sup = st["n_support_pairs"] * (9 * fft + samp) + 6 * fft * min(n_split, st["n_support_pairs"])
    out["support_stage"] = (st["ms_support"], sup, "alu")
    near = st["n_support_pairs"] * 16 * 27 * 4 * (M + 2) + N * 48 * (M + 1) * 256
    out["near_kernel"] = (st["ms_near"], near, "alu")
    out["legendre_kernel"] = (st["ms_legendre"], n_split * 10 * (nphi // 2), "alu")
    res = {}
    for k, (ms, work, bound) in out.items():
        if ms <= 0:
            continue
        ach = work / (ms * 1e-3) / 1e12
        res[k] = {"ms": ms, "bound": bound, "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s",
                  "frac": ach / fp64_peak, "algorithmic_flops": work}
    if far_split:
        # far_assemble_kernel: the matrix entries of every far pair's blocks, modes 0..M, 256 bytes each
        fb = st["n_far_pairs"] * (M + 1) * 256.0
        ach = fb / (st["ms_far_assemble"] * 1e-3) / 1e9
        res["far_assemble_kernel"] = {"ms": st["ms_far_assemble"], "bound": "hbm", "achieved": ach,
                                      "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak,
                                      "algorithmic_bytes": fb,
                                      "note": "FP64-bound in practice: the 4 x 4 block of every mode"}
        res["far_sample_kernel"] = {"ms": st["ms_far_sample"], "bound": "alu",
                                    "note": "far-pair samples on their ladder grids and their digit rows"}
        res["oz_real_gemm_kernel (far)"] = {"ms": st["ms_far_product"], "bound": "tensor",
                                            "note": "the far pairs' transforms as digit products"}
    if st.get("ms_lu_gemm", 0) > 0 and st.get("lu_gemm_bytes", 0) > 0:
        ach = st["lu_gemm_bytes"] / (st["ms_lu_gemm"] * 1e-3) / 1e9
        res["gemm_update_tc_kernel"] = {"ms": st["ms_lu_gemm"], "bound": "hbm", "achieved": ach,
                                        "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak,
                                        "algorithmic_bytes": st["lu_gemm_bytes"]}
    return res


def run_batched(args):
    """The batched workload: every body of workloads.config_batch() built and
    solved (mixed path, both plane waves) once, under a device-memory budget:
    in waves (default; each wave built by build_many, all its modes factored
    in one graph-launched LU with autotuned tiles) or one body per stream on
    args.streams concurrent streams.  Warm-up: the args.warmup smallest
    bodies, untimed.  value = wall time of the whole batch (host clock around
    the pass, device synchronised on both sides)."""
    import torch
    import workloads as W
    import paper_1810_07067_gb300 as mb
    from paper_1810_07067_gb300 import batch
    if args.impl == "reference":
        print(json.dumps({"impl": "reference", "unavailable": "the batched workload has no oracle timing "
                          "(the oracle is timed on the cylinder workload)"}))
        return
    bodies = W.config_batch()
    if args.bodies:
        bodies = bodies[:args.bodies]
    mb.cache_limit(0)                                   # bodies of distinct sizes: nothing to reuse, keep the budget whole
    free, total = torch.cuda.mem_get_info()
    budget = int(args.budget_gb * 1e9) if args.budget_gb > 0 else int(0.9 * free)
    small = sorted(bodies, key=lambda c: mb.build_bytes(c.N, c.M, 1)[0])[:max(args.warmup, 0)]

    def one_pass(group):
        if args.schedule == "waves":
            res, wall, plan, adm = batch.run_waves(group, budget, n_streams=args.streams)
            return res, wall, adm.high_water, len(plan)
        res, wall, adm = batch.run_batch(group, budget, n_streams=args.streams)
        return res, wall, adm.high_water, None

    one_pass(small)
    torch.cuda.synchronize()
    clk_path = os.path.join(_log_dir(),
                            "clocks_batched.csv")
    sampler = _clock_sampler(clk_path)
    time.sleep(0.3)
    walls = []
    for _ in range(max(args.steps, 1)):
        torch.cuda.synchronize()
        res, wall, high_water, n_waves = one_pass(bodies)
        torch.cuda.synchronize()
        walls.append(wall)
    if sampler:
        sampler.terminate()
        sampler.wait()
    wall = statistics.median(walls)
    nrhs = sum(len(c.waves) * (2 * c.M + 1) for c in bodies)
    line = {"metric": "batched: wall time to build (mixed) and solve every body of the batch under a memory budget",
            "value": wall, "unit": "s", "n_gpus": 1, "steps": len(walls), "warmup": len(small),
            "ms_per_step": wall * 1e3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "c64 factors + c128 refinement", "data": "synthetic",
            "config": {"workload": f"{len(bodies)} bodies of workloads.config_batch (random smooth bodies, "
                                   f"cylinders, cones; N {min(c.N for c in bodies)}..{max(c.N for c in bodies)}, "
                                   f"M {min(c.M for c in bodies)}..{max(c.M for c in bodies)}, k1 = 1.5 k0)",
                       "schedule": args.schedule, "streams": args.streams,
                       "waves": n_waves, "budget_gb": budget / 1e9,
                       "l2_flush": "inputs larger than L2 (every body's matrices)"},
            "bodies_per_s": len(bodies) / wall,
            "modal_solves_per_s": nrhs / wall,
            "resident_tb_total": sum(r.resident_bytes for r in res) / 1e12,
            "budget_high_water_gb": high_water / 1e9,
            "sum_assembly_s": (sum(r.build_ms for r in res) if args.schedule == "waves"
                               else sum(r.build_ms - r.lu_ms for r in res)) / 1e3,
            "sum_lu_s": (sum({r.extra.get("wave", i): r.lu_ms for i, r in enumerate(res)}.values())
                         if args.schedule == "waves" else sum(r.lu_ms for r in res)) / 1e3,
            "sum_solve_s": sum(r.solve_ms for r in res) / 1e3,
            "backward_err_max": max(r.backward_err for r in res),
            "refine_iters_max": max(r.refine_iters for r in res),
            "largest_body": max(((r.N, r.M) for r in res)),
            "gpu_launches": sum(r.launches for r in res) * len(walls),
            "clocks": _clock_summary(clk_path, 0)}
    print(json.dumps(line), flush=True)


def run_serving(args):
    """The serving workload: Poisson arrivals (default_rng(5)) at args.rate
    per second for args.duration seconds over the 32-body pool
    (workloads.config_pool), body choice Zipf(args.zipf), nrhs ~ U{1..max_rhs},
    far field on the 180 x 360 (polar x azimuth) grid per request, factors
    cached on the device under the memory budget.  Warm-up: args.warmup
    requests on the smallest body, untimed.  value = p99 latency."""
    import torch
    import workloads as W
    import paper_1810_07067_gb300 as mb
    from paper_1810_07067_gb300 import serving
    if args.impl == "reference":
        print(json.dumps({"impl": "reference", "unavailable": "the serving workload has no oracle timing "
                          "(the oracle is timed on the cylinder workload)"}))
        return
    pool = W.config_pool(32)
    mb.cache_limit(0)                                   # the admission budget accounts for every device byte
    free, _ = torch.cuda.mem_get_info()
    budget = int(args.budget_gb * 1e9) if args.budget_gb > 0 else int(0.9 * free)
    srv = serving.Server(pool, budget, precision=1, max_rhs=args.max_rhs, grid=(180, 360),
                         host_budget_bytes=int(args.host_budget_gb * 1e9))
    smallest = min(range(len(pool)), key=lambda k: srv.peaks[k])
    warm = [serving.Request(i, smallest, 0.0, np.array([[0.0, 0.0, 1.0]]), np.array([[1.0, 0.0, 0.0]]))
            for i in range(max(args.warmup, 1))]
    srv.run(warm)
    srv.close()
    reqs = serving.poisson_requests(len(pool), args.rate, args.duration, seed=5, zipf=args.zipf,
                                    max_rhs=args.max_rhs)
    clk_path = os.path.join(_log_dir(),
                            "clocks_serving.csv")
    sampler = _clock_sampler(clk_path)
    torch.cuda.synchronize()
    st = srv.run(reqs, drain_limit=args.drain)
    torch.cuda.synchronize()
    if sampler:
        sampler.terminate()
        sampler.wait()
    summ = serving.summarize(st, len(reqs), args.duration)
    line = {"metric": "serving: p99 latency (arrival to far field on the host) of a Poisson request stream",
            "value": summ["p99_latency_s"], "unit": "s", "n_gpus": 1, "steps": 1, "warmup": len(warm),
            "ms_per_step": st.wall * 1e3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "c64 factors + c128 refinement", "data": "synthetic",
            "config": {"workload": f"serving: 32-body pool (workloads.config_pool: random bodies N=1024, "
                                   f"modes -128..128, k0=10, k1=15), Poisson {args.rate:g}/s for "
                                   f"{args.duration:g} s, Zipf({args.zipf:g}) bodies, nrhs U{{1..{args.max_rhs}}}, "
                                   f"far field 180x360 per request", "budget_gb": budget / 1e9,
                       "l2_flush": "inputs larger than L2 (factors of every key)"},
            "serving": summ, "clocks": _clock_summary(clk_path, 0)}
    srv.close()
    print(json.dumps(line), flush=True)


def run_tables(args):
    """The paper's four numerical examples (Section 6, Tables 1-4): for every
    row, the body with the row's N_pts nodes and modes -N_f..N_f, the
    extinction test of eq. loop on the indirect formulation (mixed path),
    E_error = relative l2 error of E and H at random interior points, the
    build and solve times, and one more solve with a single right-hand side
    (the paper's T_add).  The paper's printed times (its CPU) and errors are
    context.  value = summed build + solve time over all rows."""
    import torch
    import workloads as W  # noqa: F401
    import paper_1810_07067_gb300 as mb
    from workloads import paper_tables as T
    from workloads.sources import current_loop_field, ring_points
    if args.impl == "reference":
        print(json.dumps({"impl": "reference", "unavailable": "the paper-table workload has no oracle timing"}))
        return
    dev = torch.device("cuda", 0)
    rows_out = []
    for ex, rows in T.EXAMPLES.items():
        for row in rows:
            cfg = T.config(ex, row)
            media, M, N = cfg.media, cfg.M, cfg.N
            k1 = media.omega * np.sqrt(complex(media.eps1) * complex(media.mu1))
            rmax = float(np.max(cfg.curve.r))
            nth = 2 * M + 2 * int(np.ceil(abs(k1) * rmax)) + 64
            pts = ring_points(cfg.curve.r, cfg.curve.z, nth)
            E, H = current_loop_field(pts.reshape(-1, 3), k1, media.omega, complex(media.mu1))
            EH = torch.tensor(np.concatenate([E, H], -1).reshape(1, N, nth, 6), device=dev)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx = mb.build(cfg.curve, media, M, mb.Options(n_phi=16, formulation=1, precision=1))
            rhs = torch.zeros((2 * M + 1, 1, 4 * N), dtype=torch.complex128, device=dev)
            ctx.rhs_fields(EH, rhs)
            x = torch.zeros_like(rhs)
            ctx.solve(rhs, x)
            torch.cuda.synchronize()
            t_total = time.perf_counter() - t0
            st = ctx.stats()
            t1 = time.perf_counter()
            x2 = torch.zeros_like(rhs)
            ctx.solve(rhs, x2)
            torch.cuda.synchronize()
            t_add = time.perf_counter() - t1
            P = T.interior_points(ex)
            out = torch.zeros((1, len(P), 6), dtype=torch.complex128, device=dev)
            ctx.eval(x, P, 1, out)
            Er, Hr = current_loop_field(P, k1, media.omega, complex(media.mu1))
            ref = np.concatenate([Er, Hr], -1)
            got = out.cpu().numpy()[0]
            err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
            ctx.close()
            rows_out.append({"example": ex, "k0": row[0], "k1": row[1], "N_f": row[2], "N_pts": row[3],
                             "n_phi": int(st["n_phi_used"]), "build_s": st["ms_build"] / 1e3,
                             "total_s": t_total, "add_s": t_add, "E_error": err,
                             "paper": {"T_kernel+T_matgen+T_solve": row[4] + row[5] + row[6], "T_add": row[7],
                                       "E_error": row[8]}})
            print(json.dumps(rows_out[-1]), file=sys.stderr, flush=True)
    tot = sum(r["total_s"] for r in rows_out)
    line = {"metric": "paper's four examples (Tables 1-4): extinction-test error and build+solve time per row",
            "value": tot, "unit": "s", "n_gpus": 1, "steps": 1, "warmup": 0, "ms_per_step": tot * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "c64 factors + c128 refinement", "data": "synthetic",
            "config": {"workload": "torus, rotated starfish, droplet, cylinder at the rows of Tables 1-4; "
                                   "current loop (0.4, 0.5, 5.0), radius 0.42; indirect formulation"},
            "rows_E_error_le_paper": sum(r["E_error"] <= r["paper"]["E_error"] for r in rows_out),
            "rows": rows_out}
    print(json.dumps(line), flush=True)


def run_single(args, cfg):
    """One body per rank: build (assembly + LU of modes 0..M) + plane-wave
    data + solve of all waves, mixed path timed over args.steps steps (the
    headline value), the FP64 path over args.fp64_steps steps beside it."""
    import torch
    import paper_1810_07067_gb300 as mb
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    # the oracle's worker pool starts (spawn) before the first GPU call
    ob = OracleBaseline(args.workload) if (ws == 1 and not args.no_cpu_baseline) else None
    stream = torch.cuda.current_stream(dev)
    M, n = cfg.M, 4 * cfg.N
    nrhs = len(cfg.waves)
    dirs = np.array([w.d for w in cfg.waves]); pols = np.array([w.e for w in cfg.waves])
    opts = {1: mb.Options(n_phi=cfg.n_phi, precision=1, refine_tol=1e-14),
            0: mb.Options(n_phi=cfg.n_phi, precision=0)}
    rhs = torch.zeros((2 * M + 1, nrhs, n), dtype=torch.complex128, device=dev)
    x = torch.zeros_like(rhs)
    # The library's cache of freed device blocks (mueller_cache_limit) is
    # raised to hold one build's buffers, so that repeated builds of the body
    # reuse their device memory, as a long-running process would, instead of
    # returning the 35 GB matrices and 69 GB digit slices to the driver and
    # mapping them again every step.
    peak_bytes, _ = mb.build_bytes(cfg.N, M, 1)
    cache_cap = max(int(1.1 * peak_bytes), 32 << 30)
    old_cap = mb.cache_limit(cache_cap)
    if old_cap > cache_cap:
        mb.cache_limit(old_cap)
        cache_cap = old_cap

    def step(prec, out=x, keep=False):
        ctx = mb.build(cfg.curve, cfg.media, M, opts[prec])
        ctx.rhs_planewave(dirs, pols, rhs)
        ctx.solve(rhs, out)
        st = ctx.stats()
        if keep:
            return st, ctx
        ctx.close()
        return st

    fp64_peak = mb.fp64_peak()
    for _ in range(args.warmup):
        step(1)
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    clk_path = os.path.join(_log_dir(), f"clocks_rank{rank}.csv")
    sampler = _clock_sampler(clk_path)
    time.sleep(0.3)
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed_step")            # lets a profiler select the timed launches
    e0.record(stream)
    stats = [step(1) for _ in range(args.steps)]
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    dev_s = e0.elapsed_time(e1) / 1e3 / args.steps
    # end to end through the public API from host inputs: build from host
    # curve arrays, plane-wave data from host directions, currents back to pinned host memory
    x_host = torch.empty((2 * M + 1, nrhs, n), dtype=torch.complex128, pin_memory=True)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx = mb.build(cfg.curve, cfg.media, M, opts[1])
        ctx.rhs_planewave(dirs, pols, rhs)
        ctx.solve(rhs, x)
        x_host.copy_(x, non_blocking=True)
        torch.cuda.synchronize(dev)
        ctx.close()
    e2e_s = (time.perf_counter() - t0) / args.steps
    # the FP64 path on the same inputs: one untimed warm-up, then fp64_steps timed steps
    x64 = torch.zeros_like(x)
    fp64 = None
    if args.fp64_steps > 0:
        step(0, x64)
        torch.cuda.synchronize(dev)
        ev0 = torch.cuda.Event(enable_timing=True); ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        st64 = [step(0, x64) for _ in range(args.fp64_steps)]
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        fp64 = {"s": ev0.elapsed_time(ev1) / 1e3 / args.fp64_steps, "steps": args.fp64_steps, "warmup": 1,
                "stages_ms": {k: round(st64[-1][k], 3) for k in
                              ("ms_legendre", "ms_far", "ms_support", "ms_near", "ms_lu", "ms_lu_gemm", "ms_solve")},
                "lu_trailing_update_tflops": st64[-1]["lu_gemm_flops"] / (st64[-1]["ms_lu_gemm"] * 1e-3) / 1e12
                if st64[-1]["ms_lu_gemm"] > 0 else None}
    if sampler:
        sampler.terminate()
        sampler.wait()
    clocks = _clock_summary(clk_path, local)
    # accuracy, untimed: both paths against the oracle's stored solution
    accuracy = None
    cond = None
    g = _golden(cfg, args.workload)
    if g is not None:
        accuracy = {}
        for prec, name in ((1, "mixed"), (0, "fp64")):
            if prec == 0 and args.fp64_steps <= 0:
                continue
            xx = torch.zeros_like(x)
            _, ctx = step(prec, xx, keep=True)
            accuracy[name] = _errors_vs_oracle(ctx, xx, g, M, dev)
            if prec == 1:
                kap = ctx.cond_estimate()
                cond = {"kappa_inf_mode0": float(kap[0]), "kappa_inf_max": float(kap.max()),
                        "mode_of_max": int(kap.argmax()), "ms": ctx.stats()["ms_cond"],
                        "kind": "Hager estimate of ||A'^-1||_inf from the complex64 factors x ||A'||_inf, "
                                "per mode (mueller_cond_estimate)"}
            ctx.close()
        accuracy["oracle"] = {"modes": [int(v) for v in g["modes"]], "waves": [int(v) for v in g["waves"]],
                              "kappa1_per_mode": ([float(v) for v in g["kappa1"]] if "kappa1" in g.files else None),
                              "noise1_per_mode": ([float(v) for v in g["noise1"]] if "noise1" in g.files else None),
                              "noise1_meaning": "relative 1-norm difference of the oracle's 32- and 24-point "
                                                "matrices (its own rounding noise)",
                              "solved_modes": len(g["solved_modes"]),
                              "oracle_backward_err_max": float(np.max(g["backward_err"])),
                              "source": "tests/golden/fullsize_%s.npz (oracle only)" % args.workload}
    if cond is None:                                    # no stored oracle solution: estimate on its own
        _, ctx = step(1, torch.zeros_like(x), keep=True)
        kap = ctx.cond_estimate()
        cond = {"kappa_inf_mode0": float(kap[0]), "kappa_inf_max": float(kap.max()), "mode_of_max": int(kap.argmax()),
                "ms": ctx.stats()["ms_cond"],
                "kind": "Hager estimate of ||A'^-1||_inf from the complex64 factors x ||A'||_inf, per mode "
                        "(mueller_cond_estimate)"}
        ctx.close()
    num = den = None
    if fp64 is not None:
        num = max(float((x[q] - x64[q]).norm()) for q in range(2 * M + 1))
        den = max(float(x64[q].norm()) for q in range(2 * M + 1))
    dev_s, e2e_s = reduce_max([dev_s, e2e_s], dist, dev)
    if rank == 0:
        st = stats[-1]
        launches = st["launches"] + st["solve_launches"] + 1  # + rhs_kernel
        hbm = _measured_peaks().get("hbm_gbs", 6790.3)
        kr = _kernel_rooflines(st, M, cfg.N, fp64_peak, hbm)
        # the dominant kernel: the longest single kernel with an algorithmic count (stages excluded)
        top = max((k for k in kr if not k.endswith("_stage") and "frac" in kr[k]), key=lambda k: kr[k]["ms"])
        roof = dict(kr[top], kernel=top)
        roof["peak_source"] = ("measured live: DFMA register loop (mueller_fp64_peak)" if roof["bound"] == "alu"
                               else "MEASURED_PEAKS.json hbm_gbs")
        roof["traffic"] = None
        roof["traffic_note"] = "per-launch DRAM bytes: profiles/ (ncu captures of this kernel)"
        h2d = 8 * 4 * cfg.N + 8 * 6 * nrhs
        d2h = 16 * (2 * M + 1) * nrhs * n
        line = {"metric": METRIC, "value": dev_s, "unit": "s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": dev_s * 1e3, "higher_is_better": False,
                "scaling": "weak", "vs_baseline": None, "dtype": "c64 LU + c128 (fp64) refinement", "data": "synthetic",
                "config": _config(cfg),
                "device_block_cache": f"{cache_cap / 2**30:.0f} GiB cap: the next build reuses one build's "
                                      "device buffers (steady state of repeated builds)",
                "bodies_per_s": job_throughput(ws, dev_s),
                "stages_ms": {k: round(st[k], 3) for k in ("ms_legendre", "ms_far", "ms_support", "ms_near",
                                                           "ms_lu", "ms_lu_gemm", "ms_solve")},
                "roofline": roof,
                "kernels": kr,
                "fp64_peak_tflops_measured": fp64_peak,
                "lu_trailing_update": {"tflops": st["lu_gemm_flops"] / (st["ms_lu_gemm"] * 1e-3) / 1e12
                                       if st["ms_lu_gemm"] > 0 else None,
                                       "ms": st["ms_lu_gemm"],
                                       "arith": "complex64 as exact 3-piece split BF16 on tcgen05, FP32 accumulation",
                                       "tile_steps_32_64_128": st["lu_tile_steps"]},
                "refine_iters": st["refine_iters"], "backward_err_max": st["backward_err_max"],
                "tensor_core_residual": ({"ms": st["ms_residual"], "launches": st["residual_launches"],
                                          "bf16_tflops": st["residual_tc_flops"] / (st["ms_residual"] * 1e-3) / 1e12,
                                          "peak_bf16_tflops": _measured_peaks().get("bf16_tflops", 1872.0),
                                          "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst)"}
                                         if st["ms_residual"] > 0 else None),
                "fp64_path": fp64,
                "mixed_over_fp64_speedup": (fp64["s"] / dev_s) if fp64 else None,
                "currents_rel_diff_mixed_vs_fp64": (num / den) if num is not None else None,
                "accuracy_vs_oracle": accuracy,
                "condition_estimate": cond,
                "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
                "gpu_launches": launches * args.steps,
                "clocks": clocks}
        if ob is not None:
            v, sample = ob.sample(20.0)
            line["cpu_baseline"] = {"value": v, "unit": "s", "cores": ob.cores, "kind": "oracle", "sample": sample}
        print(json.dumps(line), flush=True)
    if ob is not None:
        ob.close()
    if dist:
        dist.destroy_process_group()


def _measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--fp64-steps", type=int, default=2,
                    help="timed steps of the FP64 path beside the mixed headline (after one warm-up; 0 = skip)")
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="random",
                    choices=["random", "cylinder", "sphere", "small", "batched", "serving", "tables"],
                    help="random: smooth random body N=1024, M=128, n_phi=512, k0=10, k1=15 (default); "
                         "cylinder: edge-graded cylinder N=576, M=64; sphere: N=64, M=10; small: random body "
                         "N=256, M=32 (profiling captures); batched: the 72-body batch under a memory budget; "
                         "serving: Poisson request stream with a factor cache; tables: the paper's four examples")
    ap.add_argument("--bodies", type=int, default=0, help="batched: only the first K bodies (0 = all)")
    ap.add_argument("--streams", type=int, default=2, help="batched: concurrent bodies (CUDA streams)")
    ap.add_argument("--schedule", default="waves", choices=["waves", "streams"],
                    help="batched: waves = bodies grouped under the budget, each wave's modes factored in one "
                         "graph-launched LU (build_many); streams = one body per concurrent stream")
    ap.add_argument("--rate", type=float, default=200.0, help="serving: mean arrivals per second")
    ap.add_argument("--duration", type=float, default=10.0, help="serving: arrival window in seconds")
    ap.add_argument("--zipf", type=float, default=1.1, help="serving: body choice Zipf exponent (0 = uniform)")
    ap.add_argument("--max-rhs", type=int, default=256, help="serving: right-hand sides per request at most")
    ap.add_argument("--drain", type=float, default=120.0, help="serving: seconds after the last arrival to finish")
    ap.add_argument("--host-budget-gb", type=float, default=0.0,
                    help="serving: pinned host memory for factors evicted from the device (0 = none)")
    ap.add_argument("--budget-gb", type=float, default=0.0,
                    help="batched/serving: device-memory budget (0 = 90%% of the free memory)")
    args = ap.parse_args()
    if args.workload == "batched":
        run_batched(args)
        return
    if args.workload == "serving":
        run_serving(args)
        return
    if args.workload == "tables":
        run_tables(args)
        return
    cfg = _workload(args.workload)
    if args.impl == "reference":
        run_reference(args, cfg)
        return
    run_single(args, cfg)


if __name__ == "__main__":
    main()
