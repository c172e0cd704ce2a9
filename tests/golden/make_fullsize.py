"""Write the oracle's full-size reference solutions used by the GPU parity
tests and by the bench's per-mode error report.

Only the oracle (``oracle/``) computes anything here; ``workloads`` supplies
the seeded synthetic inputs.  For one named workload the script

1. assembles the per-mode Mueller matrices (eq. mullerrep, Lemma 1, the
   modal N and K operators, the near-panel rules of Section 5) row by row
   with ``oracle.system.assemble_row``, target rows spread over worker
   processes;
2. applies the L2 weighting (Section 6 remark), factors every requested mode
   with the oracle's naive partial-pivot LU and solves for the plane-wave
   data of eq. pw (``oracle.fields.modal_rhs``);
3. evaluates the far field (eq. farfieldform, magnetic current in the last
   term) of the solved currents at fixed directions;
4. for the modes whose currents are kept, also solves two seeded random
   right-hand sides (complex normal entries, numpy default_rng(7000 + m)),
   so that modes whose plane-wave data are below rounding are still
   compared on solutions of full size, and records for those modes the
   1-norm condition number of the weighted matrix and the oracle's own noise
   level, the relative 1-norm difference between the matrices its 32- and
   24-point azimuthal rules give (entries that the mode numbers m and 1/r
   factors amplify from coefficients below rounding are noise on both
   sides).

Workloads:
  cylinder  finite cylinder R = 1, H = 2, 7 dyadic levels at each edge
            (N = 576), k0 = 5, k1 = 7.5 + 0.01i, all modes -64..64, 16 plane
            waves; the far field is that of the complete solution.
  random    smooth random body (seed 1810, N = 1024), k0 = 10, k1 = 15,
            modes -128, -1, 0, 1, 64, 128, two plane waves; the far field is
            that of the listed modes' currents (the other modes set to zero).
  batch     a seeded sample of the batched workload (workloads.config_batch):
            6 of its 64 random bodies and 2 of its 8 edged bodies, drawn with
            numpy default_rng(72); modes 0, -1 and M of each, two plane waves.

Usage: python tests/golden/make_fullsize.py cylinder|random|batch [--workers K]
Writes tests/golden/fullsize_<workload>.npz (batch: fullsize_batch<index>.npz
per sampled body).  Each workload takes about 10-40 minutes on 8 cores.
"""
from __future__ import annotations

import argparse
import os
import sys
import tempfile
import time

os.environ.setdefault("OMP_NUM_THREADS", "1")
os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
os.environ.setdefault("MKL_NUM_THREADS", "1")

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

# currents kept in the file (the far field covers every solved mode)
KEEP = {
    "cylinder": dict(modes=[-64, -1, 0, 1, 32, 64], waves=[0, 1, 6, 7, 14, 15]),
    "random": dict(modes=[-128, -1, 0, 1, 64, 128], waves=[0, 1]),
}


def batch_sample():
    """Indices into workloads.config_batch() of the sampled bodies."""
    rng = np.random.default_rng(72)
    return sorted([int(v) for v in rng.choice(64, 6, replace=False)] +
                  [64 + int(v) for v in rng.choice(8, 2, replace=False)])


def workload(name):
    """(config, solved modes, kept modes and waves) of a workload name:
    cylinder, random, or batch<index> for a body of the batched workload."""
    import workloads as W
    if name == "cylinder":
        cfg = W.config_cylinder(7)
        return cfg, list(range(-cfg.M, cfg.M + 1)), KEEP["cylinder"]
    if name == "random":
        cfg = W.config_random()
        return cfg, KEEP["random"]["modes"], KEEP["random"]
    if name.startswith("batch") and name[5:].isdigit():
        cfg = W.config_batch()[int(name[5:])]
        keep = dict(modes=[-1, 0, cfg.M], waves=[0, 1])
        return cfg, keep["modes"], keep
    raise SystemExit(f"unknown workload {name}")


def far_directions():
    """48 directions: 6 polar angles x 6 azimuths plus 12 scattered ones."""
    th = (np.arange(6) + 0.5) * np.pi / 6
    ph = np.arange(6) * 2 * np.pi / 6 + 0.3
    T, Pp = np.meshgrid(th, ph, indexing="ij")
    d = np.stack([np.sin(T) * np.cos(Pp), np.sin(T) * np.sin(Pp), np.cos(T)], -1).reshape(-1, 3)
    rng = np.random.default_rng(48)
    e = rng.standard_normal((12, 3))
    e /= np.linalg.norm(e, axis=1, keepdims=True)
    return np.concatenate([d, e])


def _rows_job(args):
    name, rows, modes, path, lo_modes, lo_path = args
    from oracle import system
    cfg, _, _ = workload(name)
    A = np.load(path, mmap_mode="r+")
    A_lo = np.load(lo_path, mmap_mode="r+")
    geo = system.node_geometry(cfg.curve)
    for i in rows:
        hi, lo = system.assemble_row(cfg.curve, cfg.media, cfg.M, i, 0, modes, geo, lo_modes=lo_modes)
        A[:, 4 * i:4 * i + 4, :] = hi
        A_lo[:, 4 * i:4 * i + 4, :] = lo
    A.flush()
    A_lo.flush()
    return len(rows)


def _solve_job(args):
    name, qi, path, b, brand, lo_path, lq = args
    from oracle import system, linalg
    cfg, _, _ = workload(name)
    A = np.array(np.load(path, mmap_mode="r")[qi])
    sw = system.l2_weights(cfg.curve)
    Aw = A * sw[:, None] / sw[None, :]
    noise = None
    if lq is not None:  # 1-norm of the weighted 32- minus 24-point matrix, relative
        dA = (A - np.load(lo_path, mmap_mode="r")[lq]) * sw[:, None] / sw[None, :]
        noise = float(np.abs(dA).sum(0).max() / np.abs(Aw).sum(0).max())
        del dA
    LU, piv = linalg.lu_factor(Aw)
    bw = b * sw[:, None]
    y = linalg.lu_solve(LU, piv, bw)
    res = np.abs(Aw @ y - bw).max() / (np.abs(Aw).sum(1).max() * np.abs(y).max() + np.abs(bw).max())
    xr, kappa = None, None
    if brand is not None:
        xr = linalg.lu_solve(LU, piv, brand * sw[:, None]) / sw[:, None]
        # 1-norm condition number of the weighted matrix (LAPACK inverse; a
        # diagnostic of how far rounding-level differences can move x)
        kappa = float(np.linalg.norm(Aw, 1) * np.linalg.norm(np.linalg.inv(Aw), 1))
    return qi, y / sw[:, None], float(res), xr, kappa, noise


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("workload", choices=["cylinder", "random", "batch"])
    ap.add_argument("--workers", type=int, default=max(1, (os.cpu_count() or 2) - 1))
    ap.add_argument("--tmp", default=tempfile.gettempdir())
    args = ap.parse_args()
    names = [f"batch{i}" for i in batch_sample()] if args.workload == "batch" else [args.workload]
    for name in names:
        run(name, args)


def run(name, args):
    import multiprocessing as mp
    from oracle import fields
    cfg, modes, keep = workload(name)
    N, M, n = cfg.N, cfg.M, 4 * cfg.N
    t0 = time.time()
    path = os.path.join(args.tmp, f"oracle_A_{name}_{os.getpid()}.npy")
    lo_path = os.path.join(args.tmp, f"oracle_Alo_{name}_{os.getpid()}.npy")
    A = np.lib.format.open_memmap(path, mode="w+", dtype=np.complex128, shape=(len(modes), n, n))
    A_lo = np.lib.format.open_memmap(lo_path, mode="w+", dtype=np.complex128, shape=(len(keep["modes"]), n, n))
    del A, A_lo
    ctx = mp.get_context("spawn")
    chunks = [list(range(i, N, 4 * args.workers)) for i in range(4 * args.workers)]
    with ctx.Pool(args.workers) as pool:
        done = 0
        for k in pool.imap_unordered(_rows_job, [(name, c, modes, path, keep["modes"], lo_path)
                                                 for c in chunks if c]):
            done += k
            print(f"[{time.time() - t0:7.0f} s] assembled {done}/{N} rows", flush=True)
        b_all = fields.modal_rhs(cfg.curve, cfg.media, M, cfg.waves)     # [2M+1, n, nrhs]
        brand = {}
        for m in keep["modes"]:
            rng = np.random.default_rng(7000 + m)
            brand[m] = rng.standard_normal((n, 2)) + 1j * rng.standard_normal((n, 2))
        lqs = {m: q for q, m in enumerate(keep["modes"])}
        jobs = [(name, qi, path, b_all[m + M], brand.get(m), lo_path, lqs.get(m)) for qi, m in enumerate(modes)]
        x = np.zeros((len(modes), n, len(cfg.waves)), dtype=complex)
        xrand, kappa, noise = {}, {}, {}
        berr = np.zeros(len(modes))
        for qi, xq, res, xr, kp, nz in pool.imap_unordered(_solve_job, jobs):
            x[qi] = xq
            berr[qi] = res
            if xr is not None:
                xrand[modes[qi]] = xr
                kappa[modes[qi]] = kp
                noise[modes[qi]] = nz
            print(f"[{time.time() - t0:7.0f} s] solved mode {modes[qi]} (backward error {res:.1e})", flush=True)
    os.remove(path)
    os.remove(lo_path)
    # far field of the solved modes (the others zero)
    xf = np.zeros((2 * M + 1, n, len(cfg.waves)), dtype=complex)
    for qi, m in enumerate(modes):
        xf[m + M] = x[qi]
    dirs = far_directions()
    ff = fields.far_field(cfg.curve, cfg.media, M, xf, dirs)          # [nrhs, nd, 3]
    kq = [modes.index(m) for m in keep["modes"]]
    out = os.path.join(HERE, f"fullsize_{name}.npz")
    np.savez_compressed(
        out,
        workload=name, n_panels=cfg.curve.n_panels, closed=int(cfg.curve.closed),
        r=cfg.curve.r, z=cfg.curve.z, dr=cfg.curve.dr, dz=cfg.curve.dz,
        omega=cfg.media.omega, eps0=complex(cfg.media.eps0), mu0=complex(cfg.media.mu0),
        eps1=complex(cfg.media.eps1), mu1=complex(cfg.media.mu1), M=M, n_phi=cfg.n_phi,
        wave_d=np.array([w.d for w in cfg.waves]), wave_e=np.array([w.e for w in cfg.waves]),
        solved_modes=np.array(modes), backward_err=berr,
        modes=np.array(keep["modes"]), waves=np.array(keep["waves"]),
        x=x[kq][:, :, keep["waves"]].transpose(0, 2, 1).copy(),     # [modes, waves, 4N]
        ff_dirs=dirs, ff=ff,
        b_rand=np.stack([brand[m].T for m in keep["modes"]]),      # [modes, 2, 4N]
        x_rand=np.stack([xrand[m].T for m in keep["modes"]]),
        kappa1=np.array([kappa[m] for m in keep["modes"]]),        # 1-norm condition numbers of A'_m
        noise1=np.array([noise[m] for m in keep["modes"]]),        # ||A'_m(32-pt) - A'_m(24-pt)||_1 / ||A'_m||_1
        seconds=time.time() - t0)
    print(f"wrote {out} in {time.time() - t0:.0f} s; max oracle backward error {berr.max():.1e}")


if __name__ == "__main__":
    main()
