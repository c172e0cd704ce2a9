"""Host-side pin (no GPU) of the far pairs' grid choice (csrc/grid.cuh
compiled for the CPU; not in the paper): for non-split pairs of the
N = 1024 random body at k0 = 10, k1 = 15, M = 128, n_phi = 512, the modes
that pair_grid drops (above m_c) must be negligible and the trapezoid on its
grid of n_l points must reproduce modes 0..m_c, both judged against the
oracle's direct quadrature of the nine families (Section 4's modal
integrals) with the oracle's integrands sampled on that grid."""
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

import workloads as W
from oracle import green, system

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
EPS = 1e-17


@pytest.mark.skipif(shutil.which("nvcc") is None, reason="nvcc not found")
def test_far_pair_grid_drops_nothing_and_does_not_alias(tmp_path):
    exe = str(tmp_path / "grid_check")
    subprocess.run(["nvcc", "-O2", "-std=c++17", "-I", os.path.join(ROOT, "include"), "-o", exe,
                    os.path.join(HERE, "native", "grid_check.cu")], check=True, capture_output=True, timeout=300)
    cfg = W.config_random()
    cv, M, nphi = cfg.curve, cfg.M, cfg.n_phi
    k0, k1 = system.wavenumbers(cfg.media)
    # the build's split test: aliasing of the full grid above EPS (zeta^(nphi-M-1) > EPS)
    lmax = -math.log(EPS) / (nphi - M - 1)
    cthr = 2.0 * math.sinh(0.5 * lmax) ** 2
    rng = np.random.default_rng(3)
    pairs = []
    while len(pairs) < 48:
        i, j = (int(v) for v in rng.integers(0, cv.N, 2))
        if abs(i // 16 - j // 16) < 2:                  # self and neighbouring panels take the support points
            continue
        rt, dr0, zd = cv.r[i], cv.r[i] - cv.r[j], cv.z[i] - cv.z[j]
        if dr0 * dr0 + zd * zd < cthr * 2.0 * rt * (rt - dr0):
            continue                                     # split pairs keep the full grid and every mode
        pairs.append((i, j))
    lines = [f"{k0.real!r} {k0.imag!r} {k1.real!r} {k1.imag!r} {M} {nphi} {EPS!r} {float(cv.r[i])!r} "
             f"{float(cv.r[i] - cv.r[j])!r} {float(cv.z[i] - cv.z[j])!r} 0" for i, j in pairs]
    out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    grids = [tuple(int(v) for v in ln.split()) for ln in out.stdout.strip().split("\n")]
    assert len(grids) == len(pairs)
    worst_tail, worst_alias, smaller = 0.0, 0.0, 0
    for (i, j), (nl, mc) in zip(pairs, grids):
        assert nl % 8 == 0 and 16 <= nl <= nphi and nl >= 2 * mc + 2 and mc <= M + 1
        smaller += nl < nphi
        F = green.modal_families(cv.r[i], cv.z[i], cv.r[j], cv.z[j], k0, k1, M)     # [9, M+2], direct quadrature
        scale = np.abs(F).max(axis=1)
        if mc < M + 1:                                   # dropped modes
            worst_tail = max(worst_tail, float(np.max(np.abs(F[:, mc + 1:]).max(axis=1) / scale)))
        # trapezoid of the oracle's integrands on the pair's grid, modes 0..mc
        phi = 2.0 * np.pi * np.arange(nl) / nl
        G = green.integrands(cv.r[i], cv.z[i], cv.r[i] - cv.r[j], cv.z[i] - cv.z[j], k0, k1, phi)
        T = (2.0 * np.pi / nl) * G @ np.cos(np.outer(phi, np.arange(mc + 1)))
        worst_alias = max(worst_alias, float(np.max(np.abs(T - F[:, :mc + 1]).max(axis=1) / scale)))
    assert smaller >= len(pairs) // 2                   # the ladder is in use
    assert worst_tail <= 1e-13, worst_tail
    assert worst_alias <= 1e-13, worst_alias
