"""Host-side pin (no GPU) of the split pairs' Laplace-type coefficients
(legendre_one in csrc/green.cu, compiled for the host; Section 4.1, eqs. lm
and pm): P^_m = int_0^{2pi} cos(m phi) / rho dphi = 2 sqrt(2) Q_{m-1/2}(chi)
/ sqrt(B) and S^_m = int_0^{2pi} cos(m phi) / rho^3 dphi = -4 sqrt(2)
Q'_{m-1/2}(chi) / B^{3/2}, with B = 2 r_t r_s and rho^2 = B (chi - cos phi),
against mpmath's Legendre function of the second kind at 40 digits, on both
branches of the recurrence (forward for chi -> 1, Miller otherwise)."""
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

mpmath = pytest.importorskip("mpmath")

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1810_07067_gb300", "csrc")


@pytest.mark.skipif(shutil.which("nvcc") is None, reason="nvcc not found")
def test_laplace_coefficients_against_mpmath(tmp_path):
    obj, exe = str(tmp_path / "green.o"), str(tmp_path / "legendre_check")
    inc = ["-I", os.path.join(ROOT, "include"), "-I", CSRC]
    # host code of green.cu (device code as PTX only: nothing runs on a GPU here)
    subprocess.run(["nvcc", "-c", "-gencode", "arch=compute_103a,code=compute_103a", "-O2", "-std=c++17", *inc,
                    "-o", obj, os.path.join(CSRC, "green.cu")], check=True, capture_output=True, timeout=600)
    subprocess.run(["nvcc", "-O2", "-std=c++17", "-gencode", "arch=compute_103a,code=compute_103a", *inc, "-o", exe,
                    os.path.join(HERE, "native", "legendre_check.cu"), obj], check=True, capture_output=True,
                   timeout=600)
    # (r_t, dr, dz): chi - 1 = (dr^2 + dz^2) / (2 r_t r_s) from 1e-10 to about 3
    cases = [(1.0, 1e-5, 1e-5), (2.0, 2e-4, -1e-4), (1.0, 0.01, 0.02), (0.8, 0.1, 0.3), (0.5, -0.4, 1.0),
             (0.05, 0.01, 0.08), (1.5, 1.2, 0.5)]
    sizes = [(255, 130), (31, 12)]
    lines = [f"{rt!r} {dr!r} {dz!r} {Mq} {Ms}" for Mq, Ms in sizes for rt, dr, dz in cases]
    out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    rows = out.stdout.strip().split("\n")
    assert len(rows) == len(lines)
    worst = 0.0
    with mpmath.workdps(40):
        for (Mq, Ms), chunk in zip(sizes, (rows[:len(cases)], rows[len(cases):])):
            for (rt, dr, dz), row in zip(cases, chunk):
                v = np.array([float(t) for t in row.split()])
                P, S = v[:Mq + 1], v[Mq + 1:]
                B = 2.0 * rt * (rt - dr)
                chi = 1 + (mpmath.mpf(dr) ** 2 + mpmath.mpf(dz) ** 2) / B
                Q = lambda m, x: mpmath.re(mpmath.legenq(m - mpmath.mpf(0.5), 0, x, type=3))
                for m in sorted(set(list(range(0, Mq + 1, 9)) + [1, 2, Mq])):
                    ref = 2 * mpmath.sqrt(2) * Q(m, chi) / mpmath.sqrt(B)
                    worst = max(worst, float(abs(P[m] - ref) / abs(ref)))
                for m in sorted(set(list(range(0, Ms, 13)) + [1, Ms - 1])):
                    ref = -4 * mpmath.sqrt(2) * mpmath.diff(lambda x: Q(m, x), chi) / mpmath.mpf(B) ** 1.5
                    worst = max(worst, float(abs(S[m] - ref) / abs(ref)))
    assert worst <= 1e-13, worst
