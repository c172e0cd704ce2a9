"""Host-side pins (no GPU) of the special functions behind the split modal
kernels (csrc/special.cuh compiled for the CPU) against mpmath at 60 digits:
the seven entire functions of u = rho^2 at complex and real wavenumbers
across the switch between Taylor series and closed forms (|k rho| = 2 and 4),
the complete elliptic integral K from the complementary modulus (the Miller
recurrence's normalisation, Section 4.1) and Carlson's R_D (for E)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

mpmath = pytest.importorskip("mpmath")

HERE = os.path.dirname(os.path.abspath(__file__))


def _reference(k, su):
    """C, S, Gam, Gam2, Gamp, Sp, Spp at sqrt(u) = su from their definitions
    as functions of u: C(u) = cos(k sqrt u), S(u) = sin(k sqrt u)/sqrt u,
    Gam = C' - (C - 1)/(2u), Gam2 = (Gam(u) - Gam(0))/u, Gamp = Gam', and the
    derivatives of S, by mpmath's high-precision differentiation in u."""
    k = mpmath.mpc(k.real, k.imag)
    u0 = mpmath.mpf(su) ** 2
    Cf = lambda u: mpmath.cos(k * mpmath.sqrt(u))
    Sf = lambda u: mpmath.sin(k * mpmath.sqrt(u)) / mpmath.sqrt(u)
    Gf = lambda u: mpmath.diff(Cf, u) - (Cf(u) - 1) / (2 * u)
    gam0 = -k ** 2 / 4                                  # the limit of Gam at u = 0
    vals = [Cf(u0), Sf(u0), Gf(u0), (Gf(u0) - gam0) / u0, mpmath.diff(Gf, u0),
            mpmath.diff(Sf, u0), mpmath.diff(Sf, u0, 2)]
    return np.array([complex(v) for v in vals])


@pytest.mark.skipif(shutil.which("nvcc") is None, reason="nvcc not found")
def test_special_functions_against_mpmath(tmp_path):
    exe = str(tmp_path / "special_check")
    subprocess.run(["nvcc", "-O2", "-std=c++17", "-o", exe, os.path.join(HERE, "native", "special_check.cu")],
                   check=True, capture_output=True, timeout=300)
    rng = np.random.default_rng(7)
    pts = []
    for x in list(np.geomspace(1e-3, 40.0, 40)) + [1.999, 2.0, 2.001, 3.999, 4.0, 4.001]:
        k = float(rng.uniform(0.5, 20.0))
        pts.append((complex(k), x / k, True))
        ki = complex(k, float(rng.uniform(1e-3, 1.0)))
        pts.append((ki, x / abs(ki), False))
    lines = [f"1 {k.real!r} {float(su)!r}" if real else f"0 {k.real!r} {k.imag!r} {float(su)!r}"
             for k, su, real in pts]
    kps = list(np.geomspace(1e-6, 1.0, 25))
    lines += [f"2 {float(kp)!r}" for kp in kps]
    rd = [tuple(float(v) for v in rng.uniform(0.01, 3.0, 3)) for _ in range(25)] + [(0.0, 1.0, 2.0), (1.0, 1.0, 1.0)]
    lines += [f"3 {x!r} {y!r} {z!r}" for x, y, z in rd]
    out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    rows = out.stdout.strip().split("\n")
    assert len(rows) == len(lines)
    worst = 0.0
    for (k, su, _), row in zip(pts, rows):
        v = np.array([float(t) for t in row.split()])
        got = v[0::2] + 1j * v[1::2]
        with mpmath.workdps(60):
            ref = _reference(k, su)
        # each function against its own size, floored by its size at the
        # smallest argument times |k|^p (the natural scale of the series)
        kk = abs(k)
        scale = np.maximum(np.abs(ref), np.array([1.0, kk, kk ** 2, kk ** 4, kk ** 4, kk ** 3, kk ** 5]) * 1e-3)
        worst = max(worst, float(np.max(np.abs(got - ref) / scale)))
    assert worst <= 1e-13, worst
    for kp, row in zip(kps, rows[len(pts):len(pts) + len(kps)]):
        with mpmath.workdps(60):
            ref = float(mpmath.ellipk(1 - mpmath.mpf(kp) ** 2))
        assert abs(float(row) - ref) <= 4e-16 * ref, (kp, float(row), ref)
    for (x, y, z), row in zip(rd, rows[len(pts) + len(kps):]):
        with mpmath.workdps(60):
            ref = float(mpmath.elliprd(x, y, z))
        assert abs(float(row) - ref) <= 1e-15 * ref, (x, y, z, float(row), ref)
