"""Host-side parity (no GPU) of the Mueller 4 x 4 block arithmetic of the
far-pair assembly (csrc/block.cuh, compiled for the CPU) with the oracle's
own formulation of Lemma 1 and the modal N and K operators (Section 3;
oracle.system.operator_blocks and coefficients): random spectra of the nine
families, random target and source geometry, direct and indirect forms,
real and complex interior wavenumbers.  The specialised block (real k^2,
purely imaginary coupling coefficients, unit K factors) must equal the
general one on every case it applies to."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import system
from workloads.configs import Media

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _c(z):
    z = complex(z)
    return f"{z.real!r} {z.imag!r}"


@pytest.mark.skipif(shutil.which("nvcc") is None, reason="nvcc not found")
def test_block_arithmetic_matches_oracle(tmp_path):
    exe = str(tmp_path / "block_check")
    subprocess.run(["nvcc", "-O2", "-std=c++17", "-I", os.path.join(ROOT, "include"), "-o", exe,
                    os.path.join(HERE, "native", "block_check.cu")], check=True, capture_output=True, timeout=300)
    rng = np.random.default_rng(1810)
    cases, lines = [], []
    for q in range(240):
        form = q % 2
        k0 = float(rng.uniform(0.5, 20.0))
        if q % 4 < 2:
            k1 = complex(k0 * rng.uniform(1.1, 2.0))                                 # real: specialised block
        else:
            k1 = complex(k0 * rng.uniform(1.1, 2.0), rng.uniform(1e-3, 0.5))        # lossy interior
        med = Media.from_k(k0, k1)
        kk0, kk1 = system.wavenumbers(med)
        M = int(rng.integers(2, 40))
        m = int(rng.integers(0, M + 1))
        rt, rs = (float(v) for v in rng.uniform(0.05, 2.0, 2))
        a_t, a_s = rng.uniform(0, 2 * np.pi, 2)
        rpt, zpt, rps, zps = (float(v) for v in (np.cos(a_t), np.sin(a_t), np.cos(a_s), np.sin(a_s)))
        F = (rng.standard_normal((9, M + 2)) + 1j * rng.standard_normal((9, M + 2))) * \
            10.0 ** rng.uniform(-3, 3, (9, 1))
        cases.append((form, med, kk0, kk1, M, m, rt, rpt, zpt, rs, rps, zps, F))
        lines.append(f"{form} {med.omega!r} {_c(kk0)} {_c(kk1)} {_c(med.eps0)} {_c(med.mu0)} "
                     f"{_c(med.eps1)} {_c(med.mu1)} {M} {m} {rt!r} {rpt!r} {zpt!r} {rs!r} {rps!r} {zps!r} " +
                     " ".join(_c(v) for v in F.reshape(-1)))
    out = subprocess.run([exe], input=f"{len(cases)}\n" + "\n".join(lines) + "\n", capture_output=True,
                         text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    vals = out.stdout.split()
    pos, n_simple, worst, worst_spec = 0, 0, 0.0, 0.0
    for form, med, kk0, kk1, M, m, rt, rpt, zpt, rs, rps, zps, F in cases:
        simple = int(vals[pos]); pos += 1
        got = np.array([float(v) for v in vals[pos:pos + 64]]).reshape(2, 4, 4, 2); pos += 64
        gen = got[0, ..., 0] + 1j * got[0, ..., 1]
        spec = got[1, ..., 0] + 1j * got[1, ..., 1]
        # the oracle's block of this source point and mode, unit quadrature weight
        N0, N1, KD = system.operator_blocks(F[None], np.array([rs]), np.array([rps]), np.array([zps]),
                                            rt, rpt, zpt, kk0, kk1, np.array([m]))
        co = system.coefficients(med, form)
        om = med.omega
        x0, x1 = co["x"]; y0, y1 = co["y"]
        ref = np.zeros((4, 4), dtype=complex)
        ref[0:2, 0:2] = co["aEJ"] * KD[0, 0]
        ref[0:2, 2:4] = -1j * om * (x0 * N0[0, 0] - x1 * N1[0, 0])
        ref[2:4, 0:2] = -1j * om * (y0 * N0[0, 0] - y1 * N1[0, 0])
        ref[2:4, 2:4] = co["aHM"] * KD[0, 0]
        scale = np.abs(ref).max()
        worst = max(worst, np.abs(gen - ref).max() / scale)
        worst_spec = max(worst_spec, np.abs(spec - gen).max() / scale)
        n_simple += simple
        if np.imag(kk1) == 0.0:
            assert simple == 1, "real wavenumbers with unit vacuum parameters take the specialised block"
    assert n_simple >= 100
    assert worst <= 1e-14, worst
    assert worst_spec <= 1e-15, worst_spec
