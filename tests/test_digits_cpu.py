"""Host-side check (no GPU) of the exact fixed-point rounding behind the digit
rows of the tensor-core transforms over phi: the integer route of
csrc/digits.cuh against round-to-nearest-even of the exact product, and the
balanced base-128 digits that the BF16 products take."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.skipif(shutil.which("nvcc") is None, reason="nvcc not found")
def test_fixed_point_rounding_matches_round_to_nearest_even(tmp_path):
    exe = str(tmp_path / "digits_check")
    src = os.path.join(HERE, "native", "digits_check.cu")
    subprocess.run(["nvcc", "-O2", "-std=c++17", "-o", exe, src], check=True, capture_output=True, timeout=300)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
    assert " 0 mismatches; 0 ordering mismatches; 0 digit mismatches" in out.stdout, out.stdout
