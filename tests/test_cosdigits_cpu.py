"""Host-side check (no GPU) of the B operand of the tensor-core transform
over phi: the digits that ozaki_real_b_host (csrc/ozaki.cu, compiled for the
host) stores for the cosine matrices of every grid of the ladder sum back to
round(b / 2 * 2^56) at the operand layout the digit products read, stay
within [-64, 64] (exact in BF16) and leave the padding zero."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1810_07067_gb300", "csrc")


@pytest.mark.skipif(shutil.which("nvcc") is None, reason="nvcc not found")
def test_cosine_digits_reconstruct_exactly(tmp_path):
    obj, exe = str(tmp_path / "ozaki.o"), str(tmp_path / "cosdigits_check")
    inc = ["-I", os.path.join(ROOT, "include"), "-I", CSRC]
    ptx = ["-gencode", "arch=compute_103a,code=compute_103a"]   # device code as PTX only: nothing runs on a GPU
    subprocess.run(["nvcc", "-c", *ptx, "-O2", "-std=c++17", *inc, "-o", obj, os.path.join(CSRC, "ozaki.cu")],
                   check=True, capture_output=True, timeout=600)
    subprocess.run(["nvcc", "-O2", "-std=c++17", *ptx, *inc, "-o", exe,
                    os.path.join(HERE, "native", "cosdigits_check.cu"), obj], check=True, capture_output=True,
                   timeout=600)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
    assert " 0 violations" in out.stdout, out.stdout
