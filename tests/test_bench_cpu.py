"""Host-side checks (no GPU) of bench.py's roofline arithmetic: algorithmic
work per stage from the build's counts, achieved rate = work / device time,
fraction = achieved / peak, for a synthetic stats record."""
import math

import pytest

import bench


def _stats():
    return {"n_phi_used": 512, "n_far_pairs": 1000, "n_split_pairs": 10, "n_support_pairs": 200,
            "ms_far": 10.0, "ms_support": 5.0, "ms_near": 2.0, "ms_legendre": 1.0,
            "ms_far_assemble": 3.0, "ms_far_sample": 4.0, "ms_far_product": 2.0,
            "ms_lu_gemm": 8.0, "lu_gemm_bytes": 8e9}


def test_stage_and_kernel_rooflines():
    st, M, N, fp64, hbm = _stats(), 128, 1024, 1.05, 6790.0
    kr = bench._kernel_rooflines(st, M, N, fp64, hbm)
    n = 512
    fft, samp = 2.5 * n * math.log2(n), (n // 2 + 1) * 140
    far = 1000 * (9 * fft + samp + 256 * (M + 1))
    assert kr["far_stage"]["algorithmic_flops"] == pytest.approx(far)
    assert kr["far_stage"]["achieved"] == pytest.approx(far / 10e-3 / 1e12)
    assert kr["far_stage"]["frac"] == pytest.approx(far / 10e-3 / 1e12 / fp64)
    sup = 200 * (9 * fft + samp) + 6 * fft * 10
    assert kr["support_stage"]["algorithmic_flops"] == pytest.approx(sup)
    near = 200 * 16 * 27 * 4 * (M + 2) + N * 48 * (M + 1) * 256
    assert kr["near_kernel"]["algorithmic_flops"] == pytest.approx(near)
    assert kr["legendre_kernel"]["algorithmic_flops"] == pytest.approx(10 * 10 * (n // 2))
    fa = kr["far_assemble_kernel"]
    assert fa["algorithmic_bytes"] == pytest.approx(1000 * (M + 1) * 256)
    assert fa["achieved"] == pytest.approx(1000 * (M + 1) * 256 / 3e-3 / 1e9) and fa["unit"] == "GB/s"
    g = kr["gemm_update_tc_kernel"]
    assert g["achieved"] == pytest.approx(8e9 / 8e-3 / 1e9) and g["frac"] == pytest.approx(1000.0 / hbm)
    for k in ("far_sample_kernel", "oz_real_gemm_kernel (far)"):
        assert kr[k]["ms"] == st[{"far_sample_kernel": "ms_far_sample"}.get(k, "ms_far_product")]


def test_fused_far_path_reports_far_kernel():
    st = _stats()
    for k in ("ms_far_assemble", "ms_far_sample", "ms_far_product"):
        st[k] = 0.0
    kr = bench._kernel_rooflines(st, 128, 1024, 1.05, 6790.0)
    assert "far_kernel" in kr and "far_stage" not in kr and "far_assemble_kernel" not in kr
