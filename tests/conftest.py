import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: oracle runs longer than a few seconds")


_CACHE = {}


@pytest.fixture(scope="session")
def sphere_oracle():
    """Oracle matrices, RHS and currents for the dielectric unit sphere workload
    (4 panels x 16 nodes, modes -10..10, k0 = 1, k1 = 1.5)."""
    if "sphere" not in _CACHE:
        import numpy as np
        import workloads as W
        from oracle import system, linalg, fields
        cfg = W.config_sphere()
        A = system.assemble(cfg.curve, cfg.media, cfg.M)
        b = fields.modal_rhs(cfg.curve, cfg.media, cfg.M, cfg.waves)
        sw = system.l2_weights(cfg.curve)
        Aw = system.weight_matrix(A, sw)
        x = np.zeros_like(b)
        for q in range(2 * cfg.M + 1):
            LU, piv = linalg.lu_factor(Aw[q])
            x[q] = linalg.lu_solve(LU, piv, b[q] * sw[:, None]) / sw[:, None]
        _CACHE["sphere"] = dict(cfg=cfg, A=A, Aw=Aw, b=b, x=x, sw=sw)
    return _CACHE["sphere"]
