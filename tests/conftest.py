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


@pytest.fixture(scope="session")
def loop_oracle():
    """Oracle solution of the extinction test of the numerical examples
    (eq. loop): the sphere workload's body and media, indirect formulation
    (eq. dualmullrep), modes -12..12, boundary data from the current loop's
    k1 field sampled on the node rings (128 azimuths)."""
    if "loop" not in _CACHE:
        import numpy as np
        import workloads as W
        from workloads.sources import current_loop_field, ring_points
        from oracle import system, linalg, fields
        cfg = W.config_sphere()
        M, T = 12, 128
        _, k1 = system.wavenumbers(cfg.media)
        pts = ring_points(cfg.curve.r, cfg.curve.z, T)
        E, H = current_loop_field(pts.reshape(-1, 3), k1, cfg.media.omega, complex(cfg.media.mu1))
        EH = np.concatenate([E, H], -1).reshape(1, cfg.curve.N, T, 6)
        b = fields.modal_rhs_samples(cfg.curve, cfg.media, M, EH, formulation=1)
        A = system.assemble(cfg.curve, cfg.media, M, formulation=1)
        sw = system.l2_weights(cfg.curve)
        Aw = system.weight_matrix(A, sw)
        x = np.zeros_like(b)
        for q in range(2 * M + 1):
            LU, piv = linalg.lu_factor(Aw[q])
            x[q] = linalg.lu_solve(LU, piv, b[q] * sw[:, None]) / sw[:, None]
        rng = np.random.default_rng(3)
        d = rng.standard_normal((8, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        inner = d * rng.uniform(0.1, 0.6, (8, 1))
        outer = d * rng.uniform(1.8, 2.6, (8, 1))
        _CACHE["loop"] = dict(cfg=cfg, M=M, T=T, k1=k1, EH=EH, b=b, x=x, inner=inner, outer=outer)
    return _CACHE["loop"]
