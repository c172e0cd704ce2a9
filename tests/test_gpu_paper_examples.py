"""The paper's numerical examples (Section 6, Tables 1-4) through the GPU
path: the extinction test of eq. loop on one row of each example, with the
row's N_f and N_pts, must be at least as accurate as the error the paper
prints for that row (measured 1e-9 to 1e-14 here)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from workloads import paper_tables as T
from workloads.sources import current_loop_field, ring_points

DEV = "cuda:0"


@pytest.fixture(scope="module")
def mb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1810_07067_gb300 as m
    return m


@pytest.mark.parametrize("example,row", [("torus", 7), ("starfish", 3), ("droplet", 3), ("cylinder", 9)])
def test_extinction_error_at_most_the_papers(mb, example, row):
    r = T.EXAMPLES[example][row]
    cfg = T.config(example, r)
    media, M, N = cfg.media, cfg.M, cfg.N
    k1 = media.omega * np.sqrt(complex(media.eps1) * complex(media.mu1))
    nth = 2 * M + 2 * int(np.ceil(abs(k1) * float(np.max(cfg.curve.r)))) + 64
    pts = ring_points(cfg.curve.r, cfg.curve.z, nth)
    E, H = current_loop_field(pts.reshape(-1, 3), k1, media.omega, complex(media.mu1))
    EH = torch.tensor(np.concatenate([E, H], -1).reshape(1, N, nth, 6), device=DEV)
    ctx = mb.build(cfg.curve, media, M, mb.Options(n_phi=16, formulation=1, precision=1))
    rhs = torch.zeros((2 * M + 1, 1, 4 * N), dtype=torch.complex128, device=DEV)
    ctx.rhs_fields(EH, rhs)
    x = torch.zeros_like(rhs)
    ctx.solve(rhs, x)
    P = T.interior_points(example)
    out = torch.zeros((1, len(P), 6), dtype=torch.complex128, device=DEV)
    ctx.eval(x, P, 1, out)
    Er, Hr = current_loop_field(P, k1, media.omega, complex(media.mu1))
    ref = np.concatenate([Er, Hr], -1)
    err = np.linalg.norm(out.cpu().numpy()[0] - ref) / np.linalg.norm(ref)
    ctx.close()
    print(f"{example} row {row}: E_error {err:.2e} (paper {r[8]:.2e})")
    assert err <= r[8]


@pytest.mark.parametrize("row", [0, 3])
def test_torus_points_near_the_surface(mb, row):
    """Torus rows with few panels (4 and 10) and interior points up to half
    the tube's radii from its centre line (0.25 from the surface, below a
    panel's length): the refined evaluation must keep the paper's accuracy."""
    r = T.TORUS[row]
    cfg = T.config("torus", r)
    media, M, N = cfg.media, cfg.M, cfg.N
    k1 = media.omega * np.sqrt(complex(media.eps1) * complex(media.mu1))
    nth = 2 * M + 2 * int(np.ceil(abs(k1) * float(np.max(cfg.curve.r)))) + 64
    pts = ring_points(cfg.curve.r, cfg.curve.z, nth)
    E, H = current_loop_field(pts.reshape(-1, 3), k1, media.omega, complex(media.mu1))
    EH = torch.tensor(np.concatenate([E, H], -1).reshape(1, N, nth, 6), device=DEV)
    ctx = mb.build(cfg.curve, media, M, mb.Options(n_phi=16, formulation=1, precision=1))
    rhs = torch.zeros((2 * M + 1, 1, 4 * N), dtype=torch.complex128, device=DEV)
    ctx.rhs_fields(EH, rhs)
    x = torch.zeros_like(rhs)
    ctx.solve(rhs, x)
    P = T.interior_points("torus")
    out = torch.zeros((1, len(P), 6), dtype=torch.complex128, device=DEV)
    ctx.eval(x, P, 1, out)
    Er, Hr = current_loop_field(P, k1, media.omega, complex(media.mu1))
    ref = np.concatenate([Er, Hr], -1)
    err = np.linalg.norm(out.cpu().numpy()[0] - ref) / np.linalg.norm(ref)
    ctx.close()
    print(f"torus row {row}: E_error {err:.2e} (paper {r[8]:.2e})")
    assert err <= r[8]
