"""The four numerical examples of Section 6 (Tables 1-4): bodies, parameters
and the values the paper prints.

Each row: (k0, k1, N_f, N_pts, T_kernel, T_matgen, T_solve, T_add, E_error)
with modes -N_f..N_f, N_pts curve nodes, the paper's CPU times in seconds and
its extinction-test error (relative l2 error of E and H at a few random
points inside the body).  The bodies here use N_pts nodes as 16-node panels:
torus and starfish uniform in t, the droplet uniform with its last panel
refined five times toward the tip, the cylinder with the panels next to its
two edges refined 14 times (last panel ~1e-5, as the example states) and
the remaining panels spread over the bottom, side and top as 1 : 2 : 1.
"""
from __future__ import annotations

import numpy as np

from .configs import Config, Media
from .curves import cylinder, droplet, starfish, torus

TORUS = [  # Table 1
    (1, 2, 13, 64, 2.76, 2.98, 6.48e-2, 1.08e-2, 2.32e-9),
    (1, 5, 16, 160, 6.09, 7.95, 3.29e-1, 2.64e-2, 4.61e-9),
    (1, 10, 21, 320, 12.8, 25.1, 3.37, 8.59e-2, 3.11e-8),
    (5, 2, 13, 160, 6.13, 7.65, 3.56e-1, 3.24e-2, 1.01e-9),
    (5, 10, 21, 320, 12.7, 24.9, 2.35, 8.59e-2, 3.84e-9),
    (5, 20, 30, 640, 61.2, 138.0, 25.3, 5.85e-1, 4.63e-9),
    (10, 5, 17, 320, 13.2, 23.6, 1.97, 6.99e-2, 1.61e-9),
    (10, 20, 30, 640, 61.4, 137.0, 24.9, 5.36e-1, 2.08e-9),
    (10, 40, 45, 640, 91.4, 206.0, 34.9, 8.37e-1, 2.66e-8),
    (20, 5, 17, 320, 17.6, 27.7, 2.95, 9.8e-2, 4.78e-9),
    (20, 10, 22, 640, 60.9, 117.0, 18.3, 4.14e-1, 3.37e-9),
    (20, 40, 45, 640, 96.4, 211.0, 33.0, 8.37e-1, 1.10e-8),
]
STARFISH = [  # Table 2
    (5, 2, 10, 224, 6.47, 9.34, 4.61e-1, 3.35e-2, 1.24e-9),
    (5, 10, 16, 304, 9.49, 18.0, 1.57, 6.59e-2, 3.44e-10),
    (5, 20, 21, 464, 29.6, 61.9, 7.01, 2.06e-1, 1.51e-9),
    (10, 5, 13, 304, 9.82, 16.9, 1.78, 6.48e-2, 2.04e-10),
    (10, 20, 21, 464, 30.1, 59.4, 7.21, 2.59e-1, 9.74e-10),
    (10, 40, 30, 784, 77.3, 209.0, 39.8, 7.31e-1, 1.45e-8),
    (20, 5, 13, 464, 29.0, 49.3, 19.7, 6.99e-1, 1.05e-10),
    (20, 10, 16, 464, 29.8, 55.0, 77.8, 1.84e-1, 4.41e-10),
    (20, 40, 30, 784, 78.5, 217.0, 40.2, 8.04e-1, 4.60e-9),
    (40, 5, 13, 784, 74.1, 139.0, 20.2, 3.34e-1, 3.39e-10),
    (40, 10, 16, 784, 75.6, 155.0, 25.8, 4.46e-1, 3.58e-9),
    (40, 20, 21, 784, 77.5, 173.0, 33.2, 5.01e-1, 3.01e-9),
]
DROPLET = [  # Table 3
    (5, 2, 7, 224, 16.7, 18.9, 3.24e-1, 6.01e-2, 2.71e-10),
    (5, 10, 10, 320, 30.5, 37.2, 7.14e-1, 8.39e-2, 1.86e-9),
    (5, 20, 11, 480, 75.2, 94.3, 2.39, 1.84e-1, 5.11e-9),
    (10, 5, 9, 320, 30.5, 36.7, 5.47e-1, 7.59e-2, 1.24e-10),
    (10, 20, 11, 480, 78.0, 96.9, 2.45, 1.84e-1, 2.59e-9),
    (10, 40, 14, 800, 202.0, 279.0, 11.3, 9.27e-1, 6.76e-9),
    (20, 5, 9, 480, 72.7, 88.6, 1.97, 2.28e-1, 5.81e-10),
    (20, 10, 10, 480, 75.6, 93.4, 1.99, 2.52e-1, 1.31e-10),
    (20, 40, 14, 800, 204.0, 277.0, 11.2, 9.27e-1, 3.43e-9),
    (40, 5, 9, 800, 189.0, 239.0, 7.77, 6.07e-1, 3.48e-10),
    (40, 10, 10, 800, 192.0, 253.0, 8.19, 5.88e-1, 6.12e-10),
    (40, 20, 12, 800, 205.0, 266.0, 10.1, 8.01e-1, 1.45e-10),
]
CYLINDER = [  # Table 4
    (2, 1, 9, 1312, 106.0, 266.0, 44.6, 5.31e-1, 4.11e-9),
    (2, 5, 11, 1440, 156.0, 380.0, 71.3, 7.26e-1, 2.56e-8),
    (2, 10, 14, 1696, 218.0, 797.0, 135.0, 1.31, 9.32e-7),
    (5, 2, 10, 1440, 141.0, 358.0, 65.6, 6.63e-1, 1.54e-8),
    (5, 10, 14, 1696, 221.0, 717.0, 134.0, 1.42, 5.92e-8),
    (5, 20, 17, 2208, 344.0, 3140.0, 361.0, 2.61, 9.74e-7),
    (10, 2, 10, 1696, 194.0, 564.0, 99.2, 9.15e-1, 1.91e-8),
    (10, 5, 11, 1696, 221.0, 599.0, 107.0, 1.03, 3.95e-8),
    (10, 20, 17, 2208, 349.0, 2270.0, 362.0, 2.54, 2.24e-6),
    (20, 2, 10, 2208, 329.0, 1150.0, 219.0, 1.51, 3.54e-8),
    (20, 5, 11, 2208, 341.0, 1230.0, 238.0, 1.61, 1.39e-7),
    (20, 10, 14, 2208, 343.0, 1490.0, 296.0, 2.08, 1.32e-7),
]
EXAMPLES = {"torus": TORUS, "starfish": STARFISH, "droplet": DROPLET, "cylinder": CYLINDER}
CYL_LEVELS = 14


def body(example: str, n_pts: int):
    """The example's curve with n_pts nodes."""
    P = n_pts // 16
    if example == "torus":
        return torus(P)
    if example == "starfish":
        return starfish(P)
    if example == "droplet":
        return droplet(P - 5, 5)
    if example == "cylinder":
        B = P - 4 * CYL_LEVELS
        b0 = max(1, round(B / 4))
        return cylinder(CYL_LEVELS, 1.0, 1.0, base=(b0, B - 2 * b0, b0))
    raise ValueError(example)


def config(example: str, row) -> Config:
    k0, k1, nf, npts = row[:4]
    return Config(f"{example}_k0{k0}_k1{k1}_Nf{nf}_N{npts}", body(example, npts), Media.from_k(float(k0), float(k1)),
                  int(nf), 16, [])


def interior_points(example: str, n: int = 8, seed: int = 3) -> np.ndarray:
    """n points well inside the body (a few node spacings from the surface)."""
    rng = np.random.default_rng(seed)
    ph = rng.uniform(0, 2 * np.pi, n)
    if example == "torus":          # inside the tube (r - 2)^2 + (z / 0.5)^2 < 1, at half its size
        a = rng.uniform(0, 2 * np.pi, n); s = rng.uniform(0, 0.5, n)
        r, z = 2 + s * np.cos(a), 0.5 * s * np.sin(a)
    elif example == "starfish":     # radius < 1 in the (r, z) half-plane (the curve has R >= 1.5)
        a = rng.uniform(-0.5 * np.pi, 0.5 * np.pi, n); s = rng.uniform(0, 1.0, n)
        r, z = s * np.cos(a), s * np.sin(a)
    elif example == "droplet":      # near the widest section
        r, z = rng.uniform(0, 0.12, n), rng.uniform(-0.25, 0.1, n)
    elif example == "cylinder":
        r, z = rng.uniform(0, 0.6, n), rng.uniform(-0.6, 0.6, n)
    else:
        raise ValueError(example)
    return np.stack([r * np.cos(ph), r * np.sin(ph), z], -1)
