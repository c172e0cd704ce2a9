"""Material parameters, plane waves and the named synthetic workloads."""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .curves import Curve, sphere, cylinder, cone, random_body


@dataclass
class Media:
    """Background (0) and body (1) parameters; k_j = omega sqrt(eps_j mu_j).

    The exterior medium is medium 0 and the body medium 1, with
    eps0 = mu0 = 1, omega = k0, mu1 = 1 and eps1 = (k1/k0)^2 as the default
    reading of the numerical examples (Section 6)."""
    omega: float
    eps0: complex = 1.0
    mu0: complex = 1.0
    eps1: complex = 1.0
    mu1: complex = 1.0

    @staticmethod
    def from_k(k0: float, k1: complex) -> "Media":
        return Media(omega=float(k0), eps0=1.0, mu0=1.0, eps1=complex(k1 / k0) ** 2, mu1=1.0)


@dataclass
class PlaneWave:
    d: np.ndarray   # unit propagation direction
    e: np.ndarray   # unit electric polarisation, orthogonal to d


def plane_wave(d, p) -> PlaneWave:
    """Plane wave of eq. (pw): E ~ (d x p) x d, normalised to a unit vector."""
    d = np.asarray(d, float); d = d / np.linalg.norm(d)
    p = np.asarray(p, float)
    e = np.cross(np.cross(d, p), d)
    return PlaneWave(d, e / np.linalg.norm(e))


def paper_default_wave() -> PlaneWave:
    """Incidence angles of eq. (incidentdirection): theta1 = pi/3,
    phi1 = 2pi/3, theta2 = pi/2, phi2 = pi/3."""
    def ang(th, ph):
        return np.array([np.cos(th) * np.sin(ph), np.sin(th) * np.sin(ph), np.cos(ph)])
    return plane_wave(ang(np.pi / 3, 2 * np.pi / 3), ang(np.pi / 2, np.pi / 3))


@dataclass
class Config:
    name: str
    curve: Curve
    media: Media
    M: int
    n_phi: int
    waves: list = field(default_factory=list)

    @property
    def N(self):
        return self.curve.N


def _polar_wave(theta: float, pol: int) -> PlaneWave:
    d = np.array([np.sin(theta), 0.0, np.cos(theta)])
    e = np.array([np.cos(theta), 0.0, -np.sin(theta)]) if pol == 0 else np.array([0.0, 1.0, 0.0])
    return PlaneWave(d, e)


def config_sphere() -> Config:
    """Dielectric unit sphere: 4 panels x 16 nodes, modes -10..10, 64
    azimuthal samples, k0 = 1, k1 = 1.5, plane wave at 45 degrees (both
    polarisations)."""
    th = np.pi / 4
    return Config("sphere_N64_M10", sphere(4), Media.from_k(1.0, 1.5), 10, 64,
                  [_polar_wave(th, 0), _polar_wave(th, 1)])


def config_cylinder(levels: int = 7) -> Config:
    """Finite cylinder radius 1, height 2, edge-graded panels (N = 576 at 7
    levels), modes -64..64, 256 azimuthal samples, k0 = 5, k1 = 7.5+0.01i,
    8 polar incidence angles (j+1/2)pi/8 x 2 polarisations."""
    waves = [_polar_wave((j + 0.5) * np.pi / 8, pol) for j in range(8) for pol in (0, 1)]
    return Config(f"cylinder_N{16 * (8 + 4 * levels)}_M64", cylinder(levels),
                  Media.from_k(5.0, 7.5 + 0.01j), 64, 256, waves)


def config_random(n_panels: int = 64, seed: int = 1810, M: int = 128, n_phi: int = 512) -> Config:
    """Smooth random body, N = 16 n_panels, k0 = 10, k1 = 15."""
    from .configs import paper_default_wave  # noqa
    return Config(f"random{seed}_N{16 * n_panels}_M{M}", random_body(n_panels, seed),
                  Media.from_k(10.0, 15.0), M, n_phi, [paper_default_wave(), _polar_wave(np.pi / 4, 0)])


def config_batch(n_random: int = 64, n_edged: int = 8) -> list:
    """The batched workload: n_random smooth random bodies (seeds 0..n_random-1,
    the random-body generator) and n_edged edged bodies (seeds n_random..:
    cylinders, then cones, radius and half-height ~ U(0.5, 1.5)).  Per body,
    from default_rng(10000 + seed): N ~ U[200, 1200] rounded to whole panels
    (edged bodies: the nearest refinement level), M ~ U{32..128},
    k0 ~ U[1, 12], k1 = 1.5 k0; the paper's default plane wave and the
    45-degree wave.  n_phi is left to the solver (16 = smallest)."""
    waves = [paper_default_wave(), _polar_wave(np.pi / 4, 0)]
    out = []
    for s in range(n_random + n_edged):
        rng = np.random.default_rng(10000 + s)
        N = int(rng.uniform(200, 1200))
        M = int(rng.integers(32, 129))
        k0 = float(rng.uniform(1.0, 12.0))
        if s < n_random:
            curve = random_body(max(1, round(N / 16)), seed=s)
        else:
            R, h = float(rng.uniform(0.5, 1.5)), float(rng.uniform(0.5, 1.5))
            if s < n_random + (n_edged + 1) // 2:
                levels = max(1, round((N / 16 - 8) / 4))
                curve = cylinder(levels, R, h)
            else:
                levels = max(1, round((N / 16 - 6) / 3))
                curve = cone(levels, R, h)
        out.append(Config(f"batch{s}_{curve.name}_N{curve.N}_M{M}", curve, Media.from_k(k0, 1.5 * k0), M, 16,
                          list(waves)))
    return out


def config_pool(n_bodies: int = 32, seed0: int = 100) -> list:
    """The serving pool: n_bodies smooth random bodies as in config_random
    (64 panels, N = 1024, modes -128..128, 512 azimuthal samples, k0 = 10,
    k1 = 15), seeds seed0.. for the shape coefficients; every body is served
    at k0 = 10, so a (body, k0) key is the body."""
    return [Config(f"pool{s}_N1024_M128", random_body(64, seed=s), Media.from_k(10.0, 15.0), 128, 512, [])
            for s in range(seed0, seed0 + n_bodies)]
