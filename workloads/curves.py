"""Generating curves of bodies of revolution, sampled panel by panel.

A curve is handed to the solver as ``n_panels`` panels of ``p = 16`` nodes.
On each panel the local parameter tau runs over [-1, 1] and the nodes sit at
the 16 Gauss-Legendre points of tau.  For every node the generator records
r, z and their derivatives dr/dtau, dz/dtau (derivatives with respect to the
panel-local parameter, so the parameter need not be arclength; Section 6,
remark on non-arclength sampling).  Curves run counterclockwise in the
(r, z) half plane so that n = (z', -r') points out of the body (Section 3).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

P = 16  # nodes per panel (16th-order rules, Section 5)


def panel_nodes(p: int = P) -> np.ndarray:
    """Gauss-Legendre points on [-1, 1] where curve samples are placed."""
    x, _ = np.polynomial.legendre.leggauss(p)
    return x


@dataclass
class Curve:
    n_panels: int
    r: np.ndarray          # [N] node radius
    z: np.ndarray          # [N] node height
    dr: np.ndarray         # [N] dr/dtau (panel-local parameter)
    dz: np.ndarray         # [N] dz/dtau
    closed: bool = False   # closed curves (torus) wrap panel neighbours
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return self.n_panels * P


def _sample(panels, fun, closed=False, name="", meta=None) -> Curve:
    """Sample a parametric curve t -> (r, z, dr/dt, dz/dt) on the given
    panels [(t0, t1), ...], converting derivatives to the panel parameter."""
    x = panel_nodes()
    rs, zs, drs, dzs = [], [], [], []
    for (t0, t1) in panels:
        t = 0.5 * (t0 + t1) + 0.5 * (t1 - t0) * x
        r, z, drdt, dzdt = fun(t)
        jac = 0.5 * (t1 - t0)
        rs.append(r); zs.append(z); drs.append(drdt * jac); dzs.append(dzdt * jac)
    return Curve(len(panels), np.concatenate(rs), np.concatenate(zs),
                 np.concatenate(drs), np.concatenate(dzs), closed, name, meta or {})


def sphere(n_panels: int = 4, radius: float = 1.0) -> Curve:
    """Unit-sphere meridian r = sin t, z = -cos t, t in [0, pi] (equal panels).

    The z = -cos t sign makes the curve run from the south pole to the north
    pole, i.e. counterclockwise with the outward normal."""
    edges = np.linspace(0.0, np.pi, n_panels + 1)
    panels = list(zip(edges[:-1], edges[1:]))

    def fun(t):
        return (radius * np.sin(t), -radius * np.cos(t),
                radius * np.cos(t), radius * np.sin(t))
    return _sample(panels, fun, name=f"sphere{n_panels}")


def _dyadic(a: float, b: float, levels: int, toward_b: bool):
    """Split [a, b] dyadically `levels` times toward one end (Section 5)."""
    out = []
    lo, hi = a, b
    for _ in range(levels):
        mid = 0.5 * (lo + hi)
        if toward_b:
            out.append((lo, mid)); lo = mid
        else:
            out.append((mid, hi)); hi = mid
    out.append((lo, hi))
    if not toward_b:
        out.reverse()
    return out


def cylinder(levels: int = 7, radius: float = 1.0, half_height: float = 1.0,
             base=(2, 4, 2)) -> Curve:
    """Finite cylinder: bottom disk, side, top disk (vertices (0,-h), (R,-h),
    (R,h), (0,h)); panels next to the two edges are refined dyadically
    `levels` times toward the edge.  With the default 2/4/2 base panels and
    7 levels, N = 16 * (8 + 4*7) = 576."""
    R, h = radius, half_height
    segs = [((0.0, -h), (R, -h), base[0]), ((R, -h), (R, h), base[1]), ((R, h), (0.0, h), base[2])]
    # parameter s in [0, 1] along each segment; panels in s
    all_panels = []  # (segment index, s0, s1)
    for si, (_, _, nb) in enumerate(segs):
        edges = np.linspace(0.0, 1.0, nb + 1)
        pans = list(zip(edges[:-1], edges[1:]))
        refined = []
        for pi, (s0, s1) in enumerate(pans):
            at_end = (si in (0, 1)) and pi == nb - 1       # bottom->side, side->top edges
            at_start = (si in (1, 2)) and pi == 0
            if at_end:
                refined += _dyadic(s0, s1, levels, toward_b=True)
            elif at_start:
                refined += _dyadic(s0, s1, levels, toward_b=False)
            else:
                refined.append((s0, s1))
        all_panels += [(si, a, b) for (a, b) in refined]
    x = panel_nodes()
    rs, zs, drs, dzs = [], [], [], []
    widths = []
    for (si, s0, s1) in all_panels:
        (ra, za), (rb, zb), _ = segs[si]
        s = 0.5 * (s0 + s1) + 0.5 * (s1 - s0) * x
        rs.append(ra + (rb - ra) * s); zs.append(za + (zb - za) * s)
        jac = 0.5 * (s1 - s0)
        drs.append(np.full(P, (rb - ra) * jac)); dzs.append(np.full(P, (zb - za) * jac))
        widths.append(np.hypot(rb - ra, zb - za) * (s1 - s0))
    return Curve(len(all_panels), np.concatenate(rs), np.concatenate(zs),
                 np.concatenate(drs), np.concatenate(dzs), False, f"cylinder_L{levels}",
                 {"min_panel": float(min(widths))})


def cone(levels: int = 5, radius: float = 1.0, half_height: float = 1.0, base=(2, 4)) -> Curve:
    """Cone with its apex on the axis: bottom disk (0,-h) -> (R,-h), then the
    slant side (R,-h) -> (0,h).  The panels next to the rim edge (on both
    sides) and next to the apex are refined dyadically `levels` times toward
    them, so N = 16 * (base[0] + base[1] + 3 * levels)."""
    R, h = radius, half_height
    segs = [((0.0, -h), (R, -h), base[0]), ((R, -h), (0.0, h), base[1])]
    all_panels = []
    for si, (_, _, nb) in enumerate(segs):
        edges = np.linspace(0.0, 1.0, nb + 1)
        for pi, (s0, s1) in enumerate(zip(edges[:-1], edges[1:])):
            if si == 0 and pi == nb - 1:
                parts = _dyadic(s0, s1, levels, toward_b=True)            # toward the rim
            elif si == 1 and pi == 0:
                parts = _dyadic(s0, s1, levels, toward_b=False)           # from the rim
            elif si == 1 and pi == nb - 1:
                parts = _dyadic(s0, s1, levels, toward_b=True)            # toward the apex
            else:
                parts = [(s0, s1)]
            all_panels += [(si, a, b) for (a, b) in parts]
    x = panel_nodes()
    rs, zs, drs, dzs, widths = [], [], [], [], []
    for (si, s0, s1) in all_panels:
        (ra, za), (rb, zb), _ = segs[si]
        s = 0.5 * (s0 + s1) + 0.5 * (s1 - s0) * x
        rs.append(ra + (rb - ra) * s); zs.append(za + (zb - za) * s)
        jac = 0.5 * (s1 - s0)
        drs.append(np.full(P, (rb - ra) * jac)); dzs.append(np.full(P, (zb - za) * jac))
        widths.append(np.hypot(rb - ra, zb - za) * (s1 - s0))
    return Curve(len(all_panels), np.concatenate(rs), np.concatenate(zs),
                 np.concatenate(drs), np.concatenate(dzs), False, f"cone_L{levels}",
                 {"min_panel": float(min(widths))})


def random_body(n_panels: int = 64, seed: int = 1810, n_coef: int = 6, amp: float = 0.08) -> Curve:
    """Smooth random body r(t) = sin t (1 + sum_j a_j cos jt), z = -cos t,
    a_j ~ U(-amp, amp) drawn from numpy's default_rng(seed)."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(-amp, amp, n_coef)
    j = np.arange(1, n_coef + 1)

    def fun(t):
        t = np.asarray(t)
        s = 1.0 + (a[None, :] * np.cos(np.outer(t, j))).sum(1)
        ds = -(a[None, :] * j[None, :] * np.sin(np.outer(t, j))).sum(1)
        r = np.sin(t) * s
        dr = np.cos(t) * s + np.sin(t) * ds
        return r, -np.cos(t), dr, np.sin(t)
    edges = np.linspace(0.0, np.pi, n_panels + 1)
    return _sample(list(zip(edges[:-1], edges[1:])), fun, name=f"random{seed}",
                   meta={"a": a.tolist()})


def starfish(n_panels: int = 19) -> Curve:
    """Rotated starfish of Section 6 (Example 2): with R(t) = 2 + 0.5 cos(5 pi (t - 1))
    and psi = pi (t - 1/2), r = R cos psi, z = R sin psi, t in [0, 1], uniform
    panels in t."""
    edges = np.linspace(0.0, 1.0, n_panels + 1)

    def fun(t):
        t = np.asarray(t)
        R = 2.0 + 0.5 * np.cos(5 * np.pi * (t - 1.0))
        dR = -2.5 * np.pi * np.sin(5 * np.pi * (t - 1.0))
        ps = np.pi * (t - 0.5)
        return (R * np.cos(ps), R * np.sin(ps),
                dR * np.cos(ps) - np.pi * R * np.sin(ps), dR * np.sin(ps) + np.pi * R * np.cos(ps))
    return _sample(list(zip(edges[:-1], edges[1:])), fun, name=f"starfish{n_panels}")


def droplet(n_base: int = 15, levels: int = 5) -> Curve:
    """Droplet of Section 6 (Example 3): r = sin(pi t) cos(pi (t - 1.5)/2),
    z = sin(pi t) sin(pi (t - 1.5)/2) + 1/2, t in [1/2, 1] (a tip on the axis
    at t = 1); n_base uniform panels in t, the last one refined dyadically
    `levels` times toward the tip."""
    edges = np.linspace(0.5, 1.0, n_base + 1)
    panels = list(zip(edges[:-1], edges[1:]))
    panels = panels[:-1] + _dyadic(panels[-1][0], panels[-1][1], levels, toward_b=True)

    def fun(t):
        t = np.asarray(t)
        s, ds = np.sin(np.pi * t), np.pi * np.cos(np.pi * t)
        th = 0.5 * np.pi * (t - 1.5)
        return (s * np.cos(th), s * np.sin(th) + 0.5,
                ds * np.cos(th) - 0.5 * np.pi * s * np.sin(th), ds * np.sin(th) + 0.5 * np.pi * s * np.cos(th))
    out = _sample(panels, fun, name=f"droplet{n_base}_L{levels}")
    out.meta["min_panel_t"] = float(panels[-1][1] - panels[-1][0])
    return out


def torus(n_panels: int = 20, R: float = 2.0, a: float = 1.0, b: float = 0.5) -> Curve:
    """Torus meridian r = R + a cos t, z = b sin t (closed curve, Section 6.1)."""
    edges = np.linspace(0.0, 2 * np.pi, n_panels + 1)

    def fun(t):
        return R + a * np.cos(t), b * np.sin(t), -a * np.sin(t), b * np.cos(t)
    return _sample(list(zip(edges[:-1], edges[1:])), fun, closed=True, name=f"torus{n_panels}")
