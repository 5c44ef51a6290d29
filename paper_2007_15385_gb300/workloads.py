"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws inputs.  It holds none of the inclusion test's
arithmetic, and both the CUDA path (through the tests and ``bench.py``) and the
CPU oracle take their inputs from here.  Everything is numpy on the host;
seeds are numpy ``default_rng`` (PCG64) streams.

The paper tests random points around one polygon (Sec. 6.1) and times batches
of 10^6 points against polygons of 3 to 15 edges (Sec. 6.2); it names vehicle
collision checks, GIS and rasterisation as uses (Sec. 1).  The five workloads
below stand in for those uses; no dataset is involved.

  1. ``unit_circle_octagon``   8 vertices on the unit circle, 10^5 points in [-1.5, 1.5]^2.
  2. ``vehicle_footprint``     12 vertices on a 2.4 m x 1.0 m ellipse, lidar-like points:
                               60 % uniform in a 40 m square, 40 % in 200 Gaussian clusters.
  3. ``gis_batch``             4,096 polygons, 3..64 vertices on circles of log-uniform radius
                               [1, 100] centred in [0, 10^4]^2; each owns 10^3..10^5 points in
                               its bounding box scaled by 1.3.  ``gis_all_pairs`` draws 2^20
                               points from the first 1,024 polygons' point distributions.
  4. ``integer_hulls``         1,024 strictly convex integer hulls (4..32 vertices) in
                               [-2^20, 2^20]^2, 16,384 int32 points each: half in the bounding
                               box, a quarter on edges or vertices, a quarter one unit off an edge.
  5. ``footprint_trajectory``  the ellipse footprint at 256 SE(2) poses along a smooth random
                               trajectory over [0, 40]^2, 2^20 lidar-like obstacle points.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Workload:
    """Vertices as xy pairs with CSR offsets; points as xy pairs.

    ``point_offsets`` is set for own-polygon batches (polygon j owns points
    [point_offsets[j], point_offsets[j+1])) and None when every point meets
    every polygon.
    """
    name: str
    vertices: np.ndarray            # [sum n, 2] float32 or int32
    vertex_offsets: np.ndarray      # [P + 1] int32
    points: np.ndarray              # [M, 2] float32 or int32
    point_offsets: np.ndarray | None = None  # [P + 1] int64
    extra: dict = field(default_factory=dict)

    @property
    def num_polygons(self) -> int:
        return len(self.vertex_offsets) - 1

    @property
    def num_points(self) -> int:
        return len(self.points)

    def edges(self) -> np.ndarray:
        return np.diff(self.vertex_offsets).astype(np.int64)

    def tests(self) -> int:
        """Point x edge tests of the full-work convention (no early exit, no cull)."""
        n = self.edges()
        if self.point_offsets is not None:
            return int((np.diff(self.point_offsets) * n).sum())
        return int(self.num_points * n.sum())


def _strictly_convex_f32(v: np.ndarray) -> bool:
    """True when every turn of the float32 polygon is clearly to one side.

    Only an input filter: it rejects draws whose float32 rounding left a
    vertex nearly straight or reflex, with a wide relative margin so that
    rounding inside this check cannot matter.
    """
    d = v.astype(np.float64)
    e0 = d - np.roll(d, 1, axis=0)
    e1 = np.roll(d, -1, axis=0) - d
    p = e0[:, 0] * e1[:, 1]
    q = e0[:, 1] * e1[:, 0]
    cr = p - q
    tol = 1e-9 * (np.abs(p) + np.abs(q))
    return bool(np.all(cr > tol) or np.all(cr < -tol))


def _circle_polygon(rng, n, cx, cy, rx, ry, dtype=np.float32, tries=1000):
    for _ in range(tries):
        th = np.sort(rng.uniform(0.0, 2.0 * math.pi, n))
        v = np.stack([cx + rx * np.cos(th), cy + ry * np.sin(th)], axis=1).astype(dtype)
        if _strictly_convex_f32(v):
            return v
    raise RuntimeError("could not draw a strictly convex polygon")


def _lidar_points(rng, m, lo, hi, clusters=200, sigma=0.3, frac_uniform=0.6):
    mu = int(round(frac_uniform * m))
    mc = m - mu
    out = np.empty((m, 2), np.float32)
    out[:mu] = rng.uniform(lo, hi, size=(mu, 2)).astype(np.float32)
    centres = rng.uniform(lo, hi, size=(clusters, 2))
    which = rng.integers(0, clusters, size=mc)
    out[mu:] = (centres[which] + sigma * rng.standard_normal((mc, 2))).astype(np.float32)
    perm = rng.permutation(m)
    return out[perm]


def unit_circle_octagon(seed: int = 0, m: int = 100_000, n: int = 8) -> Workload:
    rng = np.random.default_rng(seed)
    v = _circle_polygon(rng, n, 0.0, 0.0, 1.0, 1.0)
    pts = rng.uniform(-1.5, 1.5, size=(m, 2)).astype(np.float32)
    return Workload("unit_circle_octagon", v, np.array([0, n], np.int32), pts)


def vehicle_footprint(seed: int = 1, m: int = 1 << 26, n: int = 12, shard: int = 0) -> Workload:
    """One footprint against m LiDAR-like points.  ``shard`` r > 0 keeps the
    footprint and draws its own points (one rank's share of a larger job);
    shard 0 is the single-GPU workload itself."""
    rng = np.random.default_rng(seed)
    v = _circle_polygon(rng, n, 0.0, 0.0, 2.4, 1.0)
    prng = rng if shard == 0 else np.random.default_rng([seed, 1000 + shard])
    pts = _lidar_points(prng, m, -20.0, 20.0)
    return Workload("vehicle_footprint", v, np.array([0, n], np.int32), pts)


def _gis_polygons(rng, P, n_range):
    ns = rng.integers(n_range[0], n_range[1] + 1, size=P)
    radii = np.exp(rng.uniform(0.0, math.log(100.0), size=P))
    centres = rng.uniform(0.0, 1e4, size=(P, 2))
    polys = [_circle_polygon(rng, int(ns[j]), centres[j, 0], centres[j, 1], radii[j], radii[j])
             for j in range(P)]
    voffs = np.zeros(P + 1, np.int32)
    voffs[1:] = np.cumsum([len(p) for p in polys])
    return polys, voffs


def _scaled_bbox(poly, scale=1.3):
    lo = poly.min(axis=0).astype(np.float64)
    hi = poly.max(axis=0).astype(np.float64)
    c = 0.5 * (lo + hi)
    h = 0.5 * (hi - lo) * scale
    return c - h, c + h


def gis_batch(seed: int = 2, num_polygons: int = 4096, m_range=(1_000, 100_000),
              n_range=(3, 64)) -> Workload:
    rng = np.random.default_rng(seed)
    polys, voffs = _gis_polygons(rng, num_polygons, n_range)
    ms = rng.integers(m_range[0], m_range[1] + 1, size=num_polygons)
    poffs = np.zeros(num_polygons + 1, np.int64)
    poffs[1:] = np.cumsum(ms)
    pts = np.empty((int(poffs[-1]), 2), np.float32)
    for j, poly in enumerate(polys):
        lo, hi = _scaled_bbox(poly)
        a, b = int(poffs[j]), int(poffs[j + 1])
        u = rng.random((b - a, 2), dtype=np.float32)
        pts[a:b] = (lo + u * (hi - lo)).astype(np.float32)
    return Workload("gis_batch", np.concatenate(polys), voffs, pts, poffs)


def gis_all_pairs(seed: int = 2, num_polygons: int = 1024, m: int = 1 << 20,
                  total_polygons: int = 4096, m_range=(1_000, 100_000),
                  n_range=(3, 64)) -> Workload:
    """The first ``num_polygons`` of the GIS batch against ``m`` shared points.

    The points follow the union of those polygons' own point distributions:
    a polygon is drawn in proportion to its point count, then a point uniform
    in its scaled bounding box.
    """
    rng = np.random.default_rng(seed)
    polys, _ = _gis_polygons(rng, total_polygons, n_range)
    ms = rng.integers(m_range[0], m_range[1] + 1, size=total_polygons)
    polys = polys[:num_polygons]
    ms = ms[:num_polygons].astype(np.float64)
    voffs = np.zeros(num_polygons + 1, np.int32)
    voffs[1:] = np.cumsum([len(p) for p in polys])
    rng2 = np.random.default_rng([seed, 1])
    owner = rng2.choice(num_polygons, size=m, p=ms / ms.sum())
    lo = np.empty((num_polygons, 2))
    hi = np.empty((num_polygons, 2))
    for j, poly in enumerate(polys):
        lo[j], hi[j] = _scaled_bbox(poly)
    u = rng2.random((m, 2))
    pts = (lo[owner] + u * (hi[owner] - lo[owner])).astype(np.float32)
    return Workload("gis_all_pairs", np.concatenate(polys), voffs, pts, None)


def _strict_hull_int(p: np.ndarray) -> np.ndarray:
    """Andrew's monotone chain on int64 points, collinear points dropped (CCW)."""
    pts = sorted(set(map(tuple, p.tolist())))
    if len(pts) < 3:
        return np.array(pts, np.int64)

    def cross(o, a, b):
        return (a[0] - o[0]) * (b[1] - o[1]) - (a[1] - o[1]) * (b[0] - o[0])

    lower, upper = [], []
    for q in pts:
        while len(lower) >= 2 and cross(lower[-2], lower[-1], q) <= 0:
            lower.pop()
        lower.append(q)
    for q in reversed(pts):
        while len(upper) >= 2 and cross(upper[-2], upper[-1], q) <= 0:
            upper.pop()
        upper.append(q)
    return np.array(lower[:-1] + upper[:-1], np.int64)


def integer_hulls(seed: int = 3, num_polygons: int = 1024, points_per_polygon: int = 16_384,
                  n_range=(4, 32), box: int = 1 << 20,
                  r_range=(2.0 ** 10, 2.0 ** 19)) -> Workload:
    rng = np.random.default_rng(seed)
    polys = []
    r_hi = min(r_range[1], box / 2.0)
    r_lo = min(r_range[0], r_hi / 4.0)
    while len(polys) < num_polygons:
        r = math.exp(rng.uniform(math.log(r_lo), math.log(r_hi)))
        c = rng.uniform(-box + r + 1, box - r - 1, size=2)
        k = int(rng.integers(n_range[0], n_range[1] + 1))
        th = rng.uniform(0.0, 2.0 * math.pi, k)
        raw = np.rint(np.stack([c[0] + r * np.cos(th), c[1] + r * np.sin(th)], axis=1))
        hull = _strict_hull_int(raw.astype(np.int64))
        if n_range[0] <= len(hull) <= n_range[1]:
            if rng.random() < 0.5:
                hull = hull[::-1]  # both orientations occur
            polys.append(hull)
    voffs = np.zeros(num_polygons + 1, np.int32)
    voffs[1:] = np.cumsum([len(p) for p in polys])
    m = points_per_polygon
    poffs = np.arange(num_polygons + 1, dtype=np.int64) * m
    pts = np.empty((num_polygons * m, 2), np.int64)
    kind = np.empty(num_polygons * m, np.int8)  # 0 in the box, 1 on an edge, 2 one unit off
    n_box = m // 2
    n_on = m // 4
    n_off = m - n_box - n_on
    for j, h in enumerate(polys):
        lo = h.min(axis=0)
        hi = h.max(axis=0)
        seg = pts[j * m:(j + 1) * m]
        seg[:n_box] = rng.integers(lo, hi + 1, size=(n_box, 2))
        # lattice points on edges: v_{k-1} + t (d / g), t in [0, g], g = gcd(|dx|, |dy|)
        e = rng.integers(0, len(h), size=n_on + n_off)
        a = h[e - 1]
        d = h[e] - a
        g = np.gcd(np.abs(d[:, 0]), np.abs(d[:, 1]))
        t = (rng.random(len(e)) * (g + 1)).astype(np.int64)
        on = a + (d // g[:, None]) * t[:, None]
        seg[n_box:n_box + n_on] = on[:n_on]
        off = on[n_on:].copy()
        axis = rng.integers(0, 2, size=n_off)
        sign = rng.choice(np.array([-1, 1]), size=n_off)
        off[np.arange(n_off), axis] += sign
        seg[n_box + n_on:] = off
        perm = rng.permutation(m)
        seg[:] = seg[perm]
        kind[j * m:(j + 1) * m] = np.repeat(np.array([0, 1, 2], np.int8),
                                            [n_box, n_on, n_off])[perm]
    verts = np.concatenate(polys).astype(np.int32)
    return Workload("integer_hulls", verts, voffs, pts.astype(np.int32), poffs,
                    extra={"kind": kind})


def _catmull_rom(knots: np.ndarray, samples: int):
    """Positions and tangents of a uniform Catmull-Rom cubic through the knots."""
    k = np.concatenate([2 * knots[:1] - knots[1:2], knots, 2 * knots[-1:] - knots[-2:-1]])
    segs = len(knots) - 1
    u = np.linspace(0.0, segs, samples, endpoint=False) + 0.5 * segs / samples
    i = np.minimum(u.astype(int), segs - 1)
    t = (u - i)[:, None]
    p0, p1, p2, p3 = k[i], k[i + 1], k[i + 2], k[i + 3]
    pos = 0.5 * ((2 * p1) + (-p0 + p2) * t + (2 * p0 - 5 * p1 + 4 * p2 - p3) * t ** 2
                 + (-p0 + 3 * p1 - 3 * p2 + p3) * t ** 3)
    tan = 0.5 * ((-p0 + p2) + 2 * (2 * p0 - 5 * p1 + 4 * p2 - p3) * t
                 + 3 * (-p0 + 3 * p1 - 3 * p2 + p3) * t ** 2)
    return pos, tan


def footprint_trajectory(seed: int = 4, m: int = 1 << 20, num_poses: int = 256,
                         n: int = 12, tau: float = 0.05) -> Workload:
    rng = np.random.default_rng(seed)
    v = _circle_polygon(rng, n, 0.0, 0.0, 2.4, 1.0)
    knots = rng.uniform(0.0, 40.0, size=(8, 2))
    pos, tan = _catmull_rom(knots, num_poses)
    heading = np.arctan2(tan[:, 1], tan[:, 0])
    poses = np.concatenate([pos, heading[:, None]], axis=1).astype(np.float32)
    pts = _lidar_points(rng, m, 0.0, 40.0)
    return Workload("footprint_trajectory", v, np.array([0, n], np.int32), pts,
                    extra={"poses": poses, "tau": tau})


def regular_polygon(n: int, r: float = 1.0, cx: float = 0.0, cy: float = 0.0,
                    phase: float = 0.0, dtype=np.float64) -> np.ndarray:
    th = phase + 2.0 * math.pi * np.arange(n) / n
    return np.stack([cx + r * np.cos(th), cy + r * np.sin(th)], axis=1).astype(dtype)


def chebyshev_centres(vertices: np.ndarray, vertex_offsets: np.ndarray) -> np.ndarray:
    """The centre of each convex polygon's largest inscribed circle, by a
    small linear programme per polygon (maximise r subject to
    a_k . x + r |a_k| <= b_k for every edge half-plane a_k . x <= b_k), as
    float64 [P, 2].  An interior point chosen without reference to the
    Voronoi method, for studies of the inner generator p0; solved about the
    vertex mean so that large coordinates stay well conditioned."""
    from scipy.optimize import linprog
    out = np.empty((len(vertex_offsets) - 1, 2))
    for j in range(len(vertex_offsets) - 1):
        v = vertices[vertex_offsets[j]:vertex_offsets[j + 1]].astype(np.float64)
        c = v.mean(axis=0)
        scale = np.abs(v - c).max()
        v = (v - c) / scale  # unit size: the solver's tolerances are absolute
        u = np.roll(v, 1, axis=0)
        e = v - u
        orient = 1.0 if (u[:, 0] * v[:, 1] - v[:, 0] * u[:, 1]).sum() > 0 else -1.0
        a = orient * np.stack([e[:, 1], -e[:, 0]], axis=1)
        b = orient * (e[:, 1] * u[:, 0] - e[:, 0] * u[:, 1])
        nrm = np.linalg.norm(a, axis=1)
        A = np.concatenate([a / nrm[:, None], np.ones((len(a), 1))], axis=1)
        r = linprog([0.0, 0.0, -1.0], A_ub=A, b_ub=b / nrm, bounds=[(None, None), (None, None), (0, None)],
                    method="highs")
        if r.status != 0:
            raise RuntimeError("Chebyshev centre of polygon %d: %s" % (j, r.message))
        out[j] = r.x[:2] * scale + c
    return out
