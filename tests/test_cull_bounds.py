"""The inequalities the culls and the disc filter rest on, checked with the
CPU oracle's fp64 geometry (no GPU).

* Penalty cull: with w_k the unit outward normals of a convex polygon, H the
  largest distance from p0 to an edge line and theta the largest angle
  between consecutive normals, the margin (the largest signed distance from
  the Eq. 2 bisectors, i.e. the edge lines) satisfies
  m(x) >= cos(theta / 2) |x - p0| - H.
* Disc filter: a point nearer p0 than the least distance from p0 to an edge
  line is inside (margin < 0); a point farther from p0 than every vertex is
  outside (margin > 0).
"""
import numpy as np

import oracle
from paper_2007_15385_gb300 import workloads as wl


def _polygons():
    yield wl.footprint_trajectory().vertices
    for n in (3, 4, 5, 8, 12, 17, 40, 64):
        yield wl.unit_circle_octagon(seed=900 + n, m=1, n=n).vertices
    g = wl.gis_batch(seed=901, num_polygons=40, m_range=(1, 2))
    for j in range(g.num_polygons):
        yield g.vertices[g.vertex_offsets[j]:g.vertex_offsets[j + 1]]


def _frame(v):
    _, p0 = oracle.centroid(v)
    gk = oracle.generators(v, p0)
    u = gk - p0
    d = np.linalg.norm(u, axis=1)
    w = u / d[:, None]
    cosines = (np.roll(w, 1, axis=0) * w).sum(1)
    kappa = np.sqrt(0.5 * (1.0 + cosines.min()))
    return p0, kappa, d / 2.0


def test_penalty_cull_lower_bound_on_the_margin():
    rng = np.random.default_rng(5)
    for v in _polygons():
        p0, kappa, dist = _frame(v)
        ext = np.abs(v.astype(np.float64) - p0).max()
        # points from inside the polygon to far outside, in every direction
        r = ext * rng.uniform(0.0, 30.0, 20000) ** 1.5 / 10.0
        th = rng.uniform(0.0, 2.0 * np.pi, r.size)
        pts = p0 + np.stack([r * np.cos(th), r * np.sin(th)], axis=1)
        m = oracle.margin(v, pts.astype(np.float32))
        x = pts.astype(np.float32).astype(np.float64)
        bound = kappa * np.linalg.norm(x - p0, axis=1) - dist.max()
        slack = 1e-9 * (np.abs(bound) + ext)
        assert np.all(m >= bound - slack), "margin below kappa |x - p0| - H"


def test_disc_filter_discs_about_p0():
    rng = np.random.default_rng(6)
    for v in _polygons():
        p0, _, dist = _frame(v)
        vd = v.astype(np.float64)
        r_in = dist.min()
        r_out = np.linalg.norm(vd - p0, axis=1).max()
        th = rng.uniform(0.0, 2.0 * np.pi, 4000)
        for radius, sign in ((r_in * (1.0 - 1e-6), -1.0), (r_out * (1.0 + 1e-6), 1.0)):
            rr = radius * rng.uniform(0.0, 1.0, th.size) if sign < 0 else radius * rng.uniform(1.0, 3.0, th.size)
            pts = (p0 + np.stack([rr * np.cos(th), rr * np.sin(th)], axis=1)).astype(np.float32)
            x = pts.astype(np.float64)
            keep = (np.linalg.norm(x - p0, axis=1) < r_in) if sign < 0 else (np.linalg.norm(x - p0, axis=1) > r_out)
            m = oracle.margin(v, pts)[keep]
            assert keep.sum() > 100
            assert np.all(m * sign > 0), "a point of the %s disc decided the other way" % (
                "inner" if sign < 0 else "outer")
