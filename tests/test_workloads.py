"""The seeded input generators match the recipe the design notes state for
each workload (shapes, value ranges, mixtures, convexity) and are
deterministic.  CPU only; small sizes of the same generators."""
import math

import numpy as np
import pytest

import oracle
from paper_2007_15385_gb300 import workloads as wl


def _polys(w):
    for j in range(len(w.vertex_offsets) - 1):
        yield w.vertices[w.vertex_offsets[j]:w.vertex_offsets[j + 1]]


def _twice_area(v):
    v = np.asarray(v, np.float64)
    return float(np.sum(v[:, 0] * np.roll(v[:, 1], -1) - np.roll(v[:, 0], -1) * v[:, 1]))


@pytest.mark.parametrize("gen, kw", [
    (wl.unit_circle_octagon, {"m": 1000}),
    (wl.vehicle_footprint, {"m": 1000}),
    (wl.gis_batch, {"num_polygons": 12, "m_range": (10, 200)}),
    (wl.gis_all_pairs, {"num_polygons": 12, "m": 1000}),
    (wl.integer_hulls, {"num_polygons": 6, "points_per_polygon": 64}),
    (wl.footprint_trajectory, {"m": 1000, "num_poses": 16}),
])
def test_generators_are_deterministic_and_convex(gen, kw):
    a, b = gen(**kw), gen(**kw)
    np.testing.assert_array_equal(a.vertices, b.vertices)
    np.testing.assert_array_equal(a.points, b.points)
    for v in _polys(a):
        assert oracle.polygon_status(v) == oracle.OK
    c = gen(seed=99, **kw)
    assert not np.array_equal(a.points, c.points)


def test_unit_circle_octagon_recipe():
    w = wl.unit_circle_octagon(m=20_000)
    assert w.vertices.dtype == np.float32 and w.vertices.shape == (8, 2)
    np.testing.assert_allclose(np.hypot(w.vertices[:, 0], w.vertices[:, 1]), 1.0, atol=1e-6)
    ang = np.arctan2(w.vertices[:, 1].astype(np.float64), w.vertices[:, 0].astype(np.float64)) % (2 * math.pi)
    assert np.all(np.diff(ang) > 0)  # sorted angles: counter-clockwise
    assert w.points.shape == (20_000, 2) and np.abs(w.points).max() <= 1.5


def test_vehicle_footprint_recipe():
    w = wl.vehicle_footprint(m=200_000)
    v = w.vertices.astype(np.float64)
    assert w.vertices.shape == (12, 2)
    np.testing.assert_allclose((v[:, 0] / 2.4) ** 2 + v[:, 1] ** 2, 1.0, atol=1e-5)  # on the 2.4 x 1.0 ellipse
    p = w.points.astype(np.float64)
    assert w.points.dtype == np.float32 and np.abs(p).max() <= 25.0
    # 40 % of the points sit in 200 tight clusters: on a 0.5 m grid of the
    # 40 m square the densest 10 % of the cells hold about a third of all
    # points (uniform points alone would put ~10 % there)
    cells = np.floor((p + 25.0) / 0.5).astype(np.int64)  # clusters spill a little past the square
    counts = np.bincount(cells[:, 0] * 128 + cells[:, 1], minlength=128 * 128).reshape(128, 128)
    inner = np.sort(counts[10:90, 10:90].ravel())[::-1]
    top = inner[:len(inner) // 10].sum() / len(p)
    assert 0.28 < top < 0.45
    # shuffled: no long run of points from one cluster
    d = np.hypot(*(p[1:] - p[:-1]).T)
    assert np.median(d) > 5.0
    # shards keep the footprint and draw their own points
    s1 = wl.vehicle_footprint(m=1000, shard=1)
    np.testing.assert_array_equal(s1.vertices, wl.vehicle_footprint(m=1000).vertices)


def test_gis_batch_recipe():
    w = wl.gis_batch(num_polygons=200, m_range=(1000, 3000))
    n = np.diff(w.vertex_offsets)
    assert n.min() >= 3 and n.max() <= 64
    m = np.diff(w.point_offsets)
    assert m.min() >= 1000 and m.max() <= 3000 and w.point_offsets[-1] == len(w.points)
    for j, v in enumerate(_polys(w)):
        c = v.astype(np.float64).mean(axis=0)
        assert np.all((c >= 0) & (c <= 1e4 + 100))
        r = np.hypot(*(v - c).T).max()
        assert 0.5 <= r <= 110.0
        # points uniform in the bounding box scaled by 1.3 about its centre
        q = w.points[w.point_offsets[j]:w.point_offsets[j + 1]].astype(np.float64)
        lo, hi = v.min(axis=0).astype(np.float64), v.max(axis=0).astype(np.float64)
        mid, half = (lo + hi) / 2, (hi - lo) / 2 * 1.3
        assert np.all(np.abs(q - mid) <= half * (1 + 1e-5) + 1e-3)


def test_gis_all_pairs_recipe():
    w = wl.gis_all_pairs(num_polygons=20, m=5000)
    assert len(w.vertex_offsets) == 21 and w.point_offsets is None and len(w.points) == 5000
    # the polygons are the first ones of the 4,096-polygon batch (drawn before
    # the point counts, so a batch with one point per polygon has the same ones)
    b = wl.gis_batch(m_range=(1, 1))
    np.testing.assert_array_equal(w.vertices, b.vertices[:w.vertex_offsets[-1]])


def test_integer_hulls_recipe():
    w = wl.integer_hulls(num_polygons=12, points_per_polygon=4096)
    assert w.vertices.dtype == np.int32 and w.points.dtype == np.int32
    n = np.diff(w.vertex_offsets)
    assert n.min() >= 4 and n.max() <= 32
    assert np.abs(w.vertices).max() <= 2 ** 20 and np.abs(w.points).max() <= 2 ** 20 + 1
    signs = {np.sign(_twice_area(v)) for v in _polys(w)}
    assert signs == {-1.0, 1.0} or len(list(_polys(w))) < 4  # both orientations occur
    assert np.all(np.diff(w.point_offsets) == 4096)
    # a quarter of each polygon's points lie exactly on its boundary: the
    # exact predicate holds them inside, and one unit off most of them is out
    inside, st = oracle.inside_exact_ragged(w.vertices, w.vertex_offsets, w.points, w.point_offsets)
    frac_in = inside.mean()
    assert 0.35 < frac_in < 0.95


def test_footprint_trajectory_recipe():
    w = wl.footprint_trajectory(m=4000, num_poses=64)
    P = w.extra["poses"].astype(np.float64)
    assert P.shape == (64, 3) and w.extra["tau"] == 0.05
    assert np.all((P[:, :2] >= -5) & (P[:, :2] <= 45))
    assert np.all(np.abs(P[:, 2]) <= math.pi + 1e-6)
    # heading follows the path: consecutive poses move roughly along it
    step = P[1:, :2] - P[:-1, :2]
    along = step[:, 0] * np.cos(P[:-1, 2]) + step[:, 1] * np.sin(P[:-1, 2])
    assert np.mean(along > 0) > 0.9
    assert np.abs(w.points).max() <= 45 and w.vertices.shape == (12, 2)
