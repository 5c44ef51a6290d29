"""The parallel oracle helpers give exactly the serial oracle's answers."""
import numpy as np

import oracle
import oracle_par
from paper_2007_15385_gb300 import workloads as wl


def test_inside_exact_pieces_equal_one_call():
    w = wl.vehicle_footprint(m=50_003)
    want, _ = oracle.inside_exact(w.vertices, w.points)
    assert np.array_equal(oracle_par.inside_exact(w.vertices, w.points), want)


def test_ragged_groups_equal_one_call():
    for w in (wl.gis_batch(seed=21, num_polygons=37, m_range=(0, 900)),
              wl.integer_hulls(seed=5, num_polygons=9, points_per_polygon=500)):
        want, _ = oracle.inside_exact_ragged(w.vertices, w.vertex_offsets, w.points, w.point_offsets)
        got = oracle_par.inside_exact_ragged(w.vertices, w.vertex_offsets, w.points, w.point_offsets)
        assert np.array_equal(got, want)


def test_first_hit_pieces_equal_one_call():
    w = wl.gis_all_pairs(num_polygons=40, m=7_001)
    want = oracle.first_hit_exact(w.vertices, w.vertex_offsets, w.points)
    assert np.array_equal(oracle_par.first_hit_exact(w.vertices, w.vertex_offsets, w.points), want)
