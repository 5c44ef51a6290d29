"""Pins for the CPU oracle: facts fixed by the paper and by plain geometry.

None of these retypes the oracle's own formula.  Each checks the oracle
against a closed form, an invariant, a hand-derived fixture, a brute force in
exact rationals, or an independent method, so that a dropped term, a wrong
sign, a wrong index or a transposed operand in oracle/pip_oracle.c fails at
least one of them (tests/test_oracle_mutants.py plants such mistakes).
"""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import exact_rational as er
from paper_2007_15385_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_derived_generators.txt")


def _read_golden():
    polys = {}
    cur = None
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            tok = line.split()
            if tok[0] == "polygon":
                cur = polys.setdefault(tok[1], {"v": [], "g": {}})
            elif tok[0] == "v":
                cur["v"].append([float(tok[1]), float(tok[2])])
            elif tok[0] == "area":
                cur["area"] = float(tok[1])
            elif tok[0] == "centroid":
                cur["c"] = [float(tok[1]), float(tok[2])]
            elif tok[0] == "g":
                cur["g"][int(tok[1])] = [float(tok[2]), float(tok[3])]
    return polys


# ---------------------------------------------------------------- Eq. 3-4, Alg. 3

@pytest.mark.parametrize("name", sorted(_read_golden()))
def test_golden_centroid_and_generators(name):
    p = _read_golden()[name]
    v = np.array(p["v"])
    area, c = oracle.centroid(v)
    assert area == pytest.approx(p["area"], abs=1e-12)
    np.testing.assert_allclose(c, p["c"], atol=1e-12)
    g = oracle.generators(v)
    for k, want in p["g"].items():
        np.testing.assert_allclose(g[k], want, atol=1e-12)


@pytest.mark.parametrize("n", [3, 4, 5, 7, 8, 12, 33, 64])
def test_regular_polygon_area_and_centre(n):
    r, cx, cy = 1.7, 3.25, -1.5
    v = wl.regular_polygon(n, r, cx, cy, phase=0.3)
    area, c = oracle.centroid(v)
    assert area == pytest.approx(0.5 * n * r * r * math.sin(2 * math.pi / n), rel=1e-12)
    np.testing.assert_allclose(c, [cx, cy], atol=1e-12)


def test_triangle_centroid_is_vertex_mean_and_orientation():
    rng = np.random.default_rng(11)
    for _ in range(50):
        v = rng.uniform(-5, 5, size=(3, 2))
        area, c = oracle.centroid(v)
        np.testing.assert_allclose(c, v.mean(axis=0), atol=1e-11)
        # shoelace by a determinant of edge vectors
        e1, e2 = v[1] - v[0], v[2] - v[0]
        assert area == pytest.approx(0.5 * (e1[0] * e2[1] - e1[1] * e2[0]), rel=1e-10)
        area_r, c_r = oracle.centroid(v[::-1])
        assert area_r == pytest.approx(-area, rel=1e-12)
        np.testing.assert_allclose(c_r, c, atol=1e-11)


def test_centroid_translation_covariance():
    rng = np.random.default_rng(12)
    v = wl.regular_polygon(9, 2.0, 0.1, 0.2, phase=0.4)
    v = v + rng.uniform(-0.2, 0.2, size=v.shape)
    _, c = oracle.centroid(v)
    for t in ([3, -7], [100, 25], [-64, 0]):
        _, ct = oracle.centroid(v + np.array(t, float))
        np.testing.assert_allclose(ct, c + np.array(t), atol=1e-9)


def test_centroid_of_polygon_with_collinear_vertex():
    # inserting a vertex in the middle of an edge changes neither area nor centroid
    v = np.array([[0, 0], [4, 0], [4, 2], [0, 2]], float)
    w = np.array([[0, 0], [2, 0], [4, 0], [4, 2], [0, 2]], float)
    a1, c1 = oracle.centroid(v)
    a2, c2 = oracle.centroid(w)
    assert a1 == pytest.approx(a2)
    np.testing.assert_allclose(c1, c2, atol=1e-14)


# ---------------------------------------------------------------- Eq. 6-8, Alg. 4

def _random_convex(rng, n, r=1.0, c=(0.0, 0.0), squash=1.0):
    th = np.sort(rng.uniform(0, 2 * math.pi, n))
    return np.stack([c[0] + r * np.cos(th), c[1] + squash * r * np.sin(th)], axis=1)


@pytest.mark.parametrize("seed", range(5))
def test_generators_involution_and_equidistance(seed):
    rng = np.random.default_rng(seed)
    v = _random_convex(rng, int(rng.integers(3, 12)), 2.0, (1.0, -3.0), 0.6)
    _, g0 = oracle.centroid(v)
    g = oracle.generators(v)
    n = len(v)
    for k in range(n):
        # mirroring g_k across the same edge line gives back g0
        back = oracle.generators(v, p0=g[k])[k]
        np.testing.assert_allclose(back, g0, atol=1e-12)
        # Eq. 7: the foot of the perpendicular (Eq. 6) is the midpoint
        f = oracle.foot(v, k, g0)
        np.testing.assert_allclose(f, 0.5 * (g0 + g[k]), atol=1e-12)
        # ... and it lies on edge line k, whose direction is orthogonal to g_k - g0
        a, b = v[k - 1], v[k]
        d = b - a
        cross = d[0] * (f[1] - a[1]) - d[1] * (f[0] - a[0])
        assert abs(cross) < 1e-12 * (1 + np.abs(d).sum() * np.abs(f).sum())
        assert abs(np.dot(d, g[k] - g0)) < 1e-12 * (1 + np.linalg.norm(d) * np.linalg.norm(g[k] - g0))
        # the edge endpoints are equidistant from g0 and g_k (Eq. 2)
        for q in (a, b, 0.5 * (a + b)):
            assert np.linalg.norm(q - g0) == pytest.approx(np.linalg.norm(q - g[k]), rel=1e-11)


@pytest.mark.parametrize("seed", range(5))
def test_voronoi_vertex_property(seed):
    # vertex v_k ends edge k and starts edge k+1, so it is equidistant from g0, g_k, g_{k+1}
    rng = np.random.default_rng(100 + seed)
    v = _random_convex(rng, int(rng.integers(3, 16)), 3.0, (-2.0, 5.0), 0.4)
    _, g0 = oracle.centroid(v)
    g = oracle.generators(v)
    n = len(v)
    for k in range(n):
        d0 = np.linalg.norm(v[k] - g0)
        assert np.linalg.norm(v[k] - g[k]) == pytest.approx(d0, rel=1e-11)
        assert np.linalg.norm(v[k] - g[(k + 1) % n]) == pytest.approx(d0, rel=1e-11)


@pytest.mark.parametrize("n", [3, 4, 6, 8, 12, 64])
def test_regular_polygon_generator_radius_and_angle(n):
    r, c = 1.3, np.array([0.5, -0.25])
    v = wl.regular_polygon(n, r, c[0], c[1], phase=0.1)
    g = oracle.generators(v)
    for k in range(n):
        rel = g[k] - c
        assert np.linalg.norm(rel) == pytest.approx(2 * r * math.cos(math.pi / n), rel=1e-12)
        mid = 0.5 * (v[k - 1] + v[k]) - c
        ang = math.atan2(rel[1], rel[0]) - math.atan2(mid[1], mid[0])
        assert abs(math.remainder(ang, 2 * math.pi)) < 1e-12


def test_generators_match_exact_rationals():
    rng = np.random.default_rng(7)
    v = _random_convex(rng, 7, 1.0, (0.25, 0.5)).astype(np.float32)
    area, c = er.centroid(v)
    gq = er.generators(v, c)
    a64, c64 = oracle.centroid(v)
    g64 = oracle.generators(v)
    assert a64 == pytest.approx(float(area), rel=1e-13)
    np.testing.assert_allclose(c64, [float(c[0]), float(c[1])], atol=1e-13)
    np.testing.assert_allclose(g64, [[float(x), float(y)] for x, y in gq], atol=1e-12)


# ---------------------------------------------------------------- Eq. 1, Alg. 5

def _boundary_and_near_points(v32, rng, count):
    """Vertices, edge points whose coordinates are exact in float32, and 1-ulp neighbours."""
    pts = [p for p in v32]
    n = len(v32)
    for _ in range(count):
        k = int(rng.integers(n))
        a, b = v32[k - 1].astype(np.float64), v32[k].astype(np.float64)
        t = rng.random()
        q = (a + t * (b - a)).astype(np.float32)
        pts.append(q)
        for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
            pts.append(np.array([np.nextafter(q[0], q[0] + dx * np.float32(1)) if dx else q[0],
                                 np.nextafter(q[1], q[1] + dy * np.float32(1)) if dy else q[1]],
                                np.float32))
    return np.array(pts, np.float32)


@pytest.mark.parametrize("seed", range(8))
def test_inside_exact_matches_exact_rational_voronoi(seed):
    rng = np.random.default_rng(200 + seed)
    n = int(rng.integers(3, 9))
    v = _random_convex(rng, n, 1.0, (0.1, -0.2), 0.7).astype(np.float32)
    if seed % 2:
        v = v[::-1].copy()
    if oracle.polygon_status(v) != oracle.OK:
        pytest.skip("draw not strictly convex in float32")
    pts = np.concatenate([
        rng.uniform(-1.2, 1.2, size=(150, 2)).astype(np.float32),
        _boundary_and_near_points(v, rng, 30),
    ])
    got, st = oracle.inside_exact(v, pts)
    assert st == oracle.OK
    want = er.voronoi_inclusion(v, pts)
    assert got.tolist() == want


def test_inside_exact_integer_matches_exact_rational_voronoi():
    rng = np.random.default_rng(300)
    w = wl.integer_hulls(seed=5, num_polygons=6, points_per_polygon=120,
                         n_range=(4, 9), box=1 << 12)
    for j in range(w.num_polygons):
        v = w.vertices[w.vertex_offsets[j]:w.vertex_offsets[j + 1]]
        p = w.points[w.point_offsets[j]:w.point_offsets[j + 1]]
        got, st = oracle.inside_exact(v, p)
        assert st == oracle.OK
        assert got.tolist() == er.voronoi_inclusion(v, p)
    del rng


def test_vertices_and_integer_edge_points_are_inside():
    w = wl.integer_hulls(seed=6, num_polygons=8, points_per_polygon=2000)
    for j in range(w.num_polygons):
        v = w.vertices[w.vertex_offsets[j]:w.vertex_offsets[j + 1]]
        got, _ = oracle.inside_exact(v, v.copy())
        assert got.all()
        sl = slice(w.point_offsets[j], w.point_offsets[j + 1])
        on = w.points[sl][w.extra["kind"][sl] == 1]
        assert len(on) == 500
        assert oracle.inside_exact(v, on)[0].all()


def test_outside_bbox_is_outside_and_centroid_inside():
    rng = np.random.default_rng(9)
    for _ in range(20):
        v = _random_convex(rng, int(rng.integers(3, 20)), 5.0, (2.0, 3.0), 0.3).astype(np.float32)
        if oracle.polygon_status(v) != oracle.OK:
            continue
        lo, hi = v.min(axis=0), v.max(axis=0)
        q = rng.uniform(lo - 10, hi + 10, size=(2000, 2)).astype(np.float32)
        out = (q < lo).any(axis=1) | (q > hi).any(axis=1)
        got, _ = oracle.inside_exact(v, q)
        assert not got[out].any()
        _, c = oracle.centroid(v)
        assert oracle.inside_exact(v, c.astype(np.float32)[None])[0][0] == 1


def test_monte_carlo_fraction_matches_shoelace_area():
    rng = np.random.default_rng(10)
    v = _random_convex(rng, 10, 1.0, (0.0, 0.0), 0.5).astype(np.float32)
    lo, hi = v.min(axis=0).astype(float), v.max(axis=0).astype(float)
    m = 200_000
    q = rng.uniform(lo, hi, size=(m, 2)).astype(np.float32)
    got, _ = oracle.inside_exact(v, q)
    area, _ = oracle.centroid(v)
    p = abs(area) / np.prod(hi - lo)
    sigma = math.sqrt(p * (1 - p) / m)
    assert abs(got.mean() - p) < 4 * sigma


def test_translation_and_rotation_invariance_integer():
    w = wl.integer_hulls(seed=8, num_polygons=4, points_per_polygon=4000, box=1 << 18)
    rot = lambda a: np.stack([-a[:, 1], a[:, 0]], axis=1)  # 90 degrees, exact on integers
    for j in range(w.num_polygons):
        v = w.vertices[w.vertex_offsets[j]:w.vertex_offsets[j + 1]]
        p = w.points[w.point_offsets[j]:w.point_offsets[j + 1]]
        base, _ = oracle.inside_exact(v, p)
        t = np.array([12345, -777], np.int32)
        assert (oracle.inside_exact(v + t, p + t)[0] == base).all()
        assert (oracle.inside_exact(rot(v), rot(p))[0] == base).all()


def test_translation_and_rotation_invariance_float():
    rng = np.random.default_rng(13)
    v = _random_convex(rng, 12, 3.0, (0.0, 0.0), 0.4).astype(np.float32)
    q = np.concatenate([rng.uniform(-4, 4, (3000, 2)).astype(np.float32),
                        _boundary_and_near_points(v, rng, 200)])
    base, _ = oracle.inside_exact(v, q)
    rot = lambda a: np.stack([-a[:, 1], a[:, 0]], axis=1)
    assert (oracle.inside_exact(rot(v), rot(q))[0] == base).all()
    # translation by a power of two that keeps every sum exact in float32
    t = np.array([64.0, -128.0], np.float32)
    vt, qt = v + t, q + t
    exact = ((vt - t) == v).all() and ((qt - t) == q).all()
    if exact:
        assert (oracle.inside_exact(vt, qt)[0] == base).all()


@pytest.mark.parametrize("seed", range(4))
def test_agreement_with_sign_of_offset_and_ray_crossing_off_boundary(seed):
    rng = np.random.default_rng(400 + seed)
    v = _random_convex(rng, int(rng.integers(3, 16)), 2.0, (1.0, 1.0), 0.8).astype(np.float32)
    if seed % 2:
        v = v[::-1].copy()
    q = rng.uniform(-2, 4, size=(20000, 2)).astype(np.float32)
    ex, _ = oracle.inside_exact(v, q)
    # distance to the nearest edge line, to keep clear of the boundary
    d = np.full(len(q), np.inf)
    for k in range(len(v)):
        a, b = v[k - 1].astype(float), v[k].astype(float)
        e = b - a
        cr = e[0] * (q[:, 1] - a[1]) - e[1] * (q[:, 0] - a[0])
        d = np.minimum(d, np.abs(cr) / np.linalg.norm(e))
    far = d > 1e-6
    rc = oracle.ray_crossing(v, q)
    assert (rc[far] == ex[far]).all()
    so = oracle.sign_of_offset(v, q)
    assert (so[far] == ex[far]).all()


def test_voronoi_fp64_agrees_with_exact_off_its_ambiguity_flag():
    w = wl.integer_hulls(seed=9, num_polygons=16, points_per_polygon=4000)
    flagged = 0
    for j in range(w.num_polygons):
        v = w.vertices[w.vertex_offsets[j]:w.vertex_offsets[j + 1]]
        p = w.points[w.point_offsets[j]:w.point_offsets[j + 1]]
        ex, _ = oracle.inside_exact(v, p)
        f64, amb, st = oracle.voronoi_fp64(v, p)
        assert st == oracle.OK
        ok = amb == 0
        assert (f64[ok] == ex[ok]).all()
        flagged += int(amb.sum())
    # on-edge and one-off points are the only ones near a tie
    assert flagged <= 0.6 * w.num_points


def test_voronoi_fp64_float_workload():
    w = wl.unit_circle_octagon(m=50_000)
    ex, _ = oracle.inside_exact(w.vertices, w.points)
    f64, amb, _ = oracle.voronoi_fp64(w.vertices, w.points)
    assert (f64[amb == 0] == ex[amb == 0]).all()
    assert amb.sum() == 0


# ---------------------------------------------------------------- validity readings

def test_polygon_status_readings():
    sq = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], float)
    assert oracle.polygon_status(sq) == oracle.OK
    assert oracle.polygon_status(sq[::-1]) == oracle.OK
    assert oracle.polygon_status(sq[:2]) == oracle.INVALID
    assert oracle.polygon_status([[0, 0], [1, 0], [1, 0], [0, 1]]) == oracle.DEGENERATE
    assert oracle.polygon_status([[0, 0], [1, 0], [2, 0]]) == oracle.DEGENERATE
    assert oracle.polygon_status([[0, 0], [2, 0], [1, 0.2], [2, 2], [0, 2]]) == oracle.NONCONVEX
    # collinear vertex: allowed
    assert oracle.polygon_status([[0, 0], [1, 0], [2, 0], [2, 2], [0, 2]]) == oracle.OK
    # spike that folds back along an edge
    assert oracle.polygon_status([[0, 0], [4, 0], [4, 4], [0, 4], [0, 6], [0, 4.5]]) != oracle.OK
    # pentagram: every turn the same way, but it winds twice
    pent = wl.regular_polygon(5, 1.0)[[0, 2, 4, 1, 3]]
    assert oracle.polygon_status(pent) == oracle.NONCONVEX
    assert oracle.polygon_status([[0, 0], [1, np.nan], [1, 1]]) == oracle.NONFINITE


def test_nan_point_is_outside():
    sq = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], np.float32)
    q = np.array([[np.nan, 0.5], [0.5, np.inf], [0.5, 0.5]], np.float32)
    got, _ = oracle.inside_exact(sq, q)
    assert got.tolist() == [0, 0, 1]


# ---------------------------------------------------------------- margin (Eq. 2)

def test_margin_axis_square_is_linf_distance():
    sq = np.array([[-1, -1], [1, -1], [1, 1], [-1, 1]], float)
    rng = np.random.default_rng(14)
    q = rng.uniform(-3, 3, size=(5000, 2))
    m = oracle.margin(sq, q)
    np.testing.assert_allclose(m, np.abs(q).max(axis=1) - 1.0, atol=1e-12)


def test_margin_zero_on_edges_and_bounded_by_euclidean_distance():
    rng = np.random.default_rng(15)
    v = _random_convex(rng, 9, 2.0, (0.5, 0.5), 0.5)
    for k in range(len(v)):
        t = rng.random()
        q = v[k - 1] + t * (v[k] - v[k - 1])
        assert abs(oracle.margin(v, q[None])[0]) < 1e-12
    q = rng.uniform(-4, 5, size=(3000, 2))
    m = oracle.margin(v, q)
    inside, _ = oracle.inside_exact(v.astype(np.float32), q.astype(np.float32))
    # outside: the largest violated line distance is at most the Euclidean distance
    # to the polygon, taken here as the distance to its nearest edge segment
    def seg_dist(p):
        best = np.inf
        for k in range(len(v)):
            a, b = v[k - 1], v[k]
            t = np.clip(np.dot(p - a, b - a) / np.dot(b - a, b - a), 0, 1)
            best = min(best, np.linalg.norm(p - (a + t * (b - a))))
        return best
    for i in range(0, 3000, 7):
        d = seg_dist(q[i])
        if m[i] > 1e-9:
            assert m[i] <= d + 1e-12
        elif m[i] < -1e-9:
            # inside: minus the margin is the distance to the nearest edge line
            assert -m[i] == pytest.approx(d, rel=1e-9, abs=1e-12)
    assert ((m <= 1e-9) | (inside == 0)).all()


# ---------------------------------------------------------------- penalty gradient

def _penalty_case(seed=16, npts=400, nposes=3):
    rng = np.random.default_rng(seed)
    v = _random_convex(rng, 7, 2.0, (0.0, 0.0), 0.5)
    poses = np.stack([rng.uniform(-0.5, 0.5, nposes), rng.uniform(-0.5, 0.5, nposes),
                      rng.uniform(-math.pi, math.pi, nposes)], axis=1)
    q = rng.uniform(-3, 3, size=(npts, 2))
    return v, poses, q


def _margin_terms(v, poses, q):
    """Per (pose, point): the top-two margin terms, to skip points near an argmax switch."""
    gaps = []
    for tx, ty, th in poses:
        c, s = math.cos(th), math.sin(th)
        u = q - [tx, ty]
        b = np.stack([c * u[:, 0] + s * u[:, 1], -s * u[:, 0] + c * u[:, 1]], axis=1)
        terms = []
        for k in range(len(v)):
            a, e = v[k - 1], v[k] - v[k - 1]
            nrm = np.array([e[1], -e[0]]) / np.linalg.norm(e)
            area, _ = oracle.centroid(v)
            nrm = nrm if area > 0 else -nrm
            terms.append((b - a) @ nrm)
        terms = np.sort(np.array(terms), axis=0)
        gaps.append(terms[-1] - terms[-2])
    return np.array(gaps)


def test_centroid_and_generator_vjps_match_central_differences():
    rng = np.random.default_rng(19)
    v = _random_convex(rng, 6, 1.5, (0.3, -0.2), 0.6)
    n = len(v)
    G0 = rng.standard_normal(2)
    Gk = rng.standard_normal((n, 2))
    p0 = oracle.centroid(v)[1] + rng.uniform(-0.1, 0.1, 2)
    dv_c = oracle.centroid_vjp(v, G0)
    dp0, dv_g = oracle.generators_vjp(v, p0, Gk)
    h = 1e-6
    f_c = lambda w: G0 @ oracle.centroid(w)[1]
    f_g = lambda w, p: (Gk * oracle.generators(w, p0=p)).sum()
    for i in range(n):
        for d in range(2):
            vp, vm = v.copy(), v.copy()
            vp[i, d] += h
            vm[i, d] -= h
            assert dv_c[i, d] == pytest.approx((f_c(vp) - f_c(vm)) / (2 * h), rel=1e-6, abs=1e-8)
            assert dv_g[i, d] == pytest.approx((f_g(vp, p0) - f_g(vm, p0)) / (2 * h), rel=1e-6, abs=1e-8)
    for d in range(2):
        pp, pm = p0.copy(), p0.copy()
        pp[d] += h
        pm[d] -= h
        assert dp0[d] == pytest.approx((f_g(v, pp) - f_g(v, pm)) / (2 * h), rel=1e-6, abs=1e-8)


def test_penalty_gradient_matches_central_differences():
    v, poses, q = _penalty_case()
    tau = 0.3
    gaps = _margin_terms(v, poses, q)
    keep = (gaps > 1e-3).all(axis=0)
    q = q[keep]
    loss, gv, gp = oracle.penalty(v, poses, q, tau)
    assert loss == pytest.approx(oracle.penalty_loss(v, poses, q, tau), rel=1e-13)
    h = 1e-6
    for i in range(v.shape[0]):
        for d in range(2):
            vp, vm = v.copy(), v.copy()
            vp[i, d] += h
            vm[i, d] -= h
            fd = (oracle.penalty_loss(vp, poses, q, tau) - oracle.penalty_loss(vm, poses, q, tau)) / (2 * h)
            assert gv[i, d] == pytest.approx(fd, rel=1e-5, abs=1e-6 * max(1.0, abs(loss)))
    for j in range(poses.shape[0]):
        for d in range(3):
            pp, pm = poses.copy(), poses.copy()
            pp[j, d] += h
            pm[j, d] -= h
            fd = (oracle.penalty_loss(v, pp, q, tau) - oracle.penalty_loss(v, pm, q, tau)) / (2 * h)
            assert gp[j, d] == pytest.approx(fd, rel=1e-5, abs=1e-6 * max(1.0, abs(loss)))


def test_penalty_vertex_gradient_equals_point_to_line_closed_form():
    """Each margin term is the distance to an edge line, which does not depend on
    the centroid: the centroid path through Eq. 3-4 and Eq. 8 must cancel, and
    the total must equal the gradient of the line distance with respect to the
    edge's two endpoints."""
    v, poses, q = _penalty_case(seed=17, npts=300, nposes=2)
    tau = 0.25
    loss, gv, _ = oracle.penalty(v, poses, q, tau)
    area, _ = oracle.centroid(v)
    sgn = 1.0 if area > 0 else -1.0
    want = np.zeros_like(v)
    for tx, ty, th in poses:
        c, s = math.cos(th), math.sin(th)
        u = q - [tx, ty]
        b = np.stack([c * u[:, 0] + s * u[:, 1], -s * u[:, 0] + c * u[:, 1]], axis=1)
        best = np.full(len(q), -np.inf)
        arg = np.zeros(len(q), int)
        for k in range(len(v)):
            a, e = v[k - 1], v[k] - v[k - 1]
            d = sgn * (e[1] * (b[:, 0] - a[0]) - e[0] * (b[:, 1] - a[1])) / np.linalg.norm(e)
            upd = d > best
            best[upd] = d[upd]
            arg[upd] = k
        gm = -1.0 / (1.0 + np.exp(best / tau)) / tau
        for i in range(len(q)):
            k = arg[i]
            a, bb = v[k - 1], v[k]
            e = bb - a
            L = np.linalg.norm(e)
            x = b[i]
            # d = sgn * (e x (x - a)) / |e| with e x w = e1 w2... written for (ex, ey)
            cr = sgn * (e[1] * (x[0] - a[0]) - e[0] * (x[1] - a[1]))
            # partials of cr wrt a and b
            dcr_da = sgn * np.array([-e[1] + (x[1] - a[1]) * 1.0 - 0.0, e[0] - (x[0] - a[0])])
            # careful derivation: cr = sgn*((by-ay)(x0-ax) - (bx-ax)(x1-ay))
            dcr_da = sgn * np.array([-(bb[1] - a[1]) + (x[1] - a[1]), -(x[0] - a[0]) + (bb[0] - a[0])])
            dcr_db = sgn * np.array([-(x[1] - a[1]), (x[0] - a[0])])
            dL_da = -e / L
            dL_db = e / L
            dd_da = dcr_da / L - cr * dL_da / L ** 2
            dd_db = dcr_db / L - cr * dL_db / L ** 2
            want[k - 1] += gm[i] * dd_da
            want[k] += gm[i] * dd_db
    np.testing.assert_allclose(gv, want, rtol=1e-9, atol=1e-9 * np.abs(want).max())


def test_penalty_translation_invariance():
    v, poses, q = _penalty_case(seed=18, npts=200, nposes=3)
    tau = 0.2
    l0, gv0, gp0 = oracle.penalty(v, poses, q, tau)
    t = np.array([5.5, -3.25])
    poses_t = poses.copy()
    poses_t[:, :2] += t
    l1, gv1, gp1 = oracle.penalty(v, poses_t, q + t, tau)
    assert l1 == pytest.approx(l0, rel=1e-12)
    np.testing.assert_allclose(gv1, gv0, rtol=1e-8, atol=1e-10)
    np.testing.assert_allclose(gp1, gp0, rtol=1e-8, atol=1e-10)


def _round_f32(fr):
    """Exact rational -> nearest float32, ties to even (checked against neighbours)."""
    from fractions import Fraction
    f = np.float32(float(fr))
    best = None
    for cand in (np.nextafter(f, np.float32(-np.inf)), f, np.nextafter(f, np.float32(np.inf))):
        d = abs(Fraction(float(cand)) - fr)
        key = (d, int(np.frombuffer(np.float32(cand).tobytes(), np.uint32)[0]) & 1)
        if best is None or key < best[0]:
            best = (key, cand)
    return best[1]


def test_raster_centres_are_one_rounding_of_the_exact_grid():
    from fractions import Fraction
    rng = np.random.default_rng(21)
    for _ in range(6):
        x0, y0 = (np.float32(v) for v in rng.uniform(-1e4, 1e4, 2))
        dx, dy = (np.float32(v) for v in rng.uniform(1e-3, 7.0, 2))
        W, H = 37, 5
        got = oracle.raster_centres(W, H, x0, y0, dx, dy).reshape(H, W, 2)
        for c in range(W):
            want = _round_f32(Fraction(c) * Fraction(float(dx)) + Fraction(float(x0)))
            assert got[0, c, 0] == want
        for r in range(H):
            want = _round_f32(Fraction(r) * Fraction(float(dy)) + Fraction(float(y0)))
            assert (got[r, :, 1] == want).all()


def _rect(x0, y0, x1, y1, cw):
    v = [[x0, y0], [x1, y0], [x1, y1], [x0, y1]]
    return v[::-1] if cw else v


def _in_rect(r, p):
    """Closed membership of points p in an axis-aligned rectangle, by plain comparisons."""
    (x0, y0, x1, y1) = r
    return (p[:, 0] >= x0) & (p[:, 0] <= x1) & (p[:, 1] >= y0) & (p[:, 1] <= y1)


def test_first_hit_and_ragged_on_rectangles_against_plain_comparisons():
    """Axis-aligned rectangles (both orientations) hold a point iff its
    coordinates lie within their bounds, closed; the first hit is the lowest
    such index.  Coordinates on a 1/16 lattice put many points exactly on
    edges and corners.  A non-convex and a zero-area polygon in the list hold
    nothing."""
    rng = np.random.default_rng(31)
    rects, polys = [], []
    for j in range(14):
        x0, y0 = (rng.integers(0, 64, 2) / 8.0)
        w, h = (rng.integers(1, 40, 2) / 8.0)
        rects.append((x0, y0, x0 + w, y0 + h))
        polys.append(_rect(x0, y0, x0 + w, y0 + h, cw=bool(j % 2)))
    bad = [[[0, 0], [8, 0], [4, 1], [8, 8], [0, 8]],  # non-convex: holds nothing
           [[0, 0], [4, 4], [8, 8]]]                   # zero area: holds nothing
    polys = polys[:5] + bad + polys[5:]
    rects = rects[:5] + [None, None] + rects[5:]
    verts = np.concatenate([np.array(p, np.float32) for p in polys])
    voffs = np.zeros(len(polys) + 1, np.int32)
    voffs[1:] = np.cumsum([len(p) for p in polys])
    pts = (rng.integers(-8, 13 * 16, size=(3000, 2)) / 16.0).astype(np.float32)
    hit = oracle.first_hit_exact(verts, voffs, pts)
    want = np.full(len(pts), -1)
    for j in range(len(polys) - 1, -1, -1):  # lowest index wins
        if rects[j] is not None:
            want[_in_rect(rects[j], pts.astype(np.float64))] = j
    np.testing.assert_array_equal(hit, want)
    assert (want >= 0).sum() > 500 and (want == -1).sum() > 100
    # ragged: each polygon against its own points, drawn on the 1/16 lattice
    # of its rectangle widened by 1/8 (most inside, many on the boundary)
    counts = rng.integers(0, 300, size=len(polys))
    poffs = np.zeros(len(polys) + 1, np.int64)
    poffs[1:] = np.cumsum(counts)
    own = np.empty((int(poffs[-1]), 2), np.float32)
    for j in range(len(polys)):
        x0, y0, x1, y1 = rects[j] if rects[j] is not None else (0.0, 0.0, 8.0, 8.0)
        ix = rng.integers(int(x0 * 16) - 2, int(x1 * 16) + 3, size=counts[j])
        iy = rng.integers(int(y0 * 16) - 2, int(y1 * 16) + 3, size=counts[j])
        own[poffs[j]:poffs[j + 1]] = np.stack([ix, iy], axis=1) / 16.0
    got, _ = oracle.inside_exact_ragged(verts, voffs, own, poffs)
    assert got.mean() > 0.5
    for j in range(len(polys)):
        sl = slice(poffs[j], poffs[j + 1])
        exp = np.zeros(counts[j], bool) if rects[j] is None else _in_rect(rects[j], own[sl].astype(np.float64))
        np.testing.assert_array_equal(got[sl].astype(bool), exp)
