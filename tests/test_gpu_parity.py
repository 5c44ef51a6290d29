"""GPU parity: libpip (through the C ABI) against the CPU oracle.

Masks and first-hit ids must be bit-exact against exact closed-polygon
membership (oracle.inside_exact / first_hit_exact) on every point: small
cases and the full-size workloads alike, the latter in the launch
configuration the benchmark times, with the oracle spread over every host
core (tests/oracle_par.py).
"""
import math

import numpy as np
import pytest
import torch

import oracle
import oracle_par
from paper_2007_15385_gb300 import binding as B
from paper_2007_15385_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

GUARD = 64
GUARD_WORD = -0x21524111  # 0xDEADBEEF as int32


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.lib()
    yield


def dev():
    return torch.device("cuda:0")


def guarded(n_words, dtype=torch.int32):
    buf = torch.full((n_words + 2 * GUARD,), GUARD_WORD, dtype=dtype, device=dev())
    return buf, buf[GUARD:GUARD + n_words]


def check_guards(buf):
    g = buf.cpu().numpy()
    assert (g[:GUARD] == GUARD_WORD).all() and (g[-GUARD:] == GUARD_WORD).all(), "guard zone written"


def run_test(w, mode=B.PIP_MASK, points_offset=0):
    """Runs pip_test on workload w; returns (inside uint8[M] or None, first_hit or None, refine)."""
    v = torch.from_numpy(np.ascontiguousarray(w.vertices)).to(dev())
    vo = torch.from_numpy(np.ascontiguousarray(w.vertex_offsets)).to(dev())
    M = w.num_points
    flat = np.zeros(2 * (M + points_offset), w.points.dtype)
    flat[2 * points_offset:] = w.points.reshape(-1)
    pbuf = torch.from_numpy(flat).to(dev())
    p = pbuf[2 * points_offset:]
    po = None
    if w.point_offsets is not None:
        po = torch.from_numpy(np.ascontiguousarray(w.point_offsets)).to(dev())
    t = B.pip_prepare(v, vo, max_points=M)
    nwords = (M + 31) // 32
    mbuf, mask = guarded(nwords)
    hbuf = hit = None
    if mode & B.PIP_FIRST_HIT:
        hbuf, hit = guarded(M)
    B.pip_test(t, p, po, mode=mode, mask=mask if mode & B.PIP_MASK else None, first_hit=hit)
    st, refine = B.pip_get_status(t)
    inside = None
    if mode & B.PIP_MASK:
        check_guards(mbuf)
        words = mask.cpu().numpy().view(np.uint32)
        if M % 32:
            assert words[-1] >> (M % 32) == 0, "bits past num_points must be 0"
        inside = np.unpackbits(words.view(np.uint8), bitorder="little")[:M]
    fh = None
    if hit is not None:
        check_guards(hbuf)
        fh = hit.cpu().numpy()
    t.close()
    return inside, fh, refine, st


def oracle_own(w):
    if w.point_offsets is None:
        out, st = oracle.inside_exact(w.vertices, w.points)
        return out
    out, st = oracle.inside_exact_ragged(w.vertices, w.vertex_offsets, w.points, w.point_offsets)
    return out


def assert_same(got, want, what):
    bad = np.nonzero(got != want)[0]
    assert len(bad) == 0, "%s: %d mismatches, first at %s" % (what, len(bad), bad[:10].tolist())


# ----------------------------------------------------------------- small, every point

def test_octagon_full_size():
    w = wl.unit_circle_octagon()
    got, _, refine, st = run_test(w)
    assert st == B.PIP_OK
    assert_same(got, oracle_own(w), "octagon")


@pytest.mark.parametrize("n", list(range(3, 16)))
def test_paper_sweep_polygons(n):
    """The polygons of the paper's edge-count sweep (n = 3..15, random angles on
    the unit circle, points around it), as bench.py's paper_sweep times them."""
    w = wl.unit_circle_octagon(seed=100 + n, m=60_001, n=n)
    got, _, _, st = run_test(w)
    assert st == B.PIP_OK
    assert_same(got, oracle_own(w), "sweep n=%d" % n)


@pytest.mark.parametrize("m", [1, 31, 33, 63, 64, 65, 257, 100_003])
def test_vehicle_footprint_ragged_tails(m):
    w = wl.vehicle_footprint(m=m)
    got, _, _, _ = run_test(w)
    assert_same(got, oracle_own(w), "footprint m=%d" % m)


def test_vehicle_footprint_million_unaligned_points():
    # points start 8 bytes past a 16-byte boundary: the non-vector load path
    w = wl.vehicle_footprint(m=1_000_003)
    got, _, _, _ = run_test(w, points_offset=1)
    assert_same(got, oracle_own(w), "footprint unaligned")


def test_empty_point_set():
    w = wl.vehicle_footprint(m=0)
    got, _, refine, st = run_test(w)
    assert got.size == 0 and refine == 0


def test_gis_batch_small():
    w = wl.gis_batch(seed=12, num_polygons=64, m_range=(100, 5000))
    got, _, refine, st = run_test(w)
    assert st == B.PIP_OK
    assert_same(got, oracle_own(w), "gis small")


def test_gis_batch_with_empty_and_tiny_polygons():
    w = wl.gis_batch(seed=13, num_polygons=40, m_range=(0, 70))
    got, _, _, _ = run_test(w)
    assert_same(got, oracle_own(w), "gis tiny")


@pytest.mark.parametrize("ints", [False, True])
def test_batch_with_more_polygons_than_one_pass_of_the_setup_kernels(ints):
    """12,000 polygons: the one-block item prefix takes 12 passes of 1,024
    polygons, and the item fill (one warp per polygon, at most 8 blocks of 8
    warps per SM) loops over the polygons."""
    if ints:
        w = wl.integer_hulls(seed=62, num_polygons=12000, points_per_polygon=24)
    else:
        w = wl.gis_batch(seed=61, num_polygons=12000, m_range=(0, 40))
    got, _, _, st = run_test(w)
    assert st == B.PIP_OK
    assert_same(got, oracle_own(w), "12,000 polygons")


def test_gis_batch_unaligned_points():
    # points 8 bytes past a 16-byte boundary: the batch runs without bulk copies
    w = wl.gis_batch(seed=17, num_polygons=48, m_range=(10, 3000))
    got, _, _, st = run_test(w, points_offset=1)
    assert st == B.PIP_OK
    assert_same(got, oracle_own(w), "gis unaligned")


@pytest.mark.parametrize("n", [4, 12, 16, 40])
def test_every_stream_variant_matches_the_oracle_and_autotune_picks_one(n):
    # every tile shape of the one-polygon kernel, for each edge-count variant
    # (registers up to 16 edges, shared memory above), ragged tail included
    rng = np.random.default_rng(70 + n)
    v = wl._circle_polygon(rng, n, 0.5, -0.25, 2.4, 1.0)
    pts = rng.uniform(-3.0, 3.0, size=(200_003, 2)).astype(np.float32)
    w = wl.Workload("variants", v, np.array([0, n], np.int32), pts)
    want = oracle_own(w)
    t = B.pip_prepare(torch.from_numpy(v).to(dev()), torch.from_numpy(w.vertex_offsets).to(dev()),
                      max_points=w.num_points)
    p = torch.from_numpy(pts).to(dev())
    mbuf, mask = guarded((w.num_points + 31) // 32)
    for var in range(B.pip_stream_variant_count()):
        B.pip_set_stream_variant(t, var)
        mask.fill_(-1)
        B.pip_test(t, p, mask=mask)
        st, _ = B.pip_get_status(t)
        assert st == B.PIP_OK
        check_guards(mbuf)
        got = np.unpackbits(mask.cpu().numpy().view(np.uint8), bitorder="little")[:w.num_points]
        assert_same(got, want, "stream variant %d, %d edges" % (var, n))
    best, ms = B.pip_autotune_stream(t, p, mask, reps=2)
    assert 0 <= best < B.pip_stream_variant_count() and ms > 0
    t.close()


def test_every_stream_variant_at_many_tiles_per_cta():
    # enough points that every CTA of the one-polygon kernel streams many
    # tiles (more than any variant's L2 prefetch distance) and ends on a
    # ragged, odd tail
    w = wl.vehicle_footprint(m=12_000_001)
    want = oracle_par.inside_exact(w.vertices, w.points)
    t = B.pip_prepare(torch.from_numpy(w.vertices).to(dev()), torch.from_numpy(w.vertex_offsets).to(dev()),
                      max_points=w.num_points)
    p = torch.from_numpy(w.points).to(dev())
    mbuf, mask = guarded((w.num_points + 31) // 32)
    for var in range(B.pip_stream_variant_count()):
        B.pip_set_stream_variant(t, var)
        mask.fill_(-1)
        B.pip_test(t, p, mask=mask)
        st, _ = B.pip_get_status(t)
        assert st == B.PIP_OK
        check_guards(mbuf)
        got = np.unpackbits(mask.cpu().numpy().view(np.uint8), bitorder="little")[:w.num_points]
        assert_same(got, want, "stream variant %d, 12,000,001 points" % var)
    t.close()


@pytest.mark.parametrize("ints", [False, True])
def test_every_batch_variant_matches_the_oracle_and_autotune_picks_one(ints):
    w = (wl.integer_hulls(seed=20, num_polygons=24, points_per_polygon=2000) if ints
         else wl.gis_batch(seed=21, num_polygons=40, m_range=(0, 9000)))
    want = oracle_own(w)
    dev_ = dev()
    t = B.pip_prepare(torch.from_numpy(w.vertices).to(dev_), torch.from_numpy(w.vertex_offsets).to(dev_),
                      max_points=w.num_points)
    p = torch.from_numpy(w.points).to(dev_)
    po = torch.from_numpy(w.point_offsets).to(dev_)
    mbuf, mask = guarded((w.num_points + 31) // 32)
    for v in range(B.pip_batch_variant_count()):
        B.pip_set_batch_variant(t, v)
        mask.fill_(-1)
        B.pip_test(t, p, po, mask=mask)
        st, _ = B.pip_get_status(t)
        assert st == B.PIP_OK
        check_guards(mbuf)
        got = np.unpackbits(mask.cpu().numpy().view(np.uint8), bitorder="little")[:w.num_points]
        assert_same(got, want, "batch variant %d" % v)
    best, ms = B.pip_autotune_batch(t, p, po, mask, reps=2)
    assert 0 <= best < B.pip_batch_variant_count() and ms > 0
    t.close()


def test_ragged_invalid_polygons_hold_nothing():
    sq = [[0, 0], [4, 0], [4, 4], [0, 4]]
    polys = [sq, [[0, 0], [2, 0], [1, 0.2], [2, 2], [0, 2]], [[0, 0], [1, 0], [2, 0]], sq,
             [[0, 0], [1, 0], [1, 0], [0, 1]], sq]
    verts = np.concatenate([np.array(p, np.float32) for p in polys])
    voffs = np.zeros(len(polys) + 1, np.int32)
    voffs[1:] = np.cumsum([len(p) for p in polys])
    rng = np.random.default_rng(18)
    counts = [5000, 37, 4100, 3, 900, 6000]  # shared mask words between neighbours
    poffs = np.zeros(len(polys) + 1, np.int64)
    poffs[1:] = np.cumsum(counts)
    pts = rng.uniform(-1, 5, size=(int(poffs[-1]), 2)).astype(np.float32)
    w = wl.Workload("invalid_ragged", verts, voffs, pts, poffs)
    got, _, _, st = run_test(w)
    want = oracle_own(w)
    assert_same(got, want, "ragged invalid")
    for j in (1, 2, 4):
        assert not got[poffs[j]:poffs[j + 1]].any()


def test_ragged_offsets_that_do_not_cover_the_points_are_rejected():
    w = wl.gis_batch(seed=19, num_polygons=8, m_range=(100, 400))
    v = torch.from_numpy(w.vertices).to(dev())
    vo = torch.from_numpy(w.vertex_offsets).to(dev())
    t = B.pip_prepare(v, vo, max_points=w.num_points)
    bad = w.point_offsets.copy()
    bad[-1] -= 1  # the last offset must be the number of points
    B.pip_test(t, torch.from_numpy(w.points).to(dev()), torch.from_numpy(bad).to(dev()))
    worst, _ = B.pip_get_status(t)
    assert worst == B.PIP_E_INVALID_ARG
    t.close()


def test_all_pairs_first_hit_small():
    w = wl.gis_all_pairs(seed=14, num_polygons=96, m=30_011, total_polygons=96)
    got, fh, refine, st = run_test(w, mode=B.PIP_MASK | B.PIP_FIRST_HIT)
    want = oracle.first_hit_exact(w.vertices, w.vertex_offsets, w.points)
    assert_same(fh, want, "first hit")
    assert_same(got, (want >= 0).astype(np.uint8), "all-pairs mask")


@pytest.mark.parametrize("ints", [False, True])
def test_all_pairs_culled_first_hit(ints):
    if ints:
        h = wl.integer_hulls(seed=31, num_polygons=40, points_per_polygon=700)
        w = wl.Workload("int_all_pairs", h.vertices, h.vertex_offsets, h.points, None)
    else:
        w = wl.gis_all_pairs(seed=32, num_polygons=96, m=40_003, total_polygons=96)
    got, fh, refine, st = run_test(w, mode=B.PIP_MASK | B.PIP_FIRST_HIT | B.PIP_CULL)
    want = oracle.first_hit_exact(w.vertices, w.vertex_offsets, w.points)
    assert_same(fh, want, "culled first hit")
    assert_same(got, (want >= 0).astype(np.uint8), "culled mask")


def test_all_pairs_mask_only():
    w = wl.gis_all_pairs(seed=15, num_polygons=40, m=5_000, total_polygons=40)
    got, _, _, _ = run_test(w, mode=B.PIP_MASK)
    want = oracle.first_hit_exact(w.vertices, w.vertex_offsets, w.points)
    assert_same(got, (want >= 0).astype(np.uint8), "all-pairs mask only")


def test_integer_hulls_small():
    w = wl.integer_hulls(seed=16, num_polygons=48, points_per_polygon=3000)
    want = oracle_own(w)
    # 16-byte aligned points: decided exactly in the batch kernel, nothing refined
    got, _, refine, st = run_test(w)
    assert st == B.PIP_OK
    assert_same(got, want, "integer hulls, exact batch kernel")
    assert refine == 0
    # 8-byte aligned points: float32 filter, then the int64 refine, where the
    # on-edge and one-off points dominate the queue
    got, _, refine, st = run_test(w, points_offset=1)
    assert st == B.PIP_OK
    assert_same(got, want, "integer hulls, filter and refine")
    assert refine > 0.2 * w.num_points


def test_integer_points_beyond_float_range():
    v = np.array([[-1000, -1000], [1000, -1000], [1000, 1000], [-1000, 1000]], np.int32)
    pts = np.array([[0, 0], [1000, 0], [1001, 0], [2 ** 30, 5], [-2 ** 31, 0], [2 ** 31 - 1, 2 ** 31 - 1],
                    [1000, 1000], [-1000, -1001]], np.int32)
    w = wl.Workload("big", v, np.array([0, 4], np.int32), pts)
    got, _, _, _ = run_test(w)
    assert_same(got, oracle_own(w), "big ints")


def test_ragged_integer_points_at_the_int32_limits():
    # the batch refine's int64 test: a fast path for |p| < 2^30 and a general
    # one beyond; points at both sides of that limit and at the int32 extremes,
    # many exactly on edges (integer polygons, integer points)
    sq = np.array([[-1000, -1000], [1000, -1000], [1000, 1000], [-1000, 1000]], np.int32)
    tri = np.array([[0, 0], [2 ** 24, 0], [0, 2 ** 24]], np.int32)
    big = 2 ** 30
    extreme = [[0, 0], [1000, 0], [1001, 0], [big - 1, 5], [big, 5], [-big, 0], [-big - 1, 0],
               [-2 ** 31, 0], [2 ** 31 - 1, 2 ** 31 - 1], [1000, 1000], [-1000, -1001], [0, -1000]]
    rng = np.random.default_rng(60)
    on_edge = np.stack([rng.integers(0, 2 ** 24, 500), np.zeros(500, np.int64)], 1)
    diag = rng.integers(0, 2 ** 24, 500)
    on_hyp = np.stack([diag, 2 ** 24 - diag], 1)
    pts_sq = np.array(extreme * 3, np.int64)
    pts_tri = np.concatenate([np.array(extreme, np.int64), on_edge, on_hyp, on_hyp + [0, 1], on_hyp - [1, 0]])
    pts = np.concatenate([pts_sq, pts_tri]).astype(np.int32)
    verts = np.concatenate([sq, tri])
    voffs = np.array([0, 4, 7], np.int32)
    poffs = np.array([0, len(pts_sq), len(pts)], np.int64)
    w = wl.Workload("int_limits", verts, voffs, pts, poffs)
    want = oracle_own(w)
    got, _, refine, st = run_test(w)  # exact in the batch kernel
    assert st == B.PIP_OK and refine == 0
    assert_same(got, want, "int32 limits, exact batch")
    got, _, refine, st = run_test(w, points_offset=1)  # filter and refine
    assert st == B.PIP_OK and refine > 1000
    assert_same(got, want, "int32 limits, filter and refine")


@pytest.mark.parametrize("shape", ["footprint", "needle"])
def test_single_bound_around_the_l1_ball_and_far_away(shape):
    """The one-polygon kernel decides with one bound per polygon when prepare
    proves it valid (a convex polygon whose smallest angle and generator
    distances are not tiny) and with the per-point bound otherwise (the needle:
    a 1e-6 rad vertex).  Points just beyond each vertex (where |x| + |y| leaves
    the vertices' L1 ball), along rays out to huge distances, and on a grid."""
    rng = np.random.default_rng(61)
    if shape == "footprint":
        v = wl.vehicle_footprint(m=16).vertices
    else:
        v = np.array([[0, 0], [1000, 0], [1000, 0.001]], np.float32)
    c = v.astype(np.float64).mean(0)
    pts = []
    for p in v.astype(np.float64):
        d = p - c
        for s in (1 + 2.0 ** -np.arange(1, 24)).tolist() + [1 - 2.0 ** -20, 1.0, 1.5, 3.0]:
            pts.append(c + s * d)
            pts.append(c + s * d + rng.normal(0, 1e-6, 2) * np.abs(d).max())
    for ang in rng.uniform(0, 2 * np.pi, 200):
        for r in (10.0, 1e3, 1e6, 1e12, 1e30):
            pts.append(c + r * np.array([np.cos(ang), np.sin(ang)]))
    big = np.float32(3.4e38)
    pts += [[big, big], [-big, big], [big, 0], [0, -big]]
    lo, hi = v.min(0) - 1.0, v.max(0) + 1.0
    pts += list(rng.uniform(lo, hi, size=(50_000, 2)))
    w = wl.Workload("l1ball", v, np.array([0, len(v)], np.int32), np.array(pts, np.float32))
    got, _, _, st = run_test(w)
    assert_same(got, oracle_own(w), "single bound, %s" % shape)


@pytest.mark.parametrize("chunks", [1, 3, 8])
def test_host_call_in_pieces_matches_the_oracle(chunks):
    w = wl.vehicle_footprint(m=1_000_003)
    t = B.pip_prepare(torch.from_numpy(w.vertices).to(dev()), torch.from_numpy(w.vertex_offsets).to(dev()),
                      max_points=w.num_points)
    ph = torch.from_numpy(w.points).pin_memory()
    pd = torch.empty(w.points.shape, dtype=torch.float32, device=dev())
    nw = (w.num_points + 31) // 32
    md = torch.empty(nw, dtype=torch.int32, device=dev())
    mh = torch.full((nw,), -1, dtype=torch.int32).pin_memory()
    B.pip_test_host(t, ph, pd, md, mh, chunks=chunks)
    torch.cuda.synchronize()
    words = mh.numpy().view(np.uint32)
    assert words[-1] >> (w.num_points % 32) == 0
    got = np.unpackbits(words.view(np.uint8), bitorder="little")[:w.num_points]
    assert_same(got, oracle_own(w), "host call, %d pieces" % chunks)
    t.close()


def test_host_call_all_pairs_and_integer_points():
    """pip_test_host through the C ABI for several polygons (inside any) and
    for integer points, against the oracle."""
    w = wl.gis_all_pairs(num_polygons=30, m=50_011)
    ints = wl.integer_hulls(seed=24, num_polygons=1, points_per_polygon=40_000)
    for v, vo, pts, want in ((w.vertices, w.vertex_offsets, w.points,
                              (oracle.first_hit_exact(w.vertices, w.vertex_offsets, w.points) >= 0).astype(np.uint8)),
                             (ints.vertices, ints.vertex_offsets, ints.points, oracle_own(ints))):
        t = B.pip_prepare(torch.from_numpy(v).to(dev()), torch.from_numpy(vo).to(dev()), max_points=len(pts))
        ph = torch.from_numpy(pts).pin_memory()
        pd = torch.empty(pts.shape, dtype=ph.dtype, device=dev())
        nw = (len(pts) + 31) // 32
        md = torch.empty(nw, dtype=torch.int32, device=dev())
        mh = torch.full((nw,), -1, dtype=torch.int32).pin_memory()
        B.pip_test_host(t, ph, pd, md, mh, chunks=5)
        torch.cuda.synchronize()
        got = np.unpackbits(mh.numpy().view(np.uint8), bitorder="little")[:len(pts)]
        assert_same(got, want, "host call")
        t.close()


def test_nonfinite_points_are_outside():
    v = wl.regular_polygon(6, 1.0).astype(np.float32)
    pts = np.array([[0, 0], [np.nan, 0], [0, np.inf], [-np.inf, np.inf], [np.inf, np.inf],
                    [np.nan, np.nan], [0.5, 0.1]], np.float32)
    w = wl.Workload("nan", v, np.array([0, 6], np.int32), pts)
    got, _, _, _ = run_test(w)
    assert got.tolist() == [1, 0, 0, 0, 0, 0, 1]


@pytest.mark.parametrize("n", [3, 4, 5, 17, 33, 63, 64])
@pytest.mark.parametrize("cw", [False, True])
def test_vertex_counts_and_orientation(n, cw):
    rng = np.random.default_rng(n)
    v = wl._circle_polygon(rng, n, 3.0, -2.0, 1.7, 0.9)
    if cw:
        v = v[::-1].copy()
    pts = rng.uniform(-1, 6, size=(20_000, 2)).astype(np.float32) + np.array([0, -5], np.float32)
    w = wl.Workload("n", v, np.array([0, n], np.int32), pts)
    got, _, _, st = run_test(w)
    assert st == B.PIP_OK
    assert_same(got, oracle_own(w), "n=%d cw=%s" % (n, cw))


def _edge_sweep(v, rng, per_edge=200, ulps=3):
    out = [v]
    n = len(v)
    for k in range(n):
        a, b = v[k - 1].astype(np.float64), v[k].astype(np.float64)
        t = rng.random(per_edge)
        q = (a + t[:, None] * (b - a)).astype(np.float32)
        out.append(q)
        for dx in range(-ulps, ulps + 1):
            for dy in range(-ulps, ulps + 1):
                if dx == 0 and dy == 0:
                    continue
                qq = q.copy()
                for _ in range(abs(dx)):
                    qq[:, 0] = np.nextafter(qq[:, 0], np.float32(np.sign(dx) * np.inf))
                for _ in range(abs(dy)):
                    qq[:, 1] = np.nextafter(qq[:, 1], np.float32(np.sign(dy) * np.inf))
                out.append(qq)
    return np.concatenate(out).astype(np.float32)


@pytest.mark.parametrize("centre", [(0.0, 0.0), (1e4, -3e3), (1e6, 1e6)])
def test_ulp_sweep_around_edges(centre):
    rng = np.random.default_rng(17)
    v = wl._circle_polygon(rng, 9, centre[0], centre[1], 2.5, 1.0)
    pts = _edge_sweep(v, rng)
    w = wl.Workload("ulp", v, np.array([0, len(v)], np.int32), pts)
    got, _, refine, st = run_test(w)
    assert st == B.PIP_OK
    assert_same(got, oracle_own(w), "ulp sweep at %s" % (centre,))
    assert refine > 0


def test_sliver_polygons_exact_or_rejected():
    rng = np.random.default_rng(18)
    for s in (1e-2, 1e-4, 1e-6):
        v = np.array([[0, 0], [1000, 0], [2000, s * 1000], [1000, s * 2000]], np.float32)
        if oracle.polygon_status(v) != oracle.OK:
            continue
        pts = np.concatenate([_edge_sweep(v, rng, 50, 2),
                              rng.uniform([-10, -1], [2010, 25], size=(5000, 2)).astype(np.float32)])
        w = wl.Workload("sliver", v, np.array([0, 4], np.int32), pts)
        got, _, _, st = run_test(w)
        if st == B.PIP_OK:
            assert_same(got, oracle_own(w), "sliver %g" % s)
        else:
            assert st == B.PIP_E_DEGENERATE and not got.any()


def test_invalid_polygons_report_status_and_hold_nothing():
    sq = [[0, 0], [4, 0], [4, 4], [0, 4]]
    polys = [
        sq,                                           # ok
        [[0, 0], [2, 0], [1, 0.2], [2, 2], [0, 2]],   # non-convex
        [[0, 0], [1, 0], [1, 0], [0, 1]],             # repeated vertex
        [[0, 0], [1, 0], [2, 0]],                     # zero area
        [[0, 0], [1, np.nan], [1, 1]],                # NaN vertex
        list(wl.regular_polygon(5, 1.0)[[0, 2, 4, 1, 3]]),  # winds twice
        sq,
    ]
    verts = np.concatenate([np.array(p, np.float32) for p in polys])
    voffs = np.zeros(len(polys) + 1, np.int32)
    voffs[1:] = np.cumsum([len(p) for p in polys])
    v = torch.from_numpy(verts).to(dev())
    vo = torch.from_numpy(voffs).to(dev())
    t = B.pip_prepare(v, vo, max_points=1000)
    st = B.pip_get_polygon_status(t)
    want = [oracle.polygon_status(np.array(p, np.float64)) for p in polys]
    assert st.tolist() == want
    worst, _ = B.pip_get_status(t)
    assert worst == max(want)
    # every point is offered to every polygon: only the two squares hold any
    pts = np.array([[1, 1], [0.5, 0.5], [3, 3], [0, 0]], np.float32)
    _, fh = B.pip_test(t, torch.from_numpy(pts).to(dev()), mode=B.PIP_FIRST_HIT | B.PIP_MASK)
    assert fh.cpu().numpy().tolist() == [0, 0, 0, 0]
    t.close()


def test_polygon_vertex_count_limits():
    v = torch.from_numpy(wl.regular_polygon(70, 1.0).astype(np.float32)).to(dev())
    vo = torch.tensor([0, 2, 70], dtype=torch.int32, device=dev())
    t = B.pip_prepare(v, vo, max_points=10)
    st = B.pip_get_polygon_status(t)
    assert st.tolist() == [B.PIP_E_INVALID_ARG, B.PIP_E_INVALID_ARG]
    t.close()


def test_capacity_is_enforced():
    w = wl.vehicle_footprint(m=100)
    v = torch.from_numpy(w.vertices).to(dev())
    vo = torch.from_numpy(w.vertex_offsets).to(dev())
    t = B.pip_prepare(v, vo, max_points=50)
    p = torch.from_numpy(w.points).to(dev())
    with pytest.raises(B.PipError) as e:
        B.pip_test(t, p)
    assert e.value.status == B.PIP_E_CAPACITY
    t.close()


def test_prepare_tables_match_oracle():
    w = wl.gis_batch(seed=19, num_polygons=50, m_range=(1, 2))
    v = torch.from_numpy(w.vertices).to(dev())
    vo = torch.from_numpy(w.vertex_offsets).to(dev())
    t = B.pip_prepare(v, vo, max_points=1)
    tab = B.pip_export_tables(t)
    for j in range(w.num_polygons):
        vv = w.vertices[w.vertex_offsets[j]:w.vertex_offsets[j + 1]]
        area, c = oracle.centroid(vv)
        g = oracle.generators(vv, c)
        scale = np.abs(vv).max() + 1.0
        np.testing.assert_allclose(tab["g0"][j], c, atol=1e-12 * scale, rtol=0)
        gk = tab["gk"][w.vertex_offsets[j]:w.vertex_offsets[j + 1]]
        np.testing.assert_allclose(gk, g, atol=1e-10 * scale, rtol=0)
        o = tab["origin"][j].astype(np.float64)
        np.testing.assert_allclose(o, c, rtol=2 ** -23)
        cf = tab["coef"][w.vertex_offsets[j]:w.vertex_offsets[j + 1]].astype(np.float64)
        wk = 2 * (g - c)
        tk = ((g - o) ** 2).sum(1) - ((c - o) ** 2).sum()
        tol_w = 2 ** -22 * np.abs(wk).max() + 1e-9 * scale
        np.testing.assert_allclose(cf[:, :2], wk, atol=tol_w, rtol=0)
        np.testing.assert_allclose(cf[:, 2], tk, atol=2 ** -22 * np.abs(tk).max() + 1e-9 * scale ** 2, rtol=0)
    t.close()


def test_margin_matches_oracle():
    w = wl.vehicle_footprint(m=50_001)
    v = torch.from_numpy(w.vertices).to(dev())
    vo = torch.from_numpy(w.vertex_offsets).to(dev())
    p = torch.from_numpy(w.points).to(dev())
    t = B.pip_prepare(v, vo, max_points=w.num_points)
    got = B.pip_margin(t, p).cpu().numpy().astype(np.float64)
    want = oracle.margin(w.vertices, w.points)
    # float32 evaluation relative to o: a few ulps of |x| and |t|
    tol = 8 * 2 ** -24 * (np.abs(w.points).max(axis=1) + 4.0)
    assert np.all(np.abs(got - want) <= tol)
    # sign agrees with the exact mask wherever the margin is clearly away from 0
    inside = oracle_own(w)
    far = np.abs(want) > 1e-5
    assert ((want[far] <= 0) == inside[far].astype(bool)).all()
    t.close()


@pytest.mark.parametrize("ints", [False, True])
def test_margin_pipelined_equals_register_streaming(ints):
    """16-byte aligned points take the pipelined margin kernel, points 8 bytes
    past a boundary the register-streaming one; both evaluate the same float32
    terms in the same order, so the margins are identical, and within the
    float32 bound of the oracle.  70,001 points: 18 tiles and an odd last
    point outside the bulk copies."""
    if ints:
        h = wl.integer_hulls(seed=63, num_polygons=1, points_per_polygon=70_001)
        verts, pts = h.vertices, h.points
    else:
        w = wl.vehicle_footprint(m=70_001, seed=64)
        verts, pts = w.vertices, w.points
    M = len(pts)
    t = B.pip_prepare(torch.from_numpy(verts).to(dev()), torch.tensor([0, len(verts)], dtype=torch.int32,
                                                                      device=dev()), max_points=M)
    flat = torch.from_numpy(np.ascontiguousarray(pts).reshape(-1)).to(dev())
    shifted = torch.zeros(2 * M + 2, dtype=flat.dtype, device=dev())
    shifted[2:] = flat
    assert flat.data_ptr() % 16 == 0 and shifted[2:].data_ptr() % 16 == 8
    a = B.pip_margin(t, flat).cpu().numpy()
    b = B.pip_margin(t, shifted[2:]).cpu().numpy()
    np.testing.assert_array_equal(a.view(np.uint32), b.view(np.uint32))
    want = oracle.margin(verts, pts)
    # float32 terms relative to o: a few ulps of |x| and of the edge offsets
    tol = 16 * 2 ** -24 * (np.abs(np.asarray(pts, np.float64)).max(axis=1) + 2 * np.abs(verts).max() + 4.0)
    assert np.all(np.abs(a.astype(np.float64) - want) <= tol)
    t.close()


@pytest.mark.parametrize("M", [1, 2, 3, 33, 4095, 4097])
def test_margin_pipelined_small_and_ragged_sizes(M):
    """Point counts around one slice and one tile, odd and even, on the
    pipelined margin kernel: identical to the register-streaming kernel."""
    w = wl.vehicle_footprint(m=M, seed=66)
    t = B.pip_prepare(torch.from_numpy(w.vertices).to(dev()), torch.from_numpy(w.vertex_offsets).to(dev()),
                      max_points=M)
    flat = torch.from_numpy(np.ascontiguousarray(w.points).reshape(-1)).to(dev())
    shifted = torch.zeros(2 * M + 2, dtype=flat.dtype, device=dev())
    shifted[2:] = flat
    a = B.pip_margin(t, flat).cpu().numpy()
    b = B.pip_margin(t, shifted[2:]).cpu().numpy()
    np.testing.assert_array_equal(a.view(np.uint32), b.view(np.uint32))
    want = oracle.margin(w.vertices, w.points)
    tol = 16 * 2 ** -24 * (np.abs(w.points.astype(np.float64)).max(axis=1) + 2 * np.abs(w.vertices).max() + 4.0)
    assert np.all(np.abs(a.astype(np.float64) - want) <= tol)
    t.close()


def test_margin_ragged_and_all_pairs():
    w = wl.gis_batch(seed=20, num_polygons=30, m_range=(10, 3000))
    v = torch.from_numpy(w.vertices).to(dev())
    vo = torch.from_numpy(w.vertex_offsets).to(dev())
    p = torch.from_numpy(w.points).to(dev())
    po = torch.from_numpy(w.point_offsets).to(dev())
    t = B.pip_prepare(v, vo, max_points=w.num_points)
    got = B.pip_margin(t, p, po).cpu().numpy().astype(np.float64)
    for j in range(w.num_polygons):
        sl = slice(w.point_offsets[j], w.point_offsets[j + 1])
        vv = w.vertices[w.vertex_offsets[j]:w.vertex_offsets[j + 1]]
        want = oracle.margin(vv, w.points[sl])
        tol = 16 * 2 ** -24 * (np.abs(w.points[sl] - vv.mean(0)).max(axis=1) + np.abs(vv).max() * 1e-3 + 1.0) * 64
        assert np.all(np.abs(got[sl] - want) <= tol), j
    # all pairs: the smallest margin over the polygons
    sub = w.points[:2000]
    allm = B.pip_margin(t, torch.from_numpy(sub).to(dev())).cpu().numpy()
    want = np.min([oracle.margin(w.vertices[w.vertex_offsets[j]:w.vertex_offsets[j + 1]], sub)
                   for j in range(w.num_polygons)], axis=0)
    np.testing.assert_allclose(allm, want, atol=0.05, rtol=1e-4)
    t.close()


def _distance_to_edges(v, q):
    d = np.full(len(q), np.inf)
    for k in range(len(v)):
        a, b = v[k - 1].astype(float), v[k].astype(float)
        e = b - a
        cr = e[0] * (q[:, 1] - a[1]) - e[1] * (q[:, 0] - a[0])
        d = np.minimum(d, np.abs(cr) / np.linalg.norm(e))
    return d


def _float32_decidable(verts, pts, chunk=1 << 18):
    """Points at which the float32 comparators must agree with the oracle's
    fp64 Alg. 1 / Alg. 2: for every edge k the cross product
    c = (q_y - y_{k-1}) dV_x - (q_x - x_{k-1}) dV_y lies farther from 0 than
    16 u (|q_y dV_x| + |q_x dV_y| + |y_{k-1} dV_x| + |x_{k-1} dV_y|), u = 2^-24,
    a bound on the float32 evaluation error of LHS - RHS (either form)."""
    v = np.asarray(verts, np.float64)
    vm = np.roll(v, 1, axis=0)
    dv = v - vm
    out = np.empty(len(pts), bool)
    for a in range(0, len(pts), chunk):
        q = np.asarray(pts[a:a + chunk], np.float64)
        lhs = q[:, 1:2] * dv[:, 0] - q[:, 0:1] * dv[:, 1]
        rhs = vm[:, 1] * dv[:, 0] - vm[:, 0] * dv[:, 1]
        bound = 2.0 ** -20 * (np.abs(q[:, 1:2] * dv[:, 0]) + np.abs(q[:, 0:1] * dv[:, 1])
                              + np.abs(vm[:, 1] * dv[:, 0]) + np.abs(vm[:, 0] * dv[:, 1]))
        out[a:a + chunk] = (np.abs(lhs - rhs) > bound).all(axis=1)
    return out


def _comparator_checks(got_by_name, verts, pts):
    """Element-by-element checks of the three comparators on one polygon's
    points; returns the number of points left out by the float32 band."""
    ok32 = _float32_decidable(verts, pts)
    want = {"pip_test_sign_of_offset": oracle.sign_of_offset(verts, pts),
            "pip_test_ray_crossing": oracle.ray_crossing(verts, pts)}
    for name in want:
        assert_same(got_by_name[name][ok32], want[name][ok32], name + " vs the oracle's literal listing")
    isin, amb, st = oracle.voronoi_fp64(verts, pts)
    keep = amb == 0
    assert_same(got_by_name["pip_test_voronoi_fp64"][keep], isin[keep], "fp64 Alg. 5 vs the oracle's")
    return int((~ok32).sum())


COMPARATORS = (B.pip_test_sign_of_offset, B.pip_test_ray_crossing, B.pip_test_voronoi_fp64)


def test_comparators_match_the_oracle_listings():
    w = wl.vehicle_footprint(m=300_001)
    v = torch.from_numpy(w.vertices).to(dev())
    vo = torch.from_numpy(w.vertex_offsets).to(dev())
    p = torch.from_numpy(w.points).to(dev())
    t = B.pip_prepare(v, vo, max_points=w.num_points)
    got = {fn.__name__: B.unpack_mask(fn(t, p), w.num_points).cpu().numpy() for fn in COMPARATORS}
    left_out = _comparator_checks(got, w.vertices, w.points)
    assert left_out < w.num_points // 1000
    t.close()


def test_comparators_ragged_match_the_oracle_listings():
    w = wl.gis_batch(seed=21, num_polygons=20, m_range=(50, 2000))
    v = torch.from_numpy(w.vertices).to(dev())
    vo = torch.from_numpy(w.vertex_offsets).to(dev())
    p = torch.from_numpy(w.points).to(dev())
    po = torch.from_numpy(w.point_offsets).to(dev())
    t = B.pip_prepare(v, vo, max_points=w.num_points)
    got = {fn.__name__: B.unpack_mask(fn(t, p, po), w.num_points).cpu().numpy() for fn in COMPARATORS}
    left_out = 0
    for j in range(w.num_polygons):
        a, b = w.point_offsets[j], w.point_offsets[j + 1]
        vv = w.vertices[w.vertex_offsets[j]:w.vertex_offsets[j + 1]]
        left_out += _comparator_checks({k: g[a:b] for k, g in got.items()}, vv, w.points[a:b])
    # coordinates near 10^4 and polygons of radius 1..100: the float32 band
    # around the smallest polygons is a few percent of their points
    assert left_out < w.num_points // 10
    t.close()


@pytest.mark.parametrize("n", [3, 8, 13, 16, 40])
@pytest.mark.parametrize("offset", [0, 1])
def test_comparators_every_edge_count_and_alignment(n, offset):
    """Sign of offset, ray crossing and fp64 Alg. 5 on one polygon: the
    pipelined kernel's register variants (up to 16 edges), its shared-memory
    variant (40 edges), and the register-streaming kernel for points that are
    8 but not 16 bytes aligned; element by element against the oracle."""
    w = wl.unit_circle_octagon(seed=200 + n, m=70_001, n=n)
    v = torch.from_numpy(w.vertices).to(dev())
    vo = torch.from_numpy(w.vertex_offsets).to(dev())
    flat = np.zeros(2 * (w.num_points + offset), np.float32)
    flat[2 * offset:] = w.points.reshape(-1)
    p = torch.from_numpy(flat).to(dev())[2 * offset:]
    t = B.pip_prepare(v, vo, max_points=w.num_points)
    got = {fn.__name__: B.unpack_mask(fn(t, p), w.num_points).cpu().numpy() for fn in COMPARATORS}
    left_out = _comparator_checks(got, w.vertices, w.points)
    assert left_out < w.num_points // 100
    t.close()


def test_comparators_ragged_replay_from_a_cuda_graph():
    w = wl.gis_batch(seed=23, num_polygons=40, m_range=(0, 3000))
    v = torch.from_numpy(w.vertices).to(dev())
    vo = torch.from_numpy(w.vertex_offsets).to(dev())
    p = torch.from_numpy(w.points).to(dev())
    po = torch.from_numpy(w.point_offsets).to(dev())
    t = B.pip_prepare(v, vo, max_points=w.num_points)
    for fn in COMPARATORS:
        eager = B.unpack_mask(fn(t, p, po), w.num_points).cpu().numpy()
        out = torch.zeros((w.num_points + 31) // 32, dtype=torch.int32, device=dev())
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            fn(t, p, po, mask=out)
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            fn(t, p, po, mask=out)
        out.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert_same(B.unpack_mask(out, w.num_points).cpu().numpy(), eager, fn.__name__ + " graph replay")
    t.close()


def _early_cases():
    yield "footprint, 12 edges", wl.vehicle_footprint(seed=50, m=1_000_003)
    for n in (3, 5, 16, 40):
        yield "%d-gon" % n, wl.unit_circle_octagon(seed=300 + n, m=200_001, n=n)
    hull = wl.integer_hulls(seed=51, num_polygons=1, points_per_polygon=100_000)
    yield "integer points, float polygon", wl.Workload("h", hull.vertices.astype(np.float32),
                                                       hull.vertex_offsets, hull.points)
    yield "gis batch", wl.gis_batch(seed=52, num_polygons=60, m_range=(0, 20_000))
    yield "integer batch", wl.integer_hulls(seed=53, num_polygons=20, points_per_polygon=5_000)


def test_early_exit_equals_full_work_and_the_oracle():
    """PIP_EARLY_EXIT stops a warp once all its points are decided outside;
    the masks must be those of the full-work test and of the oracle."""
    for name, w in _early_cases():
        v = torch.from_numpy(w.vertices).to(dev())
        vo = torch.from_numpy(w.vertex_offsets).to(dev())
        p = torch.from_numpy(w.points).to(dev())
        po = torch.from_numpy(w.point_offsets).to(dev()) if w.point_offsets is not None else None
        t = B.pip_prepare(v, vo, max_points=w.num_points)
        full, _ = B.pip_test(t, p, po)
        early, _ = B.pip_test(t, p, po, mode=B.PIP_MASK | B.PIP_EARLY_EXIT)
        got_full = B.unpack_mask(full, w.num_points).cpu().numpy()
        got_early = B.unpack_mask(early, w.num_points).cpu().numpy()
        assert_same(got_early, got_full, name + ": early exit vs full work")
        assert_same(got_early, oracle_own(w), name + ": early exit vs the oracle")
        t.close()


def _sliver(seed, width):
    # a thin triangle 500 long at coordinates ~1e3 (float32 ulp 6e-5): the
    # thinner ones put o = float32(p0) within ulps of the long edges
    rng = np.random.default_rng(seed)
    a = rng.uniform(-1e3, 1e3, 2)
    d = rng.normal(size=2)
    d /= np.linalg.norm(d)
    v = np.array([a, a + 500.0 * d, a + 250.0 * d + width * np.array([-d[1], d[0]])], np.float32)
    return v


def test_disc_bounds_hold_exactly():
    """The disc thresholds, in exact rationals: tout >= R^2 (1 + u)^4 with R
    the largest distance from o to a vertex, and tin <= r^2 (1 - u)^4 with r
    the least distance from o to an edge line, o strictly inside (tin > 0);
    (1 +- u)^4 bounds the kernels' rounding of d2 = fl(x x + fl(y y)) of
    x = fl(p - o).  Invalid polygons hold (0, -inf)."""
    from fractions import Fraction as Fr
    u = Fr(1, 1 << 24)
    polys = [wl.vehicle_footprint(seed=60, m=2), wl.gis_batch(seed=61, num_polygons=300, m_range=(1, 2)),
             wl.integer_hulls(seed=62, num_polygons=60, points_per_polygon=2)]
    sl = [_sliver(70 + i, wd) for i, wd in enumerate((1e-2, 3e-3, 1e-3, 3e-4, 2e-4, 1e-4, 1e-4, 1e-4))]
    polys.append(wl.Workload("slivers", np.concatenate(sl), np.arange(0, 3 * len(sl) + 1, 3, dtype=np.int32),
                             np.zeros((1, 2), np.float32)))
    polys.append(wl.Workload("invalid", np.array([[0, 0], [1, 0], [2, 0], [0, 0], [1, 1], [0, 1]], np.float32),
                             np.array([0, 3, 6], np.int32), np.zeros((1, 2), np.float32)))
    seen_inner = seen_no_inner = 0
    for w in polys:
        t = B.pip_prepare(torch.from_numpy(w.vertices).to(dev()), torch.from_numpy(w.vertex_offsets).to(dev()),
                          max_points=1)
        ex = B.pip_export_tables(t)
        status = B.pip_get_polygon_status(t)
        t.close()
        for j in range(w.num_polygons):
            tin, tout = (float(x) for x in ex["disc"][j])
            if status[j] != B.PIP_OK:
                assert tin == 0.0 and tout == -math.inf
                continue
            vv = [(Fr(float(x)), Fr(float(y))) for x, y in w.vertices[w.vertex_offsets[j]:w.vertex_offsets[j + 1]]]
            ox, oy = Fr(float(ex["origin"][j][0])), Fr(float(ex["origin"][j][1]))
            R2 = max((x - ox) ** 2 + (y - oy) ** 2 for x, y in vv)
            assert Fr(tout) >= R2 * (1 + u) ** 4, (w.name, j)
            if tin == 0.0:
                seen_no_inner += 1
                continue
            seen_inner += 1
            area2 = sum(vv[k - 1][0] * vv[k][1] - vv[k][0] * vv[k - 1][1] for k in range(len(vv)))
            sigma = 1 if area2 > 0 else -1
            for k in range(len(vv)):
                (xm, ym), (xk, yk) = vv[k - 1], vv[k]
                a, b = yk - ym, xm - xk
                L = a * (ox - xk) + b * (oy - yk)
                assert -sigma * L > 0, (w.name, j, k)
                assert Fr(tin) <= L * L / (a * a + b * b) * (1 - u) ** 4, (w.name, j, k)
    assert seen_inner > 300


def _disc_points(w, rng):
    """The workload's points plus points at the two thresholds' radii (a few
    ulps either side, many directions), o itself, the vertices, edge
    midpoints and non-finite or huge coordinates."""
    t = B.pip_prepare(torch.from_numpy(w.vertices).to(dev()), torch.from_numpy(w.vertex_offsets).to(dev()),
                      max_points=1)
    ex = B.pip_export_tables(t)
    t.close()
    o = ex["origin"][0].astype(np.float64)
    tin, tout = (float(x) for x in ex["disc"][0])
    th = rng.uniform(0, 2 * np.pi, 4096)
    extra = [w.points.astype(np.float32)]
    for T in (tin, tout):
        if T > 0 and np.isfinite(T):
            for f in (1 - 8e-7, 1 - 1e-7, 1.0, 1 + 1e-7, 1 + 8e-7):
                r = math.sqrt(T) * f
                extra.append(np.stack([o[0] + r * np.cos(th), o[1] + r * np.sin(th)], 1).astype(np.float32))
    v = w.vertices.astype(np.float64)
    extra.append(v.astype(np.float32))
    extra.append(((v + np.roll(v, -1, 0)) / 2).astype(np.float32))
    extra.append(np.array([o, [np.nan, 0], [0, np.inf], [-np.inf, 1], [1e30, -1e30], [3e38, 3e38]], np.float32))
    pts = np.concatenate(extra).astype(np.float32)
    return wl.Workload(w.name, w.vertices, w.vertex_offsets, rng.permutation(pts))


def _disc_cases():
    rng = np.random.default_rng(57)
    yield "footprint, 12 edges", _disc_points(wl.vehicle_footprint(seed=58, m=1_000_003), rng)
    for n in (3, 5, 8, 16, 17, 40, 64):
        yield "%d-gon" % n, _disc_points(wl.unit_circle_octagon(seed=310 + n, m=200_001, n=n), rng)
    far = wl.unit_circle_octagon(seed=330, m=300_001, n=12)
    far = wl.Workload("off origin", far.vertices * 3.0 + np.float32(5000.0), far.vertex_offsets,
                      far.points * 3.0 + np.float32(5000.0))
    yield "12-gon away from the origin", _disc_points(far, rng)
    yield "sliver", _disc_points(wl.Workload("sliver", _sliver(80, 1e-2), np.array([0, 3], np.int32),
                                             rng.uniform(-1e3, 1e3, (300_001, 2)).astype(np.float32)), rng)
    hull = wl.integer_hulls(seed=59, num_polygons=1, points_per_polygon=300_001)
    pts = hull.points.copy()
    pts[::97] = rng.integers(-(1 << 30), 1 << 30, size=pts[::97].shape)  # beyond float32's exact integers
    yield "integer points", wl.Workload("h", hull.vertices.astype(np.float32), hull.vertex_offsets, pts)


def test_disc_filter_equals_full_work_and_the_oracle():
    """PIP_DISC decides the points inside the inner disc or outside the outer
    one without their edges; the masks must be those of the full-work test
    and of the oracle, at and around both thresholds and on the odd tail."""
    for name, w in _disc_cases():
        v = torch.from_numpy(w.vertices).to(dev())
        vo = torch.from_numpy(w.vertex_offsets).to(dev())
        p = torch.from_numpy(np.ascontiguousarray(w.points)).to(dev())
        t = B.pip_prepare(v, vo, max_points=w.num_points)
        full, _ = B.pip_test(t, p)
        disc, _ = B.pip_test(t, p, mode=B.PIP_MASK | B.PIP_DISC)
        st, _ = B.pip_get_status(t)
        assert st == B.PIP_OK
        got_full = B.unpack_mask(full, w.num_points).cpu().numpy()
        got_disc = B.unpack_mask(disc, w.num_points).cpu().numpy()
        assert_same(got_disc, got_full, name + ": disc filter vs full work")
        assert_same(got_disc, oracle_own(w), name + ": disc filter vs the oracle")
        with pytest.raises(RuntimeError):
            B.pip_test(t, p, mode=B.PIP_MASK | B.PIP_DISC | B.PIP_EARLY_EXIT)
        t.close()


def _batch_disc_cases():
    rng = np.random.default_rng(61)
    g = wl.gis_batch(seed=62, num_polygons=80, m_range=(0, 20_000))
    yield "gis batch", g
    # the same polygons with points on both radii of every polygon, its
    # vertices and a few non-finite points, each polygon's own range
    ex_t = B.pip_prepare(torch.from_numpy(g.vertices).to(dev()), torch.from_numpy(g.vertex_offsets).to(dev()),
                         max_points=1)
    ex = B.pip_export_tables(ex_t)
    ex_t.close()
    pts, offs = [], [0]
    for j in range(g.num_polygons):
        o = ex["origin"][j].astype(np.float64)
        tin, tout = (float(x) for x in ex["disc"][j])
        th = rng.uniform(0, 2 * np.pi, 300)
        own = [g.points[g.point_offsets[j]:g.point_offsets[j + 1]]]
        for T in (tin, tout):
            if T > 0:
                for f in (1 - 4e-7, 1.0, 1 + 4e-7):
                    r = math.sqrt(T) * f
                    own.append(np.stack([o[0] + r * np.cos(th), o[1] + r * np.sin(th)], 1).astype(np.float32))
        own.append(g.vertices[g.vertex_offsets[j]:g.vertex_offsets[j + 1]])
        own.append(np.array([[np.nan, o[1]], [o[0], np.inf]], np.float32))
        q = rng.permutation(np.concatenate(own).astype(np.float32))
        pts.append(q)
        offs.append(offs[-1] + len(q))
    yield "gis batch at the radii", wl.Workload("radii", g.vertices, g.vertex_offsets, np.concatenate(pts),
                                                np.array(offs, np.int64))
    h = wl.integer_hulls(seed=63, num_polygons=30, points_per_polygon=6_000)
    pts = h.points.copy()
    pts[::89] = rng.integers(-(1 << 30), 1 << 30, size=pts[::89].shape)
    yield "integer points, float polygons", wl.Workload("hf", h.vertices.astype(np.float32), h.vertex_offsets,
                                                        pts, h.point_offsets)


def test_batch_disc_filter_every_variant_equals_full_work_and_the_oracle():
    """The batch kernel's disc filter, at every tile shape: the masks of the
    full-work test and of the oracle."""
    for name, w in _batch_disc_cases():
        v = torch.from_numpy(w.vertices).to(dev())
        vo = torch.from_numpy(w.vertex_offsets).to(dev())
        p = torch.from_numpy(np.ascontiguousarray(w.points)).to(dev())
        po = torch.from_numpy(w.point_offsets).to(dev())
        want = oracle_own(w)
        t = B.pip_prepare(v, vo, max_points=w.num_points)
        for var in range(B.pip_batch_variant_count()):
            B.pip_set_batch_variant(t, var)
            full, _ = B.pip_test(t, p, po)
            disc, _ = B.pip_test(t, p, po, mode=B.PIP_MASK | B.PIP_DISC)
            st, _ = B.pip_get_status(t)
            assert st == B.PIP_OK
            got_full = B.unpack_mask(full, w.num_points).cpu().numpy()
            got_disc = B.unpack_mask(disc, w.num_points).cpu().numpy()
            assert_same(got_disc, got_full, "%s, variant %d: disc filter vs full work" % (name, var))
            assert_same(got_disc, want, "%s, variant %d: disc filter vs the oracle" % (name, var))
        t.close()


@pytest.mark.parametrize("kind", ["centroid", "vertex_mean", "chebyshev"])
def test_inner_generator_choices_give_the_oracle_masks(kind):
    """Any interior point may be p0 (Sec. 3): with the vertex mean or the
    Chebyshev centre instead of the centroid the tables hold that p0 and its
    mirrors (Eq. 8 about it, against the oracle's generators), and the masks
    are still exact closed-polygon membership."""
    for w in (wl.gis_batch(seed=54, num_polygons=40, m_range=(100, 5000)),
              wl.integer_hulls(seed=55, num_polygons=12, points_per_polygon=4000),
              wl.vehicle_footprint(seed=56, m=100_003)):
        v = torch.from_numpy(w.vertices).to(dev())
        vo = torch.from_numpy(w.vertex_offsets).to(dev())
        if kind == "centroid":
            want_p0 = np.stack([oracle.centroid(w.vertices[w.vertex_offsets[j]:w.vertex_offsets[j + 1]])[1]
                                for j in range(w.num_polygons)])
            t = B.pip_prepare_p0(v, vo, w.num_points, B.PIP_P0_CENTROID)
        elif kind == "vertex_mean":
            want_p0 = np.stack([w.vertices[w.vertex_offsets[j]:w.vertex_offsets[j + 1]].astype(np.float64).mean(0)
                                for j in range(w.num_polygons)])
            t = B.pip_prepare_p0(v, vo, w.num_points, B.PIP_P0_VERTEX_MEAN)
        else:
            want_p0 = wl.chebyshev_centres(w.vertices, w.vertex_offsets)
            t = B.pip_prepare_p0(v, vo, w.num_points, B.PIP_P0_GIVEN, torch.from_numpy(want_p0).to(dev()))
        st, _ = B.pip_get_status(t)
        assert st == B.PIP_OK
        ex = B.pip_export_tables(t)
        g0, gk = ex["g0"], ex["gk"]
        scale = np.abs(w.vertices.astype(np.float64)).max() + 1.0
        assert np.abs(g0 - want_p0).max() <= 1e-12 * scale
        for j in range(w.num_polygons):
            vv = w.vertices[w.vertex_offsets[j]:w.vertex_offsets[j + 1]]
            ref = oracle.generators(vv, want_p0[j])
            assert np.abs(gk[w.vertex_offsets[j]:w.vertex_offsets[j + 1]] - ref).max() <= 1e-10 * scale
        p = torch.from_numpy(w.points).to(dev())
        po = torch.from_numpy(w.point_offsets).to(dev()) if w.point_offsets is not None else None
        mask, _ = B.pip_test(t, p, po)
        assert_same(B.unpack_mask(mask, w.num_points).cpu().numpy(), oracle_own(w), "%s, p0 = %s" % (w.name, kind))
        t.close()


def test_inner_generator_outside_the_polygon_is_degenerate():
    sq = np.array([[0, 0], [4, 0], [4, 4], [0, 4]], np.float32)
    v = torch.from_numpy(sq).to(dev())
    vo = torch.tensor([0, 4], dtype=torch.int32, device=dev())
    for p0 in ([5.0, 1.0], [4.0, 2.0], [float("nan"), 1.0]):  # outside, on an edge, not finite
        t = B.pip_prepare_p0(v, vo, 16, B.PIP_P0_GIVEN, torch.tensor([p0], dtype=torch.float64, device=dev()))
        st, _ = B.pip_get_status(t)
        assert st == B.PIP_E_DEGENERATE
        t.close()


def test_tuning_cache_round_trip(tmp_path):
    """pip_set_tuning_cache: the first autotune times the variants and records
    the winner under (kernel, GPU name, shape); the next one on the same shape
    takes the recorded entry, even one edited by hand, without timing."""
    import json
    path = str(tmp_path / "tuning.json")
    B.pip_set_tuning_cache(path)
    try:
        w = wl.gis_batch(seed=57, num_polygons=30, m_range=(1000, 20000))
        v, vo = torch.from_numpy(w.vertices).to(dev()), torch.from_numpy(w.vertex_offsets).to(dev())
        p, po = torch.from_numpy(w.points).to(dev()), torch.from_numpy(w.point_offsets).to(dev())
        t = B.pip_prepare(v, vo, max_points=w.num_points)
        mask = torch.empty((w.num_points + 31) // 32, dtype=torch.int32, device=dev())
        best, ms = B.pip_autotune_batch(t, p, po, mask, reps=2)
        entries = json.load(open(path))
        (key, rec), = entries.items()
        assert key.startswith("batch|") and "polygons=30" in key and "points=%d" % w.num_points in key
        assert rec["variant"] == best
        other = (best + 1) % B.lib().pip_batch_variant_count()
        entries[key] = {"variant": other, "ms": 1.5}
        json.dump(entries, open(path, "w"))
        again, ms2 = B.pip_autotune_batch(t, p, po, mask, reps=2)
        assert again == other and ms2 == pytest.approx(1.5)
        got, _ = B.pip_test(t, p, po, mask=mask)
        assert_same(B.unpack_mask(got, w.num_points).cpu().numpy(), oracle_own(w), "cached tile shape")
        t.close()
        one = wl.vehicle_footprint(seed=58, m=1 << 20)
        t1 = B.pip_prepare(torch.from_numpy(one.vertices).to(dev()), torch.from_numpy(one.vertex_offsets).to(dev()),
                           max_points=one.num_points)
        p1 = torch.from_numpy(one.points).to(dev())
        m1 = torch.empty((one.num_points + 31) // 32, dtype=torch.int32, device=dev())
        sbest, _ = B.pip_autotune_stream(t1, p1, m1, reps=2)
        assert len(json.load(open(path))) == 2
        assert B.pip_autotune_stream(t1, p1, m1, reps=2)[0] == sbest
        t1.close()
    finally:
        B.pip_set_tuning_cache(None)


def test_repeated_calls_reset_the_refine_queue():
    w = wl.integer_hulls(seed=22, num_polygons=8, points_per_polygon=1000)
    v = torch.from_numpy(w.vertices).to(dev())
    vo = torch.from_numpy(w.vertex_offsets).to(dev())
    p = torch.from_numpy(w.points).to(dev())
    po = torch.from_numpy(w.point_offsets).to(dev())
    t = B.pip_prepare(v, vo, max_points=w.num_points)
    want = oracle_own(w)
    counts = []
    for _ in range(3):
        mask, _ = B.pip_test(t, p, po)
        counts.append(B.pip_get_status(t)[1])
        assert_same(B.unpack_mask(mask, w.num_points).cpu().numpy(), want, "repeat")
    assert counts[0] == counts[1] == counts[2]
    t.close()


def test_cuda_graph_capture_of_pip_test():
    w = wl.gis_batch(seed=23, num_polygons=16, m_range=(100, 4000))
    v = torch.from_numpy(w.vertices).to(dev())
    vo = torch.from_numpy(w.vertex_offsets).to(dev())
    p = torch.from_numpy(w.points).to(dev())
    po = torch.from_numpy(w.point_offsets).to(dev())
    t = B.pip_prepare(v, vo, max_points=w.num_points)
    mask = torch.zeros((w.num_points + 31) // 32, dtype=torch.int32, device=dev())
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        B.pip_test(t, p, po, mask=mask, stream=s)  # warm-up outside capture
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    mask.zero_()
    with torch.cuda.graph(g):
        B.pip_test(t, p, po, mask=mask)
    g.replay()
    torch.cuda.synchronize()
    got = B.unpack_mask(mask, w.num_points).cpu().numpy()
    assert_same(got, oracle_own(w), "graph replay")
    t.close()


def test_cuda_graph_capture_of_pip_margin():
    """One polygon, aligned points: the pipelined margin kernel replayed from a
    CUDA graph gives the eager call's margins exactly."""
    w = wl.vehicle_footprint(m=20_001, seed=65)
    t = B.pip_prepare(torch.from_numpy(w.vertices).to(dev()), torch.from_numpy(w.vertex_offsets).to(dev()),
                      max_points=w.num_points)
    p = torch.from_numpy(w.points).to(dev())
    eager = B.pip_margin(t, p).cpu().numpy()
    out = torch.zeros(w.num_points, dtype=torch.float32, device=dev())
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        B.pip_margin(t, p, out=out, stream=s)  # warm-up outside capture
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    out.zero_()
    with torch.cuda.graph(g):
        B.pip_margin(t, p, out=out)
    g.replay()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy().view(np.uint32), eager.view(np.uint32))
    t.close()


# ----------------------------------------------------------------- full size, sampled

def test_vehicle_footprint_full_size_every_point():
    w = wl.vehicle_footprint()
    got, _, refine, st = run_test(w)
    assert st == B.PIP_OK
    assert_same(got, oracle_par.inside_exact(w.vertices, w.points), "footprint, all 2^26 points")


def test_vehicle_footprint_disc_filter_full_size_every_point():
    w = wl.vehicle_footprint()
    t = B.pip_prepare(torch.from_numpy(w.vertices).to(dev()), torch.from_numpy(w.vertex_offsets).to(dev()),
                      max_points=w.num_points)
    mask, _ = B.pip_test(t, torch.from_numpy(w.points).to(dev()), mode=B.PIP_MASK | B.PIP_DISC)
    st, _ = B.pip_get_status(t)
    assert st == B.PIP_OK
    got = B.unpack_mask(mask, w.num_points).cpu().numpy()
    t.close()
    assert_same(got, oracle_par.inside_exact(w.vertices, w.points), "footprint with the disc filter, all 2^26 points")


def test_gis_batch_full_size_every_point():
    w = wl.gis_batch()
    got, _, refine, st = run_test(w)
    assert st == B.PIP_OK
    want = oracle_par.inside_exact_ragged(w.vertices, w.vertex_offsets, w.points, w.point_offsets)
    assert_same(got, want, "gis batch, all %d points" % w.num_points)


def test_gis_batch_disc_filter_full_size_every_point():
    w = wl.gis_batch()
    t = B.pip_prepare(torch.from_numpy(w.vertices).to(dev()), torch.from_numpy(w.vertex_offsets).to(dev()),
                      max_points=w.num_points)
    mask, _ = B.pip_test(t, torch.from_numpy(w.points).to(dev()), torch.from_numpy(w.point_offsets).to(dev()),
                         mode=B.PIP_MASK | B.PIP_DISC)
    st, _ = B.pip_get_status(t)
    assert st == B.PIP_OK
    got = B.unpack_mask(mask, w.num_points).cpu().numpy()
    t.close()
    want = oracle_par.inside_exact_ragged(w.vertices, w.vertex_offsets, w.points, w.point_offsets)
    assert_same(got, want, "gis batch with the disc filter, all points")


def test_all_pairs_full_size_every_point():
    w = wl.gis_all_pairs()
    got, fh, _, _ = run_test(w, mode=B.PIP_FIRST_HIT | B.PIP_MASK)
    want = oracle_par.first_hit_exact(w.vertices, w.vertex_offsets, w.points)
    assert_same(fh, want, "all pairs first hit, all 2^20 points")
    assert_same(got, (want >= 0).astype(np.uint8), "all pairs mask")


def test_all_pairs_culled_equals_full_work_at_full_size():
    w = wl.gis_all_pairs()
    got_f, fh_f, _, _ = run_test(w, mode=B.PIP_FIRST_HIT | B.PIP_MASK)
    got_c, fh_c, _, _ = run_test(w, mode=B.PIP_FIRST_HIT | B.PIP_MASK | B.PIP_CULL)
    assert_same(fh_c, fh_f, "culled vs full work, every point")
    assert_same(got_c, got_f, "culled vs full work mask")


def test_integer_hulls_full_size_every_point():
    w = wl.integer_hulls()
    got, _, refine, st = run_test(w)
    assert st == B.PIP_OK
    want = oracle_par.inside_exact_ragged(w.vertices, w.vertex_offsets, w.points, w.point_offsets)
    assert_same(got, want, "integer hulls, all 2^24 points")
