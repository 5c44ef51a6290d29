"""pip_test_single_noalloc: the single-polygon test for callers that cannot allocate.

Some callers cannot call cudaMalloc when they test points -- a collision check
inside a fixed-rate control loop cannot absorb its latency and implicit
synchronisation, and a plug-in whose host owns the device memory pool is not
allowed to allocate at all.  pip_test_single_noalloc serves them from a static
scratch array inside libpip.  These tests call it through the C ABI and check
that it gives exactly the mask of the allocating path (pip_prepare + pip_test)
and of the oracle, on two calls in a row, so that nothing left in the shared
scratch by one call leaks into the next, and on mixed point and vertex types,
unaligned points and the largest point count.

This file sorts last so that a run stopping at the first failure has already
run every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2007_15385_gb300 import binding as B
from paper_2007_15385_gb300 import workloads as wl


def _mask_via_tables(verts, pts):
    v = torch.from_numpy(verts).cuda()
    vo = torch.tensor([0, len(verts)], dtype=torch.int32, device="cuda")
    p = torch.from_numpy(pts).cuda()
    t = B.pip_prepare(v, vo, max_points=len(pts))
    mask, _ = B.pip_test(t, p)
    torch.cuda.synchronize()
    st, refined = B.pip_get_status(t)
    out = mask.cpu().numpy().copy()
    t.close()
    return out, st, refined


def _mask_noalloc(verts, pts, offset_points=0):
    v = torch.from_numpy(verts).cuda()
    flat = np.zeros(2 * (len(pts) + offset_points), pts.dtype)
    flat[2 * offset_points:] = pts.reshape(-1)
    p = torch.from_numpy(flat).cuda()[2 * offset_points:]
    mask = torch.full(((len(pts) + 31) // 32,), -1, dtype=torch.int32, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    B.pip_test_single_noalloc(v, p, mask, status)
    torch.cuda.synchronize()
    return mask.cpu().numpy().copy(), int(status.item())


@pytest.mark.gpu
def test_noalloc_matches_pip_test_on_two_calls_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    # call 1: an integer hull whose on-edge and one-off points fill the refine queue
    w1 = wl.integer_hulls(seed=31, num_polygons=1, points_per_polygon=200_000)
    # call 2: a float footprint with fewer points than call 1 left in the queue
    w2 = wl.vehicle_footprint(seed=32, m=100_003)
    for w in (w1, w2):
        want, st_want, refined = _mask_via_tables(w.vertices, w.points)
        got, st_got = _mask_noalloc(w.vertices, w.points)
        assert st_want == B.PIP_OK and st_got == B.PIP_OK
        assert got.shape == want.shape
        bad = np.nonzero(got != want)[0]
        assert len(bad) == 0, "%s: %d mask words differ" % (w.name, len(bad))
        want_oracle, _ = oracle.inside_exact(w.vertices, w.points)
        bad = np.nonzero(_unpack(got, w.num_points) != want_oracle)[0]
        assert len(bad) == 0, "%s: %d points differ from the oracle" % (w.name, len(bad))
    assert refined >= 0


def _unpack(words, m):
    return np.unpackbits(words.view(np.uint8), bitorder="little")[:m]


def _mixed_cases():
    rng = np.random.default_rng(33)
    hull = wl.integer_hulls(seed=34, num_polygons=1, points_per_polygon=4096)
    # int32 vertices, float32 points: the hull's own points shifted by 0, 1/2 or 1/4
    fpts = (hull.points.astype(np.float64) + rng.choice([0.0, 0.5, 0.25], size=hull.points.shape))
    yield "int32 vertices, float32 points", hull.vertices, fpts.astype(np.float32)
    # float32 vertices, int32 points: a footprint scaled to integer units
    fp = wl.vehicle_footprint(seed=35, m=4096)
    fv = (fp.vertices.astype(np.float64) * 1000.0).astype(np.float32)
    ipts = np.rint(fp.points.astype(np.float64) * 1000.0).astype(np.int32)
    yield "float32 vertices, int32 points", fv, ipts


@pytest.mark.gpu
def test_noalloc_mixed_dtypes_unaligned_points_and_the_largest_size_match_the_oracle():
    """The cases its two refine kernels meet: mixed vertex and point types,
    points 8 but not 16 bytes aligned, and exactly the largest point count;
    each compared with pip_prepare + pip_test and with the oracle directly."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cases = list(_mixed_cases())
    big = wl.vehicle_footprint(seed=36, m=B.NOALLOC_MAX_POINTS)
    cases.append(("2^20 float32 points", big.vertices, big.points))
    ints = wl.integer_hulls(seed=37, num_polygons=1, points_per_polygon=B.NOALLOC_MAX_POINTS)
    cases.append(("2^20 int32 points", ints.vertices, ints.points))
    for name, verts, pts in cases:
        want_oracle, ost = oracle.inside_exact(verts, pts)
        assert ost == oracle.OK
        want_tables, st_t, _ = _mask_via_tables(verts, pts)
        for off in (0, 1):
            got, st = _mask_noalloc(verts, pts, offset_points=off)
            assert st == B.PIP_OK and st_t == B.PIP_OK
            assert np.array_equal(got, want_tables), "%s (offset %d): differs from pip_test" % (name, off)
            bad = np.nonzero(_unpack(got, len(pts)) != want_oracle)[0]
            assert len(bad) == 0, "%s (offset %d): %d points differ from the oracle" % (name, off, len(bad))


@pytest.mark.gpu
def test_noalloc_reports_an_invalid_polygon():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    v = np.array([[0, 0], [2, 0], [1, 0.2], [2, 2], [0, 2]], np.float32)  # non-convex
    pts = np.array([[1, 1], [0.5, 1.5]], np.float32)
    got, st = _mask_noalloc(v, pts)
    assert st == B.PIP_E_NONCONVEX
    assert got.tolist() == [0]


def test_noalloc_rejects_more_points_than_its_scratch_holds():
    B.lib()
    st = B.lib().pip_test_single_noalloc(8, B.PIP_F32, 4, 8, B.PIP_F32, B.NOALLOC_MAX_POINTS + 1,
                                         8, None, None)
    assert st == B.PIP_E_CAPACITY
    st = B.lib().pip_test_single_noalloc(8, B.PIP_F32, 65, 8, B.PIP_F32, 10, 8, None, None)
    assert st == B.PIP_E_INVALID_ARG


@pytest.mark.gpu
def test_noalloc_wrapper_rejects_short_or_mistyped_buffers():
    """The binding checks what the C call cannot: the mask's type and length
    and the status word's, before anything is enqueued."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    w = wl.vehicle_footprint(seed=38, m=1000)
    v = torch.from_numpy(w.vertices).cuda()
    p = torch.from_numpy(w.points).cuda()
    short = torch.zeros((1000 + 31) // 32 - 1, dtype=torch.int32, device="cuda")
    with pytest.raises(ValueError):
        B.pip_test_single_noalloc(v, p, short)
    wrong = torch.zeros((1000 + 31) // 32, dtype=torch.int64, device="cuda")
    with pytest.raises(ValueError):
        B.pip_test_single_noalloc(v, p, wrong)
    mask = torch.zeros((1000 + 31) // 32, dtype=torch.int32, device="cuda")
    with pytest.raises(ValueError):
        B.pip_test_single_noalloc(v, p, mask, torch.zeros(1, dtype=torch.float32, device="cuda"))
    with pytest.raises(ValueError):
        B.pip_test_single_noalloc(v, p, mask, torch.zeros(1, dtype=torch.int32))
