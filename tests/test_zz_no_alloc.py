"""pip_test_single_noalloc: the single-polygon test for callers that cannot allocate.

Some callers cannot call cudaMalloc when they test points -- a collision check
inside a fixed-rate control loop cannot absorb its latency and implicit
synchronisation, and a plug-in whose host owns the device memory pool is not
allowed to allocate at all.  pip_test_single_noalloc serves them from a static
scratch array inside libpip.  These tests call it through the C ABI and check
that it gives exactly the mask of the allocating path (pip_prepare + pip_test),
on two calls in a row, so that nothing left in the shared scratch by one call
leaks into the next.

This file sorts last so that a run stopping at the first failure has already
run every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest
import torch

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


def _mask_noalloc(verts, pts):
    v = torch.from_numpy(verts).cuda()
    p = torch.from_numpy(pts).cuda()
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
    assert refined >= 0


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
