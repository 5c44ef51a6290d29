"""GPU parity of pip_rasterize: per-pixel first hit and coverage mask at the
float32 pixel centres, element by element against the oracle's exact first
hit at the same centres (oracle.raster_centres, pinned on CPU)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2007_15385_gb300 import binding as B
from paper_2007_15385_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.lib()
    yield


def _dev():
    return torch.device("cuda", 0)


def _tables(verts, voffs, capacity):
    return B.pip_prepare(torch.from_numpy(np.ascontiguousarray(verts)).to(_dev()),
                         torch.from_numpy(np.ascontiguousarray(voffs)).to(_dev()), max_points=capacity)


def _want(verts, voffs, W, H, x0, y0, dx, dy):
    c = oracle.raster_centres(W, H, x0, y0, dx, dy)
    return oracle.first_hit_exact(verts, voffs, c).reshape(H, W)


def _mask_of(ids):
    H, W = ids.shape
    wpr = (W + 31) // 32
    bits = np.zeros((H, wpr * 32), np.uint8)
    bits[:, :W] = ids >= 0
    return np.packbits(bits, axis=1, bitorder="little").view(np.uint32)


def _check(verts, voffs, W, H, x0, y0, dx, dy, what):
    t = _tables(verts, voffs, W * H)
    ids, mask = B.pip_rasterize(t, W, H, x0, y0, dx, dy)
    st, _ = B.pip_get_status(t)
    got = ids.cpu().numpy()
    want = _want(verts, voffs, W, H, x0, y0, dx, dy)
    bad = np.argwhere(got != want)
    assert bad.size == 0, "%s: %d pixels differ, first (r, c) %s got %d want %d" % (
        what, len(bad), bad[0], got[tuple(bad[0])], want[tuple(bad[0])])
    np.testing.assert_array_equal(mask.cpu().numpy().view(np.uint32), _mask_of(want))
    t.close()
    return want, st


def test_gis_polygons_on_a_non_dyadic_grid():
    w = wl.gis_batch(seed=51, num_polygons=80, m_range=(10, 20))
    # the frame covers the polygons' domain; dx is not a power of two
    want, _ = _check(w.vertices, w.vertex_offsets, 257, 131, -3.0, 11.0, np.float32(1e4 / 257),
                     np.float32(1e4 / 131), "gis")
    assert (want >= 0).any() and (want < 0).any()


def test_integer_polygons_with_centres_on_edges_and_vertices():
    # integer vertices, centres on the integer lattice: many centres lie
    # exactly on edges and vertices (closed: inside), the exact refine decides
    h = wl.integer_hulls(seed=52, num_polygons=14, points_per_polygon=64, box=400, r_range=(20.0, 150.0))
    want, _ = _check(h.vertices, h.vertex_offsets, 800, 800, -400.0, -400.0, 1.0, 1.0, "integer lattice")
    assert (want >= 0).sum() > 1000


def test_overlaps_take_the_lowest_index_and_invalid_polygons_hold_nothing():
    sq = lambda x, y, s: [[x, y], [x + s, y], [x + s, y + s], [x, y + s]]
    polys = [
        [[0, 0], [2, 0], [1, 0.2], [2, 2], [0, 2]],  # non-convex: holds nothing
        sq(1, 1, 4),
        sq(3, 3, 4),       # overlaps the first square
        sq(0.5, 0.5, 8),   # under both
        [[0, 0], [1, 0], [2, 0]],  # zero area
    ]
    verts = np.concatenate([np.array(p, np.float32) for p in polys])
    voffs = np.zeros(len(polys) + 1, np.int32)
    voffs[1:] = np.cumsum([len(p) for p in polys])
    want, st = _check(verts, voffs, 40, 40, 0.125, 0.125, 0.25, 0.25, "overlaps")
    assert set(np.unique(want)) <= {-1, 1, 2, 3}
    assert (want == 2).any() and (want == 3).any()


@pytest.mark.parametrize("W,H", [(1, 1), (63, 47), (64, 48), (65, 49), (130, 97)])
def test_frame_sizes_around_the_tile(W, H):
    w = wl.gis_batch(seed=53, num_polygons=60, m_range=(10, 20))
    _check(w.vertices, w.vertex_offsets, W, H, 0.0, 0.0, np.float32(1e4 / W), np.float32(1e4 / H),
           "frame %dx%d" % (W, H))


def test_bad_grid_and_capacity():
    w = wl.gis_batch(seed=54, num_polygons=8, m_range=(10, 20))
    t = _tables(w.vertices, w.vertex_offsets, 100)
    ws = torch.empty(1 << 16, dtype=torch.uint8, device=_dev())
    ids = torch.empty(10 * 10, dtype=torch.int32, device=_dev())
    L = B.lib()
    assert L.pip_rasterize(t, 10, 10, 0.0, 0.0, 0.0, 1.0, ids.data_ptr(), None, ws.data_ptr(), ws.numel(),
                           None) == B.PIP_E_INVALID_ARG
    assert L.pip_rasterize(t, 10, 10, 0.0, 0.0, 1.0, float("nan"), ids.data_ptr(), None, ws.data_ptr(),
                           ws.numel(), None) == B.PIP_E_INVALID_ARG
    assert L.pip_rasterize(t, 10, 10, 0.0, 0.0, 1.0, 1.0, None, None, ws.data_ptr(), ws.numel(),
                           None) == B.PIP_E_INVALID_ARG
    assert L.pip_rasterize(t, 10, 10, 0.0, 0.0, 1.0, 1.0, ids.data_ptr(), None, ws.data_ptr(), 0,
                           None) == B.PIP_E_INVALID_ARG
    big = torch.empty(11 * 10, dtype=torch.int32, device=_dev())
    assert L.pip_rasterize(t, 11, 10, 0.0, 0.0, 1.0, 1.0, big.data_ptr(), None, ws.data_ptr(), ws.numel(),
                           None) == B.PIP_E_CAPACITY
    t.close()


def test_graph_capture_of_pip_rasterize():
    w = wl.gis_batch(seed=55, num_polygons=40, m_range=(10, 20))
    W, H = 200, 150
    t = _tables(w.vertices, w.vertex_offsets, W * H)
    ids = torch.empty((H, W), dtype=torch.int32, device=_dev())
    mask = torch.empty((H, (W + 31) // 32), dtype=torch.int32, device=_dev())
    ws = torch.empty(B.pip_raster_workspace_bytes(t.num_polygons, W, H) + 16, dtype=torch.uint8, device=_dev())
    args = (t, W, H, 0.0, 0.0, np.float32(1e4 / W), np.float32(1e4 / H))
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        B.pip_rasterize(*args, first_hit=ids, mask=mask, workspace=ws, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    ids.fill_(-7)
    with torch.cuda.graph(g):
        B.pip_rasterize(*args, first_hit=ids, mask=mask, workspace=ws)
    g.replay()
    torch.cuda.synchronize()
    want = _want(w.vertices, w.vertex_offsets, W, H, *args[3:])
    np.testing.assert_array_equal(ids.cpu().numpy(), want)
    t.close()


def test_full_frame_sampled():
    """The benchmark's frame: the 4,096 GIS polygons on 3840 x 2160 pixels."""
    w = wl.gis_batch()
    W, H = 3840, 2160
    dx, dy = np.float32(1e4 / W), np.float32(1e4 / H)
    t = _tables(w.vertices, w.vertex_offsets, W * H)
    ids, mask = B.pip_rasterize(t, W, H, 0.0, 0.0, dx, dy)
    got = ids.cpu().numpy()
    np.testing.assert_array_equal(mask.cpu().numpy().view(np.uint32), _mask_of(got))
    rng = np.random.default_rng(56)
    # pixels of covered tiles weigh in: half the sample where got >= 0
    cov = np.argwhere(got >= 0)
    pick = np.concatenate([rng.choice(H * W, 2000, replace=False),
                           np.ravel_multi_index(cov[rng.choice(len(cov), 2000, replace=False)].T, (H, W))])
    c = oracle.raster_centres(W, H, 0.0, 0.0, dx, dy)[pick]
    want = oracle.first_hit_exact(w.vertices, w.vertex_offsets, c)
    np.testing.assert_array_equal(got.ravel()[pick], want)
    t.close()
