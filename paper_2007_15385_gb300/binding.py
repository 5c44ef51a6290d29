"""Thin Python binding of libpip (include/pip.h), same names as the C ABI.

Argument marshalling only: every step of the inclusion test runs in the CUDA
kernels of libpip.so.  PyTorch supplies device memory and the current stream.
There is no fallback: if libpip.so is missing or a CUDA device is absent the
calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpip.so")

PIP_OK = 0
PIP_E_INVALID_ARG = 1
PIP_E_DEGENERATE = 2
PIP_E_NONCONVEX = 3
PIP_E_NONFINITE = 4
PIP_E_CUDA = 5
PIP_E_TIMEOUT = 6
PIP_E_CAPACITY = 7
PIP_F32 = 0
PIP_I32 = 1
PIP_MASK = 1
PIP_FIRST_HIT = 2
PIP_CULL = 4  # all pairs: skip polygons by bounding box, stop early (same results)
PIP_P0_CENTROID = 0
PIP_P0_VERTEX_MEAN = 1
PIP_P0_GIVEN = 2
PIP_EARLY_EXIT = 8  # one polygon / batch: warp-uniform early break over spread edges (same results)
PIP_PENALTY_CULL = 1  # penalty: pairs provably beyond 120 tau of every edge line left out (same results)
PIP_DISC = 16  # one polygon / batch: points decided by the inner / outer discs about the origin skip their edges (same results)

# every symbol include/pip.h declares, with (restype, argtypes)
_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_INT = ctypes.c_int
SIGNATURES = {
    "pip_prepare": (_INT, [_P, _INT, _P, _I32, _I32, _I64, _P, ctypes.POINTER(_P)]),
    "pip_prepare_p0": (_INT, [_P, _INT, _P, _I32, _I32, _I64, _I32, _P, _P, ctypes.POINTER(_P)]),
    "pip_test": (_INT, [_P, _P, _INT, _I64, _P, _INT, _P, _P, _P]),
    "pip_margin": (_INT, [_P, _P, _INT, _I64, _P, _P, _P]),
    "pip_get_status": (_INT, [_P, _P, ctypes.POINTER(_I64)]),
    "pip_get_polygon_status": (_INT, [_P, _P, _P]),
    "pip_export_tables": (_INT, [_P, _P, _P, _P, _P, _P, _P, _P]),
    "pip_destroy": (None, [_P]),
    "pip_timing": (_INT, [_P, _INT]),
    "pip_timing_read": (_INT, [_P, ctypes.POINTER(_I32), ctypes.POINTER(ctypes.c_double),
                                ctypes.POINTER(ctypes.c_double)]),
    "pip_num_polygons": (_I32, [_P]),
    "pip_total_vertices": (_I32, [_P]),
    "pip_status_string": (ctypes.c_char_p, [_INT]),
    "pip_test_sign_of_offset": (_INT, [_P, _P, _I64, _P, _P, _P]),
    "pip_test_ray_crossing": (_INT, [_P, _P, _I64, _P, _P, _P]),
    "pip_test_voronoi_fp64": (_INT, [_P, _P, _I64, _P, _P, _P]),
    "pip_test_single_noalloc": (_INT, [_P, _INT, _I32, _P, _INT, _I64, _P, _P, _P]),
    "pip_stream_variant_count": (_I32, []),
    "pip_selftest_wait_timeout": (_INT, [_P, _P, _I64, _P]),
    "pip_fma_peak": (_INT, [_I32, _I32, _P, _I64, _P, ctypes.POINTER(_I64)]),
    "pip_test_host": (_INT, [_P, _P, _INT, _I64, _P, _P, _P, _I32, _P]),
    "pip_set_tuning_cache": (_INT, [ctypes.c_char_p]),
    "pip_raster_workspace_bytes": (ctypes.c_size_t, [_I32, _I32, _I32]),
    "pip_rasterize": (_INT, [_P, _I32, _I32, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                             _P, _P, _P, ctypes.c_size_t, _P]),
    "pip_batch_variant_count": (_I32, []),
    "pip_set_batch_variant": (_INT, [_P, _I32]),
    "pip_autotune_batch": (_INT, [_P, _P, _INT, _I64, _P, _P, _I32, _P, ctypes.POINTER(_I32),
                                  ctypes.POINTER(ctypes.c_float)]),
    "pip_penalty_workspace_bytes": (ctypes.c_size_t, [_I32, _I32, _I64]),
    "pip_penalty_forward": (_INT, [_P, _I32, _P, _I32, _P, _I64, ctypes.c_float, _P, _I32, _P,
                                    ctypes.c_size_t, _P]),
    "pip_penalty_backward": (_INT, [_P, _I32, _P, _I32, _P, _I64, ctypes.c_float, _P, _P, _P, _I32, _P,
                                     ctypes.c_size_t, _P]),
    "pip_set_stream_variant": (_INT, [_P, _I32]),
    "pip_autotune_stream": (_INT, [_P, _P, _INT, _I64, _P, _I32, _P, ctypes.POINTER(_I32),
                                    ctypes.POINTER(ctypes.c_float)]),
}

_lib = None
_lock = threading.Lock()


class PipError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = lib().pip_status_string(status).decode() if _lib is not None else str(status)
        super().__init__("%s: %s (status %d)" % (where, msg, status))


def lib() -> ctypes.CDLL:
    """Loads libpip.so (built by paper_2007_15385_gb300.build); raises if it is absent."""
    global _lib
    if _lib is None:
        with _lock:
            if _lib is None:
                if not os.path.exists(LIB_PATH):
                    raise ImportError("libpip.so is not built (%s); run "
                                      "`python -m paper_2007_15385_gb300.build`" % LIB_PATH)
                L = ctypes.CDLL(LIB_PATH)
                for name, (res, args) in SIGNATURES.items():
                    f = getattr(L, name)
                    f.restype = res
                    f.argtypes = args
                _lib = L
    return _lib


def _check(status: int, where: str):
    if status != PIP_OK:
        raise PipError(status, where)


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float32:
        return PIP_F32
    if t.dtype == torch.int32:
        return PIP_I32
    raise TypeError("vertices and points are float32 or int32 xy pairs, got %s" % t.dtype)


def _dev(t: torch.Tensor, name: str) -> torch.Tensor:
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    return t


class Tables:
    """Owns one pip_tables handle; released with pip_destroy."""

    def __init__(self, handle: ctypes.c_void_p, num_polygons: int, total_vertices: int,
                 max_points: int, device: torch.device):
        self.handle = handle
        self.num_polygons = num_polygons
        self.total_vertices = total_vertices
        self.max_points = max_points
        self.device = device

    def close(self):
        if self.handle:
            lib().pip_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def _as_parameter_(self):
        if not self.handle:
            raise ValueError("tables already destroyed")
        return self.handle


def pip_prepare(vertices: torch.Tensor, vertex_offsets: torch.Tensor, max_points: int,
                stream=None) -> Tables:
    """Polygon -> Voronoi generator tables (Eq. 3-4, Eq. 8)."""
    _dev(vertices, "vertices")
    _dev(vertex_offsets, "vertex_offsets")
    if vertex_offsets.dtype != torch.int32:
        raise TypeError("vertex_offsets must be int32")
    P = vertex_offsets.numel() - 1
    V = vertices.numel() // 2
    h = ctypes.c_void_p()
    _check(lib().pip_prepare(vertices.data_ptr(), _dtype_code(vertices), vertex_offsets.data_ptr(),
                             P, V, int(max_points), _stream(stream), ctypes.byref(h)), "pip_prepare")
    return Tables(h, P, V, int(max_points), vertices.device)


def pip_prepare_p0(vertices: torch.Tensor, vertex_offsets: torch.Tensor, max_points: int, p0_kind: int,
                   p0: torch.Tensor | None = None, stream=None) -> Tables:
    """pip_prepare with another inner generator: PIP_P0_CENTROID, PIP_P0_VERTEX_MEAN, or
    PIP_P0_GIVEN with p0 a float64 CUDA tensor [num_polygons, 2] of interior points."""
    _dev(vertices, "vertices")
    _dev(vertex_offsets, "vertex_offsets")
    if vertex_offsets.dtype != torch.int32:
        raise TypeError("vertex_offsets must be int32")
    P = vertex_offsets.numel() - 1
    V = vertices.numel() // 2
    ptr = None
    if p0_kind == PIP_P0_GIVEN:
        if p0 is None:
            raise ValueError("PIP_P0_GIVEN needs p0")
        _dev(p0, "p0")
        if p0.dtype != torch.float64 or p0.numel() != 2 * P or p0.device != vertices.device:
            raise ValueError("p0 must be float64 [num_polygons, 2] on the vertices' device")
        ptr = p0.data_ptr()
    h = ctypes.c_void_p()
    _check(lib().pip_prepare_p0(vertices.data_ptr(), _dtype_code(vertices), vertex_offsets.data_ptr(), P, V,
                                int(max_points), int(p0_kind), ptr, _stream(stream), ctypes.byref(h)),
           "pip_prepare_p0")
    tables = Tables(h, P, V, int(max_points), vertices.device)
    tables._keep_p0 = p0  # read by the prepare kernel, which may still be running
    return tables


def pip_test(tables: Tables, points: torch.Tensor, point_offsets: torch.Tensor | None = None,
             mode: int = PIP_MASK, mask: torch.Tensor | None = None,
             first_hit: torch.Tensor | None = None, stream=None):
    """Voronoi inclusion (Alg. 5).  Returns (mask uint32 words or None, first_hit or None)."""
    _dev(points, "points")
    M = points.numel() // 2
    if mode & PIP_MASK and mask is None:
        mask = torch.empty((M + 31) // 32, dtype=torch.int32, device=points.device)
    if mode & PIP_FIRST_HIT and first_hit is None:
        first_hit = torch.empty(M, dtype=torch.int32, device=points.device)
    offs = 0
    if point_offsets is not None:
        _dev(point_offsets, "point_offsets")
        if point_offsets.dtype != torch.int64:
            raise TypeError("point_offsets must be int64")
        offs = point_offsets.data_ptr()
    _check(lib().pip_test(tables, points.data_ptr() if M else None, _dtype_code(points), M,
                          offs or None, mode, mask.data_ptr() if mask is not None else None,
                          first_hit.data_ptr() if first_hit is not None else None,
                          _stream(stream)), "pip_test")
    return (mask if mode & PIP_MASK else None), (first_hit if mode & PIP_FIRST_HIT else None)


def pip_margin(tables: Tables, points: torch.Tensor, point_offsets: torch.Tensor | None = None,
               out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Signed Voronoi margin (Eq. 2 bisector distance), > 0 outside."""
    _dev(points, "points")
    M = points.numel() // 2
    if out is None:
        out = torch.empty(M, dtype=torch.float32, device=points.device)
    offs = None
    if point_offsets is not None:
        _dev(point_offsets, "point_offsets")
        offs = point_offsets.data_ptr()
    _check(lib().pip_margin(tables, points.data_ptr() if M else None, _dtype_code(points), M, offs,
                            out.data_ptr() if M else None, _stream(stream)), "pip_margin")
    return out


def pip_get_status(tables: Tables, stream=None) -> tuple[int, int]:
    """(worst polygon status, refine count of the last pip_test); synchronizes."""
    cnt = ctypes.c_int64(0)
    st = lib().pip_get_status(tables, _stream(stream), ctypes.byref(cnt))
    if st == PIP_E_CUDA:
        raise PipError(st, "pip_get_status")
    return int(st), int(cnt.value)


def pip_get_polygon_status(tables: Tables, stream=None):
    import numpy as np
    out = np.zeros(tables.num_polygons, np.int32)
    _check(lib().pip_get_polygon_status(tables, out.ctypes.data_as(ctypes.c_void_p), _stream(stream)),
           "pip_get_polygon_status")
    return out


def pip_timing(tables: Tables, enable: bool = True):
    """Turns per-call CUDA-event timing of the bulk and refine kernels on or off."""
    _check(lib().pip_timing(tables, 1 if enable else 0), "pip_timing")


def pip_timing_read(tables: Tables) -> tuple[int, float, float]:
    """(timed calls, summed bulk-kernel ms, summed refine-kernel ms); synchronizes, resets."""
    calls = ctypes.c_int32(0)
    b = ctypes.c_double(0.0)
    r = ctypes.c_double(0.0)
    _check(lib().pip_timing_read(tables, ctypes.byref(calls), ctypes.byref(b), ctypes.byref(r)),
           "pip_timing_read")
    return int(calls.value), float(b.value), float(r.value)


def pip_stream_variant_count() -> int:
    return int(lib().pip_stream_variant_count())


def pip_set_stream_variant(tables: Tables, variant: int):
    _check(lib().pip_set_stream_variant(tables, int(variant)), "pip_set_stream_variant")


def pip_autotune_stream(tables: Tables, points: torch.Tensor, mask: torch.Tensor, reps: int = 5,
                        stream=None) -> tuple[int, float]:
    """Times every tile shape of the pipelined kernel on these inputs; keeps the fastest."""
    _dev(points, "points")
    best = ctypes.c_int32(-1)
    ms = ctypes.c_float(0.0)
    _check(lib().pip_autotune_stream(tables, points.data_ptr(), _dtype_code(points),
                                     points.numel() // 2, mask.data_ptr(), int(reps),
                                     _stream(stream), ctypes.byref(best), ctypes.byref(ms)),
           "pip_autotune_stream")
    return int(best.value), float(ms.value)


def pip_batch_variant_count() -> int:
    return int(lib().pip_batch_variant_count())


def pip_set_batch_variant(tables: Tables, variant: int):
    _check(lib().pip_set_batch_variant(tables, int(variant)), "pip_set_batch_variant")


def pip_autotune_batch(tables: Tables, points: torch.Tensor, point_offsets: torch.Tensor,
                       mask: torch.Tensor, reps: int = 3, stream=None) -> tuple[int, float]:
    """Times every tile shape of the pipelined batch kernel on this batch; keeps the fastest."""
    _dev(points, "points")
    _dev(point_offsets, "point_offsets")
    best = ctypes.c_int32(-1)
    ms = ctypes.c_float(0.0)
    _check(lib().pip_autotune_batch(tables, points.data_ptr(), _dtype_code(points), points.numel() // 2,
                                    point_offsets.data_ptr(), mask.data_ptr(), int(reps), _stream(stream),
                                    ctypes.byref(best), ctypes.byref(ms)), "pip_autotune_batch")
    return int(best.value), float(ms.value)


def pip_export_tables(tables: Tables, stream=None) -> dict:
    import numpy as np
    P, V = tables.num_polygons, tables.total_vertices
    g0 = np.zeros((P, 2))
    gk = np.zeros((V, 2))
    coef = np.zeros((V, 4), np.float32)
    origin = np.zeros((P, 2), np.float32)
    bound = np.zeros((P, 2), np.float32)
    disc = np.zeros((P, 2), np.float32)
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    _check(lib().pip_export_tables(tables, ptr(g0), ptr(gk), ptr(coef), ptr(origin), ptr(bound), ptr(disc),
                                   _stream(stream)), "pip_export_tables")
    return {"g0": g0, "gk": gk, "coef": coef, "origin": origin, "bound": bound, "disc": disc}


def _cmp(fn: str, tables: Tables, points: torch.Tensor, point_offsets=None, mask=None, stream=None):
    _dev(points, "points")
    if points.dtype != torch.float32:
        raise TypeError("the comparators take float32 points")
    M = points.numel() // 2
    if mask is None:
        mask = torch.empty((M + 31) // 32, dtype=torch.int32, device=points.device)
    offs = point_offsets.data_ptr() if point_offsets is not None else None
    _check(getattr(lib(), fn)(tables, points.data_ptr() if M else None, M, offs,
                              mask.data_ptr() if M else None, _stream(stream)), fn)
    return mask


def pip_test_sign_of_offset(tables, points, point_offsets=None, mask=None, stream=None):
    """Alg. 2 in float32 on the GPU."""
    return _cmp("pip_test_sign_of_offset", tables, points, point_offsets, mask, stream)


def pip_test_ray_crossing(tables, points, point_offsets=None, mask=None, stream=None):
    """Alg. 1 in float32 on the GPU."""
    return _cmp("pip_test_ray_crossing", tables, points, point_offsets, mask, stream)


def pip_test_voronoi_fp64(tables, points, point_offsets=None, mask=None, stream=None):
    """Alg. 5 literally in fp64 on the GPU (unbatched)."""
    return _cmp("pip_test_voronoi_fp64", tables, points, point_offsets, mask, stream)


def unpack_mask(mask: torch.Tensor, num_points: int) -> torch.Tensor:
    """uint32 words (LSB first) -> uint8 [num_points] on the same device (torch ops: output
    formatting only, not part of the test)."""
    w = mask.to(torch.int64) & 0xFFFFFFFF
    bits = (w.unsqueeze(1) >> torch.arange(32, device=mask.device)) & 1
    return bits.reshape(-1)[:num_points].to(torch.uint8)


def pip_test_host(tables: Tables, points_host: torch.Tensor, device_points: torch.Tensor,
                  device_mask: torch.Tensor, mask_host: torch.Tensor, stream=None, chunks: int = 8):
    """End-to-end call on host buffers through the C ABI's pip_test_host (one polygon or all
    pairs, mask only): pinned host points -> device staging buffer -> pip_test -> pinned host
    mask, in `chunks` pieces so that the copy of one piece overlaps the test and the read-back
    of the previous one.  The caller provides the staging buffers; nothing is allocated per
    call.  Returns mask_host (complete once the stream has run)."""
    for t_, nm in ((points_host, "points_host"), (mask_host, "mask_host")):
        if t_.is_cuda or not t_.is_contiguous():
            raise ValueError("%s must be a contiguous host tensor" % nm)
    _dev(device_points, "device_points")
    _dev(device_mask, "device_mask")
    M = points_host.numel() // 2
    if device_points.numel() < 2 * M or device_mask.numel() < (M + 31) // 32 or mask_host.numel() < (M + 31) // 32:
        raise ValueError("staging or result buffers are smaller than the points need")
    if device_points.dtype != points_host.dtype:
        raise TypeError("device_points must have the host points' dtype")
    _check(lib().pip_test_host(tables, points_host.data_ptr(), _dtype_code(points_host), M,
                               device_points.data_ptr(), device_mask.data_ptr(), mask_host.data_ptr(),
                               int(chunks), _stream(stream)), "pip_test_host")
    return mask_host


NOALLOC_MAX_POINTS = 1 << 20


def pip_raster_workspace_bytes(num_polygons: int, width: int, height: int) -> int:
    return int(lib().pip_raster_workspace_bytes(int(num_polygons), int(width), int(height)))


def pip_rasterize(tables: Tables, width: int, height: int, x0: float, y0: float, dx: float, dy: float,
                  first_hit: torch.Tensor | None = None, mask: torch.Tensor | None = None,
                  workspace: torch.Tensor | None = None, want_ids: bool = True, want_mask: bool = True,
                  stream=None):
    """Pixel coverage: (ids int32 [height, width] or None, mask int32 [height, ceil(width / 32)] or None).
    Pixel (c, r) has the float32 centre (fma(c, dx, x0), fma(r, dy, y0))."""
    dev = tables.device
    wpr = (width + 31) // 32
    if want_ids and first_hit is None:
        first_hit = torch.empty((height, width), dtype=torch.int32, device=dev)
    if want_mask and mask is None:
        mask = torch.empty((height, wpr), dtype=torch.int32, device=dev)
    need = pip_raster_workspace_bytes(tables.num_polygons, width, height)
    if workspace is None:
        workspace = torch.empty(max(need, 16), dtype=torch.uint8, device=dev)
    _check(lib().pip_rasterize(tables, int(width), int(height), float(x0), float(y0), float(dx), float(dy),
                               first_hit.data_ptr() if first_hit is not None else None,
                               mask.data_ptr() if mask is not None else None, workspace.data_ptr(),
                               workspace.numel() * workspace.element_size(), _stream(stream)), "pip_rasterize")
    return first_hit, mask


def pip_selftest_wait_timeout(tables: Tables, limit_cycles: int, stream=None) -> None:
    """Queue the self-test of a device-side wait that never completes (bounded by
    ``limit_cycles`` SM cycles); the next pip_get_status reports PIP_E_TIMEOUT."""
    scratch = torch.zeros(4096, dtype=torch.uint8, device=tables.device)
    _check(lib().pip_selftest_wait_timeout(tables, scratch.data_ptr(), int(limit_cycles), _stream(stream)),
           "pip_selftest_wait_timeout")
    tables._keep = scratch  # the copy reads it until the kernel ends


def pip_set_tuning_cache(path: str | None) -> None:
    """The autotuners' JSON cache file (None turns it off)."""
    _check(lib().pip_set_tuning_cache(os.fsencode(path) if path else None), "pip_set_tuning_cache")


def pip_fma_peak(sink: torch.Tensor, blocks_per_sm: int = 8, iters: int = 4096, stream=None) -> int:
    """Queue the pure float32 FMA kernel on the current device; returns the FMAs it performs
    (the caller times it).  ``sink`` is a float32 CUDA tensor of at least blocks x 256 elements."""
    _dev(sink, "sink")
    fmas = ctypes.c_int64(0)
    _check(lib().pip_fma_peak(int(blocks_per_sm), int(iters), sink.data_ptr(), sink.numel(), _stream(stream),
                              ctypes.byref(fmas)), "pip_fma_peak")
    return int(fmas.value)


def pip_test_single_noalloc(vertices: torch.Tensor, points: torch.Tensor, mask: torch.Tensor,
                            status: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """One polygon against points with no device allocation inside the call (for callers that
    cannot allocate: fixed-rate control loops, hosts that own the memory pool).  The caller
    passes every buffer; scratch is a static array inside libpip shared by all calls.  Every
    tensor must live on the same CUDA device; the call runs with that device current."""
    named = [(vertices, "vertices"), (points, "points"), (mask, "mask")]
    if status is not None:
        named.append((status, "status"))
    for t_, nm in named:
        _dev(t_, nm)
    device = vertices.device
    for t_, nm in named:
        if t_.device != device:
            raise ValueError("%s is on %s, vertices on %s: all tensors must share one device"
                             % (nm, t_.device, device))
    M = points.numel() // 2
    if mask.dtype != torch.int32 or mask.numel() < (M + 31) // 32:
        raise ValueError("mask must be int32 with at least ceil(num_points / 32) = %d words"
                         % ((M + 31) // 32))
    if status is not None and (status.dtype != torch.int32 or status.numel() < 1):
        raise ValueError("status must be an int32 tensor of at least one element")
    with torch.cuda.device(device):
        _check(lib().pip_test_single_noalloc(vertices.data_ptr(), _dtype_code(vertices),
                                             vertices.numel() // 2, points.data_ptr() if M else None,
                                             _dtype_code(points), M, mask.data_ptr() if M else None,
                                             status.data_ptr() if status is not None else None,
                                             _stream(stream)), "pip_test_single_noalloc")
    return mask


def pip_penalty_workspace_bytes(num_vertices: int, num_poses: int, num_points: int) -> int:
    return int(lib().pip_penalty_workspace_bytes(num_vertices, num_poses, num_points))


def _penalty_ws(vertices, poses, points):
    nb = pip_penalty_workspace_bytes(vertices.numel() // 2, poses.numel() // 3, points.numel() // 2)
    return torch.empty(nb, dtype=torch.uint8, device=vertices.device)


def pip_penalty_forward(vertices: torch.Tensor, poses: torch.Tensor, points: torch.Tensor, tau: float,
                        workspace: torch.Tensor | None = None, stream=None, cull: bool = False) -> torch.Tensor:
    """Collision penalty sum softplus(-margin/tau) over poses x points; fp64 scalar tensor.
    cull: leave out the pairs whose terms are exactly 0 in float32 (PIP_PENALTY_CULL)."""
    for t_, nm in ((vertices, "vertices"), (poses, "poses"), (points, "points")):
        _dev(t_, nm)
        if t_.dtype != torch.float32:
            raise TypeError("%s must be float32" % nm)
    ws = workspace if workspace is not None else _penalty_ws(vertices, poses, points)
    loss = torch.empty(1, dtype=torch.float64, device=vertices.device)
    _check(lib().pip_penalty_forward(vertices.data_ptr(), vertices.numel() // 2, poses.data_ptr(),
                                     poses.numel() // 3, points.data_ptr(), points.numel() // 2,
                                     float(tau), loss.data_ptr(), PIP_PENALTY_CULL if cull else 0,
                                     ws.data_ptr(), ws.numel(), _stream(stream)), "pip_penalty_forward")
    return loss[0]


def pip_penalty_backward(vertices: torch.Tensor, poses: torch.Tensor, points: torch.Tensor, tau: float,
                         grad_loss: torch.Tensor | None = None, workspace: torch.Tensor | None = None,
                         stream=None, cull: bool = False):
    """(d loss/d vertices [n, 2] fp64, d loss/d poses [P, 3] fp64), scaled by grad_loss.
    cull: leave out the pairs whose gradient is exactly 0 in float32 (PIP_PENALTY_CULL)."""
    ws = workspace if workspace is not None else _penalty_ws(vertices, poses, points)
    gv = torch.empty((vertices.numel() // 2, 2), dtype=torch.float64, device=vertices.device)
    gp = torch.empty((poses.numel() // 3, 3), dtype=torch.float64, device=vertices.device)
    go = None
    if grad_loss is not None:
        go = grad_loss.detach().to(device=vertices.device, dtype=torch.float32).reshape(1).contiguous()
    _check(lib().pip_penalty_backward(vertices.data_ptr(), vertices.numel() // 2, poses.data_ptr(),
                                      poses.numel() // 3, points.data_ptr(), points.numel() // 2,
                                      float(tau), go.data_ptr() if go is not None else None,
                                      gv.data_ptr(), gp.data_ptr(), PIP_PENALTY_CULL if cull else 0,
                                      ws.data_ptr(), ws.numel(), _stream(stream)), "pip_penalty_backward")
    return gv, gp


class CollisionPenalty(torch.autograd.Function):
    """L = sum_pose sum_point softplus(-margin(R^T (p - t)) / tau) with hand-written CUDA
    forward and backward kernels; gradients for the footprint vertices and the poses (the
    obstacle points are data).  The generator tables are rebuilt in backward.  cull: leave
    out the pairs whose terms and gradients are exactly 0 in float32 (PIP_PENALTY_CULL)."""

    @staticmethod
    def forward(ctx, vertices, poses, points, tau: float, cull: bool = False):
        v = vertices.detach().contiguous()
        p = poses.detach().contiguous()
        q = points.detach().contiguous()
        ctx.save_for_backward(v, p, q)
        ctx.tau = float(tau)
        ctx.cull = bool(cull)
        return pip_penalty_forward(v, p, q, ctx.tau, cull=ctx.cull)

    @staticmethod
    def backward(ctx, grad_out):
        v, p, q = ctx.saved_tensors
        gv, gp = pip_penalty_backward(v, p, q, ctx.tau, grad_loss=grad_out, cull=ctx.cull)
        return gv.to(v.dtype), gp.to(p.dtype), None, None, None


def collision_penalty(vertices, poses, points, tau: float, cull: bool = False):
    return CollisionPenalty.apply(vertices, poses, points, tau, cull)
