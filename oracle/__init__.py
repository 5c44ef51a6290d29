"""CPU oracle for the Voronoi point-inclusion test (arXiv 2007.15385).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s ``cpu_baseline`` / ``--impl reference`` leg may import this
package.  The CUDA library and its Python binding never import, link or call
anything under ``oracle/``; the two share no code.

The arithmetic lives in ``pip_oracle.c`` (plain C, fp64, exact expansions and
128-bit integers), compiled here with gcc into ``liborc.so`` and called through
ctypes.  ``exact_rational.py`` holds a second, independent restatement in
exact rationals for tiny inputs, used only to pin this one.

What each function follows, and what pins it (tests/test_oracle_*.py):

=====================  ===============================  ==========================================
function               follows                          pinned by
=====================  ===============================  ==========================================
centroid               Eq. 3-4, Alg. 3                  regular n-gon area and centre, triangle mean,
                                                        orientation, integer translation, golden file
generators             Eq. 8, Alg. 4                    involution, Eq. 7 midpoint, Voronoi-vertex
                                                        equidistance, regular n-gon 2 r cos(pi/n),
                                                        Eq. 6 foot, golden file (unit square)
inside_exact           Eq. 1 via the identity           exact-rational Alg. 5 brute force (boundary
                       |x-p_k|^2-|x-p_0|^2 =            points included), vertices/edge points in,
                       4 L_k(p_0) L_k(x)/(a^2+b^2)      bbox outside, area Monte Carlo, translation
                                                        and 90-degree rotation invariance
inside_exact_ragged,   inside_exact per own polygon;    axis-aligned rectangles (both orientations)
first_hit_exact        lowest polygon index holding     against plain coordinate comparisons,
                       the point (closed)               lattice points on edges and corners;
                                                        non-convex and zero-area polygons hold nothing
raster_centres         pixel centres x0 + c dx,         exact rationals rounded once to float32
                       one rounding (C fmaf)
voronoi_fp64           Alg. 5 literally (fp64)          agreement with inside_exact off its own
                                                        ambiguity flag
sign_of_offset         Alg. 2 literally (fp64)          agreement with inside_exact off-boundary
ray_crossing           Alg. 1 (+x ray, odd = inside)    agreement with inside_exact off-boundary
margin                 Eq. 2 bisector distance          axis square = L-inf distance, zero on edge
                                                        lines, <= Euclidean distance outside
penalty (+ gradient)   softplus(-margin/tau) summed     central finite differences of penalty_loss,
                       over poses and points            closed-form point-to-line gradient,
                                                        translation invariance
polygon_status         convexity / degeneracy readings  hand-built bad polygons
=====================  ===============================  ==========================================

No function here is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pip_oracle.c")
_LIB = os.path.join(_HERE, "liborc.so")
# Tests that plant a mistake in a copy of pip_oracle.c point this at the copy.
_LIB_OVERRIDE = os.environ.get("PIP_ORACLE_LIB_OVERRIDE")

OK, INVALID, DEGENERATE, NONCONVEX, NONFINITE = 0, 1, 2, 3, 4
F32, I32 = 0, 1

_lib = None


def build(force: bool = False) -> str:
    """Compile pip_oracle.c into liborc.so with gcc (plain C11, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
             "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _get():
    global _lib
    if _lib is None:
        if _LIB_OVERRIDE:
            lib = ctypes.CDLL(_LIB_OVERRIDE)
        else:
            build()
            lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i32, i64, d = ctypes.c_int, ctypes.c_int64, ctypes.c_double
        sig = {
            "orc_polygon_status": (i32, [P, P, i32]),
            "orc_centroid": (None, [P, P, i32, P, P, P]),
            "orc_generators": (None, [P, P, i32, d, d, P, P]),
            "orc_foot": (None, [P, P, i32, i32, d, d, P, P]),
            "orc_voronoi_fp64": (i32, [P, i32, i32, P, i32, i64, P, P]),
            "orc_inside_exact": (i32, [P, i32, i32, P, i32, i64, P]),
            "orc_inside_exact_ragged": (i32, [P, i32, P, i32, P, i32, P, P]),
            "orc_first_hit_exact": (i32, [P, i32, P, i32, P, i32, i64, P]),
            "orc_raster_centres": (None, [i32, i32, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                          ctypes.c_float, P]),
            "orc_sign_of_offset": (None, [P, P, i32, P, i64, P]),
            "orc_ray_crossing": (None, [P, P, i32, P, i64, P]),
            "orc_margin": (i32, [P, P, i32, P, i64, P]),
            "orc_penalty": (i32, [P, P, i32, P, i32, P, i64, d, P, P, P]),
            "orc_penalty_loss": (i32, [P, P, i32, P, i32, P, i64, d, P]),
            "orc_generators_vjp": (None, [P, P, i32, d, d, P, P, P, P, P]),
            "orc_centroid_vjp": (None, [P, P, i32, d, d, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _xy64(v) -> tuple[np.ndarray, np.ndarray]:
    v = np.asarray(v, dtype=np.float64).reshape(-1, 2)
    return np.ascontiguousarray(v[:, 0]), np.ascontiguousarray(v[:, 1])


def _dtype_code(a: np.ndarray) -> int:
    if a.dtype == np.float32:
        return F32
    if a.dtype == np.int32:
        return I32
    raise TypeError("oracle inputs are float32 or int32 xy pairs, got %s" % a.dtype)


def polygon_status(verts) -> int:
    x, y = _xy64(verts)
    return int(_get().orc_polygon_status(_ptr(x), _ptr(y), len(x)))


def centroid(verts) -> tuple[float, np.ndarray]:
    """Eq. 3-4 / Alg. 3 in fp64: (signed area, centroid)."""
    x, y = _xy64(verts)
    a, cx, cy = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _get().orc_centroid(_ptr(x), _ptr(y), len(x), ctypes.byref(a), ctypes.byref(cx),
                        ctypes.byref(cy))
    return a.value, np.array([cx.value, cy.value])


def generators(verts, p0=None) -> np.ndarray:
    """Eq. 8 / Alg. 4 in fp64: outer generators [n, 2]; g[k] mirrors p0 across edge k."""
    x, y = _xy64(verts)
    if p0 is None:
        p0 = centroid(verts)[1]
    gx = np.empty(len(x))
    gy = np.empty(len(x))
    _get().orc_generators(_ptr(x), _ptr(y), len(x), float(p0[0]), float(p0[1]), _ptr(gx), _ptr(gy))
    return np.stack([gx, gy], axis=1)


def foot(verts, k: int, p0) -> np.ndarray:
    """Eq. 6: foot of the perpendicular from p0 to edge line k."""
    x, y = _xy64(verts)
    fx, fy = ctypes.c_double(), ctypes.c_double()
    _get().orc_foot(_ptr(x), _ptr(y), len(x), k, float(p0[0]), float(p0[1]),
                    ctypes.byref(fx), ctypes.byref(fy))
    return np.array([fx.value, fy.value])


def voronoi_fp64(verts: np.ndarray, pts: np.ndarray):
    """Alg. 5 literally in fp64.  Returns (isin uint8[m], ambiguous uint8[m], status)."""
    verts = np.ascontiguousarray(verts)
    pts = np.ascontiguousarray(pts)
    m = pts.size // 2
    isin = np.zeros(m, np.uint8)
    amb = np.zeros(m, np.uint8)
    st = _get().orc_voronoi_fp64(_ptr(verts), _dtype_code(verts), verts.size // 2, _ptr(pts),
                                 _dtype_code(pts), m, _ptr(isin), _ptr(amb))
    return isin, amb, int(st)


def inside_exact(verts: np.ndarray, pts: np.ndarray):
    """Exact closed-polygon membership (what Alg. 5 reaches).  Returns (uint8[m], status)."""
    verts = np.ascontiguousarray(verts)
    pts = np.ascontiguousarray(pts)
    m = pts.size // 2
    out = np.zeros(m, np.uint8)
    st = _get().orc_inside_exact(_ptr(verts), _dtype_code(verts), verts.size // 2, _ptr(pts),
                                 _dtype_code(pts), m, _ptr(out))
    return out, int(st)


def inside_exact_ragged(verts, voffs, pts, poffs):
    """Own-polygon batch: polygon j decides its own points [poffs[j], poffs[j+1])."""
    verts = np.ascontiguousarray(verts)
    pts = np.ascontiguousarray(pts)
    voffs = np.ascontiguousarray(voffs, dtype=np.int32)
    poffs = np.ascontiguousarray(poffs, dtype=np.int64)
    out = np.zeros(int(poffs[-1]), np.uint8)
    st = _get().orc_inside_exact_ragged(_ptr(verts), _dtype_code(verts), _ptr(voffs),
                                        len(voffs) - 1, _ptr(pts), _dtype_code(pts),
                                        _ptr(poffs), _ptr(out))
    return out, int(st)


def first_hit_exact(verts, voffs, pts):
    """All pairs: lowest polygon index holding each point, or -1."""
    verts = np.ascontiguousarray(verts)
    pts = np.ascontiguousarray(pts)
    voffs = np.ascontiguousarray(voffs, dtype=np.int32)
    m = pts.size // 2
    out = np.empty(m, np.int32)
    _get().orc_first_hit_exact(_ptr(verts), _dtype_code(verts), _ptr(voffs), len(voffs) - 1,
                               _ptr(pts), _dtype_code(pts), m, _ptr(out))
    return out


def raster_centres(width, height, x0, y0, dx, dy) -> np.ndarray:
    """Pixel centres of the rasterisation grid, float32 [height * width, 2] row-major."""
    out = np.empty((int(width) * int(height), 2), np.float32)
    _get().orc_raster_centres(int(width), int(height), float(x0), float(y0), float(dx), float(dy), _ptr(out))
    return out


def sign_of_offset(verts, pts) -> np.ndarray:
    """Alg. 2 literally, fp64."""
    x, y = _xy64(verts)
    q = np.ascontiguousarray(np.asarray(pts, dtype=np.float64).reshape(-1, 2))
    out = np.zeros(len(q), np.uint8)
    _get().orc_sign_of_offset(_ptr(x), _ptr(y), len(x), _ptr(q), len(q), _ptr(out))
    return out


def ray_crossing(verts, pts) -> np.ndarray:
    """Alg. 1 literally, fp64, odd crossing count = inside."""
    x, y = _xy64(verts)
    q = np.ascontiguousarray(np.asarray(pts, dtype=np.float64).reshape(-1, 2))
    out = np.zeros(len(q), np.uint8)
    _get().orc_ray_crossing(_ptr(x), _ptr(y), len(x), _ptr(q), len(q), _ptr(out))
    return out


def margin(verts, pts) -> np.ndarray:
    """Signed Voronoi margin (largest bisector distance), fp64."""
    x, y = _xy64(verts)
    q = np.ascontiguousarray(np.asarray(pts, dtype=np.float64).reshape(-1, 2))
    out = np.zeros(len(q))
    st = _get().orc_margin(_ptr(x), _ptr(y), len(x), _ptr(q), len(q), _ptr(out))
    if st != OK:
        raise ValueError("invalid polygon (status %d)" % st)
    return out


def penalty(verts, poses, pts, tau: float):
    """Loss, d loss / d vertices [n, 2], d loss / d poses [P, 3]; all fp64."""
    x, y = _xy64(verts)
    poses = np.ascontiguousarray(np.asarray(poses, dtype=np.float64).reshape(-1, 3))
    q = np.ascontiguousarray(np.asarray(pts, dtype=np.float64).reshape(-1, 2))
    loss = ctypes.c_double()
    gv = np.zeros((len(x), 2))
    gp = np.zeros_like(poses)
    st = _get().orc_penalty(_ptr(x), _ptr(y), len(x), _ptr(poses), len(poses), _ptr(q), len(q),
                            float(tau), ctypes.byref(loss), _ptr(gv), _ptr(gp))
    if st != OK:
        raise ValueError("invalid polygon (status %d)" % st)
    return loss.value, gv, gp


def penalty_loss(verts, poses, pts, tau: float) -> float:
    x, y = _xy64(verts)
    poses = np.ascontiguousarray(np.asarray(poses, dtype=np.float64).reshape(-1, 3))
    q = np.ascontiguousarray(np.asarray(pts, dtype=np.float64).reshape(-1, 2))
    loss = ctypes.c_double()
    st = _get().orc_penalty_loss(_ptr(x), _ptr(y), len(x), _ptr(poses), len(poses), _ptr(q),
                                 len(q), float(tau), ctypes.byref(loss))
    if st != OK:
        raise ValueError("invalid polygon (status %d)" % st)
    return loss.value


def generators_vjp(verts, p0, G):
    """d/dp0 and d/dv of sum_k G[k] . p_k(p0, v) (Eq. 8).  Returns (dp0 [2], dv [n, 2])."""
    x, y = _xy64(verts)
    G = np.ascontiguousarray(np.asarray(G, dtype=np.float64).reshape(-1, 2))
    gx, gy = np.ascontiguousarray(G[:, 0]), np.ascontiguousarray(G[:, 1])
    g0x, g0y = ctypes.c_double(0.0), ctypes.c_double(0.0)
    dv = np.zeros((len(x), 2))
    _get().orc_generators_vjp(_ptr(x), _ptr(y), len(x), float(p0[0]), float(p0[1]), _ptr(gx),
                              _ptr(gy), ctypes.byref(g0x), ctypes.byref(g0y), _ptr(dv))
    return np.array([g0x.value, g0y.value]), dv


def centroid_vjp(verts, G0):
    """d/dv of G0 . p0(v) (Eq. 3-4).  Returns dv [n, 2]."""
    x, y = _xy64(verts)
    dv = np.zeros((len(x), 2))
    _get().orc_centroid_vjp(_ptr(x), _ptr(y), len(x), float(G0[0]), float(G0[1]), _ptr(dv))
    return dv
