"""The oracle over every host core, for full-size parity checks.

Each helper cuts the work into contiguous pieces (points, or whole polygons
with their own points) and runs the oracle's C functions on one thread per
piece; those calls release the GIL, so the pieces run in parallel.  Nothing
here computes any part of the method: it only splits and concatenates.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

import oracle


def _threads() -> int:
    return max(1, os.cpu_count() or 1)


def inside_exact(verts, pts) -> np.ndarray:
    """oracle.inside_exact on every point, in contiguous pieces."""
    pts = np.ascontiguousarray(pts)
    pieces = np.array_split(np.arange(len(pts)), 4 * _threads())
    with ThreadPoolExecutor(_threads()) as ex:
        parts = list(ex.map(lambda ix: oracle.inside_exact(verts, pts[ix[0]:ix[-1] + 1])[0]
                            if len(ix) else np.zeros(0, np.uint8), pieces))
    return np.concatenate(parts)


def inside_exact_ragged(verts, voffs, pts, poffs) -> np.ndarray:
    """oracle.inside_exact_ragged on every point: groups of whole polygons,
    each group with its vertex and point ranges re-based to zero."""
    voffs = np.asarray(voffs, np.int64)
    poffs = np.asarray(poffs, np.int64)
    P = len(voffs) - 1
    # cut the polygons where the running point count crosses equal shares
    cuts = np.searchsorted(poffs, np.linspace(0, poffs[-1], 4 * _threads() + 1)[1:-1])
    bounds = np.unique(np.concatenate([[0], np.clip(cuts, 0, P), [P]]))

    def run(a, b):
        vo = (voffs[a:b + 1] - voffs[a]).astype(np.int32)
        po = poffs[a:b + 1] - poffs[a]
        v = verts[voffs[a]:voffs[b]]
        q = pts[poffs[a]:poffs[b]]
        return oracle.inside_exact_ragged(v, vo, q, po)[0]

    with ThreadPoolExecutor(_threads()) as ex:
        parts = list(ex.map(lambda ab: run(*ab), zip(bounds[:-1], bounds[1:])))
    return np.concatenate(parts) if parts else np.zeros(0, np.uint8)


def first_hit_exact(verts, voffs, pts) -> np.ndarray:
    """oracle.first_hit_exact on every point, in contiguous pieces."""
    pts = np.ascontiguousarray(pts)
    pieces = np.array_split(np.arange(len(pts)), 4 * _threads())
    with ThreadPoolExecutor(_threads()) as ex:
        parts = list(ex.map(lambda ix: oracle.first_hit_exact(verts, voffs, pts[ix[0]:ix[-1] + 1])
                            if len(ix) else np.zeros(0, np.int32), pieces))
    return np.concatenate(parts)
