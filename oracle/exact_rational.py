"""Alg. 3-5 of arXiv 2007.15385 in exact rational arithmetic, for tiny inputs.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  This is a second,
independent restatement of the paper's method, used to pin the C oracle: the
centroid of Eq. 3-4, the mirrored generators of Eq. 8 and the closed Voronoi
test of Alg. 5 (M_0 <= M_j for all j), all with ``fractions.Fraction`` so that
no rounding happens anywhere.  Pure-Python loops: keep n <= 16 and a few
thousand points.
"""
from __future__ import annotations

from fractions import Fraction


def _xy(verts):
    return [(Fraction(float(x)), Fraction(float(y))) for x, y in verts]


def centroid(verts):
    """Eq. 3-4: (signed area, (cx, cy)) exactly."""
    v = _xy(verts)
    n = len(v)
    s = Fraction(0)
    sx = Fraction(0)
    sy = Fraction(0)
    for k in range(n):
        xm, ym = v[k - 1]
        xk, yk = v[k]
        det = xm * yk - xk * ym
        s += det
        sx += (xm + xk) * det
        sy += (ym + yk) * det
    area = s / 2
    return area, (sx / (6 * area), sy / (6 * area))


def generators(verts, p0):
    """Eq. 8: the mirror of p0 across each edge line, exactly."""
    v = _xy(verts)
    n = len(v)
    out = []
    for k in range(n):
        xm, ym = v[k - 1]
        xk, yk = v[k]
        a = yk - ym
        b = xm - xk
        c = -(a * xk + b * yk)
        s = a * a + b * b
        px = ((b * b - a * a) * p0[0] - 2 * a * b * p0[1] - 2 * c * a) / s
        py = (-2 * a * b * p0[0] + (a * a - b * b) * p0[1] - 2 * c * b) / s
        out.append((px, py))
    return out


def voronoi_inclusion(verts, pts):
    """Alg. 5 with exact generators: 1 if |q - p0|^2 <= |q - p_k|^2 for every k."""
    _, p0 = centroid(verts)
    gens = generators(verts, p0)
    res = []
    for qx, qy in pts:
        qx = Fraction(float(qx))
        qy = Fraction(float(qy))
        m0 = (qx - p0[0]) ** 2 + (qy - p0[1]) ** 2
        res.append(int(all(m0 <= (qx - gx) ** 2 + (qy - gy) ** 2 for gx, gy in gens)))
    return res
