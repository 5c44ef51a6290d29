// pip_prepare_kernel.cuh -- the polygon -> generator-table kernel (Eq. 3-4,
// Eq. 8, expanded Eq. 11), shared by the translation units that launch it.
// Internal linkage: each includer gets its own copy.
#pragma once

#include <math.h>

#include "pip_internal.cuh"

using namespace pip;

namespace {

__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_max(double v)
{
    for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ double warp_min(double v)
{
    for (int o = 16; o; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ void load_vertex(const void *verts, int vdtype, int64_t i, double &x,
                                            double &y)
{
    if (vdtype == PIP_I32) {
        const int32_t *q = (const int32_t *)verts;
        x = (double)q[2 * i];
        y = (double)q[2 * i + 1];
    } else {
        const float *f = (const float *)verts;
        x = (double)f[2 * i];
        y = (double)f[2 * i + 1];
    }
}

__device__ __forceinline__ float round_up_f32(double v) { return __double2float_ru(v); }

// p0_kind: the inner generator (any interior point serves, Sec. 3):
// kP0Centroid the centroid of Eq. 3-4 (the paper's choice), kP0VertexMean the
// mean of the vertices, kP0Given p0_given[j] (absolute coordinates, e.g. the
// Chebyshev centre).  Whichever is taken must be clearly inside every edge
// line (checked below; otherwise PIP_E_DEGENERATE).
constexpr int kP0Centroid = 0, kP0VertexMean = 1, kP0Given = 2;

__global__ void __launch_bounds__(256) prepare_kernel(
    const void *__restrict__ verts, int vdtype, const int32_t *__restrict__ voffs, int P, int V,
    double2 *__restrict__ g0_out, double2 *__restrict__ gk_out, float4 *__restrict__ coef,
    float4 *__restrict__ coefn, PolyInfo *__restrict__ poly, int32_t *__restrict__ worst,
    int p0_kind = kP0Centroid, const double2 *__restrict__ p0_given = nullptr)
{
    const int lane = threadIdx.x & 31;
    const int j = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
    if (j >= P) return;  // warp-uniform

    const int voff = voffs[j];
    const int vend = voffs[j + 1];
    const int n = vend - voff;
    const bool range_ok = voff >= 0 && vend <= V && vend >= voff;
    int status = PIP_OK;
    if (!range_ok || n < kMinEdges || n > kMaxEdges) status = PIP_E_INVALID_ARG;

    double sx = 0.0, sy = 0.0;  // shift origin: vertex 0
    double S = 0.0, Cx = 0.0, Cy = 0.0, D = 0.0, Mx = 0.0, My = 0.0;
    int wraps[2] = {0, 0};  // vertices where the edge direction turns across angle 0, ccw / cw
    float bb[4] = {INFINITY, INFINITY, -INFINITY, -INFINITY};
    bool nonfinite = false, zero_edge = false, int_bad = false, fold = false;
    bool pos = false, neg = false;

    if (status == PIP_OK) {
        load_vertex(verts, vdtype, voff, sx, sy);
#pragma unroll
        for (int slot = 0; slot < 2; ++slot) {
            const int k = lane + 32 * slot;
            if (k >= n) continue;
            const int km = k == 0 ? n - 1 : k - 1;
            const int kp = k == n - 1 ? 0 : k + 1;
            double xm, ym, xk, yk, xp, yp;
            load_vertex(verts, vdtype, voff + km, xm, ym);
            load_vertex(verts, vdtype, voff + k, xk, yk);
            load_vertex(verts, vdtype, voff + kp, xp, yp);
            if (!isfinite(xk) || !isfinite(yk)) nonfinite = true;
            if (vdtype == PIP_I32 && (fabs(xk) > kIntLimit || fabs(yk) > kIntLimit)) int_bad = true;
            if (xk == xm && yk == ym) zero_edge = true;
            bb[0] = fminf(bb[0], (float)xk);
            bb[1] = fminf(bb[1], (float)yk);
            bb[2] = fmaxf(bb[2], (float)xk);
            bb[3] = fmaxf(bb[3], (float)yk);
            // Eq. 3-4 in coordinates relative to v_0
            const double uxm = xm - sx, uym = ym - sy, uxk = xk - sx, uyk = yk - sy;
            const double det = uxm * uyk - uxk * uym;
            Mx += uxk;  // vertex mean, relative to v_0
            My += uyk;
            S += det;
            Cx += (uxm + uxk) * det;
            Cy += (uym + uyk) * det;
            D = fmax(D, fmax(fabs(uxk), fabs(uyk)));
            // turn at vertex k (exact sign)
            const int o = orient_sign_exact(xm, ym, xk, yk, xp, yp);
            pos |= o > 0;
            neg |= o < 0;
            const double ex = xk - xm, ey = yk - ym, fx = xp - xk, fy = yp - yk;
            const double dt = ex * fx + ey * fy;
            if (o == 0 && !(dt > 0.0)) fold = true;
            // Winding of the edge direction: with every turn the same way
            // (each less than pi), the direction crosses angle 0 once per full
            // revolution, at the vertex where it passes from the lower
            // half-plane of directions [-pi, 0) to the upper one [0, pi)
            // (ccw) or back (cw).  Decided by comparisons of the coordinates
            // alone, so exact.
            const bool up_in = yk > ym || (yk == ym && xk > xm);
            const bool up_out = yp > yk || (yp == yk && xp > xk);
            wraps[0] += !up_in && up_out;
            wraps[1] += up_in && !up_out;
        }
        S = warp_sum(S);
        Cx = warp_sum(Cx);
        Cy = warp_sum(Cy);
        Mx = warp_sum(Mx);
        My = warp_sum(My);
        wraps[0] = __reduce_add_sync(0xffffffffu, wraps[0]);
        wraps[1] = __reduce_add_sync(0xffffffffu, wraps[1]);
        D = warp_max(D);
        nonfinite = __any_sync(0xffffffffu, nonfinite);
        int_bad = __any_sync(0xffffffffu, int_bad);
        zero_edge = __any_sync(0xffffffffu, zero_edge);
        fold = __any_sync(0xffffffffu, fold);
        pos = __any_sync(0xffffffffu, pos);
        neg = __any_sync(0xffffffffu, neg);
        for (int c = 0; c < 4; ++c) {
            double v = (double)bb[c];
            v = c < 2 ? warp_min(v) : warp_max(v);
            bb[c] = (float)v;
        }
        if (nonfinite) status = PIP_E_NONFINITE;
        else if (int_bad) status = PIP_E_INVALID_ARG;
        else if (zero_edge) status = PIP_E_DEGENERATE;
        else if (!pos && !neg) status = PIP_E_DEGENERATE;           // all collinear: zero area
        else if ((pos && neg) || fold) status = PIP_E_NONCONVEX;
        else if (wraps[pos ? 0 : 1] != 1) status = PIP_E_NONCONVEX;  // winds twice or more
        else if (!(S * (pos ? 1.0 : -1.0) > 0.0)) status = PIP_E_DEGENERATE;
    }

    const int sigma = pos ? 1 : -1;
    double g0x = 0.0, g0y = 0.0;
    if (status == PIP_OK) {
        if (p0_kind == kP0VertexMean) {
            g0x = Mx / n;
            g0y = My / n;
        } else if (p0_kind == kP0Given) {
            const double2 q = p0_given[j];
            g0x = q.x - sx;
            g0y = q.y - sy;
            if (!isfinite(g0x) || !isfinite(g0y)) status = PIP_E_DEGENERATE;
        } else {
            g0x = Cx / (3.0 * S);  // Eq. 4: sum / (6 A), 2A = S
            g0y = Cy / (3.0 * S);
        }
    }

    // Eq. 8 generators; the centroid must sit strictly inside every edge line
    double gkx[2] = {0.0, 0.0}, gky[2] = {0.0, 0.0};
    double G = fmax(fabs(g0x), fabs(g0y));
    bool not_interior = false;
    if (status == PIP_OK) {
#pragma unroll
        for (int slot = 0; slot < 2; ++slot) {
            const int k = lane + 32 * slot;
            if (k >= n) continue;
            const int km = k == 0 ? n - 1 : k - 1;
            double xm, ym, xk, yk;
            load_vertex(verts, vdtype, voff + km, xm, ym);
            load_vertex(verts, vdtype, voff + k, xk, yk);
            xm -= sx; ym -= sy; xk -= sx; yk -= sy;
            const double a = yk - ym;
            const double b = xm - xk;
            const double c = -(a * xk + b * yk);
            const double L0 = a * g0x + b * g0y + c;
            // interior: L_k(p0) has the sign opposite to the orientation, clearly
            if (!(sigma * L0 < 0.0) ||
                fabs(L0) <= ldexp((fabs(a) + fabs(b)) * (G + D), -40))
                not_interior = true;
            const double s2 = a * a + b * b;
            const double w11 = b * b - a * a, w12 = -2.0 * a * b, w22 = a * a - b * b;
            gkx[slot] = (w11 * g0x + w12 * g0y - 2.0 * c * a) / s2;
            gky[slot] = (w12 * g0x + w22 * g0y - 2.0 * c * b) / s2;
            G = fmax(G, fmax(fabs(gkx[slot]), fabs(gky[slot])));
        }
        G = warp_max(G);
        if (__any_sync(0xffffffffu, not_interior)) status = PIP_E_DEGENERATE;
    }

    PolyInfo info;
    info.voff = range_ok ? voff : 0;
    info.n = (range_ok && n >= 0) ? n : 0;
    info.status = status;
    info.orient = status == PIP_OK ? sigma : 0;
    info.bbox[0] = bb[0];
    info.bbox[1] = bb[1];
    info.bbox[2] = bb[2];
    info.bbox[3] = bb[3];
    info.tin = 0.f;
    info.tout = -INFINITY;

    if (status != PIP_OK) {
        // an invalid polygon contains nothing: s_k = -inf for its slots
        if (range_ok && n <= kMaxEdges) {
            for (int k = lane; k < n; k += 32) {
                coef[voff + k] = make_float4(0.f, 0.f, -INFINITY, 0.f);
                coefn[voff + k] = make_float4(0.f, 0.f, -INFINITY, 0.f);
                gk_out[voff + k] = make_double2(NAN, NAN);
            }
        }
        if (lane == 0) {
            info.ox = info.oy = 0.f;
            info.beta0 = info.beta1 = 0.f;
            info.gerr = 0.0;
            poly[j] = info;
            g0_out[j] = make_double2(NAN, NAN);
            atomicMax(worst, status);
        }
        return;
    }

    // local origin o = float32(p0), and o relative to the shift; when the
    // centroid is no farther from (0, 0) than the polygon's own extent, o is
    // (0, 0) itself and the kernels skip the subtraction
    const double g0ax = g0x + sx, g0ay = g0y + sy;
    const bool at_zero = fmax(fabs(g0ax), fabs(g0ay)) <= D;
    const float ox = at_zero ? 0.f : (float)g0ax, oy = at_zero ? 0.f : (float)g0ay;
    const double olx = (double)ox - sx, oly = (double)oy - sy;

    float tmax = 0.f, w1 = 0.f;
    double A = fmax(fabs(g0ax), fabs(g0ay));
#pragma unroll
    for (int slot = 0; slot < 2; ++slot) {
        const int k = lane + 32 * slot;
        if (k >= n) continue;
        const double dx = gkx[slot] - g0x, dy = gky[slot] - g0y;       // p_k - p0
        const double qx = gkx[slot] + g0x - 2.0 * olx;                  // p_k + p0 - 2 o
        const double qy = gky[slot] + g0y - 2.0 * oly;
        const double t = dx * qx + dy * qy;  // |p_k - o|^2 - |p0 - o|^2
        const float4 cf = make_float4((float)(2.0 * dx), (float)(2.0 * dy), (float)t, 0.f);
        coef[voff + k] = cf;
        const double nd = sqrt(dx * dx + dy * dy);
        coefn[voff + k] = make_float4((float)(dx / nd), (float)(dy / nd), (float)(t / (2.0 * nd)), 0.f);
        const double ax = gkx[slot] + sx, ay = gky[slot] + sy;
        gk_out[voff + k] = make_double2(ax, ay);
        A = fmax(A, fmax(fabs(ax), fabs(ay)));
        tmax = fmaxf(tmax, fabsf(cf.z));
        w1 = fmaxf(w1, fabsf(cf.x) + fabsf(cf.y));
    }
    tmax = (float)warp_max((double)tmax);
    w1 = (float)warp_max((double)w1);
    A = warp_max(A);

    // Disc bounds about o.  Outer: R^2 = max_k |v_k - o|^2 (v_k - o exact in
    // fp64: both are float32 values relative to the shift).  Inner: r = min_k
    // dist(o, edge line k), less the fp64 rounding of the line's value at o;
    // r <= 0 (o on or outside an edge line after rounding) leaves no inner disc.
    double R2 = 0.0, rin = INFINITY;
#pragma unroll
    for (int slot = 0; slot < 2; ++slot) {
        const int k = lane + 32 * slot;
        if (k >= n) continue;
        const int km = k == 0 ? n - 1 : k - 1;
        double xm, ym, xk, yk;
        load_vertex(verts, vdtype, voff + km, xm, ym);
        load_vertex(verts, vdtype, voff + k, xk, yk);
        xm -= sx; ym -= sy; xk -= sx; yk -= sy;
        const double vx = xk - olx, vy = yk - oly;
        R2 = fmax(R2, vx * vx + vy * vy);
        const double a = yk - ym, b = xm - xk;  // exact: differences of float32 values
        // L(o) = a (o - v_k)_x + b (o - v_k)_y, the line through v_k; inside: -sigma L > 0
        const double L = a * (olx - xk) + b * (oly - yk);
        const double eL = ldexp(fabs(a) * (fabs(olx) + fabs(xk)) + fabs(b) * (fabs(oly) + fabs(yk)), -49);
        const double d = (-sigma * L - eL) / (sqrt(a * a + b * b) * (1.0 + ldexp(1.0, -48)));
        rin = fmin(rin, d);
    }
    R2 = warp_max(R2);
    rin = warp_min(rin);

    if (lane == 0) {
        // Error bound of the float32 test, |computed s_k - exact s_k| <= B:
        // FMA chain 2.01u(|t| + |w|_1 |x|_inf), point rounding u |w|_1 |x|_inf,
        // coefficient rounding u(|t| + |w|_1 |x|_inf), fp64 construction error
        // E per coordinate of the generators; every constant doubled.  The
        // kernels use B = beta0 + beta1 (|x| + |y|) or beta1 max(|x|, |y|),
        // both at least beta0 + beta1 |x|_inf.
        const double u = ldexp(1.0, -24);
        const double E = ldexp(G + D, -40);
        const double b0 = 8.0 * u * tmax + 64.0 * E * (G + D) + ldexp(1.0, -120);
        const double b1 = 10.0 * u * w1 + 32.0 * E;
        info.ox = ox;
        info.oy = oy;
        info.beta0 = round_up_f32(b0);
        info.beta1 = round_up_f32(b1);
        info.gerr = E + ldexp(A, -51);
        // The kernels' d2 = fl(x x + fl(y y)) of x = fl(p - o) (or of p
        // itself when o = 0) lies within (1 +- u)^4 of the exact |p - o|^2
        // (normal range); 16u of slack, directed rounding of the thresholds,
        // and no inner disc at or below 2^-100 (subnormal squares)
        const double tin = rin > 0.0 ? rin * rin * (1.0 - 16.0 * u) : 0.0;
        info.tin = tin > ldexp(1.0, -100) ? __double2float_rd(tin) : 0.f;
        info.tout = R2 > ldexp(1.0, -100) ? round_up_f32(R2 * (1.0 + 16.0 * u)) : INFINITY;
        poly[j] = info;
        g0_out[j] = make_double2(g0ax, g0ay);
    }
}

// Integer polygons, for the exact refine: per edge k the start vertex
// v_{k-1} and the edge vector oriented by the polygon's turn, e_k = orient
// (v_k - v_{k-1}), so that p is inside (closed) iff cross(e_k, p - v_{k-1}) >= 0
// for every k.  |v| <= 2^24 keeps e_k in int32.  One warp per polygon;
// invalid polygons get nothing (the refine reads their status first).
__global__ void int_edge_kernel(const PolyInfo *__restrict__ poly, const int2 *__restrict__ verts, int P,
                                int4 *__restrict__ iedge)
{
    const int lane = threadIdx.x & 31;
    const int j = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
    if (j >= P) return;
    const PolyInfo pi = poly[j];
    if (pi.status != PIP_OK) return;
    for (int k = lane; k < pi.n; k += 32) {
        const int km = k == 0 ? pi.n - 1 : k - 1;
        const int2 a = verts[pi.voff + km], b = verts[pi.voff + k];
        iedge[pi.voff + k] = make_int4(a.x, a.y, pi.orient * (b.x - a.x), pi.orient * (b.y - a.y));
    }
}

// Integer polygons, for the exact batch test: per polygon a fixed-stride row
// of kPadStride edges, edge k as (e_x, -e_y, -C) with e = orient (v_k - v_{k-1})
// and C = e_x y_{k-1} - e_y x_{k-1}, so that
//     cross_k(p) = e_x (p_y - y_{k-1}) - e_y (p_x - x_{k-1}) = e_x p_y - e_y p_x - C
// is two 32 x 32 -> 64-bit multiply-adds, and p is inside (closed) iff every
// cross_k(p) >= 0.  |v| <= 2^24 and |p| < 2^31 keep every term below 2^57.
// Rows past n are zero (cross = 0: neutral); invalid polygons are skipped by
// their status.  The same edges also go to `fpad` as float32 (a_x, a_y, e_x, e_y),
// a = v_{k-1}, exact for polygons within +-2^22 (the float32 form of the exact
// test in the batch kernel).
__global__ void int_pad_kernel(const PolyInfo *__restrict__ poly, const int2 *__restrict__ verts, int P,
                               int4 *__restrict__ ipad, float4 *__restrict__ fpad)
{
    const int lane = threadIdx.x & 31;
    const int j = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
    if (j >= P) return;
    const PolyInfo pi = poly[j];
    const int n = pi.status == PIP_OK ? pi.n : 0;
    for (int k = lane; k < kPadStride; k += 32) {
        int4 r = make_int4(0, 0, 0, 0);
        float4 f = make_float4(0.f, 0.f, 0.f, 0.f);
        if (k < n) {
            const int km = k == 0 ? n - 1 : k - 1;
            const int2 a = verts[pi.voff + km], b = verts[pi.voff + k];
            const int ex = pi.orient * (b.x - a.x), ey = pi.orient * (b.y - a.y);
            const long long negC = (long long)ey * a.x - (long long)ex * a.y;
            r = make_int4(ex, -ey, (int)(unsigned)(negC & 0xffffffffll), (int)(negC >> 32));
            f = make_float4((float)a.x, (float)a.y, (float)ex, (float)ey);
        }
        ipad[(size_t)j * kPadStride + k] = r;
        fpad[(size_t)j * kPadStride + k] = f;
    }
}

}  // namespace
