/*
 * pip_oracle.c -- CPU oracle for the Voronoi point-inclusion test of
 * Zengin & Sezer, "A Novel Point Inclusion Test for Convex Polygons Based on
 * Voronoi Tessellations" (arXiv 2007.15385).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and
 * bench.py's cpu_baseline / reference leg may load this file.  The CUDA
 * library never links, includes or calls it, and it shares no code, header,
 * table or constant with the CUDA library.
 *
 * Everything here is plain and slow on purpose: one point at a time, one edge
 * at a time, in the order the paper states its steps.  Compile with
 * -ffp-contract=off so that the compiler does not fuse a*b+c behind our back.
 *
 * Conventions (the readings of the paper that this file takes):
 *   - A polygon has n >= 3 vertices v_0..v_{n-1}; edge k joins v_{k-1} and v_k
 *     (indices cyclic).  This is the paper's "rolled" vertex array V' (Alg. 1-4)
 *     written with an index shift.
 *   - Generator 0 is the centroid (Eq. 4); generator k (k = 1..n) is the
 *     centroid mirrored across edge k (Eq. 8).  Arrays of outer generators are
 *     0-based: g[k] belongs to edge k.
 *   - The boundary is closed: Eq. 1 and Alg. 5 use "<=", so a point on an edge
 *     is inside.
 *   - A point with a NaN or infinite coordinate is outside.
 *
 * Parity status of each function is listed in the header of oracle/__init__.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_INVALID 1
#define ORC_DEGENERATE 2
#define ORC_NONCONVEX 3
#define ORC_NONFINITE 4

/* ------------------------------------------------------------------------ */
/* Exact sign of a sum of products, by floating-point expansions.            */
/* Shewchuk, "Adaptive Precision Floating-Point Arithmetic and Fast Robust    */
/* Geometric Predicates", Discrete Comput. Geom. 18 (1997): Two-Sum (Thm 7),  */
/* the exact product error (here through a fused multiply-add), and           */
/* Grow-Expansion (Thm 10).  The sign of a nonoverlapping expansion is the    */
/* sign of its largest nonzero component.  Exact as long as no product        */
/* underflows or overflows, which holds for every float32 or int32 input.     */
/* ------------------------------------------------------------------------ */

static void two_sum(double a, double b, double *s, double *e)
{
    double x = a + b;
    double bv = x - a;
    double av = x - bv;
    *s = x;
    *e = (a - av) + (b - bv);
}

/* Add b into the expansion e[0..len); returns the new length (len + 1). */
static int grow_expansion(double *e, int len, double b)
{
    double q = b;
    for (int i = 0; i < len; i++) {
        double h;
        two_sum(q, e[i], &q, &h);
        e[i] = h;
    }
    e[len] = q;
    return len + 1;
}

static int expansion_sign(const double *e, int len)
{
    for (int i = len - 1; i >= 0; i--)
        if (e[i] != 0.0) return e[i] > 0.0 ? 1 : -1;
    return 0;
}

/* Add the exact value of s*u*v (s = +1 or -1) to the expansion. */
static int grow_product(double *e, int len, double s, double u, double v)
{
    double p = u * v;
    double err = fma(u, v, -p); /* exact: u*v = p + err */
    len = grow_expansion(e, len, s * err);
    len = grow_expansion(e, len, s * p);
    return len;
}

/* Exact sign of the cross product (b - a) x (c - a), i.e. of
 *   (bx - ax)(cy - ay) - (by - ay)(cx - ax)
 * = bx*cy - bx*ay - ax*cy - by*cx + by*ax + ay*cx      (the ax*ay terms cancel)
 * This is the two-point line form (Eq. 5) of the line through a and b,
 * evaluated at c.  Positive when c is left of the directed line a -> b. */
static int orient_exact(double ax, double ay, double bx, double by, double cx, double cy)
{
    double e[12];
    int len = 0;
    len = grow_product(e, len, +1.0, bx, cy);
    len = grow_product(e, len, -1.0, bx, ay);
    len = grow_product(e, len, -1.0, ax, cy);
    len = grow_product(e, len, -1.0, by, cx);
    len = grow_product(e, len, +1.0, by, ax);
    len = grow_product(e, len, +1.0, ay, cx);
    return expansion_sign(e, len);
}

/* Exact sign of the dot product (b - a) . (c - b). */
static int dot_sign_exact(double ax, double ay, double bx, double by, double cx, double cy)
{
    /* (bx-ax)(cx-bx) + (by-ay)(cy-by)
     * = bx*cx - bx*bx - ax*cx + ax*bx + by*cy - by*by - ay*cy + ay*by */
    double e[16];
    int len = 0;
    len = grow_product(e, len, +1.0, bx, cx);
    len = grow_product(e, len, -1.0, bx, bx);
    len = grow_product(e, len, -1.0, ax, cx);
    len = grow_product(e, len, +1.0, ax, bx);
    len = grow_product(e, len, +1.0, by, cy);
    len = grow_product(e, len, -1.0, by, by);
    len = grow_product(e, len, -1.0, ay, cy);
    len = grow_product(e, len, +1.0, ay, by);
    return expansion_sign(e, len);
}

/* Exact sign of twice the signed area, sum_k det[v_{k-1} v_k] (Eq. 3). */
static int area_sign_exact(const double *x, const double *y, int n)
{
    double *e = (double *)malloc(sizeof(double) * (size_t)(4 * n + 4));
    int len = 0;
    for (int k = 0; k < n; k++) {
        int km = (k + n - 1) % n;
        len = grow_product(e, len, +1.0, x[km], y[k]);
        len = grow_product(e, len, -1.0, x[k], y[km]);
    }
    int s = expansion_sign(e, len);
    free(e);
    return s;
}

static int sgn_cmp(double a, double b) { return (a > b) - (a < b); }

/* ------------------------------------------------------------------------ */
/* Polygon validity.  The paper assumes a convex polygon (Sec. 3) and does   */
/* not say what happens otherwise; the readings here: a repeated consecutive  */
/* vertex or zero area is degenerate (Eq. 8 and Eq. 4 divide by zero), and a  */
/* polygon that turns both ways, folds back on itself, or winds more than     */
/* once is non-convex.  All decisions are exact.                              */
/* ------------------------------------------------------------------------ */
int orc_polygon_status(const double *x, const double *y, int n)
{
    if (n < 3) return ORC_INVALID;
    for (int i = 0; i < n; i++)
        if (!isfinite(x[i]) || !isfinite(y[i])) return ORC_NONFINITE;
    for (int k = 0; k < n; k++) {
        int km = (k + n - 1) % n;
        if (x[k] == x[km] && y[k] == y[km]) return ORC_DEGENERATE;
    }
    int sigma = area_sign_exact(x, y, n);
    if (sigma == 0) return ORC_DEGENERATE;
    /* every turn is to the same side as the area, or straight ahead */
    for (int k = 0; k < n; k++) {
        int km = (k + n - 1) % n, kp = (k + 1) % n;
        int t = orient_exact(x[km], y[km], x[k], y[k], x[kp], y[kp]);
        if (t == -sigma) return ORC_NONCONVEX;
        if (t == 0 && dot_sign_exact(x[km], y[km], x[k], y[k], x[kp], y[kp]) <= 0)
            return ORC_NONCONVEX; /* folds back */
    }
    /* the edge directions sweep around once: the sign of dx (and of dy)
     * changes at most twice around the polygon */
    for (int axis = 0; axis < 2; axis++) {
        const double *c = axis == 0 ? x : y;
        int first = 0, prev = 0, changes = 0;
        for (int k = 0; k < n; k++) {
            int km = (k + n - 1) % n;
            int s = sgn_cmp(c[k], c[km]);
            if (s == 0) continue;
            if (first == 0) first = s;
            else if (s != prev) changes++;
            prev = s;
        }
        if (first != 0 && prev != first) changes++;
        if (changes > 2) return ORC_NONCONVEX;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Alg. 3 (CalculateCentroid): Eq. 3 area and Eq. 4 centroid, in fp64.       */
/*   A_k = V'_x V_y - V_x V'_y = x_{k-1} y_k - x_k y_{k-1}                    */
/*   a   = (1/2) sum_k A_k                                                    */
/*   mu  = sum_k (v_k + v_{k-1}) A_k / (6 a)                                  */
/* ------------------------------------------------------------------------ */
void orc_centroid(const double *x, const double *y, int n,
                  double *area, double *cx, double *cy)
{
    double a = 0.0, sx = 0.0, sy = 0.0;
    for (int k = 0; k < n; k++) {
        int km = (k + n - 1) % n;
        double Ak = x[km] * y[k] - x[k] * y[km];
        a += Ak;
        sx += (x[k] + x[km]) * Ak;
        sy += (y[k] + y[km]) * Ak;
    }
    a *= 0.5;
    *area = a;
    *cx = sx / (6.0 * a);
    *cy = sy / (6.0 * a);
}

/* ------------------------------------------------------------------------ */
/* Alg. 4 (CalculateGenerators) / Eq. 8, in fp64.  For edge k:               */
/*   a = V_y - V'_y,  b = V'_x - V_x,  c = -(a V_x + b V_y)                   */
/*   W = [[b^2 - a^2, -2ab], [-2ab, a^2 - b^2]]                               */
/*   p_k = (W p_0 - 2 c [a; b]) / (a^2 + b^2)                                  */
/* ------------------------------------------------------------------------ */
void orc_generators(const double *x, const double *y, int n, double g0x, double g0y,
                    double *gx, double *gy)
{
    for (int k = 0; k < n; k++) {
        int km = (k + n - 1) % n;
        double a = y[k] - y[km];
        double b = x[km] - x[k];
        double c = -(a * x[k] + b * y[k]);
        double w11 = b * b - a * a, w12 = -2.0 * a * b;
        double w21 = -2.0 * a * b, w22 = a * a - b * b;
        double d1 = w11 * g0x + w12 * g0y;
        double d2 = w21 * g0x + w22 * g0y;
        double e1 = -2.0 * c * a;
        double e2 = -2.0 * c * b;
        double s = a * a + b * b;
        gx[k] = (d1 + e1) / s;
        gy[k] = (d2 + e2) / s;
    }
}

/* Eq. 6: foot of the perpendicular from p0 to edge line k. */
void orc_foot(const double *x, const double *y, int n, int k, double p0x, double p0y,
              double *fx, double *fy)
{
    int km = (k + n - 1) % n;
    double a = y[k] - y[km];
    double b = x[km] - x[k];
    double c = -(a * x[k] + b * y[k]);
    double s = a * a + b * b;
    *fx = (b * b * p0x - a * b * p0y - c * a) / s;
    *fy = (-a * b * p0x + a * a * p0y - c * b) / s;
}

static void to_double_xy(const void *xy, int dtype, int64_t i, double *px, double *py)
{
    if (dtype == 0) {
        const float *f = (const float *)xy;
        *px = (double)f[2 * i];
        *py = (double)f[2 * i + 1];
    } else {
        const int32_t *q = (const int32_t *)xy;
        *px = (double)q[2 * i];
        *py = (double)q[2 * i + 1];
    }
}

/* ------------------------------------------------------------------------ */
/* Alg. 5 (VoronoiInclusion) literally, in fp64.                             */
/*   Delta_jk = q_k - P_j,  M_jk = sum Delta^2,  IsIn = M_0 <= M_j for all j. */
/* dtype 0 = float32 xy pairs, 1 = int32 xy pairs (vertices and points).      */
/* amb[i] = 1 marks a point whose fp64 comparison is within this oracle's own */
/* error estimate of a tie (|M_j - M_0| <= 2^-36 (M_0 + M_j + R^2), R the     */
/* largest coordinate involved); there the fp64 decision is not trusted.      */
/* Returns a status code; isin is left untouched for an invalid polygon.     */
/* ------------------------------------------------------------------------ */
int orc_voronoi_fp64(const void *vxy, int vdtype, int n, const void *pxy, int pdtype,
                     int64_t m, uint8_t *isin, uint8_t *amb)
{
    if (n < 3) return ORC_INVALID;
    double *x = (double *)malloc(sizeof(double) * (size_t)n * 4);
    double *y = x + n, *gx = x + 2 * n, *gy = x + 3 * n;
    for (int k = 0; k < n; k++) to_double_xy(vxy, vdtype, k, &x[k], &y[k]);
    int st = orc_polygon_status(x, y, n);
    if (st != ORC_OK) { free(x); return st; }
    double area, g0x, g0y;
    orc_centroid(x, y, n, &area, &g0x, &g0y);
    orc_generators(x, y, n, g0x, g0y, gx, gy);
    double R = fmax(fabs(g0x), fabs(g0y));
    for (int k = 0; k < n; k++) {
        R = fmax(R, fmax(fabs(x[k]), fabs(y[k])));
        R = fmax(R, fmax(fabs(gx[k]), fabs(gy[k])));
    }
    for (int64_t i = 0; i < m; i++) {
        double qx, qy;
        to_double_xy(pxy, pdtype, i, &qx, &qy);
        if (!isfinite(qx) || !isfinite(qy)) {
            isin[i] = 0;
            if (amb) amb[i] = 0;
            continue;
        }
        double Rq = fmax(R, fmax(fabs(qx), fabs(qy)));
        double d0x = qx - g0x, d0y = qy - g0y;
        double M0 = d0x * d0x + d0y * d0y;
        int in = 1, ambig = 0;
        for (int k = 0; k < n; k++) {
            double dx = qx - gx[k], dy = qy - gy[k];
            double Mk = dx * dx + dy * dy;
            if (!(M0 <= Mk)) in = 0;
            if (fabs(Mk - M0) <= ldexp(M0 + Mk + Rq * Rq, -36)) ambig = 1;
        }
        isin[i] = (uint8_t)in;
        if (amb) amb[i] = (uint8_t)ambig;
    }
    free(x);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* The exact result that Alg. 5 reaches.  For an interior inner generator    */
/* p0 and its mirror p_k across edge line L_k(x) = a x1 + b x2 + c,           */
/*   |x - p_k|^2 - |x - p0|^2 = 4 L_k(p0) L_k(x) / (a^2 + b^2),               */
/* and L_k(p0) has the polygon's orientation sign for every k, so Eq. 1 holds */
/* exactly when x is on the inner side of, or on, every edge line: the closed */
/* convex polygon.  That is what this function decides, with exact signs.    */
/* out[i] = 1 inside (boundary included), 0 outside.                          */
/* ------------------------------------------------------------------------ */
static int inside_exact_d(const double *x, const double *y, int n, int sigma,
                          double qx, double qy)
{
    if (!isfinite(qx) || !isfinite(qy)) return 0;
    for (int k = 0; k < n; k++) {
        int km = (k + n - 1) % n;
        int s = orient_exact(x[km], y[km], x[k], y[k], qx, qy);
        if (s == -sigma) return 0;
    }
    return 1;
}

/* exact integer version: every quantity is an int32 difference product, held
 * in 128-bit integers, so no rounding happens at all */
static int inside_exact_i(const int32_t *v, int n, int sigma, int32_t qx, int32_t qy)
{
    for (int k = 0; k < n; k++) {
        int km = (k + n - 1) % n;
        __int128 ex = (__int128)v[2 * k] - v[2 * km];
        __int128 ey = (__int128)v[2 * k + 1] - v[2 * km + 1];
        __int128 dx = (__int128)qx - v[2 * km];
        __int128 dy = (__int128)qy - v[2 * km + 1];
        __int128 cr = ex * dy - ey * dx;
        int s = (cr > 0) - (cr < 0);
        if (s == -sigma) return 0;
    }
    return 1;
}

int orc_inside_exact(const void *vxy, int vdtype, int n, const void *pxy, int pdtype,
                     int64_t m, uint8_t *out)
{
    if (n < 3) return ORC_INVALID;
    double *x = (double *)malloc(sizeof(double) * (size_t)n * 2);
    double *y = x + n;
    for (int k = 0; k < n; k++) to_double_xy(vxy, vdtype, k, &x[k], &y[k]);
    int st = orc_polygon_status(x, y, n);
    if (st != ORC_OK) { free(x); return st; }
    int sigma = area_sign_exact(x, y, n);
    for (int64_t i = 0; i < m; i++) {
        if (vdtype == 1 && pdtype == 1) {
            const int32_t *q = (const int32_t *)pxy;
            out[i] = (uint8_t)inside_exact_i((const int32_t *)vxy, n, sigma, q[2 * i], q[2 * i + 1]);
        } else {
            double qx, qy;
            to_double_xy(pxy, pdtype, i, &qx, &qy);
            out[i] = (uint8_t)inside_exact_d(x, y, n, sigma, qx, qy);
        }
    }
    free(x);
    return ORC_OK;
}

/* Own-polygon batches: polygon j owns points [poffs[j], poffs[j+1]) and
 * vertices [voffs[j], voffs[j+1]).  Returns the first bad status, if any,
 * after deciding every valid polygon. */
int orc_inside_exact_ragged(const void *vxy, int vdtype, const int32_t *voffs, int P,
                            const void *pxy, int pdtype, const int64_t *poffs, uint8_t *out)
{
    int worst = ORC_OK;
    for (int j = 0; j < P; j++) {
        size_t vb = vdtype == 0 ? sizeof(float) : sizeof(int32_t);
        size_t pb = pdtype == 0 ? sizeof(float) : sizeof(int32_t);
        const char *v = (const char *)vxy + 2 * vb * (size_t)voffs[j];
        const char *p = (const char *)pxy + 2 * pb * (size_t)poffs[j];
        int st = orc_inside_exact(v, vdtype, voffs[j + 1] - voffs[j], p, pdtype,
                                  poffs[j + 1] - poffs[j], out + poffs[j]);
        if (st != ORC_OK && worst == ORC_OK) worst = st;
    }
    return worst;
}

/* All-pairs first hit: for each point, the lowest polygon index whose closed
 * polygon holds it, or -1.  Invalid polygons hold nothing. */
int orc_first_hit_exact(const void *vxy, int vdtype, const int32_t *voffs, int P,
                        const void *pxy, int pdtype, int64_t m, int32_t *out)
{
    int total = voffs[P];
    double *x = (double *)malloc(sizeof(double) * (size_t)(2 * total + 2));
    double *y = x + total + 1;
    int *sigma = (int *)malloc(sizeof(int) * (size_t)(P + 1));
    for (int i = 0; i < total; i++) to_double_xy(vxy, vdtype, i, &x[i], &y[i]);
    for (int j = 0; j < P; j++) {
        int n = voffs[j + 1] - voffs[j];
        int st = orc_polygon_status(x + voffs[j], y + voffs[j], n);
        sigma[j] = st == ORC_OK ? area_sign_exact(x + voffs[j], y + voffs[j], n) : 0;
    }
    for (int64_t i = 0; i < m; i++) {
        out[i] = -1;
        for (int j = 0; j < P; j++) {
            if (sigma[j] == 0) continue;
            int n = voffs[j + 1] - voffs[j];
            int in;
            if (vdtype == 1 && pdtype == 1) {
                const int32_t *q = (const int32_t *)pxy;
                in = inside_exact_i((const int32_t *)vxy + 2 * voffs[j], n, sigma[j],
                                    q[2 * i], q[2 * i + 1]);
            } else {
                double qx, qy;
                to_double_xy(pxy, pdtype, i, &qx, &qy);
                in = inside_exact_d(x + voffs[j], y + voffs[j], n, sigma[j], qx, qy);
            }
            if (in) { out[i] = j; break; }
        }
    }
    free(x);
    free(sigma);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Alg. 2 (SignOfOffsetInclusion), literally, in fp64.                        */
/*   dV = V - V';  LHS = Q_y dV_x - Q_x dV_y;  RHS = V'_y dV_x - V'_x dV_y;   */
/*   D = LHS < RHS;  IsIn = (sum_k D_k mod n) == 0                             */
/* ------------------------------------------------------------------------ */
void orc_sign_of_offset(const double *x, const double *y, int n, const double *q,
                        int64_t m, uint8_t *isin)
{
    for (int64_t i = 0; i < m; i++) {
        double qx = q[2 * i], qy = q[2 * i + 1];
        int sumD = 0;
        for (int k = 0; k < n; k++) {
            int km = (k + n - 1) % n;
            double dvx = x[k] - x[km], dvy = y[k] - y[km];
            double lhs = qy * dvx - qx * dvy;
            double rhs = y[km] * dvx - x[km] * dvy;
            sumD += (lhs < rhs) ? 1 : 0;
        }
        isin[i] = (uint8_t)((sumD % n) == 0);
    }
}

/* ------------------------------------------------------------------------ */
/* Alg. 1 (CrossingInclusion), literally, in fp64, with a +x ray.            */
/*   InRange = (V_y > Q_y) xor (V'_y > Q_y);  GoingUp = V_y > V'_y;            */
/*   OnLeft  = GoingUp ? LHS > RHS : LHS < RHS;  Crossing = InRange and OnLeft */
/* The listing ends with "sum mod 2 = 0"; the text of Sec. 2.1 says an odd    */
/* count means inside, which this function follows.                           */
/* ------------------------------------------------------------------------ */
void orc_ray_crossing(const double *x, const double *y, int n, const double *q,
                      int64_t m, uint8_t *isin)
{
    for (int64_t i = 0; i < m; i++) {
        double qx = q[2 * i], qy = q[2 * i + 1];
        int crossings = 0;
        for (int k = 0; k < n; k++) {
            int km = (k + n - 1) % n;
            double dvx = x[k] - x[km], dvy = y[k] - y[km];
            int in_range = (y[k] > qy) != (y[km] > qy);
            int going_up = y[k] > y[km];
            double lhs = qy * dvx - qx * dvy;
            double rhs = y[km] * dvx - x[km] * dvy;
            int on_left = going_up ? (lhs > rhs) : (lhs < rhs);
            crossings += (in_range && on_left) ? 1 : 0;
        }
        isin[i] = (uint8_t)((crossings % 2) == 1);
    }
}

/* ------------------------------------------------------------------------ */
/* Signed Voronoi margin, in fp64.  The paper defines edge k as the points    */
/* equidistant from p0 and p_k (Eq. 2); the signed distance of x from that     */
/* bisector is (|x - p0|^2 - |x - p_k|^2) / (2 |p_k - p0|).  The margin is the */
/* largest of these over k: positive outside, <= 0 inside, in length units.   */
/* ------------------------------------------------------------------------ */
int orc_margin(const double *x, const double *y, int n, const double *q, int64_t m,
               double *out)
{
    int st = orc_polygon_status(x, y, n);
    if (st != ORC_OK) return st;
    double *gx = (double *)malloc(sizeof(double) * (size_t)n * 2);
    double *gy = gx + n;
    double area, g0x, g0y;
    orc_centroid(x, y, n, &area, &g0x, &g0y);
    orc_generators(x, y, n, g0x, g0y, gx, gy);
    for (int64_t i = 0; i < m; i++) {
        double qx = q[2 * i], qy = q[2 * i + 1];
        double best = -INFINITY;
        for (int k = 0; k < n; k++) {
            double n0 = (qx - g0x) * (qx - g0x) + (qy - g0y) * (qy - g0y);
            double nk = (qx - gx[k]) * (qx - gx[k]) + (qy - gy[k]) * (qy - gy[k]);
            double D = sqrt((gx[k] - g0x) * (gx[k] - g0x) + (gy[k] - g0y) * (gy[k] - g0y));
            double mk = (n0 - nk) / (2.0 * D);
            if (mk > best) best = mk;
        }
        out[i] = best;
    }
    free(gx);
    return ORC_OK;
}

/* Vector-Jacobian product of Eq. 8 (written as p_k = p0 - 2 L_k(p0) (a, b) / (a^2 + b^2),
 * L_k(p0) = a p0x + b p0y + c, a = y_k - y_{k-1}, b = x_{k-1} - x_k,
 * c = x_k y_{k-1} - x_{k-1} y_k).  Given G_k = dL/dp_k, adds dL/dp0 into *G0x, *G0y
 * and dL/dv into grad_v[n][2]. */
void orc_generators_vjp(const double *x, const double *y, int n, double g0x, double g0y,
                        const double *Gkx, const double *Gky, double *G0x, double *G0y,
                        double *grad_v)
{
    for (int k = 0; k < n; k++) {
        int km = (k + n - 1) % n;
        double a = y[k] - y[km], b = x[km] - x[k];
        double cc = -(a * x[k] + b * y[k]);
        double sq = a * a + b * b;
        double Lk = a * g0x + b * g0y + cc;
        double Gx = Gkx[k], Gy = Gky[k];
        double nG = a * Gx + b * Gy; /* (a,b) . G */
        /* dp_k/dp0 = I - 2 (a,b)(a,b)^T / s */
        *G0x += Gx - 2.0 * a * nG / sq;
        *G0y += Gy - 2.0 * b * nG / sq;
        /* dp_k/da = -2 [ p0x (a,b)/s + L e_x/s - 2a L (a,b)/s^2 ] */
        double dLa = -2.0 * (g0x * nG / sq + Lk * Gx / sq - 2.0 * a * Lk * nG / (sq * sq));
        double dLb = -2.0 * (g0y * nG / sq + Lk * Gy / sq - 2.0 * b * Lk * nG / (sq * sq));
        double dLc = -2.0 * nG / sq;
        /* a, b, c as functions of v_{k-1} and v_k */
        grad_v[2 * k + 1] += dLa;          /* da/dy_k = 1 */
        grad_v[2 * km + 1] -= dLa;         /* da/dy_{k-1} = -1 */
        grad_v[2 * km] += dLb;             /* db/dx_{k-1} = 1 */
        grad_v[2 * k] -= dLb;              /* db/dx_k = -1 */
        grad_v[2 * k] += dLc * y[km];      /* dc/dx_k = y_{k-1} */
        grad_v[2 * km + 1] += dLc * x[k];  /* dc/dy_{k-1} = x_k */
        grad_v[2 * km] += dLc * -y[k];     /* dc/dx_{k-1} = -y_k */
        grad_v[2 * k + 1] += dLc * -x[km]; /* dc/dy_k = -x_{k-1} */
    }
}

/* Vector-Jacobian product of Eq. 3-4: p0 = C / (3 S), S = sum det_k,
 * C = sum (v_{k-1} + v_k) det_k, det_k = x_{k-1} y_k - x_k y_{k-1}.
 * Given G0 = dL/dp0, adds dL/dv into grad_v[n][2]. */
void orc_centroid_vjp(const double *x, const double *y, int n, double G0x, double G0y,
                      double *grad_v)
{
    double area, g0x, g0y;
    orc_centroid(x, y, n, &area, &g0x, &g0y);
    double S = 2.0 * area;
    double lx = G0x / (3.0 * S), ly = G0y / (3.0 * S);
    double mu = -(G0x * g0x + G0y * g0y) / S;
    for (int k = 0; k < n; k++) {
        int km = (k + n - 1) % n;
        double xm = x[km], ym = y[km], xk = x[k], yk = y[k];
        double det = xm * yk - xk * ym;
        double sx = xm + xk, sy = ym + yk;
        /* d det / d(xm, ym, xk, yk) = (yk, -xk, -ym, xm) */
        double dd[4] = {yk, -xk, -ym, xm};
        /* d (sx det) adds det to d/dxm and d/dxk; d (sy det) adds det to d/dym, d/dyk */
        grad_v[2 * km] += lx * (det + sx * dd[0]) + ly * (sy * dd[0]) + mu * dd[0];
        grad_v[2 * km + 1] += lx * (sx * dd[1]) + ly * (det + sy * dd[1]) + mu * dd[1];
        grad_v[2 * k] += lx * (det + sx * dd[2]) + ly * (sy * dd[2]) + mu * dd[2];
        grad_v[2 * k + 1] += lx * (sx * dd[3]) + ly * (det + sy * dd[3]) + mu * dd[3];
    }
}

/* ------------------------------------------------------------------------ */
/* Collision penalty and its gradient, in fp64.                               */
/*   L = sum_pose sum_point softplus(-m(x) / tau),  x = R(theta)^T (p - t)     */
/* m is the margin above.  The gradient flows back through the margin of the  */
/* edge that attains the maximum (lowest k among ties), through the mirrored  */
/* generators (Eq. 8, as p_k = p0 - 2 L_k(p0) (a, b) / (a^2 + b^2)) and       */
/* through the centroid (Eq. 3-4).                                             */
/* poses: [P][3] = (tx, ty, theta).  grad_v: [n][2].  grad_pose: [P][3].      */
/* ------------------------------------------------------------------------ */
static double softplus(double z) { return z > 0 ? z + log1p(exp(-z)) : log1p(exp(z)); }
static double sigmoid(double z) { return z >= 0 ? 1.0 / (1.0 + exp(-z)) : exp(z) / (1.0 + exp(z)); }

int orc_penalty(const double *x, const double *y, int n, const double *poses, int P,
                const double *q, int64_t m, double tau,
                double *loss, double *grad_v, double *grad_pose)
{
    int st = orc_polygon_status(x, y, n);
    if (st != ORC_OK) return st;
    double *gx = (double *)malloc(sizeof(double) * (size_t)n * 4);
    double *gy = gx + n, *Gkx = gx + 2 * n, *Gky = gx + 3 * n;
    double area, g0x, g0y;
    orc_centroid(x, y, n, &area, &g0x, &g0y);
    orc_generators(x, y, n, g0x, g0y, gx, gy);
    for (int k = 0; k < n; k++) Gkx[k] = Gky[k] = 0.0;
    double G0x = 0.0, G0y = 0.0, L = 0.0;

    for (int j = 0; j < P; j++) {
        double tx = poses[3 * j], ty = poses[3 * j + 1], th = poses[3 * j + 2];
        double c = cos(th), s = sin(th);
        double gtx = 0.0, gty = 0.0, gth = 0.0;
        for (int64_t i = 0; i < m; i++) {
            double ux = q[2 * i] - tx, uy = q[2 * i + 1] - ty;
            double bx = c * ux + s * uy;  /* R^T (p - t) */
            double by = -s * ux + c * uy;
            int kb = -1;
            double best = -INFINITY, bestN = 0.0, bestD = 1.0;
            for (int k = 0; k < n; k++) {
                double n0 = (bx - g0x) * (bx - g0x) + (by - g0y) * (by - g0y);
                double nk = (bx - gx[k]) * (bx - gx[k]) + (by - gy[k]) * (by - gy[k]);
                double D = sqrt((gx[k] - g0x) * (gx[k] - g0x) + (gy[k] - g0y) * (gy[k] - g0y));
                double mk = (n0 - nk) / (2.0 * D);
                if (mk > best) { best = mk; kb = k; bestN = n0 - nk; bestD = D; }
            }
            L += softplus(-best / tau);
            double gm = -sigmoid(-best / tau) / tau; /* dL/dm */
            /* dm/dx = (p_k - p0) / D */
            double dmx = (gx[kb] - g0x) / bestD, dmy = (gy[kb] - g0y) / bestD;
            /* x = R^T (p - t): dx/dt = -R^T, dx/dtheta = (by, -bx) */
            gtx += gm * -(c * dmx - s * dmy);
            gty += gm * -(s * dmx + c * dmy);
            gth += gm * (dmx * by - dmy * bx);
            /* dm/dp0 = -(x - p0)/D + N (p_k - p0) / (2 D^3)
             * dm/dp_k = (x - p_k)/D - N (p_k - p0) / (2 D^3) */
            double D3 = 2.0 * bestD * bestD * bestD;
            double ex = (gx[kb] - g0x) * bestN / D3, ey = (gy[kb] - g0y) * bestN / D3;
            G0x += gm * (-(bx - g0x) / bestD + ex);
            G0y += gm * (-(by - g0y) / bestD + ey);
            Gkx[kb] += gm * ((bx - gx[kb]) / bestD - ex);
            Gky[kb] += gm * ((by - gy[kb]) / bestD - ey);
        }
        grad_pose[3 * j] = gtx;
        grad_pose[3 * j + 1] = gty;
        grad_pose[3 * j + 2] = gth;
    }
    *loss = L;

    for (int i = 0; i < 2 * n; i++) grad_v[i] = 0.0;
    orc_generators_vjp(x, y, n, g0x, g0y, Gkx, Gky, &G0x, &G0y, grad_v);
    orc_centroid_vjp(x, y, n, G0x, G0y, grad_v);
    free(gx);
    return ORC_OK;
}

/* Penalty loss only (same definition), for finite differences. */
int orc_penalty_loss(const double *x, const double *y, int n, const double *poses, int P,
                     const double *q, int64_t m, double tau, double *loss)
{
    int st = orc_polygon_status(x, y, n);
    if (st != ORC_OK) return st;
    double *mg = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    double *qb = (double *)malloc(sizeof(double) * (size_t)(2 * (m > 0 ? m : 1)));
    double L = 0.0;
    for (int j = 0; j < P; j++) {
        double tx = poses[3 * j], ty = poses[3 * j + 1], th = poses[3 * j + 2];
        double c = cos(th), s = sin(th);
        for (int64_t i = 0; i < m; i++) {
            double ux = q[2 * i] - tx, uy = q[2 * i + 1] - ty;
            qb[2 * i] = c * ux + s * uy;
            qb[2 * i + 1] = -s * ux + c * uy;
        }
        orc_margin(x, y, n, qb, m, mg);
        for (int64_t i = 0; i < m; i++) L += softplus(-mg[i] / tau);
    }
    *loss = L;
    free(mg);
    free(qb);
    return ORC_OK;
}

/* Pixel centres of a raster grid, as the rasterisation call defines them:
 * pixel (c, r) -> (fmaf(c, dx, x0), fmaf(r, dy, y0)), each rounded once to
 * float32 (C's fmaf is the correctly rounded fused multiply-add).  Row-major
 * xy pairs, out[2 (r W + c)]. */
void orc_raster_centres(int W, int H, float x0, float y0, float dx, float dy, float *out)
{
    for (int r = 0; r < H; r++) {
        const float cy = fmaf((float)r, dy, y0);
        for (int c = 0; c < W; c++) {
            out[2 * ((int64_t)r * W + c)] = fmaf((float)c, dx, x0);
            out[2 * ((int64_t)r * W + c) + 1] = cy;
        }
    }
}
