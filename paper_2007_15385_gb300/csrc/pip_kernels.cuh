// pip_kernels.cuh -- device helpers shared by the test, margin and comparator
// kernels.  Everything here has internal linkage (anonymous namespace): each
// translation unit gets its own copy.
#pragma once

#include <float.h>
#include <math.h>

#include "pip_internal.cuh"

namespace {

using namespace pip;

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

enum Mode { kSingle = 0, kRagged = 1, kAllPairs = 2 };

// ---------------------------------------------------------------------------
// Point loading: lane `lane` of a chunk holds the pairs (2q, 2q+1) with
// q = chunk_pair0 + j * 32 + lane, j < F.
// ---------------------------------------------------------------------------
template <bool INT, bool V16>
__device__ __forceinline__ void load_pair(const void *__restrict__ pts, int64_t q2, int64_t M,
                                          float &x0, float &y0, float &x1, float &y1)
{
    // q2 = index of the first (even) point of the pair
    if (q2 + 1 < M) {
        if (INT) {
            if (V16) {
                const int4 v = __ldg((const int4 *)((const int32_t *)pts + 2 * q2));
                x0 = (float)v.x; y0 = (float)v.y; x1 = (float)v.z; y1 = (float)v.w;
            } else {
                const int2 a = __ldg((const int2 *)((const int32_t *)pts + 2 * q2));
                const int2 b = __ldg((const int2 *)((const int32_t *)pts + 2 * q2 + 2));
                x0 = (float)a.x; y0 = (float)a.y; x1 = (float)b.x; y1 = (float)b.y;
            }
        } else {
            if (V16) {
                const float4 v = __ldg((const float4 *)((const float *)pts + 2 * q2));
                x0 = v.x; y0 = v.y; x1 = v.z; y1 = v.w;
            } else {
                const float2 a = __ldg((const float2 *)((const float *)pts + 2 * q2));
                const float2 b = __ldg((const float2 *)((const float *)pts + 2 * q2 + 2));
                x0 = a.x; y0 = a.y; x1 = b.x; y1 = b.y;
            }
        }
    } else if (q2 < M) {
        if (INT) {
            const int2 a = __ldg((const int2 *)((const int32_t *)pts + 2 * q2));
            x0 = (float)a.x; y0 = (float)a.y;
        } else {
            const float2 a = __ldg((const float2 *)((const float *)pts + 2 * q2));
            x0 = a.x; y0 = a.y;
        }
        x1 = y1 = 0.f;
    } else {
        x0 = y0 = x1 = y1 = 0.f;
    }
}

// Integer inputs are exact in float32 only within +-2^24; farther points go to refine.
__device__ __forceinline__ bool int_exact(float px, float py)
{
    return fabsf(px) <= (float)kIntLimit && fabsf(py) <= (float)kIntLimit;
}

// Stages one polygon's coefficients into shared memory, padded to a multiple
// of 4 with edges that never win the min (w = 0, t = +inf).  An invalid
// polygon becomes one edge with t = -inf: it contains nothing.
__device__ __forceinline__ int stage_polygon(const PolyInfo &pi, const float4 *__restrict__ coef,
                                             float4 *cs, int tid, int nthreads)
{
    const bool ok = pi.status == PIP_OK;
    const int n = ok ? pi.n : 1;
    const int npad = (n + 3) & ~3;
    for (int k = tid; k < npad; k += nthreads) {
        float4 c;
        if (!ok) c = k == 0 ? make_float4(0.f, 0.f, -INFINITY, 0.f) : make_float4(0.f, 0.f, INFINITY, 0.f);
        else c = k < n ? coef[pi.voff + k] : make_float4(0.f, 0.f, INFINITY, 0.f);
        cs[k] = c;
    }
    return npad;
}

struct Decision {
    bool in, unc;
};

__device__ __forceinline__ Decision decide(float m, float x, float y, float b0, float b1, bool valid,
                                           bool exact_input)
{
    const float B = fmaf(b1, fmaxf(fabsf(x), fabsf(y)), b0);
    Decision d;
    const bool in = (m >= B) && (m < INFINITY);
    const bool out = m < -B;
    d.in = valid && exact_input && in;
    d.unc = valid && (!exact_input || (!in && !out));
    return d;
}

template <int F>
__device__ __forceinline__ int64_t chunks_of(int64_t a, int64_t b)
{
    if (b <= a) return 0;
    return ((b - 1) / Chunk<F>::kPoints) - (a / Chunk<F>::kPoints) + 1;
}

// Single block: item prefix over polygons, reset of the counters.
template <int F>
__global__ void __launch_bounds__(1024) ragged_setup_kernel(
    const int64_t *__restrict__ poffs, int P, int64_t M, int item_chunks, int64_t *__restrict__ items,
    unsigned int *__restrict__ work, unsigned int *__restrict__ qcount, int32_t *__restrict__ worst)
{
    __shared__ int64_t warp_tot[32];
    __shared__ int64_t carry;
    __shared__ int bad;
    if (threadIdx.x == 0) { carry = 0; bad = 0; *work = 0; *qcount = 0; }
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int base = 0; base < P; base += blockDim.x) {
        const int j = base + threadIdx.x;
        int64_t cnt = 0;
        if (j < P) {
            const int64_t a = poffs[j], b = poffs[j + 1];
            if (a < 0 || b < a || b > M || (j == 0 && a != 0) || (j == P - 1 && b != M)) bad = 1;
            else cnt = (chunks_of<F>(a, b) + item_chunks - 1) / item_chunks;
        }
        // block inclusive scan
        int64_t v = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t u = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += u;
        }
        if (lane == 31) warp_tot[wid] = v;
        __syncthreads();
        if (wid == 0) {
            int64_t w = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t u = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += u;
            }
            warp_tot[lane] = w;
        }
        __syncthreads();
        const int64_t excl = carry + (wid ? warp_tot[wid - 1] : 0) + v - cnt;
        if (j < P) items[j] = excl;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = excl + cnt;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        items[P] = bad ? 0 : carry;
        if (bad) atomicMax(worst, (int)PIP_E_INVALID_ARG);
    }
}


__device__ __forceinline__ void point_d(const void *pts, int dtype, int64_t i, double &x, double &y)
{
    if (dtype == PIP_I32) {
        const int32_t *q = (const int32_t *)pts;
        x = (double)q[2 * i];
        y = (double)q[2 * i + 1];
    } else {
        const float *f = (const float *)pts;
        x = (double)f[2 * i];
        y = (double)f[2 * i + 1];
    }
}

// Exact inclusion of point i in polygon j, decided by the whole warp (every
// lane calls it with the same arguments; lane l takes edges l and l + 32).
// Integer inputs: int64 cross products.  Otherwise: the fp64 Voronoi
// comparison from the stored generators, and the exact orientation sign
// where that comparison is within its bound.
__device__ __noinline__ bool warp_inside_exact_xy(const PolyInfo &pi, int j, const double2 *__restrict__ g0tab,
                                                  const double2 *__restrict__ gk,
                                                  const void *__restrict__ verts, int vdtype, double px,
                                                  double py);

__device__ __noinline__ bool warp_inside_exact(const PolyInfo *__restrict__ poly, int j,
                                               const double2 *__restrict__ g0tab,
                                               const double2 *__restrict__ gk,
                                               const void *__restrict__ verts, int vdtype,
                                               const void *__restrict__ pts, int pdtype, int64_t i)
{
    const int lane = threadIdx.x & 31;
    const PolyInfo pi = poly[j];
    if (pi.status != PIP_OK) return false;
    const int n = pi.n, v0 = pi.voff, sigma = pi.orient;
    bool out = false;
    if (vdtype == PIP_I32 && pdtype == PIP_I32) {
        const int32_t *q = (const int32_t *)pts;
        const int64_t px = q[2 * i], py = q[2 * i + 1];
        const int32_t *v = (const int32_t *)verts;
        for (int k = lane; k < n; k += 32) {
            const int km = k == 0 ? n - 1 : k - 1;
            const int64_t ax = v[2 * (v0 + km)], ay = v[2 * (v0 + km) + 1];
            const int64_t bx = v[2 * (v0 + k)], by = v[2 * (v0 + k) + 1];
            // |b - a| <= 2^25 and |p - a| < 2^32 + 2^24: each product < 2^58
            const int64_t cr = (bx - ax) * (py - ay) - (by - ay) * (px - ax);
            if ((cr > 0 ? 1 : (cr < 0 ? -1 : 0)) == -sigma) out = true;
        }
        return !__any_sync(0xffffffffu, out);
    }
    double px, py;
    point_d(pts, pdtype, i, px, py);
    return warp_inside_exact_xy(pi, j, g0tab, gk, verts, vdtype, px, py);
}

// The same for a point given by its (float32-exact) coordinates; every lane
// passes the same point.  Float path only (fp64 Voronoi, then exact
// orientation for the edges it leaves open).
__device__ __noinline__ bool warp_inside_exact_xy(const PolyInfo &pi, int j, const double2 *__restrict__ g0tab,
                                                  const double2 *__restrict__ gk,
                                                  const void *__restrict__ verts, int vdtype, double px,
                                                  double py)
{
    const int lane = threadIdx.x & 31;
    if (pi.status != PIP_OK) return false;
    const int n = pi.n, v0 = pi.voff, sigma = pi.orient;
    bool out = false;
    if (!isfinite(px) || !isfinite(py)) return false;
    const double2 g0 = g0tab[j];
    const double e = pi.gerr;
    const double ap = fmax(fabs(px), fabs(py));
    for (int k = lane; k < n; k += 32) {
        const double2 g = gk[v0 + k];
        const double dx = g.x - g0.x, dy = g.y - g0.y;                        // p_k - p0
        const double sx = g.x + g0.x - 2.0 * px, sy = g.y + g0.y - 2.0 * py;  // p_k + p0 - 2x
        const double d = dx * sx + dy * sy;  // |x - p_k|^2 - |x - p0|^2
        const double mag = fmax(fmax(fabs(g.x), fabs(g.y)), fmax(fmax(fabs(g0.x), fabs(g0.y)), ap));
        const double bound = 8.0 * e * (fabs(sx) + fabs(sy) + fabs(dx) + fabs(dy) + 4.0 * e) +
                             ldexp((fabs(dx) + fabs(dy)) * (fabs(sx) + fabs(sy) + 4.0 * mag), -48);
        if (d < -bound) {
            out = true;
        } else if (!(d > bound)) {
            const int km = k == 0 ? n - 1 : k - 1;
            double ax, ay, bx, by;
            point_d(verts, vdtype, v0 + km, ax, ay);
            point_d(verts, vdtype, v0 + k, bx, by);
            if (orient_sign_exact(ax, ay, bx, by, px, py) == -sigma) out = true;
        }
    }
    return !__any_sync(0xffffffffu, out);
}

template <typename K>
int blocks_for(K kernel, int num_sms, int threads)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    return per_sm * num_sms;
}

}  // namespace
