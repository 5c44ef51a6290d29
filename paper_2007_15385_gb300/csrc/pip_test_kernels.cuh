// pip_test_kernels.cuh -- bulk float32 test kernels and the refine kernel,
// shared by the translation units that launch them.  Internal linkage: each
// includer gets its own copy.
#pragma once

#include "pip_kernels.cuh"

using namespace pip;

namespace {

// One warp, one chunk of 64F points [p0, p0 + 64F): evaluate, then write the
// 2F mask words and queue the uncertain points.  Points outside [lo, hi) are
// not this polygon's; words that are only partly [lo, hi_w) are merged with
// atomics (hi_w extends hi to the end of the last word for the last polygon,
// so that bits past num_points are cleared).
template <int F, bool INT, bool V16>
__device__ __forceinline__ void process_chunk(const void *__restrict__ pts, int64_t M, int64_t p0,
                                              int64_t lo, int64_t hi, int64_t hi_w,
                                              const float4 *cs, int npad, float ox, float oy,
                                              float b0, float b1, uint32_t *__restrict__ mask,
                                              uint32_t *__restrict__ queue,
                                              unsigned int *__restrict__ qcount, int lane)
{
    float x[2 * F], y[2 * F], m[2 * F];
    bool valid[2 * F], exin[2 * F];
#pragma unroll
    for (int j = 0; j < F; ++j) {
        const int64_t q2 = p0 + 2 * (j * 32 + lane);
        float px0, py0, px1, py1;
        load_pair<INT, V16>(pts, q2, M, px0, py0, px1, py1);
        valid[2 * j] = q2 >= lo && q2 < hi;
        valid[2 * j + 1] = q2 + 1 >= lo && q2 + 1 < hi;
        exin[2 * j] = INT ? int_exact(px0, py0) : true;
        exin[2 * j + 1] = INT ? int_exact(px1, py1) : true;
        x[2 * j] = px0 - ox;
        y[2 * j] = py0 - oy;
        x[2 * j + 1] = px1 - ox;
        y[2 * j + 1] = py1 - oy;
    }
#pragma unroll
    for (int i = 0; i < 2 * F; ++i) m[i] = INFINITY;
    for (int k = 0; k < npad; k += 4) {
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            const float4 c = cs[k + kk];
#pragma unroll
            for (int i = 0; i < 2 * F; ++i)
                m[i] = fminf(m[i], fmaf(-x[i], c.x, fmaf(-y[i], c.y, c.z)));
        }
    }
    const int64_t wbase = p0 >> 5;
    const unsigned lt = (1u << lane) - 1u;
    uint32_t myword = 0;
#pragma unroll
    for (int j = 0; j < F; ++j) {
        const Decision d0 = decide(m[2 * j], x[2 * j], y[2 * j], b0, b1, valid[2 * j], exin[2 * j]);
        const Decision d1 = decide(m[2 * j + 1], x[2 * j + 1], y[2 * j + 1], b0, b1, valid[2 * j + 1],
                                   exin[2 * j + 1]);
        const uint32_t be = __ballot_sync(0xffffffffu, d0.in);
        const uint32_t bo = __ballot_sync(0xffffffffu, d1.in);
        uint32_t lo_w, hi_w2;
        interleave_words(be, bo, lo_w, hi_w2);
        if (lane == 2 * j) myword = lo_w;
        if (lane == 2 * j + 1) myword = hi_w2;
        const uint32_t ue = __ballot_sync(0xffffffffu, d0.unc);
        const uint32_t uo = __ballot_sync(0xffffffffu, d1.unc);
        if (ue | uo) {
            unsigned int base = 0;
            if (lane == 0) base = atomicAdd(qcount, (unsigned)(__popc(ue) + __popc(uo)));
            base = __shfl_sync(0xffffffffu, base, 0);
            const int64_t q2 = p0 + 2 * (j * 32 + lane);
            if (d0.unc) queue[base + __popc(ue & lt)] = (uint32_t)q2;
            if (d1.unc) queue[base + __popc(ue) + __popc(uo & lt)] = (uint32_t)(q2 + 1);
        }
    }
    if (lane < 2 * F) {
        const int64_t w = wbase + lane;
        const int64_t first = w << 5;
        // bits of this word that belong to [lo, hi_w)
        uint32_t own;
        if (first >= lo && first + 32 <= hi_w) {
            own = 0xffffffffu;
        } else {
            own = 0;
            for (int b = 0; b < 32; ++b)
                if (first + b >= lo && first + b < hi_w) own |= 1u << b;
        }
        if (own == 0xffffffffu) {
            mask[w] = myword;
        } else if (own) {
            atomicAnd(&mask[w], ~own);
            atomicOr(&mask[w], myword & own);
        }
    }
}

// ---------------------------------------------------------------------------
// K2: one polygon, a flat point array.  Grid-stride over warp chunks.
// ---------------------------------------------------------------------------
template <int F, bool INT, bool V16>
__global__ void __launch_bounds__(kThreads) stream_kernel(
    const PolyInfo *__restrict__ poly, const float4 *__restrict__ coef, const void *__restrict__ pts,
    int64_t M, uint32_t *__restrict__ mask, uint32_t *__restrict__ queue,
    unsigned int *__restrict__ qcount)
{
    __shared__ float4 cs[kMaxEdges + 4];
    const PolyInfo pi = poly[0];
    const int npad = stage_polygon(pi, coef, cs, threadIdx.x, blockDim.x);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nchunks = (M + Chunk<F>::kPoints - 1) / Chunk<F>::kPoints;
    const int64_t hi_w = (M + 31) & ~(int64_t)31;
    for (int64_t c = warp; c < nchunks; c += nwarps) {
        process_chunk<F, INT, V16>(pts, M, c * Chunk<F>::kPoints, 0, M, hi_w, cs, npad, pi.ox, pi.oy,
                                   pi.beta0, pi.beta1, mask, queue, qcount, lane);
    }
}

// ---------------------------------------------------------------------------
// K3: own-polygon batch.  A work item is (polygon j, up to kItemChunks chunks
// of that polygon's point range); persistent CTAs pull items from a counter.
// ---------------------------------------------------------------------------
template <int F, bool INT, bool V16>
__global__ void __launch_bounds__(kThreads) ragged_kernel(
    const PolyInfo *__restrict__ poly, const float4 *__restrict__ coef, const void *__restrict__ pts,
    int64_t M, const int64_t *__restrict__ poffs, int P, const int64_t *__restrict__ items,
    int item_chunks, unsigned int *__restrict__ work, uint32_t *__restrict__ mask,
    uint32_t *__restrict__ queue, unsigned int *__restrict__ qcount)
{
    __shared__ float4 cs[kMaxEdges + 4];
    __shared__ int s_item_poly;
    __shared__ int64_t s_item_local;
    __shared__ int s_done;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t total = items[P];
    const int64_t hi_last = (M + 31) & ~(int64_t)31;
    for (;;) {
        if (threadIdx.x == 0) {
            const int64_t it = (int64_t)atomicAdd(work, 1u);
            s_done = it >= total;
            if (it < total) {
                // polygon j with items[j] <= it < items[j+1]
                int lo = 0, hi = P;  // invariant items[lo] <= it < items[hi]
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (items[mid] <= it) lo = mid; else hi = mid;
                }
                s_item_poly = lo;
                s_item_local = it - items[lo];
            }
        }
        __syncthreads();
        if (s_done) break;
        const int j = s_item_poly;
        const int64_t local = s_item_local;
        const PolyInfo pi = poly[j];
        const int npad = stage_polygon(pi, coef, cs, threadIdx.x, blockDim.x);
        __syncthreads();
        const int64_t a = poffs[j], b = poffs[j + 1];
        const int64_t hi_w = (j == P - 1) ? hi_last : b;
        const int64_t c0 = a / Chunk<F>::kPoints + local * item_chunks;
        const int64_t c1 = min(c0 + item_chunks, (b - 1) / Chunk<F>::kPoints + 1);
        for (int64_t c = c0 + wid; c < c1; c += kWarps) {
            process_chunk<F, INT, V16>(pts, M, c * Chunk<F>::kPoints, a, b, hi_w, cs, npad, pi.ox,
                                       pi.oy, pi.beta0, pi.beta1, mask, queue, qcount, lane);
        }
        __syncthreads();  // cs is restaged by the next item
    }
}

// ---------------------------------------------------------------------------
// K4: all pairs.  Each thread keeps PT points in registers; polygons stream
// through shared memory in chunks of kPolyChunk.  Full work: every point
// meets every polygon (no early exit, no cull).
// ---------------------------------------------------------------------------
constexpr int kPolyChunk = 32;

struct SmemPoly {
    float ox, oy, b0, b1;
    int e0, npad, pad0, pad1;
};

template <int PT, bool INT>
__global__ void __launch_bounds__(kThreads) allpairs_kernel(
    const PolyInfo *__restrict__ poly, const float4 *__restrict__ coef, int P,
    const void *__restrict__ pts, int64_t M, int32_t *__restrict__ first_hit,
    uint32_t *__restrict__ mask, uint32_t *__restrict__ queue, unsigned int *__restrict__ qcount)
{
    __shared__ float4 cs[kPolyChunk * (kMaxEdges + 4)];
    __shared__ SmemPoly sp[kPolyChunk];
    const int tid = threadIdx.x, lane = tid & 31;
    const int64_t base = (int64_t)blockIdx.x * (PT * kThreads);
    float px[PT], py[PT];
    bool valid[PT], exin[PT];
    int first[PT], func[PT];
#pragma unroll
    for (int i = 0; i < PT; ++i) {
        const int64_t p = base + i * kThreads + tid;
        valid[i] = p < M;
        px[i] = valid[i] ? load_coord(pts, INT ? PIP_I32 : PIP_F32, 2 * p) : 0.f;
        py[i] = valid[i] ? load_coord(pts, INT ? PIP_I32 : PIP_F32, 2 * p + 1) : 0.f;
        exin[i] = INT ? int_exact(px[i], py[i]) : true;
        first[i] = -1;
        func[i] = P;
    }
    for (int j0 = 0; j0 < P; j0 += kPolyChunk) {
        const int nj = min(kPolyChunk, P - j0);
        __syncthreads();
        if (tid < nj) {
            const PolyInfo pi = poly[j0 + tid];
            SmemPoly s;
            s.ox = pi.ox; s.oy = pi.oy; s.b0 = pi.beta0; s.b1 = pi.beta1;
            s.e0 = tid * (kMaxEdges + 4);
            s.npad = ((pi.status == PIP_OK ? pi.n : 1) + 3) & ~3;
            s.pad0 = s.pad1 = 0;
            sp[tid] = s;
        }
        // stage every polygon of the chunk: one warp per polygon
        for (int q = tid >> 5; q < nj; q += kWarps) {
            const PolyInfo pi = poly[j0 + q];
            stage_polygon(pi, coef, cs + q * (kMaxEdges + 4), lane, 32);
        }
        __syncthreads();
        for (int q = 0; q < nj; ++q) {
            const SmemPoly s = sp[q];
            const float4 *c = cs + s.e0;
            float x[PT], y[PT], m[PT];
#pragma unroll
            for (int i = 0; i < PT; ++i) {
                x[i] = px[i] - s.ox;
                y[i] = py[i] - s.oy;
                m[i] = INFINITY;
            }
            for (int k = 0; k < s.npad; k += 4) {
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const float4 cf = c[k + kk];
#pragma unroll
                    for (int i = 0; i < PT; ++i)
                        m[i] = fminf(m[i], fmaf(-x[i], cf.x, fmaf(-y[i], cf.y, cf.z)));
                }
            }
            const int j = j0 + q;
#pragma unroll
            for (int i = 0; i < PT; ++i) {
                const Decision d = decide(m[i], x[i], y[i], s.b0, s.b1, valid[i], exin[i]);
                if (d.in && first[i] < 0) first[i] = j;
                if (d.unc && func[i] == P) func[i] = j;
            }
        }
    }
#pragma unroll
    for (int i = 0; i < PT; ++i) {
        const int64_t p = base + i * kThreads + tid;
        const bool need = valid[i] && func[i] < (first[i] < 0 ? P : first[i]);
        if (valid[i] && first_hit) first_hit[p] = first[i];
        const uint32_t bits = __ballot_sync(0xffffffffu, first[i] >= 0);
        if (mask && lane == 0 && p < ((M + 31) & ~(int64_t)31)) mask[p >> 5] = bits;
        const uint32_t ub = __ballot_sync(0xffffffffu, need);
        if (ub) {
            unsigned int qb = 0;
            if (lane == 0) qb = atomicAdd(qcount, (unsigned)__popc(ub));
            qb = __shfl_sync(0xffffffffu, qb, 0);
            if (need) queue[qb + __popc(ub & ((1u << lane) - 1u))] = (uint32_t)p;
        }
    }
}

// ---------------------------------------------------------------------------
// K6: refine.  Persistent grid-stride over the queue; the queue length is read
// on the device, so the launch shape does not depend on it.
// ---------------------------------------------------------------------------
struct RefineArgs {
    const PolyInfo *poly;
    const float4 *coef;
    const double2 *g0;
    const double2 *gk;
    const void *verts;
    int vdtype;
    int P;
    const void *pts;
    int pdtype;
    int64_t M;
    const int64_t *poffs;
    const uint32_t *queue;
    const unsigned int *qcount;
    uint32_t *mask;
    int32_t *first_hit;
    const uint32_t *keys;  // all-pairs candidate keys (pip_test's split path)
    const uint32_t *qpoly; // own-polygon batch: the polygon of each queued point, or null
    const int4 *iedge;     // integer polygons: (v_{k-1}, oriented edge k) per edge
};

__device__ __forceinline__ void vertex_d(const void *verts, int vdtype, int64_t i, double &x, double &y)
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

// Integer polygon and point: every edge's orientation in int64 (exact),
// the point inside iff none has the opposite sign of the polygon's turn.
__device__ __forceinline__ bool inside_exact_int(const RefineArgs &A, int n, int v0, int64_t i)
{
    const int2 pq = ((const int2 *)A.pts)[i];
    const int4 *e = A.iedge + v0;  // (a, oriented edge): inside iff every cross >= 0
    // -2^30 <= p < 2^30 per coordinate (unsigned compare: no abs overflow at INT_MIN)
    if ((uint32_t)pq.x + (1u << 30) < (1u << 31) && (uint32_t)pq.y + (1u << 30) < (1u << 31)) {
        // |e| <= 2^25 and |p - a| < 2^31: each product is one 32 x 32 -> 64-bit
        // multiply (|product| < 2^56), the cross product exact
        for (int k = 0; k < n; ++k) {
            const int4 E = e[k];
            if ((int64_t)E.z * (pq.y - E.y) - (int64_t)E.w * (pq.x - E.x) < 0) return false;
        }
        return true;
    }
    const int64_t px = pq.x, py = pq.y;
    for (int k = 0; k < n; ++k) {
        const int4 E = e[k];
        // |p - a| < 2^32 + 2^24: each product < 2^58
        if ((int64_t)E.z * (py - E.y) - (int64_t)E.w * (px - E.x) < 0) return false;
    }
    return true;
}

// Exact inclusion of point i in polygon j: fp64 Voronoi first (Alg. 5 with
// the stored generators, decided where the fp64 bound allows), exact
// orientation for the edges it leaves open.
__device__ bool inside_exact(const RefineArgs &A, int j, int64_t i)
{
    const PolyInfo pi = A.poly[j];
    if (pi.status != PIP_OK) return false;
    const int n = pi.n, v0 = pi.voff, sigma = pi.orient;
    if (A.vdtype == PIP_I32 && A.pdtype == PIP_I32) return inside_exact_int(A, n, v0, i);
    double px, py;
    vertex_d(A.pts, A.pdtype, i, px, py);
    if (!isfinite(px) || !isfinite(py)) return false;
    const double2 g0 = A.g0[j];
    const double e = pi.gerr;
    const double ap = fmax(fabs(px), fabs(py));
    uint64_t open = 0;  // edges the fp64 step leaves undecided
    for (int k = 0; k < n; ++k) {
        const double2 g = A.gk[v0 + k];
        const double dx = g.x - g0.x, dy = g.y - g0.y;                   // p_k - p0
        const double sx = g.x + g0.x - 2.0 * px, sy = g.y + g0.y - 2.0 * py;  // p_k + p0 - 2x
        const double d = dx * sx + dy * sy;  // |x - p_k|^2 - |x - p0|^2
        const double mag = fmax(fmax(fabs(g.x), fabs(g.y)), fmax(fmax(fabs(g0.x), fabs(g0.y)), ap));
        const double bound = 8.0 * e * (fabs(sx) + fabs(sy) + fabs(dx) + fabs(dy) + 4.0 * e) +
                             ldexp((fabs(dx) + fabs(dy)) * (fabs(sx) + fabs(sy) + 4.0 * mag), -48);
        if (d < -bound) return false;
        if (!(d > bound)) open |= 1ull << k;
    }
    while (open) {
        const int k = __ffsll((long long)open) - 1;
        open &= open - 1;
        const int km = k == 0 ? n - 1 : k - 1;
        double ax, ay, bx, by;
        vertex_d(A.verts, A.vdtype, v0 + km, ax, ay);
        vertex_d(A.verts, A.vdtype, v0 + k, bx, by);
        if (orient_sign_exact(ax, ay, bx, by, px, py) == -sigma) return false;
    }
    return true;
}

// float32 bulk decision of one (polygon, point) pair, for the all-pairs refine
__device__ int bulk_decision(const RefineArgs &A, int j, int64_t i)
{
    const PolyInfo pi = A.poly[j];
    if (pi.status != PIP_OK) return -1;
    const bool ints = A.pdtype == PIP_I32;
    const float px = load_coord(A.pts, A.pdtype, 2 * i), py = load_coord(A.pts, A.pdtype, 2 * i + 1);
    const float x = px - pi.ox, y = py - pi.oy;
    float m = INFINITY;
    for (int k = 0; k < pi.n; ++k) {
        const float4 c = A.coef[pi.voff + k];
        m = fminf(m, fmaf(-x, c.x, fmaf(-y, c.y, c.z)));
    }
    const Decision d = decide(m, x, y, pi.beta0, pi.beta1, true, ints ? int_exact(px, py) : true);
    return d.in ? 1 : (d.unc ? 0 : -1);
}

// One thread per queued point, single or own-polygon mode.  INT: integer
// polygons and points (the int64 test is short and needs no lane
// cooperation; a small kernel keeps many threads resident to hide the loads).
template <bool INT>
__global__ void __launch_bounds__(kThreads) refine_kernel(RefineArgs A, int mode)
{
    const unsigned int count = *A.qcount;
    for (unsigned int q = blockIdx.x * blockDim.x + threadIdx.x; q < count;
         q += gridDim.x * blockDim.x) {
        const int64_t i = A.queue[q];
        int j = 0;
        if (mode == kRagged && A.qpoly) {
            j = (int)A.qpoly[q];
        } else if (mode == kRagged) {
            int lo = 0, hi = A.P;  // poffs[lo] <= i < poffs[hi]
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (A.poffs[mid] <= i) lo = mid; else hi = mid;
            }
            j = lo;
        }
        bool in;
        if (INT) {
            const PolyInfo *pi = A.poly + j;
            in = pi->status == PIP_OK && inside_exact_int(A, pi->n, pi->voff, i);
        } else {
            in = inside_exact(A, j, i);
        }
        if (in) atomicOr(&A.mask[i >> 5], 1u << (i & 31));
    }
}

constexpr int kF = 4;           // float4 loads per lane per chunk (8 points per lane)
constexpr int kItemChunks = 32; // chunks per own-polygon work item (8192 points)
constexpr int kPT = 4;          // points per thread in the all-pairs kernel

}  // namespace
