// pip_internal.cuh -- layouts and helpers shared by the libpip translation units.
//
// Device data of one pip_tables, all in one allocation (HBM):
//   verts   [V][2]  float32 or int32 copy of the caller's vertices
//   voffs   [P+1]   int32 vertex offsets
//   g0      [P]     double2 centroid p0 (Eq. 4), absolute coordinates
//   gk      [V]     double2 mirrored generator p_k of edge k (Eq. 8), absolute
//   coef    [V]     float4 (w_x, w_y, t, 0) of edge k: s_k(x) = t - x.w, x = point - o
//   coefn   [V]     float4 (w_x, w_y, t, 0) / |w|: the bisector distance of Eq. 2
//   poly    [P]     PolyInfo (origin, error bound, offsets, status)
//   queue   [cap]   uint32 indices of points sent to the refine step
//   counters        refine count, work counter, worst status
#pragma once

#include <string>

#include <cuda_runtime.h>
#include <stdint.h>

#include "pip.h"

namespace pip {

constexpr int kMaxEdges = 64;
constexpr int kMinEdges = 3;
// Row stride of the padded coefficient table: 64 edges rounded up, plus room.
constexpr int kPadStride = kMaxEdges + 4;
// the refine queue's slack for the pipelined single-polygon kernel, in points
// a SM: one tile per CTA, e.g. two CTAs of 8 consumer warps x 32 lanes x 24
// points, or one of 16 warps
constexpr int kStreamSlackPerSm = 2 * 8 * 32 * 24;
// Integer vertices must satisfy |v| <= 2^24 so that float32 holds them exactly
// and every exact cross product fits in int64.
constexpr int32_t kIntLimit = 1 << 24;

struct PolyInfo {
    float ox, oy;        // local origin o = float32(p0)
    float beta0, beta1;  // |computed s_k - exact s_k| <= beta0 + beta1 * max(|x|, |y|)
    int32_t voff, n;     // first vertex, vertex count
    int32_t status;      // pip_status of this polygon
    int32_t orient;      // +1 counter-clockwise, -1 clockwise, 0 invalid
    float bbox[4];       // xmin, ymin, xmax, ymax
    double gerr;         // per-coordinate bound on |stored p_k - exact mirror of stored p0|
    // Disc bounds about o, on the computed d2 = fl(x x + fl(y y)) of the local
    // coordinates: d2 < tin only inside the largest disc about o within the
    // polygon (strictly inside), d2 > tout only outside the smallest disc about
    // o holding every vertex (strictly outside); tin = 0, tout = -inf when the
    // polygon is invalid
    float tin, tout;
};
static_assert(sizeof(PolyInfo) == 64, "PolyInfo is 64 bytes");

// Points in one chunk of the streaming kernels: F float4 loads per lane, two
// points per float4, 32 lanes.
template <int F>
struct Chunk {
    static constexpr int kPoints = 64 * F;
    static constexpr int kWords = 2 * F;
};

__device__ __forceinline__ uint32_t spread16(uint32_t x)
{
    // bit i of the low 16 bits moves to bit 2i
    x &= 0xFFFFu;
    x = (x | (x << 8)) & 0x00FF00FFu;
    x = (x | (x << 4)) & 0x0F0F0F0Fu;
    x = (x | (x << 2)) & 0x33333333u;
    x = (x | (x << 1)) & 0x55555555u;
    return x;
}

// Ballots of the even and odd points of 32 lanes (lane l holds points 2l and
// 2l+1 of a 64-point run) -> the two mask words of that run.
__device__ __forceinline__ void interleave_words(uint32_t even, uint32_t odd, uint32_t &lo,
                                                 uint32_t &hi)
{
    lo = spread16(even) | (spread16(odd) << 1);
    hi = spread16(even >> 16) | (spread16(odd >> 16) << 1);
}

__device__ __forceinline__ float load_coord(const void *p, int dtype, int64_t idx)
{
    if (dtype == PIP_I32) return (float)((const int32_t *)p)[idx];
    return ((const float *)p)[idx];
}

}  // namespace pip

struct pip_tables {
    int device;
    int32_t P, V;
    int vdtype;
    int64_t capacity;
    int num_sms;
    void *base;
    size_t bytes;
    void *d_verts;
    int32_t *d_voffs;
    double2 *d_g0;
    double2 *d_gk;
    float4 *d_coef;
    float4 *d_coefn;
    float4 *d_coefp;             // [P][kPadStride] coefficients padded per polygon (all pairs, batch)
    int4 *d_iedge;               // [V] integer polygons: (v_{k-1}, oriented edge k); null for float ones
    int4 *d_ipad;                // [P][kPadStride] integer polygons: exact edge rows (e_x, -e_y, -C lo, -C hi),
                                 // zero past n; null for float ones
    float4 *d_fpad;              // [P][kPadStride] integer polygons: (a_x, a_y, e_x, e_y) in float32, a = v_{k-1},
                                 // e the oriented edge, zero past n; null for float ones
    // comparators (float polygons only; null for integer ones), padded like d_coefp:
    float4 *d_cmp_sign;          // [P][kPadStride] Alg. 2: (dV_y, -dV_x, -RHS, 0), LHS - RHS = t - x w_x - y w_y
    float4 *d_cmp_ray;           // [P][2 kPadStride] Alg. 1, per edge (s dV_y, -s dV_x, -s RHS, 0) and
                                 // (y_{k-1}, y_k, 0, 0), s = +1 going up, -1 otherwise; NaN past n
    double2 *d_cmp_g64;          // [P][kPadStride] fp64 Alg. 5: p_k for k < n, p0 in the last slot
    pip::PolyInfo *d_poly;
    uint32_t *d_queue;
    uint32_t *d_keys;            // [max_points] all-pairs candidate keys
    int64_t *d_items;            // [P+1] work-item prefix of the register-streaming own-polygon schedule
    unsigned int *d_qcount;      // refine queue length of the last pip_test
    unsigned int *d_work;        // next work item of the persistent kernel
    int32_t *d_worst;            // worst polygon status
    int32_t *d_error;            // runtime error of a kernel (PIP_E_TIMEOUT), sticky until read
    void *d_stream_ctr;          // counters of the pipelined kernel (zero between launches)
    unsigned int *d_batch_ctr;   // the pipelined batch kernel: next chunk, queue fill, ticket (zero
                                 // between launches)
    int stream_variant;          // tile shape of the pipelined single-polygon kernel
    int batch_variant;           // tile shape of the pipelined own-polygon batch kernel
    // one-polygon tables: a host copy of the polygon's row and coefficients,
    // passed to the pipelined kernel by value (constant bank, no registers)
    int have_host_poly;
    pip::PolyInfo h_poly;
    float4 h_coef[pip::kMaxEdges];
    float4 h_cmp_sign[pip::kMaxEdges];
    float4 h_cmp_ray[2 * pip::kMaxEdges];
    // pip_test_host: a copy stream and events, created at its first call
    cudaStream_t host_copy_stream;
    cudaEvent_t host_events[65];
    int host_ready;
    // pip_timing: event triples (before bulk, after bulk, after refine)
    int timing;
    int timed_calls;
    cudaEvent_t *events;
};

namespace pip {
constexpr int kTimingSlots = 4096;
// Records timing event `which` (0, 1, 2) of the current call when timing is on.
inline void timing_mark(const pip_tables *ct, int which, cudaStream_t s)
{
    pip_tables *t = const_cast<pip_tables *>(ct);
    if (!t->timing || t->events == nullptr) return;
    const int slot = t->timed_calls % kTimingSlots;
    cudaEventRecord(t->events[3 * slot + which], s);
    if (which == 2) t->timed_calls++;
}
}  // namespace pip

#define PIP_CUDA_TRY(expr)                                   \
    do {                                                     \
        cudaError_t _e = (expr);                             \
        if (_e != cudaSuccess) return PIP_E_CUDA;            \
    } while (0)

namespace pip {
// Host helpers implemented in pip_prepare.cu.
pip_status check_tables(const pip_tables *t);
bool aligned(const void *p, size_t a);
// Implemented in pip_test.cu: raises the dynamic shared-memory limit of the
// pipelined kernels on the current device (outside any stream capture).
cudaError_t stream_kernels_setup();
cudaError_t ragged_kernels_setup();
cudaError_t allpairs_setup();
int stream_variant_count();
// the pipelined single-polygon test (pip_stream.cu): one launch, refine inline;
// `early` the warp-uniform early break, `disc` the disc filter
cudaError_t launch_stream_pipelined(const pip_tables *t, const void *pts, bool ints, int64_t M, uint32_t *mask, bool early,
                                    bool disc, cudaStream_t s);
cudaError_t launch_stream_pipelined_i32(const pip_tables *t, const void *pts, int64_t M, uint32_t *mask, bool early,
                                        bool disc, cudaStream_t s);
cudaError_t stream_kernels_setup_i32();
// pip_tuning.cu: the autotuners' JSON cache (no-ops while no cache file is set)
std::string tuning_key(const pip_tables *t, const char *kernel, int64_t num_points, int pdtype);
bool tuning_lookup(const std::string &key, int *variant, float *ms);
void tuning_store(const std::string &key, int variant, float ms);
// pip_stream.cu: the comparators (op 1 = sign of offset, 2 = ray crossing) on
// one float polygon through the pipelined single-polygon kernel
cudaError_t launch_cmp_stream(const pip_tables *t, const float *pts, int64_t M, uint32_t *mask, int op,
                              cudaStream_t s);
// pip_test.cu: the comparators (op 1 sign of offset, 2 ray crossing, 3 fp64
// Alg. 5) on an own-polygon batch through the pipelined batch kernel
// (16-byte aligned float points; the offsets stay on the device)
cudaError_t launch_ragged_cmp(const pip_tables *t, const float *pts, int64_t M, const int64_t *poffs, uint32_t *mask,
                              int op, cudaStream_t s);
}  // namespace pip

namespace pip {

// ---------------------------------------------------------------------------
// Exact sign of a 2x2 orientation determinant in fp64 floating-point
// expansions (Shewchuk 1997, "Adaptive Precision Floating-Point Arithmetic and
// Fast Robust Geometric Predicates": exact difference, exact product via a
// fused multiply-add, and expansion growth).  Correct for any finite doubles
// whose products neither overflow nor underflow -- every float32 and int32
// input qualifies.  Written with explicit _rn intrinsics so that no
// contraction or reassociation can change a step.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void x_two_sum(double a, double b, double &s, double &e)
{
    s = __dadd_rn(a, b);
    double bv = __dsub_rn(s, a);
    double av = __dsub_rn(s, bv);
    e = __dadd_rn(__dsub_rn(a, av), __dsub_rn(b, bv));
}

__device__ __forceinline__ void x_two_diff(double a, double b, double &d, double &e)
{
    x_two_sum(a, -b, d, e);
}

// Adds v to the expansion h[0..len) (nonoverlapping, increasing magnitude),
// dropping zero components as it goes (the same paper's zero elimination), so
// that the expansion stays as short as the value needs: when the coordinate
// differences are exact (their tails zero), the determinant is two exact
// products and the expansion holds at most four terms.
__device__ __forceinline__ int x_grow(double *h, int len, double v)
{
    if (v == 0.0) return len;
    double q = v;
    int out = 0;
    for (int i = 0; i < len; ++i) {
        double s, e;
        x_two_sum(q, h[i], s, e);
        if (e != 0.0) h[out++] = e;
        q = s;
    }
    if (q != 0.0) h[out++] = q;
    return out;
}

__device__ __forceinline__ int x_add_product(double *h, int len, double a, double b, bool neg)
{
    if (a == 0.0 || b == 0.0) return len;
    double p = __dmul_rn(a, b);
    double e = __fma_rn(a, b, -p);
    if (neg) { p = -p; e = -e; }
    len = x_grow(h, len, e);
    return x_grow(h, len, p);
}

// sign of (bx - ax)(cy - ay) - (by - ay)(cx - ax): +1 when c is left of a->b
static __device__ __noinline__ int orient_sign_exact(double ax, double ay, double bx, double by,
                                              double cx, double cy)
{
    // First stage of the same paper's adaptive predicate: the determinant
    // rounded in fp64, (ax - cx)(by - cy) - (ay - cy)(bx - cx), has the exact
    // sign whenever its magnitude exceeds (3 + 16 eps) eps times the sum of
    // the two products' magnitudes (eps = 2^-53; the paper's bound for this
    // evaluation order).  Only the rest falls through to the exact expansion.
    {
        const double l = __dmul_rn(__dsub_rn(ax, cx), __dsub_rn(by, cy));
        const double r = __dmul_rn(__dsub_rn(ay, cy), __dsub_rn(bx, cx));
        const double det = __dsub_rn(l, r);
        const double bound = (3.0 + 16.0 * 0x1p-53) * 0x1p-53 * __dadd_rn(fabs(l), fabs(r));
        if (det > bound) return 1;
        if (-det > bound) return -1;
    }
    double u1, u0, v1, v0, w1, w0, z1, z0;
    x_two_diff(bx, ax, u1, u0);  // bx - ax = u1 + u0
    x_two_diff(cy, ay, v1, v0);  // cy - ay
    x_two_diff(by, ay, w1, w0);  // by - ay
    x_two_diff(cx, ax, z1, z0);  // cx - ax
    double h[16];
    int len = 0;
    len = x_add_product(h, len, u1, v1, false);
    len = x_add_product(h, len, u1, v0, false);
    len = x_add_product(h, len, u0, v1, false);
    len = x_add_product(h, len, u0, v0, false);
    len = x_add_product(h, len, w1, z1, true);
    len = x_add_product(h, len, w1, z0, true);
    len = x_add_product(h, len, w0, z1, true);
    len = x_add_product(h, len, w0, z0, true);
    // zero-free and ordered by magnitude: the last term carries the sign
    return len == 0 ? 0 : (h[len - 1] > 0.0 ? 1 : -1);
}

}  // namespace pip
