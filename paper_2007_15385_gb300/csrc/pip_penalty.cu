// pip_penalty.cu -- differentiable collision penalty of a convex footprint
// placed at SE(2) poses, through the Voronoi margin:
//
//   L = sum_pose sum_point softplus(-m(x) / tau),   x = R(theta)^T (p - t),
//   m(x) = max_k (|x - p0|^2 - |x - p_k|^2) / (2 |p_k - p0|),
//
// the largest signed distance of x from the Voronoi edges (the bisectors of
// p0 and p_k, Eq. 2), with p0, p_k the footprint's centroid (Eq. 3-4) and
// mirrored generators (Eq. 8).  The gradient flows back through the edge
// that attains the max (lowest k among ties), through Eq. 8 and through
// Eq. 3-4 to the vertices, and through the rigid transform to the poses.
// Both calls rebuild the generator tables from the vertices (nothing is kept
// between forward and backward) inside a caller-provided workspace.
//
// Layout of the work: block (tile, pose) takes one pose and kPenPoints
// points.  One thread per edge first folds each pose into the edge's
// coefficients (fp64 from the fp64 generators, kept as a rounded float32 part
// and its float32 remainder), so that a margin term is two FMAs on the world
// point; for up to 16 edges the rounded parts then sit in registers.  The
// forward pass keeps float32 partial sums per thread and reduces them in fp64
// per block; a final kernel adds the block slots in a fixed order.  In the
// backward pass only the (pose, point) pairs with a nonzero gradient (the
// points within ~87 tau of the footprint, where the float32 sigmoid has not
// underflowed) need the argmax edge and the per-edge sums; each warp queues
// those pairs in shared memory and resolves them 32 at a time, one pair per
// lane.  For each such pair the argmax edge is re-decided and its margin
// re-evaluated in float-float arithmetic (the point's exact offset from the
// pose times the two-part coefficients, every edge within the float32 terms'
// rounding bound of the max taking part), the sigmoid takes a first-order
// correction for the low part of z, and per-lane float32 slots gather each
// edge's sums, which the block adds in fp64.
#include <stdlib.h>

#include "pip_prepare_kernel.cuh"

namespace {

constexpr int kPenThreads = 256;
constexpr int kPenPoints = 32768;  // points per block

struct PenWorkspace {
    PolyInfo *poly;
    int32_t *voffs;
    int32_t *worst;
    double2 *g0;
    double2 *gk;
    float4 *coef;
    float4 *coefn;
    double *loss_part;   // [blocks]
    double *loss_stage;  // [ceil(blocks / kRedPer)]  first-level sums of loss_part
    double *pose_part;   // [3][blocks]  dL/d(t_x, t_y, theta) of the block's pose, its points only
    double *edge_part;   // [n][3][blocks]  (sum g, sum g x, sum g y) per argmax edge
    double *edge_stage;  // [n][3][kEdgeChunks]  first-level sums of edge_part
    double *pose_sum;    // [3][P]  reduced
    float4 *pose_coef;  // [P][kPoseStride]  per-pose affine forms (w'_x, w'_y, c', 0), rounded
    float4 *pose_lo;    // [P][kPoseStride]  what the rounding left: exact - rounded, in float32
    double2 *pose_rot;  // [P]  (cos theta, sin theta)
    float4 *pose_cull;  // [P]  (T_x, T_y, threshold on |p - T|^2, 0): the cull disc (PIP_PENALTY_CULL)
};

// The cull (PIP_PENALTY_CULL) leaves out the pairs whose margin is provably
// above kCullZ tau: their float32 softplus term (e^-|z| below 2^-150) and
// their gradient (the backward queues z >= -88 only) are exactly 0.
constexpr double kCullZ = 120.0;

constexpr int kPoseStride = kMaxEdges;
constexpr int kRedPer = 2048;     // loss partials per first-level reduction block
constexpr int kEdgeChunks = 16;   // first-level reduction blocks per edge sum

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t carve(void *base, int n, int P, int64_t blocks, PenWorkspace *w)
{
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align256(off + bytes);
        return (char *)base + o;
    };
    w->poly = (PolyInfo *)take(sizeof(PolyInfo));
    w->voffs = (int32_t *)take(2 * sizeof(int32_t));
    w->worst = (int32_t *)take(sizeof(int32_t));
    w->g0 = (double2 *)take(sizeof(double2));
    w->gk = (double2 *)take((size_t)n * sizeof(double2));
    w->coef = (float4 *)take((size_t)n * sizeof(float4));
    w->coefn = (float4 *)take((size_t)n * sizeof(float4));
    w->loss_part = (double *)take((size_t)blocks * sizeof(double));
    w->loss_stage = (double *)take((size_t)((blocks + kRedPer - 1) / kRedPer) * sizeof(double));
    w->pose_part = (double *)take((size_t)blocks * 3 * sizeof(double));
    w->edge_part = (double *)take((size_t)blocks * n * 3 * sizeof(double));
    w->edge_stage = (double *)take((size_t)n * 3 * kEdgeChunks * sizeof(double));
    w->pose_sum = (double *)take((size_t)P * 3 * sizeof(double));
    w->pose_coef = (float4 *)take((size_t)P * kPoseStride * sizeof(float4));
    w->pose_lo = (float4 *)take((size_t)P * kPoseStride * sizeof(float4));
    w->pose_rot = (double2 *)take((size_t)P * sizeof(double2));
    w->pose_cull = (float4 *)take((size_t)P * sizeof(float4));
    return off;
}

__global__ void pen_begin_kernel(int32_t *voffs, int32_t *worst, int n)
{
    if (threadIdx.x == 0) {
        voffs[0] = 0;
        voffs[1] = n;
        *worst = 0;
    }
}

__device__ __forceinline__ double block_sum(double v, double *red)
{
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];  // fixed order
    return s;  // meaningful in thread 0
}

// max of three (a NaN operand is ignored unless all are NaN)
__device__ __forceinline__ float fmax3(float a, float b, float c)
{
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// e^-|z| on the special-function unit (ex2), never above 1
__device__ __forceinline__ float exp_neg_abs(float z)
{
    return __expf(-fabsf(z));
}

// log(1 + e) for e in [0, 1]: with u = fl(1 + e), log(u) * e / (u - 1) is
// accurate to a few ulp even where u rounds e away (Goldberg 1991, "What
// every computer scientist should know about floating-point arithmetic",
// Theorem 4); u == 1 means log(1 + e) = e to float precision.  log(u) on the
// special-function unit (lg2).
__device__ __forceinline__ float log1p_small(float e)
{
    const float u = 1.f + e;
    return u == 1.f ? e : __logf(u) * __fdividef(e, u - 1.f);
}

// Per pose, the margin terms as affine forms of d = p - t (the point relative
// to the pose's position, world axes):
//   m_k = xb . w_k - c_k  (xb = R^T d body coordinates, w_k = (p_k - p0) / |p_k - p0|
//   the unit normal of edge k, c_k = w_k . (p0 + p_k) / 2 the edge line's
//   offset from the body origin: the bisector of Eq. 2 passes through the
//   midpoint of p0 and p_k)
//       = d . w'_k - c_k,   w'_k = R w_k,
// formed in fp64 from the fp64 generators (one block per pose, one thread per
// edge), rounded once to float32 for the bulk margin, with the float32
// remainder exact - rounded kept beside it for the float-float margin of the
// backward pass.  Keeping t out of the constant keeps it small: a rounded
// t . w' (tens of metres) would shift every margin of the pose by the same
// ~1e-6 m.  Slots past n hold w' = 0, c = +inf (m_k = -inf never attains the
// max).
__global__ void __launch_bounds__(64) pose_coef_kernel(const PolyInfo *__restrict__ poly,
                                                       const double2 *__restrict__ g0tab,
                                                       const double2 *__restrict__ gktab,
                                                       const float *__restrict__ poses, int P,
                                                       float4 *__restrict__ pose_coef, float4 *__restrict__ pose_lo,
                                                       double2 *__restrict__ pose_rot, float tau,
                                                       float4 *__restrict__ pose_cull)
{
    const int j = blockIdx.x, k = threadIdx.x;
    if (j >= P) return;
    const PolyInfo pi = poly[0];
    const int n = pi.status == PIP_OK ? pi.n : 0;
    const double th = poses[3 * j + 2];
    const double cn = cos(th), sn = sin(th);
    if (k == 0) pose_rot[j] = make_double2(cn, sn);
    for (int e = k; e < kPoseStride; e += blockDim.x) {
        float4 r = make_float4(0.f, 0.f, INFINITY, 0.f), lo = make_float4(0.f, 0.f, 0.f, 0.f);
        if (e < n) {
            const double2 g0 = g0tab[0], g = gktab[e];
            const double ux = g.x - g0.x, uy = g.y - g0.y;
            const double D = sqrt(ux * ux + uy * uy);
            const double wx = ux / D, wy = uy / D;
            const double ck = 0.5 * (wx * (g0.x + g.x) + wy * (g0.y + g.y));
            const double wpx = cn * wx - sn * wy, wpy = sn * wx + cn * wy;
            r = make_float4((float)wpx, (float)wpy, (float)ck, 0.f);
            lo = make_float4((float)(wpx - (double)r.x), (float)(wpy - (double)r.y), (float)(ck - (double)r.z), 0.f);
        }
        pose_coef[(size_t)j * kPoseStride + e] = r;
        pose_lo[(size_t)j * kPoseStride + e] = lo;
    }
    if (k == 0) {
        // The pose's cull disc.  With w_k the unit outward normals and H the
        // largest |p_k - p0| / 2 (the distance from p0 to an edge line), every
        // unit direction u meets some normal within half the largest angle
        // theta between consecutive normals, so
        //     m(x) = max_k (w_k . (x - p0) - |p_k - p0| / 2) >= kappa |x - p0| - H,
        // kappa = cos(theta / 2).  In world coordinates |x - p0| = |p - T|,
        // T = t + R p0.  A pair with |p - T| > (kCullZ tau + H) / kappa has
        // m > kCullZ tau; the threshold on the float32 d2 = fl(e_x e_x + fl(e_y e_y)),
        // e = fl(p - float32(T)), carries 2^-20 of relative slack and 2^-20 |T|_1
        // of absolute slack for the roundings of e, d2 and T.  No cull when a
        // turn is pi or more (not convex) or the footprint is invalid.
        float4 pc = make_float4(0.f, 0.f, INFINITY, 0.f);
        if (n > 0) {
            const double2 g0 = g0tab[0];
            double H = 0.0, cmin = 1.0;
            bool ok = true;
            double2 gl = gktab[n - 1];
            double qx = gl.x - g0.x, qy = gl.y - g0.y;
            double ql = sqrt(qx * qx + qy * qy);
            qx /= ql;
            qy /= ql;
            for (int e = 0; e < n; ++e) {
                const double2 g = gktab[e];
                const double ux = g.x - g0.x, uy = g.y - g0.y, D = sqrt(ux * ux + uy * uy);
                const double wx = ux / D, wy = uy / D;
                H = fmax(H, 0.5 * D);
                if (!((qx * wy - qy * wx) * pi.orient > 0.0)) ok = false;
                cmin = fmin(cmin, qx * wx + qy * wy);
                qx = wx;
                qy = wy;
            }
            const double kappa = sqrt(0.5 * (1.0 + cmin)) * (1.0 - 0x1p-40);
            const double tx = poses[3 * j], ty = poses[3 * j + 1];
            const double Tx = tx + cn * g0.x - sn * g0.y, Ty = ty + sn * g0.x + cn * g0.y;
            pc.x = (float)Tx;
            pc.y = (float)Ty;
            if (ok && kappa > 0.0) {
                const double R = (kCullZ * (double)tau + H) / kappa * (1.0 + 0x1p-20) +
                                 0x1p-20 * (fabs((double)pc.x) + fabs((double)pc.y)) + 0x1p-100;
                pc.z = __double2float_ru(R * R * (1.0 + 0x1p-20));
            }
        }
        pose_cull[j] = pc;
    }
}

// Forward: sum of softplus(-m / tau) over this block's points for its pose.
// NE > 0: the polygon has at most NE edges, coefficients in registers; NE == 0:
// any edge count, read from shared memory.  kPenUnroll points per thread in
// flight.
constexpr int kPenUnroll = 4;

template <bool B>
struct BoolTag {
    static constexpr bool value = B;
};

template <int NE>
__device__ __forceinline__ float margin_of(const float4 *cs, const float (&w)[NE > 0 ? NE : 1][3], int n,
                                           float dx, float dy)
{
    if (NE > 0) {
        float m = fmaf(dx, w[0][0], fmaf(dy, w[0][1], -w[0][2]));
#pragma unroll
        for (int k = 1; k + 1 < (NE > 0 ? NE : 2); k += 2)
            m = fmax3(m, fmaf(dx, w[k][0], fmaf(dy, w[k][1], -w[k][2])),
                      fmaf(dx, w[k + 1][0], fmaf(dy, w[k + 1][1], -w[k + 1][2])));
        if ((NE & 1) == 0)
            m = fmaxf(m, fmaf(dx, w[NE - 1][0], fmaf(dy, w[NE - 1][1], -w[NE - 1][2])));
        return m;
    }
    float m = -INFINITY;
    for (int k = 0; k < n; ++k) {
        const float4 c = cs[k];
        m = fmaxf(m, fmaf(dx, c.x, fmaf(dy, c.y, -c.z)));
    }
    return m;
}

// Backward accumulators, per edge (sum g, sum g dx, sum g dy) in shared
// memory, float32, summed over the block in fp64.  NE > 0: per lane, no
// atomics; a lane's slots are 3 NE + 1 words apart (odd), so that lanes on the
// same edge hit 32 different banks.  NE == 0 (up to 64 edges): per warp, by
// shared-memory atomics.  A lane's slot takes at most 64 terms per block (its
// share of the block's points), in practice a few: the slot sums' rounding is
// of the order of the products' own.
template <int NE>
__host__ __device__ constexpr int lane_words() { return NE > 0 ? 3 * NE + 1 : 3 * kMaxEdges; }
template <int NE>
__host__ __device__ constexpr int acc_rows() { return NE > 0 ? kPenThreads : kPenThreads / 32; }
template <int NE>
__host__ __device__ constexpr size_t acc_floats() { return (size_t)acc_rows<NE>() * lane_words<NE>(); }
// per-warp ring of queued pairs after the accumulators, three float arrays
// (p_x, p_y, m); drained at most every second pair, so it holds up to
// 31 + 2 x 32 entries
constexpr int kPenQueue = 128;
template <int NE>
constexpr size_t acc_bytes()
{
    return acc_floats<NE>() * sizeof(float) + (size_t)(kPenThreads / 32) * kPenQueue * 3 * sizeof(float);
}

// Error-free transformations (Knuth's two-sum, the FMA product error); the
// _rn intrinsics keep the compiler from fusing the roundings they rely on.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e)
{
    p = __fmul_rn(a, b);
    e = fmaf(a, b, -p);
}

// Margin of one edge in float-float: d = (px - tx, py - ty) exactly (two
// two-sums), times the two-part coefficients (hi + lo), minus c; returns
// mh + ml with |error| about 2^-44 of the largest term.
__device__ __forceinline__ void margin_ff(float px, float py, float tx, float ty, float4 hi, float4 lo,
                                         float &mh, float &ml)
{
    float dxh, dxl, dyh, dyl;
    two_sum(px, -tx, dxh, dxl);
    two_sum(py, -ty, dyh, dyl);
    float p1, e1, p2, e2, s1, e3, s2, e4;
    two_prod(dxh, hi.x, p1, e1);
    two_prod(dyh, hi.y, p2, e2);
    two_sum(p1, p2, s1, e3);
    two_sum(s1, -hi.z, s2, e4);
    float r = (e1 + e2) + (e3 + e4);
    r += fmaf(dxh, lo.x, dxl * hi.x) + fmaf(dyh, lo.y, dyl * hi.y) - lo.z;
    two_sum(s2, r, mh, ml);
}

// The argmax edge of a queued pair, decided as exactly as the float-float
// margins allow: every edge whose float32 term lies within `tol` of the
// float32 max m (tol bounds twice the terms' rounding error) is re-evaluated
// in float-float and the largest wins, the lowest k among ties.  Nearly
// always one edge qualifies.  Returns the edge and its margin (mh, ml).
template <int NE>
__device__ __forceinline__ int argmax_edge_ff(const float4 *cs, const float4 *cl,
                                              const float (&w)[NE > 0 ? NE : 1][3], int n, float px,
                                              float py, float tx, float ty, float m, float &mh, float &ml)
{
    const float dx = px - tx, dy = py - ty;  // as in the bulk pass
    // |fp32 term - exact term| <= 8u (|dx| + |dy| + |c_k| + |term|), |c_k| <= |term| + |dx| + |dy|
    const float tol = 0x1p-19f * (2.f * (fabsf(dx) + fabsf(dy)) + 2.f * fabsf(m)) + 0x1p-120f;
    const float lo = m - tol;
    // candidate edges as a bitmask (n <= 64), then one float-float margin each
    uint64_t cand = 0;
    if (NE > 0) {
#pragma unroll
        for (int k = 0; k < (NE > 0 ? NE : 1); ++k)
            if (fmaf(dx, w[k][0], fmaf(dy, w[k][1], -w[k][2])) >= lo) cand |= 1ull << k;
    } else {
        for (int k = 0; k < n; ++k) {
            const float4 c = cs[k];
            if (fmaf(dx, c.x, fmaf(dy, c.y, -c.z)) >= lo) cand |= 1ull << k;
        }
    }
    int kb = -1;
    mh = -INFINITY;
    ml = 0.f;
    while (cand) {
        const int k = __ffsll((long long)cand) - 1;  // ascending k: ties keep the lowest
        cand &= cand - 1;
        float h, l;
        margin_ff(px, py, tx, ty, cs[k], cl[k], h, l);
        if (h > mh || (h == mh && l > ml)) {
            kb = k;
            mh = h;
            ml = l;
        }
    }
    return kb;
}

// The register count is left to the compiler (58 at 12 edges, 4 blocks per
// SM): capping it at 128 or 80 measured 25 % and 14 % slower.
// CULL: each warp first tests its pairs against the pose's cull disc
// (pose_cull) and rings the pairs inside it in shared memory (p_x, p_y, after
// the backward pass's arrays); those go through the pair logic 32 at a time,
// the others add exactly 0 to the loss and nothing to the gradient.
template <int NE, bool BACKWARD>
constexpr size_t pen_smem(bool cull)
{
    return (BACKWARD ? acc_bytes<NE>() : 0) + (cull ? (size_t)(kPenThreads / 32) * 2 * kPenQueue * sizeof(float) : 0);
}

template <int NE, bool BACKWARD, bool CULL = false>
__global__ void __launch_bounds__(kPenThreads) penalty_kernel(
    const PolyInfo *__restrict__ poly, const float4 *__restrict__ pose_coef,
    const float4 *__restrict__ pose_lo, const double2 *__restrict__ pose_rot, const float *__restrict__ poses,
    const float *__restrict__ pts, int64_t M, int nv, float tau, double *__restrict__ loss_part, double *__restrict__ pose_part,
    double *__restrict__ edge_part, const float4 *__restrict__ pose_cull)
{
    constexpr int kWarps = kPenThreads / 32;
    extern __shared__ float lane_acc[];  // backward: [acc_rows][kLW] accumulators, then the warps' queues
    __shared__ double red[kWarps];
    const int n = poly[0].status == PIP_OK ? poly[0].n : 0;
    const int pose = blockIdx.y;
    const float4 *cs = pose_coef + (size_t)pose * kPoseStride;
    const float4 *cl = pose_lo + (size_t)pose * kPoseStride;
    float w[NE > 0 ? NE : 1][3];
#pragma unroll
    for (int k = 0; k < NE; ++k) {
        const float4 c = cs[k];
        w[k][0] = c.x;
        w[k][1] = c.y;
        w[k][2] = c.z;
    }
    constexpr int kLW = lane_words<NE>();
    float *my = lane_acc + (size_t)(NE > 0 ? threadIdx.x : threadIdx.x >> 5) * kLW;
    if (BACKWARD) {
        for (int e = threadIdx.x; e < acc_rows<NE>() * kLW; e += kPenThreads) lane_acc[e] = 0.f;
        __syncthreads();
    }
    const float inv_tau = 1.f / tau;
    const float ftx = poses[3 * pose], fty = poses[3 * pose + 1];

    float l_acc = 0.f;
    const int64_t p0 = (int64_t)blockIdx.x * kPenPoints;
    const int cnt = (int)(min(p0 + kPenPoints, M) - p0);  // this block's points
    const float2 *bp = (const float2 *)pts + p0;
    constexpr int kStep = kPenThreads * kPenUnroll;
    const int lane = threadIdx.x & 31;
    // Backward: the pairs with a possibly nonzero gradient, queued per warp
    // as (p_x, p_y, m) and finished 32 at a time.  Below z = -87.34 the
    // float32 e^-|z| flushes to 0, so dL/dm is exactly 0 there (kZCold leaves
    // a margin).  Head and tail count pairs (warp-uniform).  (Queuing the
    // forward pass's softplus the same way measured slower: the ballot per
    // pair costs more than the special functions it saves.)
    constexpr float kZCold = -88.f;
    float *qx = lane_acc + acc_floats<NE>() + (size_t)(threadIdx.x >> 5) * 3 * kPenQueue;
    float *qy = qx + kPenQueue, *qm = qy + kPenQueue;
    int qh = 0, qt = 0;
    // One queued pair: its argmax edge and margin in float-float, z = -m / tau
    // with its remainder, dL/dm = -sigmoid(z) / tau with the first-order term
    // sigmoid' z_lo; the edge's slot gathers g, g dx, g dy.
    auto finish = [&](int slot) {
        const float4 r = make_float4(qx[slot], qy[slot], qm[slot], 0.f);
        float mh, ml;
        const int kb = argmax_edge_ff<NE>(cs, cl, w, n, r.x, r.y, ftx, fty, r.z, mh, ml);
        if (kb < 0) return;  // a non-finite point: no gradient
        const float zh = __fmul_rn(-mh, inv_tau);
        const float zl = -(fmaf(zh, tau, mh) + ml) * inv_tau;  // z - zh
        const float e = expf(-fabsf(zh));
        const float inv = __fdividef(1.f, 1.f + e);
        const float sg = zh >= 0.f ? inv : e * inv;  // sigmoid(zh)
        const float sc = zh >= 0.f ? e * inv : inv;  // 1 - sigmoid(zh)
        const float g = -fmaf(sg * sc, zl, sg) * inv_tau;  // dL/dm
        const float dx = r.x - ftx, dy = r.y - fty;
        float *slot3 = my + 3 * kb;
        if (NE > 0) {
            slot3[0] += g;
            slot3[1] += g * dx;
            slot3[2] += g * dy;
        } else {
            atomicAdd(&slot3[0], g);
            atomicAdd(&slot3[1], g * dx);
            atomicAdd(&slot3[2], g * dy);
        }
    };

    // one (pose, point) pair; every thread of the block calls this the same
    // number of times, so that the whole warp takes part in every ballot
    auto pair = [&](float2 pt, bool valid) {
        const float dx = pt.x - ftx, dy = pt.y - fty;
        const float m = margin_of<NE>(cs, w, n, dx, dy);
        const float z = -m * inv_tau;
        if (!BACKWARD) {
            if (valid) l_acc += fmaxf(z, 0.f) + log1p_small(exp_neg_abs(z));  // softplus(z)
            return;
        }
        const bool hot = valid && !(z < kZCold);
        const unsigned bal = __ballot_sync(0xffffffffu, hot);
        if (bal) {
            const int at = (qt + __popc(bal & ((1u << lane) - 1u))) & (kPenQueue - 1);
            if (hot) {
                qx[at] = pt.x;
                qy[at] = pt.y;
                qm[at] = m;
            }
            qt += __popc(bal);
        }
    };
    // finishes whole groups of 32 queued pairs (called after every second pair)
    auto drain = [&]() {
        while (qt - qh >= 32) {
            __syncwarp();
            finish((qh + lane) & (kPenQueue - 1));
            qh += 32;
            __syncwarp();  // finished slots are refilled next
        }
    };
    // CULL: the ring of pairs inside the cull disc (holds at most 31 + 2 x 32)
    float *cx = lane_acc + (BACKWARD ? acc_bytes<NE>() / sizeof(float) : 0) + (size_t)(threadIdx.x >> 5) * 2 * kPenQueue;
    float *cy = cx + kPenQueue;
    int ch = 0, ct = 0;
    float Tx = 0.f, Ty = 0.f, Tc = INFINITY;
    if (CULL) {
        const float4 pc = pose_cull[pose];
        Tx = pc.x;
        Ty = pc.y;
        Tc = pc.z;
    }
    auto cull_pair = [&](float2 pt, bool valid) {
        const float ex = pt.x - Tx, ey = pt.y - Ty;
        const bool in = valid && !(fmaf(ex, ex, ey * ey) > Tc);  // NaN: kept
        const unsigned bal = __ballot_sync(0xffffffffu, in);
        if (bal) {
            const int at = (ct + __popc(bal & ((1u << lane) - 1u))) & (kPenQueue - 1);
            if (in) {
                cx[at] = pt.x;
                cy[at] = pt.y;
            }
            ct += __popc(bal);
        }
    };
    // whole groups of 32 ringed pairs through the pair logic (after every second pair)
    auto cull_drain = [&]() {
        while (ct - ch >= 32) {
            __syncwarp();
            const int sl = (ch + lane) & (kPenQueue - 1);
            const float2 pt = make_float2(cx[sl], cy[sl]);
            ch += 32;
            pair(pt, true);
            if (BACKWARD) drain();
        }
    };
    // Steps of kStep points, kPenUnroll per thread, with the next step's
    // points loaded into the other register set while these are evaluated.
    // FULL: a whole tile of kPenPoints, no bounds checks.
    auto tile = [&](auto full) {
        constexpr bool FULL = decltype(full)::value;
        const int steps = FULL ? kPenPoints / kStep : (cnt + kStep - 1) / kStep;
        auto load = [&](int st, float2 (&p)[kPenUnroll]) {
#pragma unroll
            for (int u = 0; u < kPenUnroll; ++u) {
                const int i = st * kStep + u * kPenThreads + (int)threadIdx.x;
                p[u] = (FULL || i < cnt) ? bp[i] : make_float2(ftx, fty);
            }
        };
        auto eval = [&](int st, const float2 (&p)[kPenUnroll]) {
#pragma unroll
            for (int u = 0; u < kPenUnroll; ++u) {
                const bool valid = FULL || st * kStep + u * kPenThreads + (int)threadIdx.x < cnt;
                if (CULL) {
                    cull_pair(p[u], valid);
                    if (u & 1) cull_drain();
                } else {
                    pair(p[u], valid);
                    if (BACKWARD && (u & 1)) drain();
                }
            }
        };
        float2 a[kPenUnroll], b[kPenUnroll];
        load(0, a);
        for (int st = 0; st < steps; st += 2) {
            if (FULL || st + 1 < steps) load(st + 1, b);
            eval(st, a);
            if (st + 2 < steps) load(st + 2, a);
            if (FULL || st + 1 < steps) eval(st + 1, b);
        }
    };
    static_assert(kPenPoints % (2 * kStep) == 0, "a full tile is an even number of steps");
    if (n > 0) {
        if (cnt == kPenPoints) tile(BoolTag<true>());
        else tile(BoolTag<false>());
        if (CULL) {
            // the last ringed pairs (fewer than 32)
            __syncwarp();
            const int rem = ct - ch;
            float2 pt = make_float2(Tx, Ty);
            if (lane < rem) pt = make_float2(cx[(ch + lane) & (kPenQueue - 1)], cy[(ch + lane) & (kPenQueue - 1)]);
            pair(pt, lane < rem);
            ch = ct;
            if (BACKWARD) drain();
        }
        if (BACKWARD) {
            __syncwarp();
            if (lane < qt - qh) finish((qh + lane) & (kPenQueue - 1));
        }
    }
    const int64_t blk = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
    const size_t nb = (size_t)gridDim.x * gridDim.y;  // blocks of the launch
    if (!BACKWARD) {
        const double s = block_sum((double)l_acc, red);
        if (threadIdx.x == 0) loss_part[blk] = s;
    } else {
        __syncthreads();
        // per (edge, component) v: warp v % 8 adds the slots of the lanes
        // (or warps), fp64, a fixed order
        __shared__ double es[kMaxEdges][3];
        const int wid = threadIdx.x >> 5;
        for (int v = wid; v < 3 * n; v += kWarps) {
            double t = 0.0;
            for (int r = lane; r < acc_rows<NE>(); r += 32) t += (double)lane_acc[(size_t)r * kLW + v];
            for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0) es[v / 3][v % 3] = t;
        }
        __syncthreads();
        __shared__ double pg[kMaxEdges][3];
        const int k = threadIdx.x;
        if (k < n) {
            const double S = es[k][0], Dx = es[k][1], Dy = es[k][2];
            const float4 c = cs[k], c2 = cl[k];
            const double wx = (double)c.x + (double)c2.x, wy = (double)c.y + (double)c2.y;
            // dm/dt = -w',  dm/dtheta = (p - t) x w' = dy w'_x - dx w'_y
            pg[k][0] = -S * wx;
            pg[k][1] = -S * wy;
            pg[k][2] = Dy * wx - Dx * wy;
            // body coordinates: xb = R^T (p - t)
            const double2 rc = pose_rot[pose];
            edge_part[(size_t)(3 * k) * nb + blk] = S;
            edge_part[(size_t)(3 * k + 1) * nb + blk] = rc.x * Dx + rc.y * Dy;
            edge_part[(size_t)(3 * k + 2) * nb + blk] = -rc.y * Dx + rc.x * Dy;
        } else if (k < nv) {
            // an invalid footprint (n = 0): zeros
            for (int c = 0; c < 3; ++c) edge_part[(size_t)(3 * k + c) * nb + blk] = 0.0;
        }
        __syncthreads();
        if (threadIdx.x < 3) {
            double v = 0.0;
            for (int e = 0; e < n; ++e) v += pg[e][threadIdx.x];  // fixed order
            pose_part[(size_t)threadIdx.x * nb + blk] = v;
        }
    }
}

// Fixed-order sums: block (b, r) adds row r's values [b L, (b + 1) L) of
// part[r][count] (a strided pass, then a tree of fixed shape) into
// out[r][gridDim.x].
__global__ void __launch_bounds__(kPenThreads) penalty_sum_kernel(const double *__restrict__ part,
                                                                  int64_t count, int64_t L,
                                                                  double *__restrict__ out)
{
    __shared__ double red[kPenThreads / 32];
    const double *row = part + (size_t)blockIdx.y * count;
    const int64_t lo = (int64_t)blockIdx.x * L, hi = min(lo + L, count);
    double s = 0.0;
    for (int64_t b = lo + threadIdx.x; b < hi; b += kPenThreads) s += row[b];
    s = block_sum(s, red);
    if (threadIdx.x == 0) out[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = s;
}

// Backward chain rule in fp64: one block, one thread per edge (n <= 64).
// Adds the edge sums' first-level slots (fixed order), then
//   per edge k (N = |x - p0|^2 - |x - p_k|^2 summed affinely, D = |p_k - p0|):
//     dL/dp0  += -(X - S p0)/D + Nsum (p_k - p0) / (2 D^3)
//     dL/dp_k  =  (X - S p_k)/D - Nsum (p_k - p0) / (2 D^3)
//   then back through Eq. 8 (p_k = p0 - 2 L_k(p0) (a, b) / (a^2 + b^2)) and
//   Eq. 3-4 (p0 = C / (3 S2)) to the vertices.  The pose gradients arrive
//   summed per pose (dL/dt = -sum g R(theta) w, dL/dtheta = sum g (p - t) x
//   R(theta) w, in world axes) and are only scaled here.  Edge k touches
//   vertices v_{k-1} and v_k; each vertex adds its two edges' shares in a
//   fixed order (no atomics).
__global__ void __launch_bounds__(64) penalty_chain_kernel(
    const float *__restrict__ verts, int n, const double2 *__restrict__ g0tab,
    const double2 *__restrict__ gk, const PolyInfo *__restrict__ poly, const float *__restrict__ poses,
    int P, const double *__restrict__ pose_sum, const double *__restrict__ edge_stage,
    const float *__restrict__ grad_out, double *__restrict__ grad_v, double *__restrict__ grad_pose)
{
    __shared__ double sG0[2][64];
    __shared__ double sgen[64][4];  // edge k's share for (v_{k-1}.x, v_{k-1}.y, v_k.x, v_k.y)
    __shared__ double scen[64][4];  // the same through the centroid
    const int k = threadIdx.x;
    const double scale = grad_out ? (double)grad_out[0] : 1.0;
    const bool ok = poly[0].status == PIP_OK;
    // pose gradients: one thread per pose, in a loop
    for (int j = k; j < P; j += blockDim.x)
        for (int c = 0; c < 3; ++c) grad_pose[3 * j + c] = ok ? scale * pose_sum[(size_t)c * P + j] : 0.0;
    double G0x = 0.0, G0y = 0.0;
    double gxm = 0.0, gym = 0.0, gxk = 0.0, gyk = 0.0;  // this edge's share of the vertex gradient
    const int km = k == 0 ? n - 1 : k - 1;
    double xm = 0.0, ym = 0.0, xk = 0.0, yk = 0.0;
    if (ok && k < n) {
        double E[3];
        for (int c = 0; c < 3; ++c) {
            double v = 0.0;
            for (int b = 0; b < kEdgeChunks; ++b) v += edge_stage[(size_t)(3 * k + c) * kEdgeChunks + b];
            E[c] = v;
        }
        const double S = E[0], X = E[1], Y = E[2];
        const double2 g0 = g0tab[0], g = gk[k];
        const double ux = g.x - g0.x, uy = g.y - g0.y;
        const double D = sqrt(ux * ux + uy * uy);
        const double rD = 1.0 / D;
        const double Nsum = 2.0 * (X * ux + Y * uy) + S * (g0.x * g0.x + g0.y * g0.y - g.x * g.x - g.y * g.y);
        const double h = 0.5 * Nsum * rD * rD * rD;  // Nsum / (2 D^3)
        const double Gkx = (X - S * g.x) * rD - h * ux;
        const double Gky = (Y - S * g.y) * rD - h * uy;
        G0x = -(X - S * g0.x) * rD + h * ux;
        G0y = -(Y - S * g0.y) * rD + h * uy;
        // Eq. 8 backward: a = y_k - y_{k-1}, b = x_{k-1} - x_k, c = x_k y_{k-1} - x_{k-1} y_k
        xm = verts[2 * km]; ym = verts[2 * km + 1]; xk = verts[2 * k]; yk = verts[2 * k + 1];
        const double a = yk - ym, b = xm - xk, c = xk * ym - xm * yk;
        const double rq = 1.0 / (a * a + b * b);
        const double L = a * g0.x + b * g0.y + c;
        const double nG = (a * Gkx + b * Gky) * rq;  // (a Gkx + b Gky) / q
        G0x += Gkx - 2.0 * a * nG;
        G0y += Gky - 2.0 * b * nG;
        // d p_k / d(a, b, c), contracted with G_k
        const double dA = -2.0 * (g0.x * nG + L * Gkx * rq - 2.0 * a * L * nG * rq);
        const double dB = -2.0 * (g0.y * nG + L * Gky * rq - 2.0 * b * L * nG * rq);
        const double dC = -2.0 * nG;
        // (a, b, c) as functions of v_{k-1} = (xm, ym) and v_k = (xk, yk)
        gxm = dB + dC * (-yk);
        gym = -dA + dC * xk;
        gxk = -dB + dC * ym;
        gyk = dA + dC * (-xm);
    }
    sG0[0][k] = G0x;
    sG0[1][k] = G0y;
    sgen[k][0] = gxm;
    sgen[k][1] = gym;
    sgen[k][2] = gxk;
    sgen[k][3] = gyk;
    __syncthreads();
    double Gx = 0.0, Gy = 0.0;
    for (int i = 0; i < n; ++i) {  // same order in every thread
        Gx += sG0[0][i];
        Gy += sG0[1][i];
    }
    // Eq. 3-4 backward: p0 = C / (3 S2), S2 = sum det_k, C = sum (v_{k-1} + v_k) det_k
    double c0 = 0.0, c1 = 0.0, c2 = 0.0, c3 = 0.0;
    if (ok && k < n) {
        double S2 = 0.0;
        for (int i = 0; i < n; ++i) {
            const int im = i == 0 ? n - 1 : i - 1;
            S2 += (double)verts[2 * im] * verts[2 * i + 1] - (double)verts[2 * i] * verts[2 * im + 1];
        }
        const double2 g0 = g0tab[0];
        const double rS = 1.0 / S2;
        const double lx = Gx * rS * (1.0 / 3.0), ly = Gy * rS * (1.0 / 3.0);
        const double mu = -(Gx * g0.x + Gy * g0.y) * rS;
        const double det = xm * yk - xk * ym;
        const double sx = xm + xk, sy = ym + yk;
        // d det / d(xm, ym, xk, yk) = (yk, -xk, -ym, xm)
        c0 = lx * (det + sx * yk) + ly * (sy * yk) + mu * yk;
        c1 = lx * (sx * -xk) + ly * (det + sy * -xk) + mu * -xk;
        c2 = lx * (det + sx * -ym) + ly * (sy * -ym) + mu * -ym;
        c3 = lx * (sx * xm) + ly * (det + sy * xm) + mu * xm;
    }
    scen[k][0] = c0;
    scen[k][1] = c1;
    scen[k][2] = c2;
    scen[k][3] = c3;
    __syncthreads();
    if (k < n) {
        // v_k ends edge k and starts edge k + 1
        const int kp = k == n - 1 ? 0 : k + 1;
        const double vx = (sgen[k][2] + sgen[kp][0]) + (scen[k][2] + scen[kp][0]);
        const double vy = (sgen[k][3] + sgen[kp][1]) + (scen[k][3] + scen[kp][1]);
        grad_v[2 * k] = ok ? scale * vx : 0.0;
        grad_v[2 * k + 1] = ok ? scale * vy : 0.0;
    }
}

// the footprint's edge count is known on the host: pick the register variant
template <bool BACKWARD, bool CULL>
void launch_penalty(int n, dim3 grid, cudaStream_t s, const PenWorkspace &w, const float *poses,
                    const float *pts, int64_t M, float tau)
{
    const int P = (int)grid.y;
    pose_coef_kernel<<<P, 64, 0, s>>>(w.poly, w.g0, w.gk, poses, P, w.pose_coef, w.pose_lo, w.pose_rot, tau,
                                      w.pose_cull);
    // the backward pass's accumulators and queues (up to 57 KiB at 16 edges,
    // 8 KiB more with the cull's rings) with the static reduction buffers
    // pass the default 48 KiB limit
#define PIP_PEN(NE)                                                                                     \
    do {                                                                                                \
        const size_t sm = pen_smem<NE, BACKWARD>(CULL);                                                 \
        if (BACKWARD)                                                                                   \
            cudaFuncSetAttribute(penalty_kernel<NE, BACKWARD, CULL>,                                    \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);                 \
        penalty_kernel<NE, BACKWARD, CULL><<<grid, kPenThreads, sm, s>>>(                               \
            w.poly, w.pose_coef, w.pose_lo, w.pose_rot, poses, pts, M, n, tau, w.loss_part, w.pose_part,  \
            w.edge_part, w.pose_cull);                                                                    \
    } while (0)
    if (n <= 4) PIP_PEN(4);
    else if (n <= 8) PIP_PEN(8);
    else if (n <= 12) PIP_PEN(12);
    else if (n <= 16) PIP_PEN(16);
    else PIP_PEN(0);
#undef PIP_PEN
}

pip_status check_args(const float *d_vertices, int32_t n, const float *d_poses, int32_t P,
                      const float *d_points, int64_t M, float tau, void *ws, size_t ws_bytes)
{
    if (d_vertices == nullptr || d_poses == nullptr || ws == nullptr) return PIP_E_INVALID_ARG;
    if (n < kMinEdges || n > kMaxEdges || P < 1 || M < 0 || !(tau > 0.f)) return PIP_E_INVALID_ARG;
    if (M > 0 && (d_points == nullptr || !aligned(d_points, 8))) return PIP_E_INVALID_ARG;
    if (!aligned(d_vertices, 8) || !aligned(d_poses, 4) || !aligned(ws, 256)) return PIP_E_INVALID_ARG;
    if (ws_bytes < pip_penalty_workspace_bytes(n, P, M)) return PIP_E_INVALID_ARG;
    return PIP_OK;
}

}  // namespace

extern "C" {

size_t pip_penalty_workspace_bytes(int32_t num_vertices, int32_t num_poses, int64_t num_points)
{
    if (num_vertices < 1 || num_poses < 1 || num_points < 0) return 0;
    const int64_t tiles = num_points > 0 ? (num_points + kPenPoints - 1) / kPenPoints : 1;
    PenWorkspace w;
    return carve(nullptr, num_vertices, num_poses, tiles * num_poses, &w) + 256;
}

pip_status pip_penalty_forward(const float *d_vertices, int32_t num_vertices, const float *d_poses,
                               int32_t num_poses, const float *d_points, int64_t num_points, float tau,
                               double *d_loss, int32_t flags, void *d_workspace, size_t workspace_bytes,
                               void *stream)
{
    pip_status st = check_args(d_vertices, num_vertices, d_poses, num_poses, d_points, num_points, tau,
                               d_workspace, workspace_bytes);
    if (st != PIP_OK) return st;
    if (d_loss == nullptr || (flags & ~PIP_PENALTY_CULL)) return PIP_E_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t tiles = num_points > 0 ? (num_points + kPenPoints - 1) / kPenPoints : 1;
    PenWorkspace w;
    carve(d_workspace, num_vertices, num_poses, tiles * num_poses, &w);
    pen_begin_kernel<<<1, 32, 0, s>>>(w.voffs, w.worst, num_vertices);
    prepare_kernel<<<1, 32, 0, s>>>(d_vertices, PIP_F32, w.voffs, 1, num_vertices, w.g0, w.gk, w.coef,
                                    w.coefn, w.poly, w.worst);
    if (flags & PIP_PENALTY_CULL)
        launch_penalty<false, true>(num_vertices, dim3((unsigned)tiles, (unsigned)num_poses), s, w, d_poses,
                                    d_points, num_points, tau);
    else
        launch_penalty<false, false>(num_vertices, dim3((unsigned)tiles, (unsigned)num_poses), s, w, d_poses,
                                     d_points, num_points, tau);
    const int64_t blocks = tiles * num_poses;
    const int64_t g = (blocks + kRedPer - 1) / kRedPer;
    penalty_sum_kernel<<<(unsigned)g, kPenThreads, 0, s>>>(w.loss_part, blocks, kRedPer, w.loss_stage);
    penalty_sum_kernel<<<1, kPenThreads, 0, s>>>(w.loss_stage, g, g, d_loss);
    return cudaGetLastError() == cudaSuccess ? PIP_OK : PIP_E_CUDA;
}

pip_status pip_penalty_backward(const float *d_vertices, int32_t num_vertices, const float *d_poses,
                                int32_t num_poses, const float *d_points, int64_t num_points, float tau,
                                const float *d_grad_loss, double *d_grad_vertices, double *d_grad_poses,
                                int32_t flags, void *d_workspace, size_t workspace_bytes, void *stream)
{
    pip_status st = check_args(d_vertices, num_vertices, d_poses, num_poses, d_points, num_points, tau,
                               d_workspace, workspace_bytes);
    if (st != PIP_OK) return st;
    if (d_grad_vertices == nullptr || d_grad_poses == nullptr || (flags & ~PIP_PENALTY_CULL))
        return PIP_E_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t tiles = num_points > 0 ? (num_points + kPenPoints - 1) / kPenPoints : 1;
    PenWorkspace w;
    carve(d_workspace, num_vertices, num_poses, tiles * num_poses, &w);
    pen_begin_kernel<<<1, 32, 0, s>>>(w.voffs, w.worst, num_vertices);
    prepare_kernel<<<1, 32, 0, s>>>(d_vertices, PIP_F32, w.voffs, 1, num_vertices, w.g0, w.gk, w.coef,
                                    w.coefn, w.poly, w.worst);
    if (flags & PIP_PENALTY_CULL)
        launch_penalty<true, true>(num_vertices, dim3((unsigned)tiles, (unsigned)num_poses), s, w, d_poses,
                                   d_points, num_points, tau);
    else
        launch_penalty<true, false>(num_vertices, dim3((unsigned)tiles, (unsigned)num_poses), s, w, d_poses,
                                    d_points, num_points, tau);
    const int64_t blocks = tiles * num_poses;
    // edge sums: kEdgeChunks slices per (edge, component); pose sums: one
    // block per (pose, component) over the pose's tiles
    penalty_sum_kernel<<<dim3(kEdgeChunks, 3 * num_vertices), kPenThreads, 0, s>>>(
        w.edge_part, blocks, (blocks + kEdgeChunks - 1) / kEdgeChunks, w.edge_stage);
    penalty_sum_kernel<<<dim3(num_poses, 3), kPenThreads, 0, s>>>(w.pose_part, blocks, tiles, w.pose_sum);
    penalty_chain_kernel<<<1, 64, 0, s>>>(d_vertices, num_vertices, w.g0, w.gk, w.poly, d_poses, num_poses,
                                          w.pose_sum, w.edge_stage, d_grad_loss, d_grad_vertices,
                                          d_grad_poses);
    return cudaGetLastError() == cudaSuccess ? PIP_OK : PIP_E_CUDA;
}

}  // extern "C"
