// pip_ragged_tma.cuh -- the pipelined own-polygon batch: many polygons, each
// with its own contiguous range of points (Alg. 5 per point against its own
// polygon only).
//
// Schedule.  The point array is cut at a fixed grid of kTile-point chunks, and
// one persistent launch works through the chunks: a CTA's producer warp takes
// the next chunk from a global counter (dynamic balance: polygons have 3 to
// 64 edges and 10^3 to 10^5 points), finds the chunk's first polygon by a
// 32-way search over the device point offsets (three dependent loads for
// 4,096 polygons), reads the next 32 offsets in one load, and packs the
// chunk's polygons, up to K of them, into a stage of the shared-memory ring:
// one bulk copy of their points (contiguous: the polygons' ranges are
// consecutive), their padded coefficient rows and their PolyInfo rows.  A
// chunk with more than K polygons takes several stages.  Before the loop
// every CTA checks a share of the offsets (non-decreasing, 0 .. M); the last
// CTA to finish resets the counters, so that one launch is the whole bulk
// test and no setup kernel is needed.
//
// Persistent CTAs, one producer warp and seven consumer warps (16 warps per SM
// at two CTAs: 128 registers a thread, 16 points per lane).  Consumers split
// the stage's points into 32*PPL-point slices on the chunk grid (one slice per
// warp, rotating over warps from stage to stage) and evaluate, for each of the
// stage's polygons that a slice meets, s_k = t_k - x w_kx - y w_ky with the
// first three edges peeled, four edges per step and an exact 0-3 edge tail.
// Mask words inside a polygon's range are stored; a word shared with a
// neighbouring polygon is written by each polygon through an AND that clears
// its own bits and an OR of its results, so the neighbours' writes commute.
// Uncertain points go to the global refine queue, decided by the refine
// launch that follows.  Integer polygons with integer points (EXACT) are
// decided exactly in the consumers instead, from the polygon's staged integer
// edge row (float32 determinants with an exact sign, or int64 beyond
// +-2^22), so that nothing is queued and no refine launch follows.
#pragma once

#include "pip_kernels.cuh"
#include "pip_tma.cuh"

namespace {

using namespace pip;

constexpr int kRaggedWarps = 7;  // consumer warps
constexpr int kRaggedThreads = (kRaggedWarps + 1) * 32;
constexpr int kMaxPack = 4;      // polygons per stage, at most

// The stage's header: its chunk, its polygons (indices and point ranges
// relative to the chunk, in order) and the consumers' rotation; np < 0 ends
// the CTA's loop.
struct RaggedHeader {
    int32_t c, np, rot, pad;
    int32_t j[kMaxPack], lo[kMaxPack], hi[kMaxPack];
};

// K: polygons per stage (1, 2 or 4).  ROWS: 16-byte entries per edge of a
// staged polygon row (2 for the ray comparator, 1 otherwise).
// DISC: each consumer warp also owns, in shared memory, PPL mask words and a
// list of up to 32 * PPL slice positions (the disc filter's undecided points).
template <int PPL, int STAGES, int K = 1, int ROWS = 1, bool DISC = false>
struct RaggedCfg {
    static constexpr int kSlice = 32 * PPL;
    static constexpr int kTile = kRaggedWarps * kSlice;  // points per chunk
    static constexpr size_t kPtsBytes = (size_t)kTile * 8;
    static constexpr size_t kCoefOff = kPtsBytes;
    static constexpr size_t kRowBytes = (size_t)ROWS * kPadStride * sizeof(float4);
    static constexpr size_t kInfoOff = kCoefOff + K * kRowBytes;
    static constexpr size_t kHdrOff = kInfoOff + K * sizeof(PolyInfo);
    static constexpr size_t kStageBytes = (kHdrOff + sizeof(RaggedHeader) + 127) & ~(size_t)127;
    static constexpr size_t kBarOff = STAGES * kStageBytes;
    static constexpr size_t kDiscOff = kBarOff + 2 * STAGES * sizeof(uint64_t);
    static constexpr size_t kDiscWarpBytes = (size_t)PPL * 4 + (size_t)kSlice * 2;
    static constexpr size_t kSmem = kDiscOff + (DISC ? kRaggedWarps * kDiscWarpBytes : 0);
    static constexpr int kFit = (int)((227 * 1024) / (kSmem + 1024));
    static constexpr int kMinBlocks = kFit < 1 ? 1 : (kFit > 2 ? 2 : kFit);
};

// The disc filter pays where the full test costs more per point than the
// filter's pass: polygons of at least this many edges (fewer take full work).
constexpr int kDiscMinEdges = 8;

// The batch kernel's counters, zero between launches: the next chunk, the
// refine queue's fill, the CTAs that have finished.
struct BatchCounters {
    unsigned int chunk, qfill, ticket;
};

// Largest j in [0, P) with poffs[j] <= x (the polygon holding point x when the
// offsets are a non-decreasing cover), by the whole warp, 32 probes a round.
__device__ __forceinline__ int find_polygon(const int64_t *__restrict__ poffs, int P, int64_t x, int lane)
{
    int lo = 0, hi = P;  // poffs[lo] <= x holds for lo = 0 (offsets start at 0)
    while (hi - lo > 1) {
        const int step = (hi - lo + 31) / 32;
        const int probe = lo + lane * step;
        const bool le = probe < hi && poffs[probe] <= x;
        const unsigned b = __ballot_sync(0xffffffffu, le) | 1u;
        const int L = 31 - __clz((int)b);
        lo = lo + L * step;
        hi = min(hi, lo + step);
    }
    return lo;
}

// The slice's PPL mask words.  Words wholly inside the polygon's range are
// stored (16-byte stores when aligned); a word shared with a neighbour gets an
// AND that clears the polygon's own bits and an OR of its results, so that
// the neighbours' writes commute and no word needs zeroing first.  A polygon
// owns its points' bits [a, b) and, when it holds the last point (bw > b),
// the bits past it up to bw (the end of the last word), which become 0.
__device__ __forceinline__ uint32_t own_bits(int64_t w0, int64_t a, int64_t bw)
{
    const int64_t lo = max(a, w0) - w0, hi = min(bw, w0 + 32) - w0;
    if (hi <= lo) return 0u;
    const uint32_t upto = hi >= 32 ? 0xffffffffu : ((1u << hi) - 1u);
    return upto & ~((1u << lo) - 1u);
}

template <int PPL, bool TAIL>
__device__ __forceinline__ void ragged_store_words(const uint32_t (&w_in)[PPL], int64_t gs, int64_t a, int64_t b,
                                                   int64_t bw, int lane, uint32_t *__restrict__ mask,
                                                   bool vec_store)
{
    uint32_t *mw = mask + (gs >> 5);
    if (!TAIL) {
        if (vec_store && (PPL % 4) == 0) {
            if (lane == 0) {
#pragma unroll
                for (int q = 0; q < PPL; q += 4)
                    *(uint4 *)(mw + q) = make_uint4(w_in[q], w_in[q + 1], w_in[q + 2], w_in[q + 3]);
            }
        } else {
            uint32_t myword = 0;
#pragma unroll
            for (int q = 0; q < PPL; ++q)
                if (lane == q) myword = w_in[q];
            if (lane < PPL) mw[lane] = myword;
        }
    } else {
        uint32_t myword = 0;
#pragma unroll
        for (int q = 0; q < PPL; ++q)
            if (lane == q) myword = w_in[q];
        if (lane < PPL) {
            const int64_t w0 = gs + 32 * lane;  // first point of this lane's word
            if (w0 >= a && w0 + 32 <= bw) {
                mw[lane] = myword;  // wholly this polygon's
            } else {
                const uint32_t own = own_bits(w0, a, bw);
                if (own) {
                    atomicAnd(&mw[lane], ~own);
                    if (myword & own) atomicOr(&mw[lane], myword & own);
                }
            }
        }
    }
}

// One consumer warp, one slice: points gs + [0, 32*PPL) of which [a, b) are
// polygon j's (TAIL: the slice is not wholly inside; the odd last point of
// the range is not in the bulk copy and is read from global memory).  An
// uncertain point is queued with its polygon (queue / qpoly).
// EARLY: the warp-uniform early break (as in the single-polygon kernel): edges
// in groups of four spread around the polygon, the warp stops once all its
// points are decided outside (min s < -B); same decisions as full work.
template <int PPL, bool INT, bool CENTER, bool TAIL, bool EARLY = false>
__device__ __forceinline__ void ragged_slice(const float4 *cs, int n, float ox, float oy, float b0, float b1,
                                             const unsigned char *rows, const void *__restrict__ pts,
                                             int64_t gs, int64_t a, int64_t b, int64_t bw, int lane,
                                             uint32_t *__restrict__ mask, bool vec_store, int j,
                                             uint32_t *__restrict__ queue, uint32_t *__restrict__ qpoly,
                                             unsigned int *__restrict__ qcount)
{
    float xs[PPL], ys[PPL], m[PPL];
    bool valid[PPL];
#pragma unroll
    for (int q = 0; q < PPL; ++q) {
        const int r = 32 * q + lane;
        const int64_t p = gs + r;
        float x = ox, y = oy;
        valid[q] = !TAIL || (p >= a && p < b);
        if (valid[q]) {
            if (TAIL && p == b - 1 && (b & 1)) {
                if (INT) {
                    x = (float)((const int32_t *)pts)[2 * p];
                    y = (float)((const int32_t *)pts)[2 * p + 1];
                } else {
                    x = ((const float *)pts)[2 * p];
                    y = ((const float *)pts)[2 * p + 1];
                }
            } else if (INT) {
                const int2 v = ((const int2 *)rows)[r];
                x = (float)v.x;
                y = (float)v.y;
            } else {
                const float2 v = ((const float2 *)rows)[r];
                x = v.x;
                y = v.y;
            }
        }
        // an integer point that float32 does not hold exactly becomes NaN: the
        // NaN-propagating min then leaves it undecided, for the exact refine
        if (INT && !int_exact(x, y)) x = __int_as_float(0x7fc00000);
        xs[q] = CENTER ? x - ox : x;
        ys[q] = CENTER ? y - oy : y;
    }
    // m = min_k s_k (NaN-propagating): three edges, then four at a time, then the rest
    if (EARLY) {
        const int G = ((n + 3) & ~3) / 4;  // rows are padded with w = 0, t = +inf
        float Bq[PPL];
#pragma unroll
        for (int q = 0; q < PPL; ++q) {
            Bq[q] = fmaf(b1, fabsf(xs[q]) + fabsf(ys[q]), b0);
            m[q] = INFINITY;
        }
        for (int g = 0; g < G; ++g) {
            const float4 c0 = cs[g], c1 = cs[G + g], c2 = cs[2 * G + g], c3 = cs[3 * G + g];
#pragma unroll
            for (int q = 0; q < PPL; ++q) {
                const float s0 = fmaf(-xs[q], c0.x, fmaf(-ys[q], c0.y, c0.z));
                const float s1 = fmaf(-xs[q], c1.x, fmaf(-ys[q], c1.y, c1.z));
                const float s2 = fmaf(-xs[q], c2.x, fmaf(-ys[q], c2.y, c2.z));
                const float s3 = fmaf(-xs[q], c3.x, fmaf(-ys[q], c3.y, c3.z));
                m[q] = fmin3_nan(fmin3_nan(m[q], s0, s1), s2, s3);
            }
            if (g + 1 < G) {
                bool out = true;
#pragma unroll
                for (int q = 0; q < PPL; ++q) out &= m[q] < -Bq[q] || !valid[q];
                if (__all_sync(0xffffffffu, out)) break;
            }
        }
    }
    if (!EARLY) {
        const float4 c0 = cs[0], c1 = cs[1], c2 = cs[2];
#pragma unroll
        for (int q = 0; q < PPL; ++q)
            m[q] = fmin3_nan(fmaf(-xs[q], c0.x, fmaf(-ys[q], c0.y, c0.z)),
                             fmaf(-xs[q], c1.x, fmaf(-ys[q], c1.y, c1.z)),
                             fmaf(-xs[q], c2.x, fmaf(-ys[q], c2.y, c2.z)));
    }
    int k = EARLY ? n : 3;
    for (; k + 4 <= n; k += 4) {
        const float4 c0 = cs[k], c1 = cs[k + 1], c2 = cs[k + 2], c3 = cs[k + 3];
#pragma unroll
        for (int q = 0; q < PPL; ++q) {
            const float s0 = fmaf(-xs[q], c0.x, fmaf(-ys[q], c0.y, c0.z));
            const float s1 = fmaf(-xs[q], c1.x, fmaf(-ys[q], c1.y, c1.z));
            const float s2 = fmaf(-xs[q], c2.x, fmaf(-ys[q], c2.y, c2.z));
            const float s3 = fmaf(-xs[q], c3.x, fmaf(-ys[q], c3.y, c3.z));
            m[q] = fmin3_nan(fmin3_nan(m[q], s0, s1), s2, s3);
        }
    }
    const int rem = n - k;  // 0 in the early-exit form
    if (rem == 1) {
        const float4 c0 = cs[k];
#pragma unroll
        for (int q = 0; q < PPL; ++q) m[q] = fmin_nan(m[q], fmaf(-xs[q], c0.x, fmaf(-ys[q], c0.y, c0.z)));
    } else if (rem == 2) {
        const float4 c0 = cs[k], c1 = cs[k + 1];
#pragma unroll
        for (int q = 0; q < PPL; ++q)
            m[q] = fmin3_nan(m[q], fmaf(-xs[q], c0.x, fmaf(-ys[q], c0.y, c0.z)),
                             fmaf(-xs[q], c1.x, fmaf(-ys[q], c1.y, c1.z)));
    } else if (rem == 3) {
        const float4 c0 = cs[k], c1 = cs[k + 1], c2 = cs[k + 2];
#pragma unroll
        for (int q = 0; q < PPL; ++q)
            m[q] = fmin3_nan(fmin_nan(m[q], fmaf(-xs[q], c0.x, fmaf(-ys[q], c0.y, c0.z))),
                             fmaf(-xs[q], c1.x, fmaf(-ys[q], c1.y, c1.z)),
                             fmaf(-xs[q], c2.x, fmaf(-ys[q], c2.y, c2.z)));
    }
    uint32_t w_in[PPL];
    bool unc[PPL];
    bool any = false;
#pragma unroll
    for (int q = 0; q < PPL; ++q) {
        // B >= beta0 + beta1 max(|x|, |y|); NaN m or infinite B is never "in"
        const float B = fmaf(b1, fabsf(xs[q]) + fabsf(ys[q]), b0);
        const bool in = (m[q] >= B) && valid[q];
        unc[q] = !(fabsf(m[q]) >= B) && valid[q];
        any |= unc[q];
        w_in[q] = __ballot_sync(0xffffffffu, in);
    }
    if (__any_sync(0xffffffffu, any)) {
        // one reservation in the global queue for the whole slice
        uint32_t u[PPL];
        unsigned int total = 0;
#pragma unroll
        for (int q = 0; q < PPL; ++q) {
            u[q] = __ballot_sync(0xffffffffu, unc[q]);
            total += (unsigned int)__popc(u[q]);
        }
        unsigned int base = 0;
        if (lane == 0) base = atomicAdd(qcount, total);
        base = __shfl_sync(0xffffffffu, base, 0);
        const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
        for (int q = 0; q < PPL; ++q) {
            if (unc[q]) {
                const unsigned int at = base + __popc(u[q] & lt);
                queue[at] = (uint32_t)(gs + 32 * q + lane);
                qpoly[at] = (uint32_t)j;
            }
            base += (unsigned int)__popc(u[q]);
        }
    }
    ragged_store_words<PPL, TAIL>(w_in, gs, a, b, bw, lane, mask, vec_store);
}

// m = min_k s_k for two points against a staged row: four edges a step, two
// partial minima per point so that the min chains stay short (NaN-propagating).
__device__ __forceinline__ void ragged_point_min2(const float4 *cs, int n, float x0, float y0, float x1, float y1,
                                                  float &m0, float &m1)
{
    float a0 = INFINITY, b0 = INFINITY, a1 = INFINITY, b1 = INFINITY;
    int k = 0;
#pragma unroll 2
    for (; k + 4 <= n; k += 4) {
        const float4 c0 = cs[k], c1 = cs[k + 1], c2 = cs[k + 2], c3 = cs[k + 3];
        a0 = fmin3_nan(a0, fmaf(-x0, c0.x, fmaf(-y0, c0.y, c0.z)), fmaf(-x0, c1.x, fmaf(-y0, c1.y, c1.z)));
        b0 = fmin3_nan(b0, fmaf(-x0, c2.x, fmaf(-y0, c2.y, c2.z)), fmaf(-x0, c3.x, fmaf(-y0, c3.y, c3.z)));
        a1 = fmin3_nan(a1, fmaf(-x1, c0.x, fmaf(-y1, c0.y, c0.z)), fmaf(-x1, c1.x, fmaf(-y1, c1.y, c1.z)));
        b1 = fmin3_nan(b1, fmaf(-x1, c2.x, fmaf(-y1, c2.y, c2.z)), fmaf(-x1, c3.x, fmaf(-y1, c3.y, c3.z)));
    }
    for (; k < n; ++k) {
        const float4 c0 = cs[k];
        a0 = fmin_nan(a0, fmaf(-x0, c0.x, fmaf(-y0, c0.y, c0.z)));
        a1 = fmin_nan(a1, fmaf(-x1, c0.x, fmaf(-y1, c0.y, c0.z)));
    }
    m0 = fmin_nan(a0, b0);
    m1 = fmin_nan(a1, b1);
}

// The disc filter (PIP_DISC) in a batch slice, as consume_slice_disc of the
// one-polygon kernel with the polygon's own thresholds (PolyInfo::tin /
// tout): a point with d2 = |p - o|^2 < tin is inside, one with d2 > tout
// outside, without its edges.  The rest are listed per warp in shared memory
// (`wlist`) and decided 64 at a time, two per lane, by the full test
// (ragged_point_min2, the float32 bound, uncertain points queued with their
// polygon); their inside bits are ORed into the warp's words (`wwords`).
template <int PPL, bool INT, bool CENTER, bool TAIL>
__device__ __forceinline__ void ragged_slice_disc(const float4 *cs, const PolyInfo &pi, const unsigned char *rows,
                                                  const void *__restrict__ pts, int64_t gs, int64_t a, int64_t b,
                                                  int64_t bw, int lane, uint32_t *__restrict__ mask, bool vec_store,
                                                  int j, uint32_t *__restrict__ queue, uint32_t *__restrict__ qpoly,
                                                  unsigned int *__restrict__ qcount, uint32_t *wwords,
                                                  uint16_t *wlist)
{
    const float ox = pi.ox, oy = pi.oy;
    // point gs + r; an integer point that float32 does not hold exactly
    // becomes NaN, so that the full test leaves it to the exact refine
    auto load = [&](int r, float &x, float &y) {
        const int64_t p = gs + r;
        if (TAIL && p == b - 1 && (b & 1)) {
            if (INT) {
                x = (float)((const int32_t *)pts)[2 * p];
                y = (float)((const int32_t *)pts)[2 * p + 1];
            } else {
                x = ((const float *)pts)[2 * p];
                y = ((const float *)pts)[2 * p + 1];
            }
        } else if (INT) {
            const int2 v = ((const int2 *)rows)[r];
            x = (float)v.x;
            y = (float)v.y;
        } else {
            const float2 v = ((const float2 *)rows)[r];
            x = v.x;
            y = v.y;
        }
        if (INT && !int_exact(x, y)) x = __int_as_float(0x7fc00000);
    };
    const uint32_t lt = (1u << lane) - 1u;
    uint32_t w_in[PPL], nb[PPL];
#pragma unroll
    for (int q = 0; q < PPL; ++q) {
        const int r = 32 * q + lane;
        const int64_t p = gs + r;
        const bool valid = !TAIL || (p >= a && p < b);
        float x = ox, y = oy;
        if (valid) load(r, x, y);
        const float xl = CENTER ? x - ox : x, yl = CENTER ? y - oy : y;
        const float d2 = fmaf(xl, xl, yl * yl);
        const bool in = valid && d2 < pi.tin;
        const bool near = valid && !in && !(d2 > pi.tout);  // NaN: the full test
        w_in[q] = __ballot_sync(0xffffffffu, in);
        nb[q] = __ballot_sync(0xffffffffu, near);
    }
    // the list: positions from the ballots alone, so the writes do not wait
    // on one another
    int cnt = 0;
#pragma unroll
    for (int q = 0; q < PPL; ++q) {
        if ((nb[q] >> lane) & 1u) wlist[cnt + __popc(nb[q] & lt)] = (uint16_t)(32 * q + lane);
        cnt += __popc(nb[q]);
    }
    if (cnt) {  // warp-uniform
        uint32_t myword = 0;
#pragma unroll
        for (int q = 0; q < PPL; ++q)
            if (lane == q) myword = w_in[q];
        if (lane < PPL) wwords[lane] = myword;
        __syncwarp();
        for (int base = 0; base < cnt; base += 64) {
            const bool act0 = base + lane < cnt, act1 = base + 32 + lane < cnt;
            const int r0 = act0 ? wlist[base + lane] : 0, r1 = act1 ? wlist[base + 32 + lane] : 0;
            float x0 = ox, y0 = oy, x1 = ox, y1 = oy;
            if (act0) load(r0, x0, y0);
            if (act1) load(r1, x1, y1);
            const float xl0 = CENTER ? x0 - ox : x0, yl0 = CENTER ? y0 - oy : y0;
            const float xl1 = CENTER ? x1 - ox : x1, yl1 = CENTER ? y1 - oy : y1;
            float m0, m1;
            ragged_point_min2(cs, pi.n, xl0, yl0, xl1, yl1, m0, m1);
            const float B0 = fmaf(pi.beta1, fabsf(xl0) + fabsf(yl0), pi.beta0);
            const float B1 = fmaf(pi.beta1, fabsf(xl1) + fabsf(yl1), pi.beta0);
            if (act0 && m0 >= B0) atomicOr(&wwords[r0 >> 5], 1u << (r0 & 31));
            if (act1 && m1 >= B1) atomicOr(&wwords[r1 >> 5], 1u << (r1 & 31));
            const bool unc0 = act0 && !(fabsf(m0) >= B0), unc1 = act1 && !(fabsf(m1) >= B1);
            const uint32_t u0 = __ballot_sync(0xffffffffu, unc0), u1 = __ballot_sync(0xffffffffu, unc1);
            if (u0 | u1) {
                unsigned int at = 0;
                if (lane == 0) at = atomicAdd(qcount, (unsigned int)(__popc(u0) + __popc(u1)));
                at = __shfl_sync(0xffffffffu, at, 0);
                if (unc0) {
                    queue[at + __popc(u0 & lt)] = (uint32_t)(gs + r0);
                    qpoly[at + __popc(u0 & lt)] = (uint32_t)j;
                }
                at += __popc(u0);
                if (unc1) {
                    queue[at + __popc(u1 & lt)] = (uint32_t)(gs + r1);
                    qpoly[at + __popc(u1 & lt)] = (uint32_t)j;
                }
            }
        }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < PPL; ++q) w_in[q] = wwords[q];
        __syncwarp();  // the words and the list are rewritten by the next slice
    }
    ragged_store_words<PPL, TAIL>(w_in, gs, a, b, bw, lane, mask, vec_store);
}

// Integer polygon and integer points, decided exactly here: no filter, no
// queue, no refine.  Edge k of the staged row is (a_x, a_y, e_x, e_y) in
// float32, a = v_{k-1}, e = orient (v_k - v_{k-1}); p is inside (closed) iff
// cross_k(p) = e_x d_y - e_y d_x >= 0 for every k, d = p - a.  With every
// vertex and the warp's points within +-2^22, a, e and d are exact in float32
// and the sign of the integer cross_k is exact from
//     w = fl(e_y d_x),  r = e_y d_x - w (one FMA, exact),
//     f = fl(e_x d_y - w) (one FMA),  cross_k ~ fl(f - r):
// if |e_x d_y - w| < 2^24, f is exact and f - r = cross_k; otherwise |f| and
// |e_x d_y - w| exceed |r| (<= 2^22, as |w| <= 2^46) by more than f's
// rounding, so f - r has the sign of cross_k.  The min over edges of those
// values is >= 0 iff the point is inside; rows past n are zero (neutral).
// A warp holding a point beyond +-2^22, or a polygon beyond it, takes the
// int64 form instead, cross_k = e_x p_y - e_y p_x - C from the polygon's
// integer row in global memory (two 32 x 32 -> 64-bit multiply-adds).
template <int PPL, bool TAIL>
__device__ __forceinline__ void ragged_slice_exact(const float4 *fs, const int4 *__restrict__ irow, int n,
                                                   bool poly_small, const unsigned char *rows,
                                                   const void *__restrict__ pts, int64_t gs, int64_t a, int64_t b,
                                                   int64_t bw, int lane, uint32_t *__restrict__ mask, bool vec_store)
{
    constexpr int kLim = 1 << 22;
    int px[PPL], py[PPL];
    bool valid[PPL];
    bool small = true;
#pragma unroll
    for (int q = 0; q < PPL; ++q) {
        const int r = 32 * q + lane;
        const int64_t p = gs + r;
        int x = 0, y = 0;
        valid[q] = !TAIL || (p >= a && p < b);
        if (valid[q]) {
            if (TAIL && p == b - 1 && (b & 1)) {
                x = ((const int32_t *)pts)[2 * p];
                y = ((const int32_t *)pts)[2 * p + 1];
            } else {
                const int2 v = ((const int2 *)rows)[r];
                x = v.x;
                y = v.y;
            }
        }
        px[q] = x;
        py[q] = y;
        small &= x >= -kLim && x <= kLim && y >= -kLim && y <= kLim;
    }
    const int npad = (n + 3) & ~3;
    uint32_t w_in[PPL];
    if (__all_sync(0xffffffffu, small && poly_small)) {
        float xs[PPL], ys[PPL], m[PPL];
#pragma unroll
        for (int q = 0; q < PPL; ++q) {
            xs[q] = (float)px[q];
            ys[q] = (float)py[q];
            m[q] = 0.f;
        }
        for (int k = 0; k < npad; k += 2) {
            const float4 c0 = fs[k], c1 = fs[k + 1];
#pragma unroll
            for (int q = 0; q < PPL; ++q) {
                const float dx0 = __fsub_rn(xs[q], c0.x), dy0 = __fsub_rn(ys[q], c0.y);
                const float w0 = __fmul_rn(c0.w, dx0);
                const float r0 = fmaf(c0.w, dx0, -w0);
                const float f0 = fmaf(c0.z, dy0, -w0);
                const float dx1 = __fsub_rn(xs[q], c1.x), dy1 = __fsub_rn(ys[q], c1.y);
                const float w1 = __fmul_rn(c1.w, dx1);
                const float r1 = fmaf(c1.w, dx1, -w1);
                const float f1 = fmaf(c1.z, dy1, -w1);
                m[q] = fmin3(m[q], __fsub_rn(f0, r0), __fsub_rn(f1, r1));
            }
        }
#pragma unroll
        for (int q = 0; q < PPL; ++q) w_in[q] = __ballot_sync(0xffffffffu, valid[q] && m[q] >= 0.f);
    } else {
        int neg[PPL];
#pragma unroll
        for (int q = 0; q < PPL; ++q) neg[q] = 0;
        for (int k = 0; k < npad; ++k) {
            const int4 e = irow[k];
            const long long c = (long long)(((unsigned long long)(unsigned)e.w << 32) | (unsigned)e.z);
#pragma unroll
            for (int q = 0; q < PPL; ++q) {
                const long long v = (long long)e.y * px[q] + ((long long)e.x * py[q] + c);
                neg[q] |= (int)(v >> 32);
            }
        }
#pragma unroll
        for (int q = 0; q < PPL; ++q) w_in[q] = __ballot_sync(0xffffffffu, valid[q] && neg[q] >= 0);
    }
    ragged_store_words<PPL, TAIL>(w_in, gs, a, b, bw, lane, mask, vec_store);
}

// What a batch slice decides: the Voronoi test (filter, or exact for integer
// inputs) or one of the comparators in the same frame (float32 points and
// polygons): sign of offset (Alg. 2), ray crossing (Alg. 1) and the literal
// fp64 Alg. 5.
constexpr int kRagVoronoi = 0, kRagSign = 1, kRagRay = 2, kRagFp64 = 3;

// A comparator slice, float32 points in absolute coordinates as in the
// listings.  Rows: sign of offset (w_x, w_y, t, 0) per edge with
// LHS - RHS = t - x w_x - y w_y; ray (w, t times the going-up sign) and
// (y_{k-1}, y_k); fp64 p_k per edge and p0 in the last slot.  Padding is NaN
// (sign, ray), so the polygon's whole rows run in groups of four edges.
template <int OP, int PPL, bool TAIL>
__device__ __forceinline__ void ragged_slice_cmp(const float4 *cs, int n, const unsigned char *rows,
                                                 const void *__restrict__ pts, int64_t gs, int64_t a, int64_t b,
                                                 int64_t bw, int lane, uint32_t *__restrict__ mask, bool vec_store)
{
    float xs[PPL], ys[PPL];
    bool valid[PPL];
#pragma unroll
    for (int q = 0; q < PPL; ++q) {
        const int r = 32 * q + lane;
        const int64_t p = gs + r;
        float x = 0.f, y = 0.f;
        valid[q] = !TAIL || (p >= a && p < b);
        if (valid[q]) {
            if (TAIL && p == b - 1 && (b & 1)) {
                x = ((const float *)pts)[2 * p];
                y = ((const float *)pts)[2 * p + 1];
            } else {
                const float2 v = ((const float2 *)rows)[r];
                x = v.x;
                y = v.y;
            }
        }
        xs[q] = x;
        ys[q] = y;
    }
    const int npad = (n + 3) & ~3;
    bool in[PPL];
    if (OP == kRagSign) {
        float mn[PPL], mx[PPL];
#pragma unroll
        for (int q = 0; q < PPL; ++q) mn[q] = mx[q] = __int_as_float(0x7fc00000);
        for (int k = 0; k < npad; k += 4) {
            const float4 c0 = cs[k], c1 = cs[k + 1], c2 = cs[k + 2], c3 = cs[k + 3];
#pragma unroll
            for (int q = 0; q < PPL; ++q) {
                const float v0 = fmaf(-xs[q], c0.x, fmaf(-ys[q], c0.y, c0.z));
                const float v1 = fmaf(-xs[q], c1.x, fmaf(-ys[q], c1.y, c1.z));
                const float v2 = fmaf(-xs[q], c2.x, fmaf(-ys[q], c2.y, c2.z));
                const float v3 = fmaf(-xs[q], c3.x, fmaf(-ys[q], c3.y, c3.z));
                mn[q] = fmin3(fmin3(mn[q], v0, v1), v2, v3);
                mx[q] = fmax3(fmax3(mx[q], v0, v1), v2, v3);
            }
        }
#pragma unroll
        for (int q = 0; q < PPL; ++q) in[q] = mn[q] >= 0.f || mx[q] < 0.f;
    } else if (OP == kRagRay) {
        uint32_t par[PPL];
#pragma unroll
        for (int q = 0; q < PPL; ++q) par[q] = 0u;
        for (int k = 0; k < npad; k += 2) {
            const float4 c0 = cs[2 * k], e0 = cs[2 * k + 1], c1 = cs[2 * k + 2], e1 = cs[2 * k + 3];
#pragma unroll
            for (int q = 0; q < PPL; ++q) {
                const float v0 = fmaf(-xs[q], c0.x, fmaf(-ys[q], c0.y, c0.z));
                const float v1 = fmaf(-xs[q], c1.x, fmaf(-ys[q], c1.y, c1.z));
                const bool s0 = (e0.y > ys[q]) != (e0.x > ys[q]);
                const bool s1 = (e1.y > ys[q]) != (e1.x > ys[q]);
                par[q] ^= (uint32_t)(s0 && v0 > 0.f) ^ (uint32_t)(s1 && v1 > 0.f);
            }
        }
#pragma unroll
        for (int q = 0; q < PPL; ++q) in[q] = par[q] != 0u;
    } else {
        const double2 *g = (const double2 *)cs;
        const double2 g0 = g[kPadStride - 1];
#pragma unroll
        for (int q = 0; q < PPL; ++q) {
            const double x = xs[q], y = ys[q];
            const double d0x = x - g0.x, d0y = y - g0.y;
            const double M0 = d0x * d0x + d0y * d0y;
            bool ok = true;
            for (int k = 0; k < n; ++k) {
                const double dx = x - g[k].x, dy = y - g[k].y;
                ok &= M0 <= dx * dx + dy * dy;
            }
            in[q] = ok;
        }
    }
    uint32_t w_in[PPL];
#pragma unroll
    for (int q = 0; q < PPL; ++q) w_in[q] = __ballot_sync(0xffffffffu, valid[q] && in[q]);
    ragged_store_words<PPL, TAIL>(w_in, gs, a, b, bw, lane, mask, vec_store);
}

// A polygon that failed validation contains no point: its whole words are
// zero, its bits of shared words are cleared.
template <int PPL>
__device__ __forceinline__ void ragged_slice_empty(int64_t gs, int64_t a, int64_t bw, int lane,
                                                   uint32_t *__restrict__ mask)
{
    if (lane < PPL) {
        const int64_t w0 = gs + 32 * lane;
        if (w0 >= a && w0 + 32 <= bw) {
            mask[(gs >> 5) + lane] = 0u;
        } else {
            const uint32_t own = own_bits(w0, a, bw);
            if (own) atomicAnd(&mask[(gs >> 5) + lane], ~own);
        }
    }
}

// EXACT (integer polygons and points): `coefp` is the table of the polygons'
// float32 edge rows (a_x, a_y, e_x, e_y) and every point is decided exactly in
// the consumers (nothing is queued); `ipad` holds the int64 rows for points or
// polygons beyond +-2^22.  OP other than kRagVoronoi: a comparator, `coefp`
// its row table (float polygons and points), nothing queued.  K: polygons per
// stage.  `qcount` receives the number of queued points (the refine's count).
// DISC: the disc filter of ragged_slice_disc (float Voronoi test only).
template <int PPL, int STAGES, bool INT, bool EXACT, int OP = kRagVoronoi, bool EARLY = false, int K = 1,
          bool DISC = false>
__global__ void __launch_bounds__(kRaggedThreads,
                                  RaggedCfg<PPL, STAGES, K, OP == kRagRay ? 2 : 1, DISC>::kMinBlocks) ragged_tma_kernel(
    const PolyInfo *__restrict__ poly, const float4 *__restrict__ coefp, const int4 *__restrict__ ipad,
    const void *__restrict__ pts, int64_t M, const int64_t *__restrict__ poffs, int P,
    BatchCounters *__restrict__ ctr, uint32_t *__restrict__ mask, uint32_t *__restrict__ queue,
    uint32_t *__restrict__ qpoly, unsigned int *__restrict__ qcount, int32_t *__restrict__ worst,
    int *__restrict__ err)
{
    using C = RaggedCfg<PPL, STAGES, K, OP == kRagRay ? 2 : 1, DISC>;
    constexpr int kSlice = C::kSlice;
    constexpr int kTile = C::kTile;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *full = (uint64_t *)(smem + C::kBarOff);
    uint64_t *empty = full + STAGES;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kRaggedWarps);
        }
        fence_mbar_init();
    }
    // this CTA's share of the offsets' check: a non-decreasing cover of [0, M)
    for (int j = blockIdx.x * blockDim.x + tid; j < P; j += gridDim.x * blockDim.x) {
        const int64_t a = poffs[j], b = poffs[j + 1];
        if (a < 0 || b < a || b > M || (j == 0 && a != 0) || (j == P - 1 && b != M))
            atomicMax(worst, (int)PIP_E_INVALID_ARG);
    }
    __syncthreads();
    const int64_t nchunks = (M + kTile - 1) / kTile;
    const int64_t last_word_end = (M + 31) & ~(int64_t)31;

    if (warp == kRaggedWarps) {
        // ---------------- producer: the whole warp finds a chunk's polygons,
        // lane 0 fills the stages
        int it = 0, s = 0;
        uint32_t ephase = 0;
        int rot = 0;
        bool fail = false;
        // chunks come in runs of consecutive chunks (guided: up to 8, fewer as the
        // work runs out), so that within a run the polygon walk continues from
        // the previous chunk instead of searching the offsets again
        unsigned int run_c = 0, run_end = 0;
        int jnext = 0;
        // the next chunk's offset window, loaded before this chunk's stages are
        // issued so that its latency hides behind the waits for free stages
        constexpr int64_t kBeyond = (int64_t)1 << 62;
        int pre_j = -1;
        int64_t pre_a = 0, pre_b = 0;
        for (;;) {
            if (run_c >= run_end) {
                unsigned int c = 0, len = 1;
                if (lane == 0) {
                    const unsigned int seen = *(volatile unsigned int *)&ctr->chunk;
                    const int64_t left = nchunks - (int64_t)seen;
                    len = (unsigned int)max((int64_t)1, min((int64_t)8, left / (16 * (int64_t)gridDim.x)));
                    c = atomicAdd(&ctr->chunk, len);
                }
                c = __shfl_sync(0xffffffffu, c, 0);
                len = __shfl_sync(0xffffffffu, len, 0);
                if ((int64_t)c >= nchunks) break;
                run_c = c;
                run_end = (unsigned int)min((int64_t)c + len, nchunks);
                jnext = find_polygon(poffs, P, (int64_t)c * kTile, lane);
            }
            const unsigned int c = run_c++;
            const int64_t c0 = (int64_t)c * kTile, c1 = min(c0 + kTile, M);
            int j = jnext;
            // the chunk's polygons, in groups of up to K non-empty ones
            while (j < P) {
                // lane i: polygon j + i and its range clipped to the chunk
                const int jj = j + lane;
                int64_t ra, rb;
                if (j == pre_j) {  // warp-uniform
                    ra = pre_a;
                    rb = pre_b;
                } else {
                    ra = jj < P ? poffs[jj] : kBeyond;
                    rb = jj < P ? poffs[jj + 1] : kBeyond;
                }
                pre_j = -1;
                const int64_t pa = jj < P ? max(ra, c0) : c1, pb = jj < P ? min(rb, c1) : c1;
                const bool starts = jj < P && ra < c1;  // meets the chunk or lies beyond it
                const bool meets = starts && pb > pa;
                const unsigned mm = __ballot_sync(0xffffffffu, meets);
                const unsigned beyond = __ballot_sync(0xffffffffu, !starts);
                // polygons before the first lane that lies beyond the chunk belong to it
                const int nlanes = beyond ? __ffs(beyond) - 1 : 32;
                unsigned todo = mm & (nlanes == 32 ? 0xffffffffu : ((1u << nlanes) - 1u));
                if (nlanes < 32 && run_c < run_end) {
                    // the next chunk of this run starts with the last polygon
                    // that starts before c1: load its window now
                    pre_j = j + max(nlanes - 1, 0);
                    const int jq = pre_j + lane;
                    pre_a = jq < P ? poffs[jq] : kBeyond;
                    pre_b = jq < P ? poffs[jq + 1] : kBeyond;
                }
                while (todo) {
                    // the next group: up to K polygons of `todo`, in order
                    int gj[K], glo[K], ghi[K];
                    int np = 0;
#pragma unroll
                    for (int q = 0; q < K; ++q) {
                        gj[q] = 0;
                        glo[q] = ghi[q] = 0;
                        if (todo) {  // warp-uniform
                            const int l = __ffs(todo) - 1;
                            todo &= todo - 1;
                            gj[q] = j + l;
                            glo[q] = (int)(__shfl_sync(0xffffffffu, pa, l) - c0);
                            ghi[q] = (int)(__shfl_sync(0xffffffffu, pb, l) - c0);
                            np = q + 1;
                        }
                    }
                    if (lane == 0) {
                        if (it >= STAGES && !mbar_wait(&empty[s], ephase, err)) fail = true;
                        if (!fail) {
                            unsigned char *st = smem + (size_t)s * C::kStageBytes;
                            RaggedHeader *h = (RaggedHeader *)(st + C::kHdrOff);
                            h->c = (int32_t)c;
                            h->np = np;
                            h->rot = rot;
#pragma unroll
                            for (int q = 0; q < K; ++q) {
                                h->j[q] = gj[q];
                                h->lo[q] = glo[q];
                                h->hi[q] = ghi[q];
                            }
                            const int lo = glo[0], hi = ghi[np - 1];
                            rot = (rot + (hi - 1) / kSlice - lo / kSlice + 1) % kRaggedWarps;
                            const int64_t sa = (c0 + lo) & ~(int64_t)1, eb = (c0 + hi) & ~(int64_t)1;
                            const uint32_t pbytes = eb > sa ? (uint32_t)((eb - sa) * 8) : 0u;
                            const uint32_t rbytes = (uint32_t)C::kRowBytes;
                            mbar_arrive_expect_tx(&full[s], pbytes + (uint32_t)np * (rbytes + (uint32_t)sizeof(PolyInfo)));
                            if (pbytes)
                                bulk_copy_g2s(st + (sa - c0) * 8, (const char *)pts + sa * 8, pbytes, &full[s]);
                            for (int q = 0; q < np; ++q) {
                                bulk_copy_g2s(st + C::kCoefOff + q * C::kRowBytes,
                                              (const char *)coefp + (size_t)gj[q] * C::kRowBytes, rbytes, &full[s]);
                                bulk_copy_g2s(st + C::kInfoOff + q * sizeof(PolyInfo), poly + gj[q],
                                              (uint32_t)sizeof(PolyInfo), &full[s]);
                            }
                            if (++s == STAGES) {
                                s = 0;
                                if (it + 1 >= 2 * STAGES) ephase ^= 1u;
                            }
                            ++it;
                        }
                    }
                    fail = __shfl_sync(0xffffffffu, fail, 0);
                    if (fail) break;
                }
                if (fail) break;
                if (nlanes < 32) {
                    // the next chunk starts with the last polygon that starts before c1
                    jnext = j + max(nlanes - 1, 0);
                    break;
                }
                j += 32;  // more than 32 polygons meet this chunk: the next window
            }
            if (j >= P) jnext = P - 1;
            if (fail) break;
        }
        if (lane == 0) {
            if (fail) {
                // gave up: let the copies already issued land before the CTA leaves
                for (int k = it > STAGES ? it - STAGES : 0; k < it; ++k)
                    mbar_wait(&full[k % STAGES], (uint32_t)((k / STAGES) & 1), err);
            } else if (it < STAGES || mbar_wait(&empty[s], ephase, err)) {
                RaggedHeader *h = (RaggedHeader *)(smem + (size_t)s * C::kStageBytes + C::kHdrOff);
                h->np = -1;
                mbar_arrive(&full[s]);  // release: the header is visible to the consumers
            }
        }
    } else {
        // ---------------- consumers
        const bool vec_store = ((uintptr_t)mask & 15) == 0;
        int s = 0;
        uint32_t fphase = 0;
        for (;;) {
            if (!mbar_wait(&full[s], fphase, err)) break;
            const unsigned char *st = smem + (size_t)s * C::kStageBytes;
            const RaggedHeader &h = *(const RaggedHeader *)(st + C::kHdrOff);  // read in place
            if (h.np < 0) break;
            const int lo0 = h.lo[0], hiN = h.hi[h.np - 1];
            const int nsl = (hiN - 1) / kSlice - lo0 / kSlice + 1;
            const int r = (warp - h.rot + kRaggedWarps) % kRaggedWarps;
            if (r < nsl) {
                const int64_t c0 = (int64_t)h.c * kTile;
                const int sl = lo0 / kSlice + r;
                const int64_t gs = c0 + (int64_t)sl * kSlice;
                const unsigned char *rows = st + (size_t)sl * kSlice * 8;
#pragma unroll 1
                for (int q = 0; q < h.np; ++q) {
                    const int64_t a = c0 + h.lo[q], b = c0 + h.hi[q];
                    if (b <= gs || a >= gs + kSlice) continue;  // this polygon misses the slice
                    const int64_t bw = b == M ? last_word_end : b;
                    const PolyInfo &pi = *(const PolyInfo *)(st + C::kInfoOff + q * sizeof(PolyInfo));
                    const float4 *cs = (const float4 *)(st + C::kCoefOff + q * C::kRowBytes);
                    const bool whole = gs >= a && gs + kSlice <= b;
                    const int j = h.j[q];
                    if (pi.status != PIP_OK) {
                        ragged_slice_empty<PPL>(gs, a, bw, lane, mask);
                    } else if (OP != kRagVoronoi) {
                        if (whole)
                            ragged_slice_cmp<OP, PPL, false>(cs, pi.n, rows, pts, gs, a, b, bw, lane, mask, vec_store);
                        else
                            ragged_slice_cmp<OP, PPL, true>(cs, pi.n, rows, pts, gs, a, b, bw, lane, mask, vec_store);
                    } else if (EXACT) {
                        const int4 *irow = ipad + (size_t)j * kPadStride;
                        const bool poly_small =
                            fmaxf(fmaxf(-pi.bbox[0], -pi.bbox[1]), fmaxf(pi.bbox[2], pi.bbox[3])) <= (float)(1 << 22);
                        if (whole)
                            ragged_slice_exact<PPL, false>(cs, irow, pi.n, poly_small, rows, pts, gs, a, b, bw, lane,
                                                           mask, vec_store);
                        else
                            ragged_slice_exact<PPL, true>(cs, irow, pi.n, poly_small, rows, pts, gs, a, b, bw, lane,
                                                          mask, vec_store);
                    } else if (DISC && pi.n >= kDiscMinEdges) {
                        unsigned char *dw = smem + C::kDiscOff + (size_t)(warp * C::kDiscWarpBytes);
                        uint32_t *wwords = (uint32_t *)dw;
                        uint16_t *wlist = (uint16_t *)(dw + PPL * 4);
                        if (!whole)
                            ragged_slice_disc<PPL, INT, true, true>(cs, pi, rows, pts, gs, a, b, bw, lane, mask,
                                                                    vec_store, j, queue, qpoly, &ctr->qfill, wwords,
                                                                    wlist);
                        else if (pi.ox == 0.f && pi.oy == 0.f)
                            ragged_slice_disc<PPL, INT, false, false>(cs, pi, rows, pts, gs, a, b, bw, lane, mask,
                                                                      vec_store, j, queue, qpoly, &ctr->qfill, wwords,
                                                                      wlist);
                        else
                            ragged_slice_disc<PPL, INT, true, false>(cs, pi, rows, pts, gs, a, b, bw, lane, mask,
                                                                     vec_store, j, queue, qpoly, &ctr->qfill, wwords,
                                                                     wlist);
                    } else if (whole) {
                        if (pi.ox == 0.f && pi.oy == 0.f)
                            ragged_slice<PPL, INT, false, false, EARLY>(cs, pi.n, 0.f, 0.f, pi.beta0, pi.beta1, rows,
                                                                        pts, gs, a, b, bw, lane, mask, vec_store, j,
                                                                        queue, qpoly, &ctr->qfill);
                        else
                            ragged_slice<PPL, INT, true, false, EARLY>(cs, pi.n, pi.ox, pi.oy, pi.beta0, pi.beta1, rows,
                                                                       pts, gs, a, b, bw, lane, mask, vec_store, j,
                                                                       queue, qpoly, &ctr->qfill);
                    } else {
                        ragged_slice<PPL, INT, true, true, EARLY>(cs, pi.n, pi.ox, pi.oy, pi.beta0, pi.beta1, rows,
                                                                  pts, gs, a, b, bw, lane, mask, vec_store, j, queue,
                                                                  qpoly, &ctr->qfill);
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
            if (++s == STAGES) {
                s = 0;
                fphase ^= 1u;
            }
        }
    }
    // the last CTA to finish hands over the queue's fill and resets the counters
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        const unsigned int t = atomicAdd(&ctr->ticket, 1u);
        if (t == gridDim.x - 1) {
            __threadfence();
            *qcount = atomicExch(&ctr->qfill, 0u);
            atomicExch(&ctr->chunk, 0u);
            atomicExch(&ctr->ticket, 0u);
        }
    }
}

}  // namespace
