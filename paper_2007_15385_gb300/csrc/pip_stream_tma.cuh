// pip_stream_tma.cuh -- the pipelined single-polygon test (the benchmark's
// hot path) and the warp-cooperative exact re-decision it calls inline.
//
// Persistent CTAs: one producer warp streams tiles of points from HBM into a
// ring of shared-memory stages with 1-D bulk copies (cp.async.bulk), each
// stage guarded by a "full" mbarrier (transaction bytes) and an "empty"
// mbarrier (one arrive per consumer warp, made as soon as the warp's points
// are in registers, so that the producer refills the stage during the edge
// math).  Consumer warps (8, or 16 in one CTA a SM) evaluate the
// expanded Eq. 11, s_k = t_k - x w_kx - y w_ky, with two FMAs per edge and
// take the "for all k" of Alg. 5 as a NaN-propagating running min; for up to
// 16 edges the coefficients sit in registers (edge count a template
// parameter), above that in shared memory.  32 decisions become one mask word
// with a ballot.  The few points whose float32 result lies within the error
// bound are decided exactly right there by the whole warp (one lane per
// edge), so one launch does the whole test.
#pragma once

#include "pip_kernels.cuh"
#include "pip_tma.cuh"

namespace {

using namespace pip;

// counters that survive between launches; the last CTA of each launch moves
// the refine count out and zeroes them, so every launch starts from zero
struct StreamCounters {
    unsigned int refine;
    unsigned int ticket;
};

// consumer warps of a CTA: 8 (two CTAs a SM), or 16 (one CTA a SM, stages of
// twice the size at the same shared memory per SM)
constexpr int kConsumerWarps = 8;

// DISC: each consumer warp also owns PPL mask words in shared memory (the
// disc filter's inside bits of the points it sends through the full test).
// CW: consumer warps.
template <int PPL, int STAGES, bool DISC = false, int CW = kConsumerWarps>
struct StreamCfg {
    static constexpr int kThreads = (CW + 1) * 32;  // the consumers and one producer warp
    static constexpr int kTile = CW * 32 * PPL;  // points per stage
    static constexpr size_t kStageBytes = (size_t)kTile * 8;
    static constexpr size_t kCoefOff = STAGES * kStageBytes;
    static constexpr int kCoef = 2 * (kMaxEdges + 4);  // float4 (w_x, w_y, t, 0), padded to 4; ray: two per edge
    static constexpr size_t kBarOff = kCoefOff + (size_t)kCoef * 16;
    static constexpr size_t kDiscOff = kBarOff + 2 * STAGES * sizeof(uint64_t);
    static constexpr size_t kDiscWarpBytes = (size_t)PPL * 4;
    static constexpr size_t kSmem = kDiscOff + (DISC ? CW * kDiscWarpBytes : 0);
    // two CTAs per SM (<= 112 registers a thread at 8 consumer warps) when
    // the shared memory allows it
    static constexpr int kFit = (int)((227 * 1024) / (kSmem + 1024));
    static constexpr int kMinBlocks = kFit < 1 ? 1 : (kFit > 2 ? 2 : kFit);
};

// What the per-edge term decides: the Voronoi test (Alg. 5, Eq. 11
// expanded), or the paper's comparators run in the same frame, sign of offset
// (Alg. 2) and ray crossing (Alg. 1), whose LHS - RHS is the same two-FMA
// affine form with other coefficients.
constexpr int kTmaVoronoi = 0, kTmaSign = 1, kTmaRay = 2;

// The polygon as launch parameters: read from the constant bank by the
// FMAs themselves (no registers, no loads).  Voronoi: edges past n carry
// w = 0, t = +inf, an invalid polygon one edge with t = -inf.  Comparators:
// (w_x, w_y, t) = (dV_y, -dV_x, -RHS) (ray: times the edge's going-up sign),
// y0 / y1 the edge's end ordinates (ray only); edges past n and an invalid
// polygon carry t = NaN, y0 = y1 = NaN.
constexpr int kParamEdges = 16;
struct StreamPoly {
    float ox, oy, b0, b1;
    int n, ok;
    float tin, tout;  // the polygon's disc bounds (PolyInfo)
    float wx[kParamEdges], wy[kParamEdges], t[kParamEdges];
    float y0[kParamEdges], y1[kParamEdges];
};

struct SliceCtx {
    const StreamPoly *sp;  // launch parameters (NE > 0)
    const float4 *cs;      // shared-memory coefficients (NE == 0)
    int npad;
};

// One consumer warp, one slice of 32 * PPL points of a stage: evaluate, write
// the slice's PPL mask words, queue the uncertain points.  TAIL: the slice may
// run past M (or hold the odd last point, which is not in the bulk copy).
// CENTER: subtract the local origin o (false when o = (0, 0)).
// EARLY: the early break of the sequential test (Sec. 5: stop at the first
// edge that already decides the point), made warp-uniform.  Edges run in
// groups of four spread around the polygon (edge i * n/4 + g of group g); after
// each group but the last, the warp stops when every one of its points already
// has min s < -B, i.e. is decided outside.  The full min could only be
// smaller, so the decisions are those of the full-work test.
// The slice's points are read from the stage once, into registers; the warp
// then hands the stage back (one arrive on `release`) before its edge math,
// so that the producer refills the stage while the warp computes.
template <int NE, int PPL, bool INT, bool CENTER, bool TAIL, bool EARLY = false>
__device__ __forceinline__ void consume_slice(const SliceCtx &cx, const unsigned char *stage,
                                              const void *__restrict__ pts, int64_t M, int64_t wfirst,
                                              int lane, uint32_t *__restrict__ mask, bool vec_store,
                                              uint32_t *__restrict__ myqueue, unsigned int *s_queued,
                                              uint64_t *release)
{
    const int nvalid = TAIL ? (int)max((int64_t)0, min((int64_t)32 * PPL, M - wfirst)) : 32 * PPL;
    const StreamPoly &sp = *cx.sp;
    float xs[PPL], ys[PPL], m[PPL];
    bool exin[PPL];
#pragma unroll
    for (int q = 0; q < PPL; ++q) {
        const int r = 32 * q + lane;
        float x = sp.ox, y = sp.oy;
        if (!TAIL || r < nvalid) {
            if (TAIL && wfirst + r == M - 1 && (M & 1)) {
                const int64_t p = M - 1;
                if (INT) {
                    x = (float)((const int32_t *)pts)[2 * p];
                    y = (float)((const int32_t *)pts)[2 * p + 1];
                } else {
                    x = ((const float *)pts)[2 * p];
                    y = ((const float *)pts)[2 * p + 1];
                }
            } else if (INT) {
                const int2 v = ((const int2 *)stage)[r];
                x = (float)v.x;
                y = (float)v.y;
            } else {
                const float2 v = ((const float2 *)stage)[r];
                x = v.x;
                y = v.y;
            }
        }
        exin[q] = INT ? int_exact(x, y) : true;
        xs[q] = CENTER ? x - sp.ox : x;  // local coordinates x = p - o
        ys[q] = CENTER ? y - sp.oy : y;
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(release);
    // m = min_k s_k, NaN-propagating so that a non-finite point stays undecided;
    // three operands per min (NE is a multiple of 4)
    if (EARLY) {
        float Bq[PPL];
#pragma unroll
        for (int q = 0; q < PPL; ++q) {
            Bq[q] = fmaf(sp.b1, fabsf(xs[q]) + fabsf(ys[q]), sp.b0);
            m[q] = INFINITY;
        }
        const int G = NE > 0 ? NE / 4 : cx.npad / 4;
        // one group of four spread edges; true when the warp may stop
        auto group = [&](int g) -> bool {
            float4 c[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int k = i * G + g;
                c[i] = NE > 0 ? make_float4(sp.wx[k], sp.wy[k], sp.t[k], 0.f) : cx.cs[k];
            }
#pragma unroll
            for (int q = 0; q < PPL; ++q) {
                const float s0 = fmaf(-xs[q], c[0].x, fmaf(-ys[q], c[0].y, c[0].z));
                const float s1 = fmaf(-xs[q], c[1].x, fmaf(-ys[q], c[1].y, c[1].z));
                const float s2 = fmaf(-xs[q], c[2].x, fmaf(-ys[q], c[2].y, c[2].z));
                const float s3 = fmaf(-xs[q], c[3].x, fmaf(-ys[q], c[3].y, c[3].z));
                m[q] = fmin3_nan(fmin3_nan(m[q], s0, s1), s2, s3);
            }
            if (g + 1 >= G) return true;
            bool out = true;
#pragma unroll
            for (int q = 0; q < PPL; ++q) out &= m[q] < -Bq[q];
            return __all_sync(0xffffffffu, out);
        };
        if (NE > 0) {
#pragma unroll
            for (int g = 0; g < (NE > 0 ? NE / 4 : 1); ++g)
                if (group(g)) break;
        } else {
            for (int g = 0; g < G; ++g)
                if (group(g)) break;
        }
    } else if (NE > 0) {
#pragma unroll
        for (int q = 0; q < PPL; ++q)
            m[q] = fmin_nan(fmaf(-xs[q], sp.wx[0], fmaf(-ys[q], sp.wy[0], sp.t[0])),
                            fmaf(-xs[q], sp.wx[1], fmaf(-ys[q], sp.wy[1], sp.t[1])));
#pragma unroll
        for (int k = 2; k < (NE > 0 ? NE : 2); k += 2) {
#pragma unroll
            for (int q = 0; q < PPL; ++q) {
                const float s1 = fmaf(-xs[q], sp.wx[k], fmaf(-ys[q], sp.wy[k], sp.t[k]));
                const float s2 = fmaf(-xs[q], sp.wx[k + 1], fmaf(-ys[q], sp.wy[k + 1], sp.t[k + 1]));
                m[q] = fmin3_nan(m[q], s1, s2);
            }
        }
    } else {
#pragma unroll
        for (int q = 0; q < PPL; ++q) m[q] = INFINITY;
        for (int k = 0; k < cx.npad; k += 4) {
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const float4 c = cx.cs[k + kk];
#pragma unroll
                for (int q = 0; q < PPL; ++q)
                    m[q] = fmin_nan(m[q], fmaf(-xs[q], c.x, fmaf(-ys[q], c.y, c.z)));
            }
        }
    }
    // decisions: one ballot per 32 points for "inside", one vote for the slice
    uint32_t w_in[PPL];
    bool unc[PPL];
    bool any = false;
#pragma unroll
    for (int q = 0; q < PPL; ++q) {
        // B >= beta0 + beta1 max(|x|, |y|), formed on the FMA pipe; a NaN or
        // infinite coordinate makes m NaN or B infinite, never "decided in"
        const float B = fmaf(sp.b1, fabsf(xs[q]) + fabsf(ys[q]), sp.b0);
        const bool valid = !TAIL || 32 * q + lane < nvalid;
        const bool in = (m[q] >= B) && (!INT || exin[q]) && valid;
        unc[q] = (!(fabsf(m[q]) >= B) || (INT && !exin[q])) && valid;
        any |= unc[q];
        w_in[q] = __ballot_sync(0xffffffffu, in);
    }
    if (__any_sync(0xffffffffu, any)) {
        // rare: queue the uncertain points; they are decided after the tile
        // loop, when the coefficient registers are free
#pragma unroll
        for (int q = 0; q < PPL; ++q) {
            const uint32_t u = __ballot_sync(0xffffffffu, unc[q]);
            if (u) {
                unsigned int base = 0;
                if (lane == 0) base = atomicAdd(s_queued, (unsigned int)__popc(u));
                base = __shfl_sync(0xffffffffu, base, 0);
                if (unc[q]) myqueue[base + __popc(u & ((1u << lane) - 1u))] = (uint32_t)(wfirst + 32 * q + lane);
            }
        }
    }
    // the slice's mask words: PPL consecutive words
    uint32_t *mw = mask + (wfirst >> 5);
    if (!TAIL && vec_store && (PPL % 4) == 0) {
        if (lane == 0) {
#pragma unroll
            for (int q = 0; q < PPL; q += 4)
                *(uint4 *)(mw + q) = make_uint4(w_in[q], w_in[q + 1], w_in[q + 2], w_in[q + 3]);
        }
    } else {
        const int nw = (nvalid + 31) >> 5;
        uint32_t myword = 0;
#pragma unroll
        for (int q = 0; q < PPL; ++q)
            if (lane == q) myword = w_in[q];
        if (lane < nw) mw[lane] = myword;
    }
}

// m = min_k s_k for one point (the full test's per-edge terms, NaN-propagating).
template <int NE>
__device__ __forceinline__ float point_min(const SliceCtx &cx, float x, float y)
{
    const StreamPoly &sp = *cx.sp;
    float m;
    if (NE > 0) {
        m = fmin_nan(fmaf(-x, sp.wx[0], fmaf(-y, sp.wy[0], sp.t[0])),
                     fmaf(-x, sp.wx[1], fmaf(-y, sp.wy[1], sp.t[1])));
#pragma unroll
        for (int k = 2; k < (NE > 0 ? NE : 2); k += 2)
            m = fmin3_nan(m, fmaf(-x, sp.wx[k], fmaf(-y, sp.wy[k], sp.t[k])),
                          fmaf(-x, sp.wx[k + 1], fmaf(-y, sp.wy[k + 1], sp.t[k + 1])));
    } else {
        m = INFINITY;
        for (int k = 0; k < cx.npad; k += 2) {
            const float4 c0 = cx.cs[k], c1 = cx.cs[k + 1];
            m = fmin3_nan(m, fmaf(-x, c0.x, fmaf(-y, c0.y, c0.z)), fmaf(-x, c1.x, fmaf(-y, c1.y, c1.z)));
        }
    }
    return m;
}

// The slice with the disc filter (PIP_DISC).  In the Voronoi picture the
// polygon is the cell of p0: no generator is nearer than p0 within half the
// distance to the nearest one, and the cell lies inside the disc through its
// farthest vertex.  Taken about the local origin o with rigorous float32
// thresholds (PolyInfo::tin / tout), a point with d2 = |x|^2 < tin is inside
// and one with d2 > tout outside, without its edges.  Each lane keeps a mask
// of its points left between the discs (in the benchmark's footprint about
// 1 %) and takes them one per pass through the full test of consume_slice
// (float32 filter, uncertain points queued for the exact decision); their
// inside bits are ORed into the warp's words in shared memory.  Decisions
// equal full work's.
template <int NE, int PPL, bool INT, bool CENTER, bool TAIL>
__device__ __forceinline__ void consume_slice_disc(const SliceCtx &cx, const unsigned char *stage,
                                                   const void *__restrict__ pts, int64_t M, int64_t wfirst,
                                                   int lane, uint32_t *__restrict__ mask, bool vec_store,
                                                   uint32_t *__restrict__ myqueue, unsigned int *s_queued,
                                                   uint32_t *wwords)
{
    static_assert(PPL <= 32, "one mask bit per point of a lane");
    const int nvalid = TAIL ? (int)max((int64_t)0, min((int64_t)32 * PPL, M - wfirst)) : 32 * PPL;
    const StreamPoly &sp = *cx.sp;
    // the point at slice position r (the odd last point is not in the bulk copy)
    auto load = [&](int r, float &x, float &y) {
        if (TAIL && wfirst + r == M - 1 && (M & 1)) {
            const int64_t p = M - 1;
            if (INT) {
                x = (float)((const int32_t *)pts)[2 * p];
                y = (float)((const int32_t *)pts)[2 * p + 1];
            } else {
                x = ((const float *)pts)[2 * p];
                y = ((const float *)pts)[2 * p + 1];
            }
        } else if (INT) {
            const int2 v = ((const int2 *)stage)[r];
            x = (float)v.x;
            y = (float)v.y;
        } else {
            const float2 v = ((const float2 *)stage)[r];
            x = v.x;
            y = v.y;
        }
    };
    uint32_t w_in[PPL];
    uint32_t nearm = 0;  // bit q: this lane's point 32 q + lane takes the full test
#pragma unroll
    for (int q = 0; q < PPL; ++q) {
        const int r = 32 * q + lane;
        const bool valid = !TAIL || r < nvalid;
        float x = sp.ox, y = sp.oy;
        if (valid) load(r, x, y);
        // an integer point that float32 does not hold exactly takes the full test
        const bool exact = INT ? int_exact(x, y) : true;
        const float xl = CENTER ? x - sp.ox : x, yl = CENTER ? y - sp.oy : y;
        const float d2 = fmaf(xl, xl, yl * yl);
        const bool in = valid && exact && d2 < sp.tin;
        // NaN d2 is neither in nor out: the full test decides it
        const bool near = valid && !in && !(exact && d2 > sp.tout);
        w_in[q] = __ballot_sync(0xffffffffu, in);
        nearm |= (uint32_t)near << q;
    }
    if (__any_sync(0xffffffffu, nearm != 0u)) {
        if (lane < PPL) wwords[lane] = 0u;
        __syncwarp();
        const uint32_t lt = (1u << lane) - 1u;
        while (__any_sync(0xffffffffu, nearm != 0u)) {
            // each lane takes its lowest pending point
            const bool act = nearm != 0u;
            const int q = act ? __ffs(nearm) - 1 : 0;
            nearm &= nearm - 1u;
            const int r = 32 * q + lane;
            float x = sp.ox, y = sp.oy;
            if (act) load(r, x, y);
            const bool exin = INT ? int_exact(x, y) : true;
            const float xl = CENTER ? x - sp.ox : x, yl = CENTER ? y - sp.oy : y;
            const float m = point_min<NE>(cx, xl, yl);
            const float B = fmaf(sp.b1, fabsf(xl) + fabsf(yl), sp.b0);
            const bool in = act && m >= B && exin;
            const bool unc = act && (!(fabsf(m) >= B) || !exin);
            if (in) atomicOr(&wwords[q], 1u << lane);
            const uint32_t u = __ballot_sync(0xffffffffu, unc);
            if (u) {
                unsigned int at = 0;
                if (lane == 0) at = atomicAdd(s_queued, (unsigned int)__popc(u));
                at = __shfl_sync(0xffffffffu, at, 0);
                if (unc) myqueue[at + __popc(u & lt)] = (uint32_t)(wfirst + r);
            }
        }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < PPL; ++q) w_in[q] |= wwords[q];
        __syncwarp();  // the words are rewritten by the next slice
    }
    // the slice's mask words: PPL consecutive words
    uint32_t *mw = mask + (wfirst >> 5);
    if (!TAIL && vec_store && (PPL % 4) == 0) {
        if (lane == 0) {
#pragma unroll
            for (int q = 0; q < PPL; q += 4)
                *(uint4 *)(mw + q) = make_uint4(w_in[q], w_in[q + 1], w_in[q + 2], w_in[q + 3]);
        }
    } else {
        const int nw = (nvalid + 31) >> 5;
        uint32_t myword = 0;
#pragma unroll
        for (int q = 0; q < PPL; ++q)
            if (lane == q) myword = w_in[q];
        if (lane < nw) mw[lane] = myword;
    }
}

// The comparators' slice (float32 points, absolute coordinates as in the
// listings): v_k = LHS_k - RHS_k = t_k - x w_kx - y w_ky per edge.  Sign of
// offset: inside when every D_k = (v_k < 0) is the same, i.e. min v >= 0 or
// max v < 0 (NaN padding ignored by the plain min / max; a NaN point is
// outside).  Ray crossing: edge k crosses the +x ray when its ends straddle y
// (y_{k-1} > y differs from y_k > y) and the signed v_k > 0; an odd count is
// inside.  NE > 0: coefficients from the launch parameters, else from shared
// memory (ray: (w_x, w_y, t, 0) and (y0, y1, 0, 0) per edge).
// Like consume_slice, the stage is handed back once the points are in registers.
template <int OP, int NE, int PPL, bool TAIL>
__device__ __forceinline__ void consume_slice_cmp(const SliceCtx &cx, const unsigned char *stage,
                                                  const void *__restrict__ pts, int64_t M, int64_t wfirst, int lane,
                                                  uint32_t *__restrict__ mask, bool vec_store, uint64_t *release)
{
    const int nvalid = TAIL ? (int)max((int64_t)0, min((int64_t)32 * PPL, M - wfirst)) : 32 * PPL;
    const StreamPoly &sp = *cx.sp;
    float xs[PPL], ys[PPL];
#pragma unroll
    for (int q = 0; q < PPL; ++q) {
        const int r = 32 * q + lane;
        float x = 0.f, y = 0.f;
        if (!TAIL || r < nvalid) {
            if (TAIL && wfirst + r == M - 1 && (M & 1)) {
                x = ((const float *)pts)[2 * (M - 1)];
                y = ((const float *)pts)[2 * (M - 1) + 1];
            } else {
                const float2 v = ((const float2 *)stage)[r];
                x = v.x;
                y = v.y;
            }
        }
        xs[q] = x;
        ys[q] = y;
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(release);
    bool in[PPL];
    if (OP == kTmaSign) {
        float mn[PPL], mx[PPL];
#pragma unroll
        for (int q = 0; q < PPL; ++q) {
            mn[q] = __int_as_float(0x7fc00000);
            mx[q] = __int_as_float(0x7fc00000);
        }
        if (NE > 0) {
#pragma unroll
            for (int k = 0; k < (NE > 0 ? NE : 2); k += 2) {
#pragma unroll
                for (int q = 0; q < PPL; ++q) {
                    const float v0 = fmaf(-xs[q], sp.wx[k], fmaf(-ys[q], sp.wy[k], sp.t[k]));
                    const float v1 = fmaf(-xs[q], sp.wx[k + 1], fmaf(-ys[q], sp.wy[k + 1], sp.t[k + 1]));
                    mn[q] = fmin3(mn[q], v0, v1);
                    mx[q] = fmax3(mx[q], v0, v1);
                }
            }
        } else {
            for (int k = 0; k < cx.npad; ++k) {
                const float4 c = cx.cs[k];
#pragma unroll
                for (int q = 0; q < PPL; ++q) {
                    const float v = fmaf(-xs[q], c.x, fmaf(-ys[q], c.y, c.z));
                    mn[q] = fminf(mn[q], v);
                    mx[q] = fmaxf(mx[q], v);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < PPL; ++q) in[q] = mn[q] >= 0.f || mx[q] < 0.f;
    } else {
        uint32_t par[PPL];
#pragma unroll
        for (int q = 0; q < PPL; ++q) par[q] = 0u;
        if (NE > 0) {
#pragma unroll
            for (int k = 0; k < (NE > 0 ? NE : 1); ++k) {
#pragma unroll
                for (int q = 0; q < PPL; ++q) {
                    const float v = fmaf(-xs[q], sp.wx[k], fmaf(-ys[q], sp.wy[k], sp.t[k]));
                    const bool straddle = (sp.y1[k] > ys[q]) != (sp.y0[k] > ys[q]);
                    par[q] ^= (uint32_t)(straddle && v > 0.f);
                }
            }
        } else {
            for (int k = 0; k < cx.npad; ++k) {
                const float4 c = cx.cs[2 * k], e = cx.cs[2 * k + 1];
#pragma unroll
                for (int q = 0; q < PPL; ++q) {
                    const float v = fmaf(-xs[q], c.x, fmaf(-ys[q], c.y, c.z));
                    const bool straddle = (e.y > ys[q]) != (e.x > ys[q]);
                    par[q] ^= (uint32_t)(straddle && v > 0.f);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < PPL; ++q) in[q] = par[q] != 0u;
    }
    uint32_t w_in[PPL];
#pragma unroll
    for (int q = 0; q < PPL; ++q) w_in[q] = __ballot_sync(0xffffffffu, in[q] && (!TAIL || 32 * q + lane < nvalid));
    uint32_t *mw = mask + (wfirst >> 5);
    if (!TAIL && vec_store && (PPL % 4) == 0) {
        if (lane == 0) {
#pragma unroll
            for (int q = 0; q < PPL; q += 4)
                *(uint4 *)(mw + q) = make_uint4(w_in[q], w_in[q + 1], w_in[q + 2], w_in[q + 3]);
        }
    } else {
        const int nw = (nvalid + 31) >> 5;
        uint32_t myword = 0;
#pragma unroll
        for (int q = 0; q < PPL; ++q)
            if (lane == q) myword = w_in[q];
        if (lane < nw) mw[lane] = myword;
    }
}

// NE > 0: the polygon has at most NE edges and the coefficients live in
// registers; NE == 0: any edge count, coefficients read from shared memory.
// OP: the Voronoi test (with its exact refine) or a comparator (no refine;
// `coef` is then the polygon's comparator row, padded with NaN).
// DISC: the disc filter of consume_slice_disc (the Voronoi test only).
// CW: consumer warps of the CTA.
template <int NE, int PPL, int STAGES, bool INT, int OP = kTmaVoronoi, bool EARLY = false, bool DISC = false,
          int CW = kConsumerWarps>
__global__ void __launch_bounds__(StreamCfg<PPL, STAGES, DISC, CW>::kThreads,
                                  StreamCfg<PPL, STAGES, DISC, CW>::kMinBlocks) stream_tma_kernel(
    const __grid_constant__ StreamPoly sp, const PolyInfo *__restrict__ poly, const float4 *__restrict__ coef,
    const double2 *__restrict__ g0tab, const double2 *__restrict__ gktab,
    const void *__restrict__ verts, int vdtype, const void *__restrict__ pts, int64_t M,
    uint32_t *__restrict__ mask, uint32_t *__restrict__ queue, StreamCounters *__restrict__ ctr,
    unsigned int *__restrict__ last_refine, int *__restrict__ err)
{
    using C = StreamCfg<PPL, STAGES, DISC, CW>;
    constexpr int kTile = C::kTile;
    extern __shared__ __align__(128) unsigned char smem[];
    float4 *cs = (float4 *)(smem + C::kCoefOff);
    uint64_t *full = (uint64_t *)(smem + C::kBarOff);
    uint64_t *empty = full + STAGES;
    __shared__ unsigned int s_refined;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n = sp.ok ? sp.n : 1;
    const int npad = (n + 3) & ~3;
    if (NE == 0 && OP != kTmaVoronoi) {
        // comparator rows (already padded with NaN past n; ray: two per edge)
        const int rows = (OP == kTmaRay ? 2 : 1) * npad;
        for (int k = tid; k < rows; k += blockDim.x) cs[k] = coef[k];  // an invalid polygon: all NaN
    } else if (NE == 0) {
        // more edges than the parameter block holds: stage them in shared memory
        const PolyInfo pi = poly[0];
        for (int k = tid; k < npad; k += blockDim.x) {
            float4 c;
            if (!sp.ok) c = k == 0 ? make_float4(0.f, 0.f, -INFINITY, 0.f) : make_float4(0.f, 0.f, INFINITY, 0.f);
            else c = k < n ? coef[pi.voff + k] : make_float4(0.f, 0.f, INFINITY, 0.f);
            cs[k] = c;
        }
    }
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], CW);
        }
        s_refined = 0;
        fence_mbar_init();
    }
    __syncthreads();

    const int64_t ntiles = (M + kTile - 1) / kTile;
    const int64_t mine = ntiles > (int64_t)blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    // this CTA's slice of the scratch queue: room for every point it owns
    const int64_t per_cta = ((ntiles + gridDim.x - 1) / gridDim.x) * kTile;
    uint32_t *myqueue = queue + (int64_t)blockIdx.x * per_cta;

    if (warp == CW) {
        // ---------------- producer: one elected lane issues the bulk copies
        if (lane == 0) {
            const int nmine = (int)mine;
            int it = 0, s = 0;
            uint32_t ephase = 0;  // parity of the empty-barrier phase to wait for
            int64_t first = (int64_t)blockIdx.x * kTile;
            const int64_t step = (int64_t)gridDim.x * kTile;
            for (; it < nmine; ++it) {
                if (it >= STAGES && !mbar_wait(&empty[s], ephase, err)) break;
                const int64_t cnt = min((int64_t)kTile, M - first);
                const uint32_t bytes = (uint32_t)(cnt * 8) & ~15u;  // an odd last point is read directly
                if (bytes) {
                    mbar_arrive_expect_tx(&full[s], bytes);
                    bulk_copy_g2s(smem + (size_t)s * C::kStageBytes, (const char *)pts + first * 8, bytes, &full[s]);
                } else {
                    mbar_arrive(&full[s]);
                }
                first += step;
                if (++s == STAGES) {
                    s = 0;
                    if (it + 1 >= 2 * STAGES) ephase ^= 1u;  // round r >= 1 waits for parity (r - 1) & 1
                }
            }
            if (it < nmine) {
                // gave up: let the copies already issued land before the CTA leaves
                for (int k = it > STAGES ? it - STAGES : 0; k < it; ++k)
                    mbar_wait(&full[k % STAGES], (uint32_t)((k / STAGES) & 1), err);
            }
        }
    } else {
        // ---------------- consumers
        // o = (0, 0) when prepare chose the origin itself: no centring needed
        const bool center = !(sp.ox == 0.f && sp.oy == 0.f);
        const bool vec_store = ((uintptr_t)mask & 15) == 0;
        SliceCtx cx{&sp, cs, npad};
        const int nmine = (int)mine;
        int s = 0;
        uint32_t fphase = 0;
        int64_t wfirst = (int64_t)blockIdx.x * kTile + warp * 32 * PPL;
        const int64_t step = (int64_t)gridDim.x * kTile;
        // slices that end before the last point (or at an even end) need no bounds logic
        const int64_t whole_end = (M & 1) ? M - 1 : M;
        for (int it = 0; it < nmine; ++it, wfirst += step) {
            if (!mbar_wait(&full[s], fphase, err)) break;
            const unsigned char *stage = smem + (size_t)s * C::kStageBytes + (size_t)warp * 32 * PPL * 8;
            const bool whole = wfirst + 32 * PPL <= whole_end;
            if (DISC && OP == kTmaVoronoi) {
                uint32_t *wwords = (uint32_t *)(smem + C::kDiscOff + (size_t)warp * C::kDiscWarpBytes);
                if (whole) {
                    if (center)
                        consume_slice_disc<NE, PPL, INT, true, false>(cx, stage, pts, M, wfirst, lane, mask,
                                                                     vec_store, myqueue, &s_refined, wwords);
                    else
                        consume_slice_disc<NE, PPL, INT, false, false>(cx, stage, pts, M, wfirst, lane, mask,
                                                                      vec_store, myqueue, &s_refined, wwords);
                } else {
                    consume_slice_disc<NE, PPL, INT, true, true>(cx, stage, pts, M, wfirst, lane, mask, vec_store,
                                                                myqueue, &s_refined, wwords);
                }
                // the near pass reads the stage again: hand it back afterwards
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[s]);
            } else if (OP != kTmaVoronoi) {
                // these hand the stage back themselves, once the points are in registers
                if (whole)
                    consume_slice_cmp<OP, NE, PPL, false>(cx, stage, pts, M, wfirst, lane, mask, vec_store,
                                                          &empty[s]);
                else
                    consume_slice_cmp<OP, NE, PPL, true>(cx, stage, pts, M, wfirst, lane, mask, vec_store,
                                                         &empty[s]);
            } else if (whole) {
                if (center)
                    consume_slice<NE, PPL, INT, true, false, EARLY>(cx, stage, pts, M, wfirst, lane, mask,
                                                                   vec_store, myqueue, &s_refined, &empty[s]);
                else
                    consume_slice<NE, PPL, INT, false, false, EARLY>(cx, stage, pts, M, wfirst, lane, mask,
                                                                    vec_store, myqueue, &s_refined, &empty[s]);
            } else {
                consume_slice<NE, PPL, INT, true, true, EARLY>(cx, stage, pts, M, wfirst, lane, mask,
                                                              vec_store, myqueue, &s_refined, &empty[s]);
            }
            if (++s == STAGES) {
                s = 0;
                fphase ^= 1u;
            }
        }
    }
    __syncthreads();
    if (OP != kTmaVoronoi) return;  // the comparators decide in float32, as the listings do
    // exact decision of this CTA's queued points, one warp per point (every
    // warp of the CTA, the producer's included); their mask words were
    // written above with the bit clear
    const unsigned int nq = s_refined;
    for (unsigned int i = warp; i < nq; i += CW + 1) {
        const int64_t p = myqueue[i];
        if (warp_inside_exact(poly, 0, g0tab, gktab, verts, vdtype, pts, INT ? PIP_I32 : PIP_F32, p) &&
            lane == 0)
            atomicOr(&mask[p >> 5], 1u << (p & 31));
    }
    if (tid == 0) {
        if (s_refined) atomicAdd(&ctr->refine, s_refined);
        __threadfence();
        const unsigned int t = atomicAdd(&ctr->ticket, 1u);
        if (t == gridDim.x - 1) {
            *last_refine = atomicExch(&ctr->refine, 0u);
            atomicExch(&ctr->ticket, 0u);
        }
    }
}

}  // namespace
