// pip_stream_tma.cuh -- the pipelined single-polygon test (the benchmark's
// hot path) and the warp-cooperative exact re-decision it calls inline.
//
// Persistent CTAs: one producer warp streams tiles of points from HBM into a
// ring of shared-memory stages with 1-D bulk copies (cp.async.bulk), each
// stage guarded by a "full" mbarrier (transaction bytes) and an "empty"
// mbarrier (one arrive per consumer warp).  Consumer warps evaluate the
// expanded Eq. 11 for two points at once with packed f32x2 FMAs, take the
// "for all k" of Alg. 5 as a 3-input NaN-propagating min, and turn 32
// decisions into one mask word with a ballot.  The few points whose float32
// result lies within the error bound are decided exactly right there by the
// whole warp (one lane per edge), so one launch does the whole test.
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

constexpr int kConsumerWarps = 8;
constexpr int kStreamThreads = (kConsumerWarps + 1) * 32;

template <int PPL, int STAGES>
struct StreamCfg {
    static constexpr int kTile = kConsumerWarps * 32 * PPL;  // points per stage
    static constexpr size_t kStageBytes = (size_t)kTile * 8;
    static constexpr size_t kCoefOff = STAGES * kStageBytes;
    static constexpr int kCab = kMaxEdges + 2;       // float4 (-wx, -wx, -wy, -wy) per edge
    static constexpr int kCtt = (kMaxEdges + 2) / 2; // float4 (t_k, t_k, t_k+1, t_k+1) per edge pair
    static constexpr size_t kBarOff = kCoefOff + (size_t)(kCab + kCtt) * 16;
    static constexpr size_t kSmem = kBarOff + 2 * STAGES * sizeof(uint64_t);
    // CTAs that fit one SM's 228 KB of shared memory (at most 3)
    static constexpr int kFit = (int)((227 * 1024) / (kSmem + 1024));
    static constexpr int kMinBlocks = kFit < 1 ? 1 : (kFit > 3 ? 3 : kFit);
};

template <int PPL, int STAGES, bool INT>
__global__ void __launch_bounds__(kStreamThreads, StreamCfg<PPL, STAGES>::kMinBlocks) stream_tma_kernel(
    const PolyInfo *__restrict__ poly, const float4 *__restrict__ coef,
    const double2 *__restrict__ g0tab, const double2 *__restrict__ gktab,
    const void *__restrict__ verts, int vdtype, const void *__restrict__ pts, int64_t M,
    uint32_t *__restrict__ mask, StreamCounters *__restrict__ ctr, unsigned int *__restrict__ last_refine,
    int *__restrict__ err)
{
    using C = StreamCfg<PPL, STAGES>;
    constexpr int kTile = C::kTile;
    extern __shared__ __align__(128) unsigned char smem[];
    float4 *cab = (float4 *)(smem + C::kCoefOff);
    float4 *ctt = cab + C::kCab;
    uint64_t *full = (uint64_t *)(smem + C::kBarOff);
    uint64_t *empty = full + STAGES;
    __shared__ unsigned int s_refined;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const PolyInfo pi = poly[0];
    const bool ok = pi.status == PIP_OK;
    const int n = ok ? pi.n : 1;
    const int npad = (n + 1) & ~1;
    for (int k = tid; k < npad; k += blockDim.x) {
        float4 c;
        if (!ok) c = k == 0 ? make_float4(0.f, 0.f, -INFINITY, 0.f) : make_float4(0.f, 0.f, INFINITY, 0.f);
        else c = k < n ? coef[pi.voff + k] : make_float4(0.f, 0.f, INFINITY, 0.f);
        cab[k] = make_float4(-c.x, -c.x, -c.y, -c.y);
        float *tt = (float *)ctt;
        tt[2 * k] = c.z;
        tt[2 * k + 1] = c.z;
    }
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kConsumerWarps);
        }
        s_refined = 0;
        fence_mbar_init();
    }
    __syncthreads();

    const int64_t ntiles = (M + kTile - 1) / kTile;
    const int64_t mine = ntiles > (int64_t)blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

    if (warp == kConsumerWarps) {
        // ---------------- producer: one elected lane issues the bulk copies
        if (lane == 0) {
            int64_t it = 0;
            for (; it < mine; ++it) {
                const int s = (int)(it % STAGES);
                if (it >= STAGES && !mbar_wait(&empty[s], (uint32_t)((it / STAGES - 1) & 1), err)) break;
                const int64_t first = ((int64_t)blockIdx.x + it * gridDim.x) * kTile;
                const int64_t cnt = min((int64_t)kTile, M - first);
                const uint32_t bytes = (uint32_t)(cnt * 8) & ~15u;  // an odd last point is read directly
                if (bytes) {
                    mbar_arrive_expect_tx(&full[s], bytes);
                    bulk_copy_g2s(smem + (size_t)s * C::kStageBytes, (const char *)pts + first * 8, bytes, &full[s]);
                } else {
                    mbar_arrive(&full[s]);
                }
            }
            if (it < mine) {
                // gave up: let the copies already issued land before the CTA leaves
                for (int64_t k = it > STAGES ? it - STAGES : 0; k < it; ++k)
                    mbar_wait(&full[k % STAGES], (uint32_t)((k / STAGES) & 1), err);
            }
        }
    } else {
        // ---------------- consumers
        const float ox = pi.ox, oy = pi.oy;
        const f2x NOX = pk(-ox, -ox), NOY = pk(-oy, -oy);
        const f2x B0P = pk(pi.beta0, pi.beta0), B1P = pk(pi.beta1, pi.beta1);
        const int64_t nwords = (M + 31) >> 5;
        unsigned int refined = 0;
        for (int64_t it = 0; it < mine; ++it) {
            const int s = (int)(it % STAGES);
            if (!mbar_wait(&full[s], (uint32_t)((it / STAGES) & 1), err)) break;
            const int64_t first = ((int64_t)blockIdx.x + it * gridDim.x) * kTile;
            const int64_t wfirst = first + warp * 32 * PPL;
            const bool tail = first + kTile > M;
            const unsigned char *stage = smem + (size_t)s * C::kStageBytes + (size_t)warp * 32 * PPL * 8;
            float px[PPL], py[PPL];
#pragma unroll
            for (int q = 0; q < PPL; ++q) {
                const int64_t p = wfirst + 32 * q + lane;
                float x = 0.f, y = 0.f;
                if (!tail || p < M) {
                    if (tail && p == M - 1 && (M & 1)) {
                        // the odd last point is not in the bulk copy
                        if (INT) {
                            x = (float)((const int32_t *)pts)[2 * p];
                            y = (float)((const int32_t *)pts)[2 * p + 1];
                        } else {
                            x = ((const float *)pts)[2 * p];
                            y = ((const float *)pts)[2 * p + 1];
                        }
                    } else if (INT) {
                        const int2 v = ((const int2 *)stage)[32 * q + lane];
                        x = (float)v.x;
                        y = (float)v.y;
                    } else {
                        const float2 v = ((const float2 *)stage)[32 * q + lane];
                        x = v.x;
                        y = v.y;
                    }
                }
                px[q] = x;
                py[q] = y;
            }
            f2x X[PPL / 2], Y[PPL / 2];
            float m[PPL];
#pragma unroll
            for (int i = 0; i < PPL / 2; ++i) {
                X[i] = fadd2(pk(px[2 * i], px[2 * i + 1]), NOX);  // x - o, rounded as in fl(x - o)
                Y[i] = fadd2(pk(py[2 * i], py[2 * i + 1]), NOY);
                m[2 * i] = INFINITY;
                m[2 * i + 1] = INFINITY;
            }
            for (int e = 0; e < npad; e += 2) {
                const float4 a0 = cab[e], a1 = cab[e + 1], tt = ctt[e >> 1];
                const f2x A0 = pk(a0.x, a0.y), Bw0 = pk(a0.z, a0.w);
                const f2x A1 = pk(a1.x, a1.y), Bw1 = pk(a1.z, a1.w);
                const f2x T0 = pk(tt.x, tt.y), T1 = pk(tt.z, tt.w);
#pragma unroll
                for (int i = 0; i < PPL / 2; ++i) {
                    // s_k = t_k - x w_kx - y w_ky for the two points of the pair
                    const f2x s0 = ffma2(X[i], A0, ffma2(Y[i], Bw0, T0));
                    const f2x s1 = ffma2(X[i], A1, ffma2(Y[i], Bw1, T1));
                    float s0l, s0h, s1l, s1h;
                    upk(s0, s0l, s0h);
                    upk(s1, s1l, s1h);
                    m[2 * i] = fmin3_nan(m[2 * i], s0l, s1l);
                    m[2 * i + 1] = fmin3_nan(m[2 * i + 1], s0h, s1h);
                }
            }
            // decisions: one ballot per 32 points for "inside", one for "uncertain"
            uint32_t w_in[PPL], w_unc[PPL];
            uint32_t any_unc = 0;
#pragma unroll
            for (int i = 0; i < PPL / 2; ++i) {
                float x0, x1, y0, y1;
                upk(X[i], x0, x1);
                upk(Y[i], y0, y1);
                const f2x N = pk(fmaxf(fabsf(x0), fabsf(y0)), fmaxf(fabsf(x1), fabsf(y1)));
                float B[2];
                upk(ffma2(N, B1P, B0P), B[0], B[1]);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int q = 2 * i + h;
                    const bool valid = !tail || wfirst + 32 * q + lane < M;
                    bool in = m[q] >= B[h];
                    bool unc = !(fabsf(m[q]) >= B[h]);
                    if (INT && !int_exact(px[q], py[q])) { in = false; unc = true; }
                    w_in[q] = __ballot_sync(0xffffffffu, in && valid);
                    w_unc[q] = __ballot_sync(0xffffffffu, unc && valid);
                    any_unc |= w_unc[q];
                }
            }
            if (any_unc) {
                // rare: the whole warp decides each uncertain point exactly
#pragma unroll
                for (int q = 0; q < PPL; ++q) {
                    uint32_t u = w_unc[q];
                    while (u) {
                        const int l = __ffs(u) - 1;
                        u &= u - 1;
                        if (warp_inside_exact(poly, 0, g0tab, gktab, verts, vdtype, pts,
                                              INT ? PIP_I32 : PIP_F32, wfirst + 32 * q + l))
                            w_in[q] |= 1u << l;
                        ++refined;
                    }
                }
            }
            uint32_t myword = 0;
#pragma unroll
            for (int q = 0; q < PPL; ++q)
                if (lane == q) myword = w_in[q];
            if (lane < PPL && (wfirst >> 5) + lane < nwords) mask[(wfirst >> 5) + lane] = myword;
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
        }
        if (lane == 0 && refined) atomicAdd(&s_refined, refined);
    }
    __syncthreads();
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
