// pip_margin_tma.cuh -- the signed margin of one polygon's points (Eq. 2
// bisector distance, normalised coefficients) in the pipelined layout of the
// single-polygon test: persistent CTAs, one producer warp bulk-copying
// (cp.async.bulk) 32 KB tiles of points into a ring of shared-memory stages
// guarded by full / empty mbarriers, eight consumer warps taking one slice of
// a stage each and writing one float per point.  The coefficients sit in
// shared memory (one broadcast load per edge for 16 points a lane), so one
// instantiation serves every edge count.  The same float32 terms as the
// register-streaming margin kernel, and an exact min: the results are
// identical.
#pragma once

#include "pip_kernels.cuh"
#include "pip_tma.cuh"

namespace {

using namespace pip;

constexpr int kMarginWarps = 8;
constexpr int kMarginThreads = (kMarginWarps + 1) * 32;

template <int PPL, int STAGES>
struct MarginCfg {
    static constexpr int kTile = kMarginWarps * 32 * PPL;  // points per stage
    static constexpr size_t kStageBytes = (size_t)kTile * 8;
    static constexpr size_t kCoefOff = STAGES * kStageBytes;
    static constexpr size_t kBarOff = kCoefOff + (size_t)(kMaxEdges + 4) * 16;
    static constexpr size_t kSmem = kBarOff + 2 * STAGES * sizeof(uint64_t);
};

// One consumer warp, one slice of 32 * PPL points starting at wfirst; the
// stage holds the points the bulk copy moved.  TAIL: the slice may run past
// M, or hold an odd last point of the set (not in the copy, read from global
// memory).  The min takes three operands at a time; min is exact, so the
// result equals the two-operand chain of the register-streaming kernel.
template <int PPL, bool INT, bool TAIL>
__device__ __forceinline__ void margin_slice(const float4 *cs, int npad, float ox, float oy,
                                             const unsigned char *stage, const void *__restrict__ pts,
                                             int64_t M, int64_t wfirst, int lane, float *__restrict__ out)
{
    const int nvalid = TAIL ? (int)max((int64_t)0, min((int64_t)32 * PPL, M - wfirst)) : 32 * PPL;
    float x[PPL], y[PPL], m[PPL];
    bool fin[PPL];
#pragma unroll
    for (int q = 0; q < PPL; ++q) {
        const int r = 32 * q + lane;
        float px = 0.f, py = 0.f;
        if (!TAIL || r < nvalid) {
            if (TAIL && wfirst + r == M - 1 && (M & 1)) {
                if (INT) {
                    px = (float)((const int32_t *)pts)[2 * (M - 1)];
                    py = (float)((const int32_t *)pts)[2 * (M - 1) + 1];
                } else {
                    px = ((const float *)pts)[2 * (M - 1)];
                    py = ((const float *)pts)[2 * (M - 1) + 1];
                }
            } else if (INT) {
                const int2 v = ((const int2 *)stage)[r];
                px = (float)v.x;
                py = (float)v.y;
            } else {
                const float2 v = ((const float2 *)stage)[r];
                px = v.x;
                py = v.y;
            }
        }
        fin[q] = isfinite(px) && isfinite(py);
        x[q] = px - ox;
        y[q] = py - oy;
        m[q] = INFINITY;
    }
    for (int k = 0; k < npad; k += 4) {
        const float4 c0 = cs[k], c1 = cs[k + 1], c2 = cs[k + 2], c3 = cs[k + 3];
#pragma unroll
        for (int q = 0; q < PPL; ++q) {
            const float s0 = fmaf(-x[q], c0.x, fmaf(-y[q], c0.y, c0.z));
            const float s1 = fmaf(-x[q], c1.x, fmaf(-y[q], c1.y, c1.z));
            const float s2 = fmaf(-x[q], c2.x, fmaf(-y[q], c2.y, c2.z));
            const float s3 = fmaf(-x[q], c3.x, fmaf(-y[q], c3.y, c3.z));
            m[q] = fmin3(fmin3(m[q], s0, s1), s2, s3);
        }
    }
#pragma unroll
    for (int q = 0; q < PPL; ++q) {
        const int r = 32 * q + lane;
        if (!TAIL || r < nvalid) out[wfirst + r] = fin[q] ? -m[q] : INFINITY;
    }
}

template <int PPL, int STAGES, bool INT>
__global__ void __launch_bounds__(kMarginThreads, 2) margin_tma_kernel(const PolyInfo *__restrict__ poly,
                                                                      const float4 *__restrict__ coefn,
                                                                      const void *__restrict__ pts, int64_t M,
                                                                      float *__restrict__ out, int *__restrict__ err)
{
    using C = MarginCfg<PPL, STAGES>;
    constexpr int kTile = C::kTile;
    extern __shared__ __align__(128) unsigned char smem[];
    float4 *cs = (float4 *)(smem + C::kCoefOff);
    uint64_t *full = (uint64_t *)(smem + C::kBarOff);
    uint64_t *empty = full + STAGES;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const PolyInfo pi = poly[0];
    const int npad = stage_polygon(pi, coefn, cs, tid, blockDim.x);
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kMarginWarps);
        }
        fence_mbar_init();
    }
    __syncthreads();

    const int64_t ntiles = (M + kTile - 1) / kTile;
    const int64_t mine = ntiles > (int64_t)blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int64_t step = (int64_t)gridDim.x * kTile;
    if (warp == kMarginWarps) {
        // producer: one lane issues the bulk copies, STAGES tiles ahead
        if (lane == 0) {
            int64_t it = 0;
            int s = 0;
            uint32_t ephase = 0;
            int64_t first = (int64_t)blockIdx.x * kTile;
            for (; it < mine; ++it) {
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
            if (it < mine) {
                // gave up: let the copies already issued land before the CTA leaves
                for (int64_t k = it > STAGES ? it - STAGES : 0; k < it; ++k)
                    mbar_wait(&full[k % STAGES], (uint32_t)((k / STAGES) & 1), err);
            }
        }
    } else {
        int s = 0;
        uint32_t fphase = 0;
        int64_t wfirst = (int64_t)blockIdx.x * kTile + warp * 32 * PPL;
        // slices that end before the last point (or at an even end) need no bounds logic
        const int64_t whole_end = (M & 1) ? M - 1 : M;
        for (int64_t it = 0; it < mine; ++it, wfirst += step) {
            if (!mbar_wait(&full[s], fphase, err)) break;
            const unsigned char *stage = smem + (size_t)s * C::kStageBytes + (size_t)warp * 32 * PPL * 8;
            if (wfirst + 32 * PPL <= whole_end)
                margin_slice<PPL, INT, false>(cs, npad, pi.ox, pi.oy, stage, pts, M, wfirst, lane, out);
            else
                margin_slice<PPL, INT, true>(cs, npad, pi.ox, pi.oy, stage, pts, M, wfirst, lane, out);
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
            if (++s == STAGES) {
                s = 0;
                fphase ^= 1u;
            }
        }
    }
}

constexpr int kMarginPPL = 16, kMarginStages = 3;

// Raises the kernel's dynamic shared-memory limit (once, from pip_prepare,
// outside any stream capture).
template <bool INT>
cudaError_t setup_margin_tma()
{
    using C = MarginCfg<kMarginPPL, kMarginStages>;
    return cudaFuncSetAttribute(margin_tma_kernel<kMarginPPL, kMarginStages, INT>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::kSmem);
}

// Launches the pipelined margin over M points of the tables' one polygon
// (16-byte aligned points).
template <bool INT>
cudaError_t launch_margin_tma(const pip_tables *t, const void *pts, int64_t M, float *out, cudaStream_t s)
{
    constexpr int kPPL = kMarginPPL, kStages = kMarginStages;
    using C = MarginCfg<kPPL, kStages>;
    auto k = margin_tma_kernel<kPPL, kStages, INT>;
    const int64_t tiles = (M + C::kTile - 1) / C::kTile;
    const int blocks = (int)max((int64_t)1, min((int64_t)2 * t->num_sms, tiles));
    k<<<blocks, kMarginThreads, C::kSmem, s>>>(t->d_poly, t->d_coefn, pts, M, out, t->d_error);
    return cudaGetLastError();
}

}  // namespace
