// pip_test.cu -- the Voronoi inclusion test (Alg. 5 with the squared-distance
// form of Eq. 10-11) on the GPU, bit-exact through a float32 filter and an
// exact refine step.
//
// Bulk kernels (float32):  per point, x = p - o and
//     s_k = fma(-x, w_kx, fma(-y, w_ky, t_k)),   m = min_k s_k,
//     inside   if m >= B(p) (and m finite),
//     outside  if m <  -B(p),
//     else     queued for refine,        B(p) = beta0 + beta1 * max(|x|, |y|).
// B bounds |computed s_k - exact s_k| for every k, so a decided point agrees
// with exact closed-polygon membership (Eq. 1).  The min over edges is the
// "for all j" of Alg. 5; 32 decisions become one mask word by warp ballot.
//
// Refine kernel: each queued point is re-decided from the fp64 generator table
// (Alg. 5 in fp64 with its own bound) and, where that is still within its
// bound, exactly: int64 cross products for integer inputs, floating-point
// expansions otherwise.
#include <float.h>
#include <math.h>

#include "pip_kernels.cuh"

using namespace pip;

#include "pip_test_kernels.cuh"
#include "pip_ragged_tma.cuh"

namespace {

template <bool INT, bool V16>
cudaError_t launch_stream(const pip_tables *t, const void *pts, int64_t M, uint32_t *mask,
                          cudaStream_t s)
{
    auto k = stream_kernel<kF, INT, V16>;
    const int64_t chunks = (M + Chunk<kF>::kPoints - 1) / Chunk<kF>::kPoints;
    const int64_t want = (chunks + kWarps - 1) / kWarps;
    const int blocks = (int)max((int64_t)1, min((int64_t)blocks_for(k, t->num_sms, kThreads), want));
    k<<<blocks, kThreads, 0, s>>>(t->d_poly, t->d_coef, pts, M, mask, t->d_queue, t->d_qcount);
    return cudaGetLastError();
}

template <bool INT, bool V16>
cudaError_t launch_ragged(const pip_tables *t, const void *pts, int64_t M, const int64_t *poffs,
                          uint32_t *mask, cudaStream_t s)
{
    ragged_setup_kernel<kF><<<1, 1024, 0, s>>>(poffs, t->P, M, kItemChunks, t->d_items, t->d_work,
                                               t->d_qcount, t->d_worst);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    auto k = ragged_kernel<kF, INT, V16>;
    k<<<blocks_for(k, t->num_sms, kThreads), kThreads, 0, s>>>(t->d_poly, t->d_coef, pts, M, poffs, t->P,
                                                     t->d_items, kItemChunks, t->d_work, mask,
                                                     t->d_queue, t->d_qcount);
    return cudaGetLastError();
}

// The pipelined own-polygon batch: setup (items, shared mask words, counters)
// then the persistent kernel.  Variants: (points per lane, ring stages); the
// item tile is 7 consumer warps x 32 lanes x points per lane.
// Variants of the pipelined batch kernel: (points per lane, ring stages,
// polygons per stage).
struct BatchVariant {
    int ppl, stages, pack;
};
constexpr BatchVariant kBatchVariants[] = {{16, 3, 1}, {16, 3, 2}, {16, 3, 4}, {16, 2, 2}, {12, 3, 2}, {12, 4, 2}};
constexpr int kNumBatchVariants = sizeof(kBatchVariants) / sizeof(kBatchVariants[0]);

template <int PPL, int STAGES, bool INT, bool EXACT, int OP = kRagVoronoi, bool EARLY = false, int K = 1,
          bool DISC = false>
cudaError_t launch_ragged_tma_one(const pip_tables *t, const void *pts, int64_t M, const int64_t *poffs,
                                  uint32_t *mask, cudaStream_t s)
{
    using C = RaggedCfg<PPL, STAGES, K, OP == kRagRay ? 2 : 1, DISC>;
    auto k = ragged_tma_kernel<PPL, STAGES, INT, EXACT, OP, EARLY, K, DISC>;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kRaggedThreads, C::kSmem) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    if (per_sm > 2) per_sm = 2;
    // the exact path stages the float32 integer edge rows in the coefficient
    // rows' place, a comparator its own rows
    const float4 *rows = OP == kRagSign ? t->d_cmp_sign
                         : OP == kRagRay ? t->d_cmp_ray
                         : OP == kRagFp64 ? (const float4 *)t->d_cmp_g64
                         : EXACT ? t->d_fpad : t->d_coefp;
    k<<<per_sm * t->num_sms, kRaggedThreads, C::kSmem, s>>>(t->d_poly, rows, t->d_ipad, pts, M, poffs, t->P,
                                                            (BatchCounters *)t->d_batch_ctr, mask, t->d_queue,
                                                            t->d_keys, t->d_qcount, t->d_worst, t->d_error);
    return cudaGetLastError();
}

// DISC: the disc-filter form of the chosen tile shape (float polygons).
template <bool INT, bool EXACT, bool DISC = false>
cudaError_t launch_ragged_tma(const pip_tables *t, const void *pts, int64_t M, const int64_t *poffs,
                              uint32_t *mask, cudaStream_t s)
{
    constexpr int V = kRagVoronoi;
    switch (t->batch_variant) {
    case 1: return launch_ragged_tma_one<16, 3, INT, EXACT, V, false, 2, DISC>(t, pts, M, poffs, mask, s);
    case 2: return launch_ragged_tma_one<16, 3, INT, EXACT, V, false, 4, DISC>(t, pts, M, poffs, mask, s);
    case 3: return launch_ragged_tma_one<16, 2, INT, EXACT, V, false, 2, DISC>(t, pts, M, poffs, mask, s);
    case 4: return launch_ragged_tma_one<12, 3, INT, EXACT, V, false, 2, DISC>(t, pts, M, poffs, mask, s);
    case 5: return launch_ragged_tma_one<12, 4, INT, EXACT, V, false, 2, DISC>(t, pts, M, poffs, mask, s);
    default: return launch_ragged_tma_one<16, 3, INT, EXACT, V, false, 1, DISC>(t, pts, M, poffs, mask, s);
    }
}

template <int PPL, int STAGES, bool INT, bool EXACT, int OP, bool EARLY, int K, bool DISC = false>
cudaError_t set_one_ragged_attr()
{
    return cudaFuncSetAttribute(ragged_tma_kernel<PPL, STAGES, INT, EXACT, OP, EARLY, K, DISC>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)RaggedCfg<PPL, STAGES, K, OP == kRagRay ? 2 : 1, DISC>::kSmem);
}

template <int PPL, int STAGES, int K>
cudaError_t set_ragged_attr()
{
    cudaError_t e = set_one_ragged_attr<PPL, STAGES, false, false, kRagVoronoi, false, K>();
    if (e == cudaSuccess) e = set_one_ragged_attr<PPL, STAGES, true, false, kRagVoronoi, false, K>();
    if (e == cudaSuccess) e = set_one_ragged_attr<PPL, STAGES, true, true, kRagVoronoi, false, K>();
    if (e == cudaSuccess) e = set_one_ragged_attr<PPL, STAGES, false, false, kRagVoronoi, false, K, true>();
    if (e == cudaSuccess) e = set_one_ragged_attr<PPL, STAGES, true, false, kRagVoronoi, false, K, true>();
    return e;
}

template <int OP>
cudaError_t set_ragged_cmp_attr()
{
    return set_one_ragged_attr<16, 3, false, false, OP, false, 2>();
}


// ---------------------------------------------------------------------------
// All pairs, split over point tiles and polygon ranges.  Each thread keeps
// AP_PT points in registers and evaluates every polygon of its block's range
// (full work: no early exit, no cull); the polygons stream through shared
// memory in chunks.  Per point the lowest "candidate" polygon -- decided
// inside, or uncertain -- is kept as the key (j << 1) | uncertain and merged
// over the ranges with atomicMin; a finalize pass turns keys into first-hit
// ids and mask words and queues the points whose lowest candidate is
// uncertain.
// ---------------------------------------------------------------------------
constexpr int kApPT = 12;
constexpr int kApThreads = 256;
constexpr int kApChunk = 32;  // polygons per shared-memory chunk
constexpr int kApSplit = 4;   // polygon ranges per point tile

// Shared memory of the all-pairs kernel: two chunk buffers, each the padded
// coefficient rows and the PolyInfo rows of kApChunk polygons.
constexpr size_t kApRowsBytes = (size_t)kApChunk * kPadStride * sizeof(float4);
constexpr size_t kApInfoBytes = (size_t)kApChunk * sizeof(PolyInfo);
constexpr size_t kApBufBytes = kApRowsBytes + kApInfoBytes;
constexpr size_t kApSmem = 2 * kApBufBytes;

// s_k(x) = t_k - x . w_k for one coefficient row (w_x, w_y, t_k, -), two roundings
__device__ __forceinline__ float ap_s(const float4 &c, float x, float y)
{
    return fmaf(-x, c.x, fmaf(-y, c.y, c.z));
}

// CULL (pip_test's PIP_CULL): a warp skips a polygon when none of its points
// that still lacks a candidate lies in the polygon's vertex bounding box (the
// polygon lies inside that box exactly, and float32 rounding of a point is
// monotone, so a skipped point is outside) and within its outer disc (the
// generator-radius cull: PolyInfo::tout, as in the disc filter); when every
// such point lies inside the polygon's inner disc (PolyInfo::tin), they are
// decided inside without the edges.  A CTA stops once every one of its points
// has a candidate in its range (a later polygon cannot lower it).  Same first
// hits for every point whose first hit lies in the range; fewer tests.
template <bool INT, bool CULL>
__global__ void __launch_bounds__(kApThreads, 2) allpairs_split_kernel(
    const PolyInfo *__restrict__ poly, const float4 *__restrict__ coefp, int P, const void *__restrict__ pts,
    int64_t M, uint32_t *__restrict__ keys, int *__restrict__ err)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t full[2];
    const int tid = threadIdx.x;
    const int64_t base = (int64_t)blockIdx.x * (kApPT * kApThreads);
    const int per = (P + gridDim.y - 1) / gridDim.y;
    const int jlo = blockIdx.y * per, jhi = min(P, jlo + per);
    const int nchunks = jhi > jlo ? (jhi - jlo + kApChunk - 1) / kApChunk : 0;
    // one elected thread streams chunks of polygons into the two buffers
    auto issue = [&](int c) {
        const int j0 = jlo + c * kApChunk;
        const int nj = min(kApChunk, jhi - j0);
        unsigned char *buf = smem + (size_t)(c & 1) * kApBufBytes;
        const uint32_t rows = (uint32_t)(nj * kPadStride * sizeof(float4));
        const uint32_t info = (uint32_t)(nj * sizeof(PolyInfo));
        mbar_arrive_expect_tx(&full[c & 1], rows + info);
        bulk_copy_g2s(buf, coefp + (size_t)j0 * kPadStride, rows, &full[c & 1]);
        bulk_copy_g2s(buf + kApRowsBytes, poly + j0, info, &full[c & 1]);
    };
    if (tid == 0) {
        mbar_init(&full[0], 1);
        mbar_init(&full[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
        if (nchunks > 0) issue(0);
        if (nchunks > 1) issue(1);
    }
    float px[kApPT], py[kApPT];
    uint32_t key[kApPT];
#pragma unroll
    for (int i = 0; i < kApPT; ++i) {
        const int64_t p = base + i * kApThreads + tid;
        px[i] = p < M ? load_coord(pts, INT ? PIP_I32 : PIP_F32, 2 * p) : 0.f;
        py[i] = p < M ? load_coord(pts, INT ? PIP_I32 : PIP_F32, 2 * p + 1) : 0.f;
        // an integer point that float32 cannot hold exactly is uncertain
        // against the first polygon of the range, which settles its key
        key[i] = (!INT || int_exact(px[i], py[i]) || jlo >= jhi) ? 0xffffffffu : ((uint32_t)jlo << 1) | 1u;
    }
    int c = 0;
    bool early = false;  // CULL: stopped after consuming chunk c - 1
    for (; c < nchunks; ++c) {
        if (!mbar_wait(&full[c & 1], (uint32_t)((c >> 1) & 1), err)) break;
        const unsigned char *buf = smem + (size_t)(c & 1) * kApBufBytes;
        const float4 *rows = (const float4 *)buf;
        const PolyInfo *info = (const PolyInfo *)(buf + kApRowsBytes);
        const int j0 = jlo + c * kApChunk;
        const int nj = min(kApChunk, jhi - j0);
        for (int q = 0; q < nj; ++q) {
            const PolyInfo &pi = info[q];
            if (pi.status != PIP_OK) continue;  // an invalid polygon contains no point
            if (CULL) {
                const float bx0 = pi.bbox[0], by0 = pi.bbox[1], bx1 = pi.bbox[2], by1 = pi.bbox[3];
                bool open = false;
#pragma unroll
                for (int i = 0; i < kApPT; ++i)
                    open |= key[i] == 0xffffffffu && px[i] >= bx0 && px[i] <= bx1 && py[i] >= by0 && py[i] <= by1;
                if (!__any_sync(0xffffffffu, open)) continue;
                // the discs about o, with d2 of x = fl(p - o) as the edge loop forms it
                bool in_disc[kApPT];
                bool between = false;
                open = false;
#pragma unroll
                for (int i = 0; i < kApPT; ++i) {
                    const float xl = px[i] - pi.ox, yl = py[i] - pi.oy;
                    const float d2 = fmaf(xl, xl, yl * yl);
                    const bool cand = key[i] == 0xffffffffu && px[i] >= bx0 && px[i] <= bx1 && py[i] >= by0 &&
                                      py[i] <= by1 && !(d2 > pi.tout);
                    in_disc[i] = cand && d2 < pi.tin;
                    open |= cand;
                    between |= cand && !in_disc[i];
                }
                if (!__any_sync(0xffffffffu, open)) continue;
                if (!__any_sync(0xffffffffu, between)) {
                    const uint32_t jj = (uint32_t)(j0 + q) << 1;
#pragma unroll
                    for (int i = 0; i < kApPT; ++i)
                        if (in_disc[i]) key[i] = jj;
                    continue;
                }
            }
            const float ox = pi.ox, oy = pi.oy;
            const int n = pi.n;  // at least 3
            const float4 *cf = rows + q * kPadStride;
            float x[kApPT], y[kApPT], m[kApPT];
            {
                const float4 c0 = cf[0], c1 = cf[1], c2 = cf[2];
#pragma unroll
                for (int i = 0; i < kApPT; ++i) {
                    x[i] = px[i] - ox;
                    y[i] = py[i] - oy;
                    m[i] = fmin3_nan(ap_s(c0, x[i], y[i]), ap_s(c1, x[i], y[i]), ap_s(c2, x[i], y[i]));
                }
            }
            int k = 3;
            for (; k + 4 <= n; k += 4) {
                const float4 c0 = cf[k], c1 = cf[k + 1], c2 = cf[k + 2], c3 = cf[k + 3];
#pragma unroll
                for (int i = 0; i < kApPT; ++i)
                    m[i] = fmin3_nan(fmin3_nan(m[i], ap_s(c0, x[i], y[i]), ap_s(c1, x[i], y[i])),
                                     ap_s(c2, x[i], y[i]), ap_s(c3, x[i], y[i]));
            }
            const int rem = n - k;  // the last 0..3 edges
            if (rem == 1) {
                const float4 c0 = cf[k];
#pragma unroll
                for (int i = 0; i < kApPT; ++i) m[i] = fmin_nan(m[i], ap_s(c0, x[i], y[i]));
            } else if (rem == 2) {
                const float4 c0 = cf[k], c1 = cf[k + 1];
#pragma unroll
                for (int i = 0; i < kApPT; ++i)
                    m[i] = fmin3_nan(m[i], ap_s(c0, x[i], y[i]), ap_s(c1, x[i], y[i]));
            } else if (rem == 3) {
                const float4 c0 = cf[k], c1 = cf[k + 1], c2 = cf[k + 2];
#pragma unroll
                for (int i = 0; i < kApPT; ++i)
                    m[i] = fmin3_nan(fmin_nan(m[i], ap_s(c0, x[i], y[i])), ap_s(c1, x[i], y[i]),
                                     ap_s(c2, x[i], y[i]));
            }
            // Most pairs are clearly outside (m <= -B); the key update runs
            // only when some lane of the warp holds a candidate.
            const float b0 = pi.beta0, b1 = pi.beta1;
            bool any = false;
#pragma unroll
            for (int i = 0; i < kApPT; ++i) any |= !(m[i] <= -fmaf(b1, fabsf(x[i]) + fabsf(y[i]), b0));
            if (__any_sync(0xffffffffu, any)) {
                const uint32_t jj = (uint32_t)(j0 + q) << 1;
#pragma unroll
                for (int i = 0; i < kApPT; ++i) {
                    const float B = fmaf(b1, fabsf(x[i]) + fabsf(y[i]), b0);
                    const bool in = m[i] >= B;
                    const bool unc = !(fabsf(m[i]) >= B);
                    if (key[i] == 0xffffffffu && (in || unc)) key[i] = jj | (in ? 0u : 1u);
                }
            }
        }
        if (CULL) {
            // every warp is done with this buffer; stop when every point has a candidate
            bool settled = true;
#pragma unroll
            for (int i = 0; i < kApPT; ++i) settled &= key[i] != 0xffffffffu || base + i * kApThreads + tid >= M;
            if (__syncthreads_and(settled)) {
                ++c;  // this chunk was consumed
                early = true;
                break;
            }
        } else {
            __syncthreads();  // every warp is done with this buffer
        }
        if (tid == 0 && c + 2 < nchunks) issue(c + 2);
    }
    if (c < nchunks && tid == 0) {
        // gave up waiting on chunk c (chunks c and c + 1 may be in flight), or
        // stopped early with chunk c in flight: let those copies land first
        const int end = min(nchunks, c + (early ? 1 : 2));
        for (int k = c; k < end; ++k) mbar_wait(&full[k & 1], (uint32_t)((k >> 1) & 1), err);
    }
#pragma unroll
    for (int i = 0; i < kApPT; ++i) {
        const int64_t p = base + i * kApThreads + tid;
        if (p < M && key[i] != 0xffffffffu) atomicMin(&keys[p], key[i]);
    }
}

// keys -> first-hit ids, mask words, refine queue
__global__ void __launch_bounds__(kThreads) allpairs_finalize_kernel(
    const uint32_t *__restrict__ keys, int64_t M, int32_t *__restrict__ first_hit, uint32_t *__restrict__ mask,
    uint32_t *__restrict__ queue, unsigned int *__restrict__ qcount)
{
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t end = (M + 31) & ~(int64_t)31;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < end; p += stride) {
        const uint32_t k = p < M ? keys[p] : 0xffffffffu;
        const bool decided_in = k != 0xffffffffu && !(k & 1u);
        const bool unc = k != 0xffffffffu && (k & 1u);
        if (p < M && first_hit) first_hit[p] = decided_in ? (int32_t)(k >> 1) : -1;
        const uint32_t w = __ballot_sync(0xffffffffu, decided_in);
        if (mask && lane == 0) mask[p >> 5] = w;
        const uint32_t u = __ballot_sync(0xffffffffu, unc);
        if (u) {
            unsigned int qb = 0;
            if (lane == 0) qb = atomicAdd(qcount, (unsigned int)__popc(u));
            qb = __shfl_sync(0xffffffffu, qb, 0);
            if (unc) queue[qb + __popc(u & ((1u << lane) - 1u))] = (uint32_t)p;
        }
    }
}

template <bool INT, bool CULL>
cudaError_t launch_allpairs(const pip_tables *t, const void *pts, int64_t M, int32_t *first_hit,
                            uint32_t *mask, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(t->d_keys, 0xff, (size_t)M * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    const int64_t tiles = (M + kApPT * kApThreads - 1) / (kApPT * kApThreads);
    const int split = t->P < kApSplit ? t->P : kApSplit;
    allpairs_split_kernel<INT, CULL><<<dim3((unsigned)tiles, (unsigned)split), kApThreads, kApSmem, s>>>(
        t->d_poly, t->d_coefp, t->P, pts, M, t->d_keys, t->d_error);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    allpairs_finalize_kernel<<<t->num_sms * 4, kThreads, 0, s>>>(t->d_keys, M, first_hit, mask, t->d_queue,
                                                                 t->d_qcount);
    return cudaGetLastError();
}

// Warp-cooperative refine for float inputs: one warp per queued point, the
// lanes split the polygon's edges (warp_inside_exact).  Own-polygon mode takes
// the polygon from the queue (or from the offsets); single mode has one.
__global__ void __launch_bounds__(kThreads) refine_warp_kernel(RefineArgs A, int mode)
{
    const int lane = threadIdx.x & 31;
    const unsigned int count = *A.qcount;
    const unsigned int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (unsigned int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < count; q += nwarps) {
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
        if (warp_inside_exact(A.poly, j, A.g0, A.gk, A.verts, A.vdtype, A.pts, A.pdtype, i) && lane == 0)
            atomicOr(&A.mask[i >> 5], 1u << (i & 31));
    }
}

// All-pairs refine, one block per queued point: warp w scans polygons
// start + 32 w + 256 r upward (float32 decision per lane, exact test by the
// whole warp for uncertain ones) and stops at its first hit or once it has
// passed the lowest hit any warp has found; that lowest hit is the answer.
__global__ void __launch_bounds__(kThreads) refine_allpairs_kernel(RefineArgs A)
{
    __shared__ int best;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int kStride = kThreads;  // polygons per round of the whole block
    const unsigned int count = *A.qcount;
    for (unsigned int q = blockIdx.x; q < count; q += gridDim.x) {
        const int64_t i = A.queue[q];
        if (threadIdx.x == 0) best = INT_MAX;
        __syncthreads();
        const int start = (int)(A.keys[i] >> 1);
        for (int base = start + 32 * warp; base < A.P; base += kStride) {
            if (base > *(volatile int *)&best) break;
            const int j = base + lane;
            const int b = j < A.P ? bulk_decision(A, j, i) : -1;
            const uint32_t in_m = __ballot_sync(0xffffffffu, b > 0);
            uint32_t cand = in_m | __ballot_sync(0xffffffffu, b == 0);
            bool found = false;
            while (cand) {
                const int l = __ffs(cand) - 1;
                cand &= cand - 1;
                if (((in_m >> l) & 1u) ||
                    warp_inside_exact(A.poly, base + l, A.g0, A.gk, A.verts, A.vdtype, A.pts, A.pdtype, i)) {
                    if (lane == 0) atomicMin(&best, base + l);
                    found = true;
                    break;
                }
            }
            if (found) break;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const int hit = best == INT_MAX ? -1 : best;
            if (A.first_hit) A.first_hit[i] = hit;
            if (A.mask && hit >= 0) atomicOr(&A.mask[i >> 5], 1u << (i & 31));
        }
        __syncthreads();  // best is reset for the next point
    }
}

}  // namespace

namespace pip {

cudaError_t ragged_kernels_setup()
{
    cudaError_t e = set_ragged_attr<16, 3, 1>();
    if (e == cudaSuccess) e = set_ragged_attr<16, 3, 2>();
    if (e == cudaSuccess) e = set_ragged_attr<16, 3, 4>();
    if (e == cudaSuccess) e = set_ragged_attr<16, 2, 2>();
    if (e == cudaSuccess) e = set_ragged_attr<12, 3, 2>();
    if (e == cudaSuccess) e = set_ragged_attr<12, 4, 2>();
    if (e == cudaSuccess) e = set_one_ragged_attr<16, 3, false, false, kRagVoronoi, true, 2>();
    if (e == cudaSuccess) e = set_one_ragged_attr<16, 3, true, false, kRagVoronoi, true, 2>();
    if (e == cudaSuccess) e = set_ragged_cmp_attr<kRagSign>();
    if (e == cudaSuccess) e = set_ragged_cmp_attr<kRagRay>();
    if (e == cudaSuccess) e = set_ragged_cmp_attr<kRagFp64>();
    return e;
}

cudaError_t launch_ragged_cmp(const pip_tables *t, const float *pts, int64_t M, const int64_t *poffs, uint32_t *mask,
                              int op, cudaStream_t s)
{
    // one tile shape: 16 points per lane, 3 stages
    if (op == kRagSign) return launch_ragged_tma_one<16, 3, false, false, kRagSign, false, 2>(t, pts, M, poffs, mask, s);
    if (op == kRagRay) return launch_ragged_tma_one<16, 3, false, false, kRagRay, false, 2>(t, pts, M, poffs, mask, s);
    return launch_ragged_tma_one<16, 3, false, false, kRagFp64, false, 2>(t, pts, M, poffs, mask, s);
}

cudaError_t allpairs_setup()
{
    const int bytes = (int)kApSmem;
    cudaError_t e = cudaFuncSetAttribute(allpairs_split_kernel<false, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(allpairs_split_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(allpairs_split_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(allpairs_split_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 bytes);
    return e;
}

}  // namespace pip

extern "C" pip_status pip_test(const pip_tables *t, const void *d_points, pip_dtype pdtype,
                               int64_t num_points, const int64_t *d_point_offsets, int mode,
                               uint32_t *d_mask, int32_t *d_first_hit, void *stream)
{
    pip_status st = check_tables(t);
    if (st != PIP_OK) return st;
    if (pdtype != PIP_F32 && pdtype != PIP_I32) return PIP_E_INVALID_ARG;
    if (num_points < 0) return PIP_E_INVALID_ARG;
    if (num_points > t->capacity) return PIP_E_CAPACITY;
    if ((mode & ~(PIP_MASK | PIP_FIRST_HIT | PIP_CULL | PIP_EARLY_EXIT | PIP_DISC)) || !(mode & (PIP_MASK | PIP_FIRST_HIT)))
        return PIP_E_INVALID_ARG;
    const bool early = (mode & PIP_EARLY_EXIT) != 0;
    const bool disc = (mode & PIP_DISC) != 0;
    if (early && disc) return PIP_E_INVALID_ARG;
    const bool want_mask = mode & PIP_MASK, want_hit = mode & PIP_FIRST_HIT;
    if (want_hit && d_point_offsets != nullptr) return PIP_E_INVALID_ARG;
    if (num_points == 0) {  // nothing to decide; the refine count of this call is 0
        PIP_CUDA_TRY(cudaMemsetAsync(t->d_qcount, 0, sizeof(unsigned int), (cudaStream_t)stream));
        return PIP_OK;
    }
    if (want_mask && d_mask == nullptr) return PIP_E_INVALID_ARG;
    if (want_hit && (d_first_hit == nullptr || d_point_offsets != nullptr)) return PIP_E_INVALID_ARG;
    if (num_points > 0 && (d_points == nullptr || !aligned(d_points, 8))) return PIP_E_INVALID_ARG;
    if (d_mask && !aligned(d_mask, 4)) return PIP_E_INVALID_ARG;
    if (d_first_hit && !aligned(d_first_hit, 4)) return PIP_E_INVALID_ARG;
    if (d_point_offsets && !aligned(d_point_offsets, 8)) return PIP_E_INVALID_ARG;
    if (!want_hit && d_point_offsets == nullptr && t->P > 1 && !want_mask) return PIP_E_INVALID_ARG;

    cudaStream_t s = (cudaStream_t)stream;
    const bool ints = pdtype == PIP_I32;
    const bool v16 = aligned(d_points, 16);
    uint32_t *mask = want_mask ? d_mask : nullptr;
    int32_t *hit = want_hit ? d_first_hit : nullptr;
    cudaError_t e = cudaSuccess;
    int kmode;

    if (d_point_offsets != nullptr) {
        kmode = kRagged;
        timing_mark(t, 0, s);
        if (num_points == 0) {
            PIP_CUDA_TRY(cudaMemsetAsync(t->d_qcount, 0, sizeof(unsigned int), s));
            return PIP_OK;
        }
        if (v16 && ints && t->vdtype == PIP_I32) {
            // integer polygons and points: uncertain points decided exactly in
            // the bulk kernel, nothing queued, no refine launch
            e = launch_ragged_tma<true, true>(t, d_points, num_points, d_point_offsets, mask, s);
            if (e != cudaSuccess) return PIP_E_CUDA;
            timing_mark(t, 1, s);
            timing_mark(t, 2, s);
            return PIP_OK;
        }
        if (v16 && early)  // the early-exit form at the default tile shape
            e = ints ? launch_ragged_tma_one<16, 3, true, false, kRagVoronoi, true, 2>(t, d_points, num_points,
                                                                                     d_point_offsets, mask, s)
                     : launch_ragged_tma_one<16, 3, false, false, kRagVoronoi, true, 2>(t, d_points, num_points,
                                                                                      d_point_offsets, mask, s);
        else if (v16 && disc)  // the disc filter at the chosen tile shape
            e = ints ? launch_ragged_tma<true, false, true>(t, d_points, num_points, d_point_offsets, mask, s)
                     : launch_ragged_tma<false, false, true>(t, d_points, num_points, d_point_offsets, mask, s);
        else if (v16)  // bulk copies want a 16-byte aligned point array
            e = ints ? launch_ragged_tma<true, false>(t, d_points, num_points, d_point_offsets, mask, s)
                     : launch_ragged_tma<false, false>(t, d_points, num_points, d_point_offsets, mask, s);
        else
            e = ints ? launch_ragged<true, false>(t, d_points, num_points, d_point_offsets, mask, s)
                     : launch_ragged<false, false>(t, d_points, num_points, d_point_offsets, mask, s);
    } else if (t->P == 1 && !want_hit && v16 && t->have_host_poly) {
        // the pipelined kernel: bulk test and exact refine in one launch
        timing_mark(t, 0, s);
        e = launch_stream_pipelined(t, d_points, ints, num_points, mask, early, disc, s);
        if (e != cudaSuccess) return PIP_E_CUDA;
        timing_mark(t, 1, s);
        timing_mark(t, 2, s);
        return PIP_OK;
    } else if (t->P == 1 && !want_hit) {
        kmode = kSingle;
        PIP_CUDA_TRY(cudaMemsetAsync(t->d_qcount, 0, sizeof(unsigned int), s));
        if (num_points == 0) return PIP_OK;
        timing_mark(t, 0, s);
        if (ints) e = v16 ? launch_stream<true, true>(t, d_points, num_points, mask, s)
                          : launch_stream<true, false>(t, d_points, num_points, mask, s);
        else e = v16 ? launch_stream<false, true>(t, d_points, num_points, mask, s)
                     : launch_stream<false, false>(t, d_points, num_points, mask, s);
    } else {
        kmode = kAllPairs;
        PIP_CUDA_TRY(cudaMemsetAsync(t->d_qcount, 0, sizeof(unsigned int), s));
        if (num_points == 0) return PIP_OK;
        timing_mark(t, 0, s);
        if (mode & PIP_CULL)
            e = ints ? launch_allpairs<true, true>(t, d_points, num_points, hit, mask, s)
                     : launch_allpairs<false, true>(t, d_points, num_points, hit, mask, s);
        else
            e = ints ? launch_allpairs<true, false>(t, d_points, num_points, hit, mask, s)
                     : launch_allpairs<false, false>(t, d_points, num_points, hit, mask, s);
    }
    if (e != cudaSuccess) return PIP_E_CUDA;
    timing_mark(t, 1, s);

    RefineArgs A{};
    A.poly = t->d_poly;
    A.coef = t->d_coef;
    A.g0 = t->d_g0;
    A.gk = t->d_gk;
    A.verts = t->d_verts;
    A.vdtype = t->vdtype;
    A.P = t->P;
    A.pts = d_points;
    A.pdtype = pdtype;
    A.M = num_points;
    A.poffs = d_point_offsets;
    A.queue = t->d_queue;
    A.qcount = t->d_qcount;
    A.mask = mask;
    A.first_hit = hit;
    A.keys = t->d_keys;
    A.iedge = t->d_iedge;
    // the pipelined batch kernel files the polygon of each queued point in the keys buffer
    A.qpoly = (kmode == kRagged && v16) ? t->d_keys : nullptr;
    if (kmode != kAllPairs && t->vdtype == PIP_I32 && pdtype == PIP_I32)
        refine_kernel<true><<<t->num_sms * 8, kThreads, 0, s>>>(A, kmode);  // int64, one thread a point
    else if (kmode == kAllPairs)
        refine_allpairs_kernel<<<t->num_sms * 2, kThreads, 0, s>>>(A);
    else
        refine_warp_kernel<<<t->num_sms * 4, kThreads, 0, s>>>(A, kmode);
    if (cudaGetLastError() != cudaSuccess) return PIP_E_CUDA;
    timing_mark(t, 2, s);
    return PIP_OK;
}

extern "C" int32_t pip_batch_variant_count(void) { return kNumBatchVariants; }

extern "C" pip_status pip_set_batch_variant(pip_tables *t, int32_t variant)
{
    pip_status st = check_tables(t);
    if (st != PIP_OK) return st;
    if (variant < 0 || variant >= kNumBatchVariants) return PIP_E_INVALID_ARG;
    t->batch_variant = variant;
    return PIP_OK;
}

extern "C" pip_status pip_autotune_batch(pip_tables *t, const void *d_points, pip_dtype pdtype,
                                         int64_t num_points, const int64_t *d_point_offsets, uint32_t *d_mask,
                                         int32_t reps, void *stream, int32_t *best_variant, float *best_ms)
{
    pip_status st = check_tables(t);
    if (st != PIP_OK) return st;
    if (num_points <= 0 || reps < 1 || d_point_offsets == nullptr || !aligned(d_points, 16))
        return PIP_E_INVALID_ARG;
    // a cached choice for this kernel, GPU and shape skips the timing runs
    const std::string key = tuning_key(t, "batch", num_points, pdtype);
    int cached = -1;
    float cached_ms = 0.f;
    if (tuning_lookup(key, &cached, &cached_ms) && cached >= 0 && cached < kNumBatchVariants) {
        t->batch_variant = cached;
        if (best_variant) *best_variant = cached;
        if (best_ms) *best_ms = cached_ms;
        return PIP_OK;
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    PIP_CUDA_TRY(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return PIP_E_CUDA;
    }
    const int keep = t->timing;
    t->timing = 0;
    int best = -1;
    float best_t = 0.f;
    pip_status out = PIP_OK;
    for (int v = 0; v < kNumBatchVariants && out == PIP_OK; ++v) {
        t->batch_variant = v;
        out = pip_test(t, d_points, pdtype, num_points, d_point_offsets, PIP_MASK, d_mask, nullptr, stream);
        if (out != PIP_OK) break;
        float ms = 0.f;
        if (cudaEventRecord(e0, s) != cudaSuccess) { out = PIP_E_CUDA; break; }
        for (int r = 0; r < reps && out == PIP_OK; ++r)
            out = pip_test(t, d_points, pdtype, num_points, d_point_offsets, PIP_MASK, d_mask, nullptr, stream);
        if (out != PIP_OK) break;
        if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            out = PIP_E_CUDA;
            break;
        }
        ms /= reps;
        if (best < 0 || ms < best_t) { best = v; best_t = ms; }
    }
    t->timing = keep;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (out != PIP_OK) return out;
    tuning_store(key, best, best_t);
    t->batch_variant = best;
    if (best_variant) *best_variant = best;
    if (best_ms) *best_ms = best_t;
    return PIP_OK;
}
