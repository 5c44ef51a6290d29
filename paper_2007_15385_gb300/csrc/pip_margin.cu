// pip_margin.cu -- signed Voronoi margin.
//
// Edge k of the Voronoi polygon is the bisector of p0 and p_k (Eq. 2).  The
// signed distance of x from it is
//     (|x - p0|^2 - |x - p_k|^2) / (2 |p_k - p0|) = x . w_k/|w_k| - t_k/|w_k|
// (x relative to o), and the margin is the largest over k: > 0 outside,
// <= 0 inside.  The normalised table (w/|w|, t/|w|) is built by pip_prepare,
// so the inner loop is the same two FMAs and a min as the inclusion test.
// A point with a non-finite coordinate gets +inf (outside).
#include "pip_kernels.cuh"
#include "pip_margin_tma.cuh"

using namespace pip;

namespace {

template <int F, bool INT, bool V16>
__device__ __forceinline__ void margin_chunk(const void *__restrict__ pts, int64_t M, int64_t p0,
                                             int64_t lo, int64_t hi, const float4 *cs, int npad,
                                             float ox, float oy, float *__restrict__ out, int lane)
{
    float x[2 * F], y[2 * F], m[2 * F];
    bool fin[2 * F];
#pragma unroll
    for (int j = 0; j < F; ++j) {
        const int64_t q2 = p0 + 2 * (j * 32 + lane);
        float px0, py0, px1, py1;
        load_pair<INT, V16>(pts, q2, M, px0, py0, px1, py1);
        fin[2 * j] = isfinite(px0) && isfinite(py0);
        fin[2 * j + 1] = isfinite(px1) && isfinite(py1);
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
#pragma unroll
    for (int j = 0; j < F; ++j) {
        const int64_t q2 = p0 + 2 * (j * 32 + lane);
        if (q2 >= lo && q2 < hi) out[q2] = fin[2 * j] ? -m[2 * j] : INFINITY;
        if (q2 + 1 >= lo && q2 + 1 < hi) out[q2 + 1] = fin[2 * j + 1] ? -m[2 * j + 1] : INFINITY;
    }
}

template <int F, bool INT, bool V16>
__global__ void __launch_bounds__(kThreads) margin_stream_kernel(
    const PolyInfo *__restrict__ poly, const float4 *__restrict__ coefn, const void *__restrict__ pts,
    int64_t M, float *__restrict__ out)
{
    __shared__ float4 cs[kMaxEdges + 4];
    const PolyInfo pi = poly[0];
    const int npad = stage_polygon(pi, coefn, cs, threadIdx.x, blockDim.x);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nchunks = (M + Chunk<F>::kPoints - 1) / Chunk<F>::kPoints;
    for (int64_t c = warp; c < nchunks; c += nwarps)
        margin_chunk<F, INT, V16>(pts, M, c * Chunk<F>::kPoints, 0, M, cs, npad, pi.ox, pi.oy, out, lane);
}

template <int F, bool INT, bool V16>
__global__ void __launch_bounds__(kThreads) margin_ragged_kernel(
    const PolyInfo *__restrict__ poly, const float4 *__restrict__ coefn, const void *__restrict__ pts,
    int64_t M, const int64_t *__restrict__ poffs, int P, const int64_t *__restrict__ items,
    int item_chunks, unsigned int *__restrict__ work, float *__restrict__ out)
{
    __shared__ float4 cs[kMaxEdges + 4];
    __shared__ int s_poly;
    __shared__ int64_t s_local;
    __shared__ int s_done;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t total = items[P];
    for (;;) {
        if (threadIdx.x == 0) {
            const int64_t it = (int64_t)atomicAdd(work, 1u);
            s_done = it >= total;
            if (it < total) {
                int lo = 0, hi = P;
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (items[mid] <= it) lo = mid; else hi = mid;
                }
                s_poly = lo;
                s_local = it - items[lo];
            }
        }
        __syncthreads();
        if (s_done) break;
        const int j = s_poly;
        const PolyInfo pi = poly[j];
        const int npad = stage_polygon(pi, coefn, cs, threadIdx.x, blockDim.x);
        __syncthreads();
        const int64_t a = poffs[j], b = poffs[j + 1];
        const int64_t c0 = a / Chunk<F>::kPoints + s_local * item_chunks;
        const int64_t c1 = min(c0 + item_chunks, (b - 1) / Chunk<F>::kPoints + 1);
        for (int64_t c = c0 + wid; c < c1; c += kWarps)
            margin_chunk<F, INT, V16>(pts, M, c * Chunk<F>::kPoints, a, b, cs, npad, pi.ox, pi.oy, out, lane);
        __syncthreads();
    }
}

// All pairs: the smallest margin over every polygon (negative when some
// polygon holds the point).
constexpr int kPolyChunk = 32;

template <int PT, bool INT>
__global__ void __launch_bounds__(kThreads) margin_allpairs_kernel(
    const PolyInfo *__restrict__ poly, const float4 *__restrict__ coefn, int P,
    const void *__restrict__ pts, int64_t M, float *__restrict__ out)
{
    __shared__ float4 cs[kPolyChunk * (kMaxEdges + 4)];
    __shared__ float4 so[kPolyChunk];  // (ox, oy, npad, 0)
    const int tid = threadIdx.x, lane = tid & 31;
    const int64_t base = (int64_t)blockIdx.x * (PT * kThreads);
    float px[PT], py[PT], best[PT];
#pragma unroll
    for (int i = 0; i < PT; ++i) {
        const int64_t p = base + i * kThreads + tid;
        px[i] = p < M ? load_coord(pts, INT ? PIP_I32 : PIP_F32, 2 * p) : 0.f;
        py[i] = p < M ? load_coord(pts, INT ? PIP_I32 : PIP_F32, 2 * p + 1) : 0.f;
        best[i] = INFINITY;
    }
    for (int j0 = 0; j0 < P; j0 += kPolyChunk) {
        const int nj = min(kPolyChunk, P - j0);
        __syncthreads();
        if (tid < nj) {
            const PolyInfo pi = poly[j0 + tid];
            so[tid] = make_float4(pi.ox, pi.oy,
                                  __int_as_float(((pi.status == PIP_OK ? pi.n : 1) + 3) & ~3), 0.f);
        }
        for (int q = tid >> 5; q < nj; q += kWarps)
            stage_polygon(poly[j0 + q], coefn, cs + q * (kMaxEdges + 4), lane, 32);
        __syncthreads();
        for (int q = 0; q < nj; ++q) {
            const float4 s = so[q];
            const int npad = __float_as_int(s.z);
            const float4 *c = cs + q * (kMaxEdges + 4);
            float x[PT], y[PT], m[PT];
#pragma unroll
            for (int i = 0; i < PT; ++i) {
                x[i] = px[i] - s.x;
                y[i] = py[i] - s.y;
                m[i] = INFINITY;
            }
            for (int k = 0; k < npad; k += 4) {
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const float4 cf = c[k + kk];
#pragma unroll
                    for (int i = 0; i < PT; ++i)
                        m[i] = fminf(m[i], fmaf(-x[i], cf.x, fmaf(-y[i], cf.y, cf.z)));
                }
            }
#pragma unroll
            for (int i = 0; i < PT; ++i) best[i] = fminf(best[i], -m[i]);
        }
    }
#pragma unroll
    for (int i = 0; i < PT; ++i) {
        const int64_t p = base + i * kThreads + tid;
        if (p < M) out[p] = (isfinite(px[i]) && isfinite(py[i])) ? best[i] : INFINITY;
    }
}

constexpr int kF = 4;
constexpr int kItemChunks = 32;
constexpr int kPT = 4;

}  // namespace

namespace pip {

// Called by pip_prepare (outside any stream capture).
cudaError_t margin_kernels_setup()
{
    cudaError_t e = setup_margin_tma<false>();
    if (e == cudaSuccess) e = setup_margin_tma<true>();
    return e;
}

}  // namespace pip

extern "C" pip_status pip_margin(const pip_tables *t, const void *d_points, pip_dtype pdtype,
                                 int64_t num_points, const int64_t *d_point_offsets, float *d_margin,
                                 void *stream)
{
    pip_status st = check_tables(t);
    if (st != PIP_OK) return st;
    if (pdtype != PIP_F32 && pdtype != PIP_I32) return PIP_E_INVALID_ARG;
    if (num_points < 0) return PIP_E_INVALID_ARG;
    if (num_points == 0) return PIP_OK;
    if (d_points == nullptr || d_margin == nullptr) return PIP_E_INVALID_ARG;
    if (!aligned(d_points, 8) || !aligned(d_margin, 4)) return PIP_E_INVALID_ARG;
    if (d_point_offsets && !aligned(d_point_offsets, 8)) return PIP_E_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const bool ints = pdtype == PIP_I32, v16 = aligned(d_points, 16);
    const int64_t M = num_points;
    if (d_point_offsets) {
        // the refine count of the last pip_test is left alone: a spare counter word
        ragged_setup_kernel<kF><<<1, 1024, 0, s>>>(d_point_offsets, t->P, M, kItemChunks, t->d_items,
                                                   t->d_work, t->d_work + 1, t->d_worst);
        PIP_CUDA_TRY(cudaGetLastError());
#define LAUNCH_MR(I, V)                                                                              \
    {                                                                                                \
        auto k = margin_ragged_kernel<kF, I, V>;                                                     \
        k<<<blocks_for(k, t->num_sms, kThreads), kThreads, 0, s>>>(                                  \
            t->d_poly, t->d_coefn, d_points, M, d_point_offsets, t->P, t->d_items, kItemChunks,       \
            t->d_work, d_margin);                                                                    \
    }
        if (ints) { if (v16) LAUNCH_MR(true, true) else LAUNCH_MR(true, false) }
        else { if (v16) LAUNCH_MR(false, true) else LAUNCH_MR(false, false) }
#undef LAUNCH_MR
    } else if (t->P == 1 && v16) {
        // 16-byte aligned points: the pipelined kernel (bulk copies through shared memory)
        PIP_CUDA_TRY(ints ? launch_margin_tma<true>(t, d_points, M, d_margin, s)
                          : launch_margin_tma<false>(t, d_points, M, d_margin, s));
    } else if (t->P == 1) {
        const int64_t chunks = (M + Chunk<kF>::kPoints - 1) / Chunk<kF>::kPoints;
#define LAUNCH_MS(I, V)                                                                              \
    {                                                                                                \
        auto k = margin_stream_kernel<kF, I, V>;                                                     \
        const int blocks = (int)max((int64_t)1, min((int64_t)blocks_for(k, t->num_sms, kThreads),    \
                                                     (chunks + kWarps - 1) / kWarps));               \
        k<<<blocks, kThreads, 0, s>>>(t->d_poly, t->d_coefn, d_points, M, d_margin);                 \
    }
        if (ints) { if (v16) LAUNCH_MS(true, true) else LAUNCH_MS(true, false) }
        else { if (v16) LAUNCH_MS(false, true) else LAUNCH_MS(false, false) }
#undef LAUNCH_MS
    } else {
        const int64_t blocks = (M + kPT * kThreads - 1) / (kPT * kThreads);
        if (ints)
            margin_allpairs_kernel<kPT, true><<<(unsigned)blocks, kThreads, 0, s>>>(t->d_poly, t->d_coefn, t->P, d_points, M, d_margin);
        else
            margin_allpairs_kernel<kPT, false><<<(unsigned)blocks, kThreads, 0, s>>>(t->d_poly, t->d_coefn, t->P, d_points, M, d_margin);
    }
    return cudaGetLastError() == cudaSuccess ? PIP_OK : PIP_E_CUDA;
}
