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

template <bool INT>
cudaError_t launch_allpairs(const pip_tables *t, const void *pts, int64_t M, int32_t *first_hit,
                            uint32_t *mask, cudaStream_t s)
{
    const int64_t blocks = (M + kPT * kThreads - 1) / (kPT * kThreads);
    allpairs_kernel<kPT, INT><<<(unsigned)blocks, kThreads, 0, s>>>(
        t->d_poly, t->d_coef, t->P, pts, M, first_hit, mask, t->d_queue, t->d_qcount);
    return cudaGetLastError();
}

}  // namespace

extern "C" pip_status pip_test(const pip_tables *t, const void *d_points, pip_dtype pdtype,
                               int64_t num_points, const int64_t *d_point_offsets, int mode,
                               uint32_t *d_mask, int32_t *d_first_hit, void *stream)
{
    pip_status st = check_tables(t);
    if (st != PIP_OK) return st;
    if (pdtype != PIP_F32 && pdtype != PIP_I32) return PIP_E_INVALID_ARG;
    if (num_points < 0) return PIP_E_INVALID_ARG;
    if (num_points > t->capacity) return PIP_E_CAPACITY;
    if ((mode & ~(PIP_MASK | PIP_FIRST_HIT)) || mode == 0) return PIP_E_INVALID_ARG;
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
        if (ints) e = v16 ? launch_ragged<true, true>(t, d_points, num_points, d_point_offsets, mask, s)
                          : launch_ragged<true, false>(t, d_points, num_points, d_point_offsets, mask, s);
        else e = v16 ? launch_ragged<false, true>(t, d_points, num_points, d_point_offsets, mask, s)
                     : launch_ragged<false, false>(t, d_points, num_points, d_point_offsets, mask, s);
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
        e = ints ? launch_allpairs<true>(t, d_points, num_points, hit, mask, s)
                 : launch_allpairs<false>(t, d_points, num_points, hit, mask, s);
    }
    if (e != cudaSuccess) return PIP_E_CUDA;
    timing_mark(t, 1, s);

    RefineArgs A;
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
    refine_kernel<<<t->num_sms * 2, kThreads, 0, s>>>(A, kmode);
    if (cudaGetLastError() != cudaSuccess) return PIP_E_CUDA;
    timing_mark(t, 2, s);
    return PIP_OK;
}
