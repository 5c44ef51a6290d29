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
#include "pip_stream_tma.cuh"

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

// Variants of the pipelined kernel: (points per lane per stage, stages,
// 3-operand min).
struct StreamVariant {
    int ppl, stages, min3;
};
constexpr StreamVariant kStreamVariants[] = {{16, 3, 0}, {16, 2, 0}, {8, 4, 0}, {8, 6, 0}};
constexpr int kNumStreamVariants = sizeof(kStreamVariants) / sizeof(kStreamVariants[0]);

template <int NE, int PPL, int STAGES, bool INT, bool MIN3>
cudaError_t launch_tma_one(const pip_tables *t, const void *pts, int64_t M, uint32_t *mask, cudaStream_t s)
{
    using C = StreamCfg<PPL, STAGES>;
    auto k = stream_tma_kernel<NE, PPL, STAGES, INT, MIN3>;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kStreamThreads, C::kSmem) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    if (per_sm > 2) per_sm = 2;  // the scratch queue holds one tile of slack per CTA, 2 CTAs per SM
    const int64_t tiles = (M + C::kTile - 1) / C::kTile;
    const int blocks = (int)max((int64_t)1, min((int64_t)per_sm * t->num_sms, tiles));
    StreamPoly sp;
    const PolyInfo &hp = t->h_poly;
    sp.ox = hp.ox;
    sp.oy = hp.oy;
    sp.b0 = hp.beta0;
    sp.b1 = hp.beta1;
    sp.ok = hp.status == PIP_OK;
    sp.n = sp.ok ? hp.n : 1;
    sp.pad0 = sp.pad1 = 0;
    for (int k = 0; k < kParamEdges; ++k) {
        float4 c = make_float4(0.f, 0.f, INFINITY, 0.f);
        if (!sp.ok) { if (k == 0) c.z = -INFINITY; }
        else if (k < sp.n) c = t->h_coef[k];
        sp.wx[k] = c.x;
        sp.wy[k] = c.y;
        sp.t[k] = c.z;
    }
    k<<<blocks, kStreamThreads, C::kSmem, s>>>(sp, t->d_poly, t->d_coef, t->d_g0, t->d_gk, t->d_verts,
                                               t->vdtype, pts, M, mask, t->d_queue,
                                               (StreamCounters *)t->d_stream_ctr, t->d_qcount, t->d_error);
    return cudaGetLastError();
}

template <int PPL, int STAGES, bool INT, bool MIN3>
cudaError_t launch_tma_ne(const pip_tables *t, const void *pts, int64_t M, uint32_t *mask, cudaStream_t s)
{
    // the polygon's edge count is known on the host from the vertex count
    const int n = t->V;
    if (n <= 4) return launch_tma_one<4, PPL, STAGES, INT, MIN3>(t, pts, M, mask, s);
    if (n <= 8) return launch_tma_one<8, PPL, STAGES, INT, MIN3>(t, pts, M, mask, s);
    if (n <= 12) return launch_tma_one<12, PPL, STAGES, INT, MIN3>(t, pts, M, mask, s);
    if (n <= 16) return launch_tma_one<16, PPL, STAGES, INT, MIN3>(t, pts, M, mask, s);
    return launch_tma_one<0, PPL, STAGES, INT, MIN3>(t, pts, M, mask, s);
}

template <int NE, int PPL, int STAGES, bool MIN3>
cudaError_t set_attr_one()
{
    const int bytes = (int)StreamCfg<PPL, STAGES>::kSmem;
    cudaError_t e = cudaFuncSetAttribute(stream_tma_kernel<NE, PPL, STAGES, false, MIN3>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(stream_tma_kernel<NE, PPL, STAGES, true, MIN3>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    return e;
}

template <int PPL, int STAGES, bool MIN3>
cudaError_t set_smem_attr()
{
    cudaError_t e = set_attr_one<4, PPL, STAGES, MIN3>();
    if (e == cudaSuccess) e = set_attr_one<8, PPL, STAGES, MIN3>();
    if (e == cudaSuccess) e = set_attr_one<12, PPL, STAGES, MIN3>();
    if (e == cudaSuccess) e = set_attr_one<16, PPL, STAGES, MIN3>();
    if (e == cudaSuccess) e = set_attr_one<0, PPL, STAGES, MIN3>();
    return e;
}

template <bool INT>
cudaError_t launch_stream_tma(const pip_tables *t, const void *pts, int64_t M, uint32_t *mask,
                              cudaStream_t s)
{
    switch (t->stream_variant) {
    case 1: return launch_tma_ne<16, 2, INT, false>(t, pts, M, mask, s);
    case 2: return launch_tma_ne<8, 4, INT, false>(t, pts, M, mask, s);
    case 3: return launch_tma_ne<8, 6, INT, false>(t, pts, M, mask, s);
    default: return launch_tma_ne<16, 3, INT, false>(t, pts, M, mask, s);
    }
}

}  // namespace

namespace pip {

cudaError_t stream_kernels_setup()
{
    cudaError_t e = set_smem_attr<16, 3, false>();
    if (e == cudaSuccess) e = set_smem_attr<16, 2, false>();
    if (e == cudaSuccess) e = set_smem_attr<8, 4, false>();
    if (e == cudaSuccess) e = set_smem_attr<8, 6, false>();
    return e;
}

int stream_variant_count() { return kNumStreamVariants; }

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
    } else if (t->P == 1 && !want_hit && v16 && t->have_host_poly) {
        // the pipelined kernel: bulk test and exact refine in one launch
        timing_mark(t, 0, s);
        e = ints ? launch_stream_tma<true>(t, d_points, num_points, mask, s)
                 : launch_stream_tma<false>(t, d_points, num_points, mask, s);
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

extern "C" int32_t pip_stream_variant_count(void) { return kNumStreamVariants; }

extern "C" pip_status pip_set_stream_variant(pip_tables *t, int32_t variant)
{
    pip_status st = check_tables(t);
    if (st != PIP_OK) return st;
    if (variant < 0 || variant >= kNumStreamVariants) return PIP_E_INVALID_ARG;
    t->stream_variant = variant;
    return PIP_OK;
}

extern "C" pip_status pip_autotune_stream(pip_tables *t, const void *d_points, pip_dtype pdtype,
                                          int64_t num_points, uint32_t *d_mask, int32_t reps,
                                          void *stream, int32_t *best_variant, float *best_ms)
{
    pip_status st = check_tables(t);
    if (st != PIP_OK) return st;
    if (t->P != 1 || num_points <= 0 || reps < 1 || !aligned(d_points, 16)) return PIP_E_INVALID_ARG;
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
    for (int v = 0; v < kNumStreamVariants && out == PIP_OK; ++v) {
        t->stream_variant = v;
        out = pip_test(t, d_points, pdtype, num_points, nullptr, PIP_MASK, d_mask, nullptr, stream);
        if (out != PIP_OK) break;
        float ms = 0.f;
        if (cudaEventRecord(e0, s) != cudaSuccess) { out = PIP_E_CUDA; break; }
        for (int r = 0; r < reps && out == PIP_OK; ++r)
            out = pip_test(t, d_points, pdtype, num_points, nullptr, PIP_MASK, d_mask, nullptr, stream);
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
    t->stream_variant = best;
    if (best_variant) *best_variant = best;
    if (best_ms) *best_ms = best_t;
    return PIP_OK;
}
