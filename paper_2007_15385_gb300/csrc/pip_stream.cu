// pip_stream.cu -- launch side of the pipelined single-polygon kernel
// (pip_stream_tma.cuh): the polygon's row and coefficients as launch
// parameters, the edge-count and tile-shape variants, and their autotuner.
#include "pip_kernels.cuh"

using namespace pip;

#include "pip_stream_tma.cuh"

namespace {

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

cudaError_t launch_stream_pipelined(const pip_tables *t, const void *pts, bool ints, int64_t M, uint32_t *mask,
                                    cudaStream_t s)
{
    return ints ? launch_stream_tma<true>(t, pts, M, mask, s) : launch_stream_tma<false>(t, pts, M, mask, s);
}

}  // namespace pip

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
