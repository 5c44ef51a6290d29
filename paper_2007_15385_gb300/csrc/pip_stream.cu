// pip_stream.cu -- the pipelined single-polygon test for float32 points, the
// dispatch by point type, and the tile-shape API and autotuner.
#include <limits>

#include "pip_stream_launch.cuh"

using namespace pip;

namespace {

// The comparators run at one tile shape, the headline's default (16 points
// per lane, 3 stages).
constexpr int kCmpPPL = 16, kCmpStages = 3;

template <int NE, int OP>
cudaError_t launch_cmp_one(const pip_tables *t, const float *pts, int64_t M, uint32_t *mask, cudaStream_t s)
{
    using C = StreamCfg<kCmpPPL, kCmpStages>;
    auto k = stream_tma_kernel<NE, kCmpPPL, kCmpStages, false, OP>;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, C::kThreads, C::kSmem) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    if (per_sm > 2) per_sm = 2;
    const int64_t tiles = (M + C::kTile - 1) / C::kTile;
    const int blocks = (int)max((int64_t)1, min((int64_t)per_sm * t->num_sms, tiles));
    StreamPoly sp;
    const PolyInfo &hp = t->h_poly;
    sp.ox = sp.oy = sp.b0 = sp.b1 = 0.f;
    sp.ok = hp.status == PIP_OK;
    sp.n = sp.ok ? hp.n : 1;
    sp.tin = 0.f;
    sp.tout = -INFINITY;
    const float qnan = std::numeric_limits<float>::quiet_NaN();
    for (int e = 0; e < kParamEdges; ++e) {
        float4 c = make_float4(0.f, 0.f, qnan, 0.f), y = make_float4(qnan, qnan, 0.f, 0.f);
        if (sp.ok && e < sp.n) {
            c = OP == kTmaSign ? t->h_cmp_sign[e] : t->h_cmp_ray[2 * e];
            if (OP == kTmaRay) y = t->h_cmp_ray[2 * e + 1];
        }
        sp.wx[e] = c.x;
        sp.wy[e] = c.y;
        sp.t[e] = c.z;
        sp.y0[e] = y.x;
        sp.y1[e] = y.y;
    }
    const float4 *rows = OP == kTmaSign ? t->d_cmp_sign : t->d_cmp_ray;
    k<<<blocks, C::kThreads, C::kSmem, s>>>(sp, t->d_poly, rows, t->d_g0, t->d_gk, t->d_verts, t->vdtype, pts,
                                               M, mask, t->d_queue, (StreamCounters *)t->d_stream_ctr, t->d_qcount,
                                               t->d_error);
    return cudaGetLastError();
}

template <int OP>
cudaError_t launch_cmp_ne(const pip_tables *t, const float *pts, int64_t M, uint32_t *mask, cudaStream_t s)
{
    const int n = t->V;
    if (n <= 4) return launch_cmp_one<4, OP>(t, pts, M, mask, s);
    if (n <= 8) return launch_cmp_one<8, OP>(t, pts, M, mask, s);
    if (n <= 12) return launch_cmp_one<12, OP>(t, pts, M, mask, s);
    if (n <= 16) return launch_cmp_one<16, OP>(t, pts, M, mask, s);
    return launch_cmp_one<0, OP>(t, pts, M, mask, s);
}

template <int OP>
cudaError_t set_cmp_attr()
{
    const int bytes = (int)StreamCfg<kCmpPPL, kCmpStages>::kSmem;
    cudaError_t e = cudaFuncSetAttribute(stream_tma_kernel<4, kCmpPPL, kCmpStages, false, OP>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(stream_tma_kernel<8, kCmpPPL, kCmpStages, false, OP>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(stream_tma_kernel<12, kCmpPPL, kCmpStages, false, OP>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(stream_tma_kernel<16, kCmpPPL, kCmpStages, false, OP>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(stream_tma_kernel<0, kCmpPPL, kCmpStages, false, OP>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    return e;
}

}  // namespace

namespace pip {

cudaError_t stream_kernels_setup()
{
    cudaError_t e = setup_stream_type<false>();
    if (e == cudaSuccess) e = stream_kernels_setup_i32();
    if (e == cudaSuccess) e = set_cmp_attr<kTmaSign>();
    if (e == cudaSuccess) e = set_cmp_attr<kTmaRay>();
    return e;
}

cudaError_t launch_cmp_stream(const pip_tables *t, const float *pts, int64_t M, uint32_t *mask, int op,
                              cudaStream_t s)
{
    return op == kTmaSign ? launch_cmp_ne<kTmaSign>(t, pts, M, mask, s) : launch_cmp_ne<kTmaRay>(t, pts, M, mask, s);
}

int stream_variant_count() { return kNumStreamVariants; }

cudaError_t launch_stream_pipelined(const pip_tables *t, const void *pts, bool ints, int64_t M, uint32_t *mask,
                                    bool early, bool disc, cudaStream_t s)
{
    return ints ? launch_stream_pipelined_i32(t, pts, M, mask, early, disc, s)
                : launch_stream_type<false>(t, pts, M, mask, early, disc, s);
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
    // a cached choice for this kernel, GPU and shape skips the timing runs
    const std::string key = tuning_key(t, "stream", num_points, pdtype);
    int cached = -1;
    float cached_ms = 0.f;
    if (tuning_lookup(key, &cached, &cached_ms) && cached >= 0 && cached < kNumStreamVariants) {
        t->stream_variant = cached;
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
    tuning_store(key, best, best_t);
    t->stream_variant = best;
    if (best_variant) *best_variant = best;
    if (best_ms) *best_ms = best_t;
    return PIP_OK;
}
