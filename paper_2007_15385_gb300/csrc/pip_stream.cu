// pip_stream.cu -- the pipelined single-polygon test for float32 points, the
// dispatch by point type, and the tile-shape API and autotuner.
#include "pip_stream_launch.cuh"

using namespace pip;

namespace pip {

cudaError_t stream_kernels_setup()
{
    cudaError_t e = setup_stream_type<false>();
    if (e == cudaSuccess) e = stream_kernels_setup_i32();
    return e;
}

int stream_variant_count() { return kNumStreamVariants; }

cudaError_t launch_stream_pipelined(const pip_tables *t, const void *pts, bool ints, int64_t M, uint32_t *mask,
                                    cudaStream_t s)
{
    return ints ? launch_stream_pipelined_i32(t, pts, M, mask, s) : launch_stream_type<false>(t, pts, M, mask, s);
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
