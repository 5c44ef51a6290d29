// pip_stream_launch.cuh -- launch side of the pipelined single-polygon kernel
// (pip_stream_tma.cuh): the polygon's row and coefficients as launch
// parameters, the edge-count and tile-shape variants.  Included by
// pip_stream.cu (float32 points) and pip_stream_i32.cu (int32 points), so that
// the two sets of instantiations compile in parallel.
#pragma once

#include "pip_kernels.cuh"
#include "pip_stream_tma.cuh"

namespace {

using namespace pip;


// Variants of the pipelined kernel: (points per lane per stage, stages,
// consumer warps).  Since a consumer warp hands its stage back once the
// points are in registers, fewer and larger stages (bigger bulk copies) pay;
// the last shape is one CTA of 16 consumer warps a SM with 96 KB stages.
struct StreamVariant {
    int ppl, stages, warps;
};
constexpr StreamVariant kStreamVariants[] = {{16, 3, 8}, {16, 2, 8}, {24, 2, 8}, {20, 2, 8}, {24, 2, 16}};
constexpr int kNumStreamVariants = sizeof(kStreamVariants) / sizeof(kStreamVariants[0]);
// the refine queue's slack (pip_prepare) holds kStreamSlackPerSm points a SM:
// one tile per CTA at the CTAs a SM that launch_tma_one allows
static_assert(StreamCfg<24, 2, false, 16>::kTile <= kStreamSlackPerSm, "a stream tile larger than the slack");

template <int NE, int PPL, int STAGES, bool INT, bool EARLY = false, bool DISC = false, int CW = kConsumerWarps>
cudaError_t launch_tma_one(const pip_tables *t, const void *pts, int64_t M, uint32_t *mask, cudaStream_t s)
{
    using C = StreamCfg<PPL, STAGES, DISC, CW>;
    auto k = stream_tma_kernel<NE, PPL, STAGES, INT, kTmaVoronoi, EARLY, DISC, CW>;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, C::kThreads, C::kSmem) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    // the scratch queue holds one tile of slack per CTA: kStreamSlackPerSm points a SM
    if (per_sm > kStreamSlackPerSm / C::kTile) per_sm = kStreamSlackPerSm / C::kTile;
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
    sp.tin = sp.ok ? hp.tin : 0.f;
    sp.tout = sp.ok ? hp.tout : -INFINITY;
    for (int k = 0; k < kParamEdges; ++k) {
        float4 c = make_float4(0.f, 0.f, INFINITY, 0.f);
        if (!sp.ok) { if (k == 0) c.z = -INFINITY; }
        else if (k < sp.n) c = t->h_coef[k];
        sp.wx[k] = c.x;
        sp.wy[k] = c.y;
        sp.t[k] = c.z;
    }
    k<<<blocks, C::kThreads, C::kSmem, s>>>(sp, t->d_poly, t->d_coef, t->d_g0, t->d_gk, t->d_verts,
                                            t->vdtype, pts, M, mask, t->d_queue,
                                            (StreamCounters *)t->d_stream_ctr, t->d_qcount, t->d_error);
    return cudaGetLastError();
}

template <int PPL, int STAGES, bool INT, bool EARLY = false, bool DISC = false, int CW = kConsumerWarps>
cudaError_t launch_tma_ne(const pip_tables *t, const void *pts, int64_t M, uint32_t *mask, cudaStream_t s)
{
    // the polygon's edge count is known on the host from the vertex count
    const int n = t->V;
    if (n <= 4) return launch_tma_one<4, PPL, STAGES, INT, EARLY, DISC, CW>(t, pts, M, mask, s);
    if (n <= 8) return launch_tma_one<8, PPL, STAGES, INT, EARLY, DISC, CW>(t, pts, M, mask, s);
    if (n <= 12) return launch_tma_one<12, PPL, STAGES, INT, EARLY, DISC, CW>(t, pts, M, mask, s);
    if (n <= 16) return launch_tma_one<16, PPL, STAGES, INT, EARLY, DISC, CW>(t, pts, M, mask, s);
    return launch_tma_one<0, PPL, STAGES, INT, EARLY, DISC, CW>(t, pts, M, mask, s);
}

template <int NE, int PPL, int STAGES, bool INT, bool EARLY = false, bool DISC = false, int CW = kConsumerWarps>
cudaError_t set_attr_one()
{
    return cudaFuncSetAttribute(stream_tma_kernel<NE, PPL, STAGES, INT, kTmaVoronoi, EARLY, DISC, CW>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)StreamCfg<PPL, STAGES, DISC, CW>::kSmem);
}

template <int PPL, int STAGES, bool INT, bool EARLY = false, bool DISC = false, int CW = kConsumerWarps>
cudaError_t set_smem_attr()
{
    cudaError_t e = set_attr_one<4, PPL, STAGES, INT, EARLY, DISC, CW>();
    if (e == cudaSuccess) e = set_attr_one<8, PPL, STAGES, INT, EARLY, DISC, CW>();
    if (e == cudaSuccess) e = set_attr_one<12, PPL, STAGES, INT, EARLY, DISC, CW>();
    if (e == cudaSuccess) e = set_attr_one<16, PPL, STAGES, INT, EARLY, DISC, CW>();
    if (e == cudaSuccess) e = set_attr_one<0, PPL, STAGES, INT, EARLY, DISC, CW>();
    return e;
}

template <bool INT, bool DISC = false>
cudaError_t launch_stream_tma(const pip_tables *t, const void *pts, int64_t M, uint32_t *mask,
                              cudaStream_t s)
{
    switch (t->stream_variant) {
    case 1: return launch_tma_ne<16, 2, INT, false, DISC>(t, pts, M, mask, s);
    case 2: return launch_tma_ne<24, 2, INT, false, DISC>(t, pts, M, mask, s);
    case 3: return launch_tma_ne<20, 2, INT, false, DISC>(t, pts, M, mask, s);
    case 4: return launch_tma_ne<24, 2, INT, false, DISC, 16>(t, pts, M, mask, s);
    default: return launch_tma_ne<16, 3, INT, false, DISC>(t, pts, M, mask, s);
    }
}

template <bool INT>
cudaError_t set_all_attr()
{
    cudaError_t e = set_smem_attr<16, 3, INT, true>();  // the early-exit mode's one tile shape
    // the disc filter's forms of the four tile shapes
    if (e == cudaSuccess) e = set_smem_attr<16, 3, INT, false, true>();
    if (e == cudaSuccess) e = set_smem_attr<16, 2, INT, false, true>();
    if (e == cudaSuccess) e = set_smem_attr<24, 2, INT, false, true>();
    if (e == cudaSuccess) e = set_smem_attr<20, 2, INT, false, true>();
    if (e == cudaSuccess) e = set_smem_attr<24, 2, INT, false, true, 16>();
    if (e == cudaSuccess) e = set_smem_attr<16, 3, INT>();
    if (e == cudaSuccess) e = set_smem_attr<16, 2, INT>();
    if (e == cudaSuccess) e = set_smem_attr<24, 2, INT>();
    if (e == cudaSuccess) e = set_smem_attr<20, 2, INT>();
    if (e == cudaSuccess) e = set_smem_attr<24, 2, INT, false, false, 16>();
    return e;
}

// One point type: the pipelined kernel (or its disc-filter form) at the
// chosen tile shape; the early-exit mode at the default shape (16 points per
// lane, 3 stages).
template <bool INT>
cudaError_t launch_stream_type(const pip_tables *t, const void *pts, int64_t M, uint32_t *mask, bool early,
                               bool disc, cudaStream_t s)
{
    if (disc) return launch_stream_tma<INT, true>(t, pts, M, mask, s);
    if (early) return launch_tma_ne<16, 3, INT, true>(t, pts, M, mask, s);
    return launch_stream_tma<INT>(t, pts, M, mask, s);
}

template <bool INT>
cudaError_t setup_stream_type()
{
    return set_all_attr<INT>();
}

}  // namespace
