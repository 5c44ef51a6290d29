// pip_noalloc.cu -- pip_test_single_noalloc: the single-polygon inclusion test
// with no device allocation at all.
//
// Who needs this: callers that cannot call cudaMalloc when they test points.
// A vehicle's collision checker running in a fixed-rate control loop cannot
// afford cudaMalloc's latency and implicit synchronisation; a plug-in hosted
// by an application that owns the device memory pool (or a safety-certified
// deployment with a fixed memory budget) is not allowed to allocate at all.
// pip_prepare allocates its tables and refine queue, so such callers get this
// entry point instead: it builds the polygon's tables and runs the float32
// bulk test and the exact refine exactly as pip_prepare + pip_test do, but
// every scratch byte lives in one file-scope __device__ array below.
//
// Limits and sharing: one polygon of 3..64 vertices and at most
// kNoAllocMaxPoints points per call (the refine queue must hold every point
// in the worst case).  The array exists once per GPU that loads the library,
// for the life of the process; every call shares it and it keeps the last
// call's contents, so each call clears its counters first, and calls that
// overlap on the GPU (different streams, or different host threads without
// ordering) race on it.  The scratch address is looked up once per device and
// kept; cudaDeviceReset destroys the context that holds the array, so after a
// reset this entry point must not be called again in the same process.
#include <mutex>

#include "pip_prepare_kernel.cuh"
#include "pip_test_kernels.cuh"

namespace {

constexpr int64_t kNoAllocMaxPoints = int64_t(1) << 20;

struct NoAllocScratch {
    PolyInfo poly;
    double2 g0;
    int32_t worst;
    unsigned int qcount;
    int32_t voffs[2];
    double2 gk[kMaxEdges];
    float4 coef[kMaxEdges];
    float4 coefn[kMaxEdges];
    int4 iedge[kMaxEdges];
    uint32_t queue[kNoAllocMaxPoints];
};

// The scratch itself: about 4 MiB per GPU.  In host code this name is only a
// host-side stand-in; its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
NoAllocScratch *g_scratch_ptr[kMaxDevices] = {};
int g_num_sms[kMaxDevices] = {};

// Once per device, with that device current: the device address of the
// scratch array and the SM count.
pip_status setup_device(int dev, NoAllocScratch **scratch, int *num_sms)
{
    if (dev < 0 || dev >= kMaxDevices) return PIP_E_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (g_scratch_ptr[dev] == nullptr) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || ptr == nullptr)
            return PIP_E_CUDA;
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
            return PIP_E_CUDA;
        g_scratch_ptr[dev] = (NoAllocScratch *)ptr;
        g_num_sms[dev] = sms;
    }
    *scratch = g_scratch_ptr[dev];
    *num_sms = g_num_sms[dev];
    return PIP_OK;
}

// Clears what must start at zero and states the one polygon's offsets.
__global__ void noalloc_begin_kernel(NoAllocScratch *s, int32_t n)
{
    if (threadIdx.x == 0) {
        s->voffs[0] = 0;
        s->voffs[1] = n;
        s->worst = 0;
        s->qcount = 0;
    }
}

}  // namespace

extern "C" pip_status pip_test_single_noalloc(const void *d_vertices, pip_dtype vdtype,
                                              int32_t num_vertices, const void *d_points,
                                              pip_dtype pdtype, int64_t num_points,
                                              uint32_t *d_mask, int32_t *d_status, void *stream)
{
    if (vdtype != PIP_F32 && vdtype != PIP_I32) return PIP_E_INVALID_ARG;
    if (pdtype != PIP_F32 && pdtype != PIP_I32) return PIP_E_INVALID_ARG;
    if (num_vertices < kMinEdges || num_vertices > kMaxEdges) return PIP_E_INVALID_ARG;
    if (d_vertices == nullptr || !aligned(d_vertices, 8)) return PIP_E_INVALID_ARG;
    if (num_points < 0) return PIP_E_INVALID_ARG;
    if (num_points > kNoAllocMaxPoints) return PIP_E_CAPACITY;
    if (num_points > 0 && (d_points == nullptr || !aligned(d_points, 8))) return PIP_E_INVALID_ARG;
    if (num_points > 0 && (d_mask == nullptr || !aligned(d_mask, 4))) return PIP_E_INVALID_ARG;
    if (d_status != nullptr && !aligned(d_status, 4)) return PIP_E_INVALID_ARG;

    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return PIP_E_CUDA;
    NoAllocScratch *s = nullptr;
    int num_sms = 0;
    pip_status st = setup_device(dev, &s, &num_sms);
    if (st != PIP_OK) return st;

    cudaStream_t cs = (cudaStream_t)stream;
    noalloc_begin_kernel<<<1, 32, 0, cs>>>(s, num_vertices);
    prepare_kernel<<<1, 32, 0, cs>>>(d_vertices, vdtype, s->voffs, 1, num_vertices, &s->g0, s->gk,
                                     s->coef, s->coefn, &s->poly, &s->worst);
    if (vdtype == PIP_I32) int_edge_kernel<<<1, 32, 0, cs>>>(&s->poly, (const int2 *)d_vertices, 1, s->iedge);
    PIP_CUDA_TRY(cudaGetLastError());
    if (d_status != nullptr)
        PIP_CUDA_TRY(cudaMemcpyAsync(d_status, &s->worst, sizeof(int32_t), cudaMemcpyDeviceToDevice, cs));
    if (num_points == 0) return PIP_OK;

    const bool ints = pdtype == PIP_I32, v16 = aligned(d_points, 16);
    const int64_t chunks = (num_points + Chunk<kF>::kPoints - 1) / Chunk<kF>::kPoints;
    const int64_t want = (chunks + kWarps - 1) / kWarps;
#define NOALLOC_STREAM(I, V)                                                                        \
    {                                                                                               \
        auto k = stream_kernel<kF, I, V>;                                                           \
        const int blocks = (int)max((int64_t)1, min((int64_t)blocks_for(k, num_sms, kThreads), want)); \
        k<<<blocks, kThreads, 0, cs>>>(&s->poly, s->coef, d_points, num_points, d_mask, s->queue,    \
                                       &s->qcount);                                                 \
    }
    if (ints) { if (v16) NOALLOC_STREAM(true, true) else NOALLOC_STREAM(true, false) }
    else { if (v16) NOALLOC_STREAM(false, true) else NOALLOC_STREAM(false, false) }
#undef NOALLOC_STREAM
    PIP_CUDA_TRY(cudaGetLastError());

    RefineArgs A{};
    A.poly = &s->poly;
    A.coef = s->coef;
    A.g0 = &s->g0;
    A.gk = s->gk;
    A.verts = d_vertices;
    A.vdtype = vdtype;
    A.P = 1;
    A.pts = d_points;
    A.pdtype = pdtype;
    A.M = num_points;
    A.poffs = nullptr;
    A.queue = s->queue;
    A.qcount = &s->qcount;
    A.mask = d_mask;
    A.first_hit = nullptr;
    A.iedge = s->iedge;
    // as pip_test: int64 cross products, one thread a point, when both inputs
    // are int32; otherwise the per-thread fp64 Voronoi form with the exact
    // orientation predicate behind it
    if (vdtype == PIP_I32 && pdtype == PIP_I32)
        refine_kernel<true><<<num_sms * 8, kThreads, 0, cs>>>(A, kSingle);
    else
        refine_kernel<false><<<num_sms * 2, kThreads, 0, cs>>>(A, kSingle);
    PIP_CUDA_TRY(cudaGetLastError());
    return PIP_OK;
}
