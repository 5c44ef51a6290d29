// pip_host.cu -- pip_test_host: the inclusion test end to end on host
// buffers (points in host memory, mask back to host memory), for callers
// outside a GPU framework.  The paper has no counterpart; it is the
// transfer-overlapped form of pip_prepare's tables + pip_test.
//
// The points move in pieces on a copy stream of the tables' own; piece i's
// test waits on an event of its copy and runs on the caller's stream, then
// its mask words are read back on that stream.  So the copy of piece i + 1
// overlaps the test and read-back of piece i, and the host link, not the
// kernel, sets the pace.  One cudaMemcpyAsync per piece and direction.
#include "pip_internal.cuh"

using namespace pip;

extern "C" pip_status pip_test_host(pip_tables *t, const void *h_points, pip_dtype pdtype, int64_t num_points,
                                    void *d_points, uint32_t *d_mask, uint32_t *h_mask, int32_t pieces,
                                    void *stream)
{
    pip_status st = check_tables(t);
    if (st != PIP_OK) return st;
    if (pdtype != PIP_F32 && pdtype != PIP_I32) return PIP_E_INVALID_ARG;
    if (num_points < 0 || pieces < 1 || pieces > 64) return PIP_E_INVALID_ARG;
    if (num_points == 0) return pip_test(t, d_points, pdtype, 0, nullptr, PIP_MASK, d_mask, nullptr, stream);
    if (h_points == nullptr || d_points == nullptr || d_mask == nullptr || h_mask == nullptr)
        return PIP_E_INVALID_ARG;
    if (!aligned(d_points, 16) || !aligned(d_mask, 16) || !aligned(h_mask, 4)) return PIP_E_INVALID_ARG;
    if (num_points > t->capacity) return PIP_E_CAPACITY;
    if (!t->host_ready) {
        PIP_CUDA_TRY(cudaStreamCreateWithFlags(&t->host_copy_stream, cudaStreamNonBlocking));
        for (int i = 0; i < 65; ++i)
            PIP_CUDA_TRY(cudaEventCreateWithFlags(&t->host_events[i], cudaEventDisableTiming));
        t->host_ready = 1;
    }
    cudaStream_t s = (cudaStream_t)stream, cs = t->host_copy_stream;
    // the staging buffers are free once the caller's earlier work is done
    PIP_CUDA_TRY(cudaEventRecord(t->host_events[64], s));
    PIP_CUDA_TRY(cudaStreamWaitEvent(cs, t->host_events[64], 0));
    // pieces start at multiples of 128 points: whole, 16-byte aligned mask words
    int64_t piece = (num_points + pieces - 1) / pieces;
    piece = ((piece + 127) / 128) * 128;
    const char *hp = (const char *)h_points;
    char *dp = (char *)d_points;
    int i = 0;
    for (int64_t a = 0; a < num_points; a += piece, ++i) {
        const int64_t b = a + piece < num_points ? a + piece : num_points;
        PIP_CUDA_TRY(cudaMemcpyAsync(dp + a * 8, hp + a * 8, (size_t)(b - a) * 8, cudaMemcpyHostToDevice, cs));
        PIP_CUDA_TRY(cudaEventRecord(t->host_events[i], cs));
        PIP_CUDA_TRY(cudaStreamWaitEvent(s, t->host_events[i], 0));
        st = pip_test(t, dp + a * 8, pdtype, b - a, nullptr, PIP_MASK, d_mask + a / 32, nullptr, stream);
        if (st != PIP_OK) return st;
        const int64_t w0 = a / 32, w1 = (b + 31) / 32;
        PIP_CUDA_TRY(cudaMemcpyAsync(h_mask + w0, d_mask + w0, (size_t)(w1 - w0) * 4, cudaMemcpyDeviceToHost, s));
    }
    return PIP_OK;
}
