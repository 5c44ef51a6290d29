// pip_calibrate.cu -- pip_fma_peak: a pure float32 FMA kernel, the measured
// denominator of the FP32 roofline that the dense all-pairs test and the
// penalty kernels are reported against.  The paper has no counterpart.
//
// Every thread runs 8 independent FMA chains (x = x * a + b) in an unrolled
// loop of 16 steps, 128 FMAs per iteration against 3 loop instructions, with
// 8 blocks of 256 threads per SM, so that the FMA pipe, not latency or issue
// of other instructions, sets the rate.  With a in (0, 1) the chains converge
// to b / (1 - a) and never reach denormals or infinities.  The sum of the
// chains is stored only when it equals a value it never takes, which keeps
// the compiler from removing the work without writing anything.
#include "pip_internal.cuh"

namespace {

constexpr int kPeakThreads = 256;
constexpr int kPeakChains = 8;
constexpr int kPeakUnroll = 16;

__global__ void __launch_bounds__(kPeakThreads) fma_peak_kernel(float *__restrict__ sink, int iters, float a,
                                                                 float b)
{
    float x[kPeakChains];
#pragma unroll
    for (int i = 0; i < kPeakChains; ++i) x[i] = (float)(threadIdx.x & 7) * 0.125f + (float)i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < kPeakUnroll; ++r) {
#pragma unroll
            for (int i = 0; i < kPeakChains; ++i) x[i] = fmaf(x[i], a, b);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kPeakChains; ++i) s += x[i];
    if (s == -1.0f) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" pip_status pip_fma_peak(int32_t blocks_per_sm, int32_t iters, float *d_sink, int64_t sink_floats,
                                   void *stream, int64_t *fmas)
{
    if (blocks_per_sm < 1 || blocks_per_sm > 64 || iters < 1 || d_sink == nullptr || fmas == nullptr)
        return PIP_E_INVALID_ARG;
    int dev = 0, sms = 0;
    PIP_CUDA_TRY(cudaGetDevice(&dev));
    PIP_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t blocks = (int64_t)blocks_per_sm * sms;
    if (sink_floats < blocks * kPeakThreads) return PIP_E_INVALID_ARG;
    fma_peak_kernel<<<(unsigned)blocks, kPeakThreads, 0, (cudaStream_t)stream>>>(d_sink, iters, 0.9999f,
                                                                                  1e-4f);
    PIP_CUDA_TRY(cudaGetLastError());
    *fmas = blocks * kPeakThreads * (int64_t)iters * kPeakUnroll * kPeakChains;
    return PIP_OK;
}
