// pip_selftest.cu -- the failure path of the pipelined kernels, exercised
// without a fault: a bounded mbarrier wait that nothing completes.
//
// One CTA, one thread does the work: it arms barrier `copied` for a 4 KiB
// bulk copy and starts it, then waits on barrier `never` (count 1, nobody
// arrives) with the caller's cycle limit.  mbar_wait_limit gives up, records
// PIP_E_TIMEOUT in the error word and returns false; the thread then waits,
// bounded by the kernels' own limit, for its copy to land -- the same drain a
// producer does before it leaves -- and the CTA exits normally.
#include "pip_tma.cuh"

using namespace pip;

namespace {

constexpr uint32_t kSelftestBytes = 4096;

__global__ void __launch_bounds__(32) selftest_wait_kernel(const void *__restrict__ src, long long limit,
                                                           int *__restrict__ err)
{
    __shared__ __align__(128) unsigned char buf[kSelftestBytes];
    __shared__ uint64_t bars[2];
    uint64_t *copied = &bars[0], *never = &bars[1];
    if (threadIdx.x == 0) {
        mbar_init(copied, 1);
        mbar_init(never, 1);
        fence_mbar_init();
    }
    __syncwarp();
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(copied, kSelftestBytes);
        bulk_copy_g2s(buf, src, kSelftestBytes, copied);
        if (!mbar_wait_limit(never, 0u, err, limit)) {
            // gave up (PIP_E_TIMEOUT recorded): let the copy in flight land
            mbar_wait(copied, 0u, err);
        }
    }
    __syncwarp();
}

}  // namespace

extern "C" pip_status pip_selftest_wait_timeout(pip_tables *t, const void *d_scratch, int64_t limit_cycles,
                                                void *stream)
{
    pip_status st = check_tables(t);
    if (st != PIP_OK) return st;
    if (d_scratch == nullptr || !aligned(d_scratch, 16) || limit_cycles < 1 || limit_cycles > (1ll << 31))
        return PIP_E_INVALID_ARG;
    selftest_wait_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(d_scratch, (long long)limit_cycles, t->d_error);
    return cudaGetLastError() == cudaSuccess ? PIP_OK : PIP_E_CUDA;
}
