// pip_stream_i32.cu -- the pipelined single-polygon test for int32 points
// (instantiations compiled apart from the float32 ones).
#include "pip_stream_launch.cuh"

namespace pip {

cudaError_t stream_kernels_setup_i32() { return setup_stream_type<true>(); }

cudaError_t launch_stream_pipelined_i32(const pip_tables *t, const void *pts, int64_t M, uint32_t *mask,
                                        bool early, bool disc, cudaStream_t s)
{
    return launch_stream_type<true>(t, pts, M, mask, early, disc, s);
}

}  // namespace pip
