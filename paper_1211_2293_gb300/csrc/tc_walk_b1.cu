// tc_walk_b1.cu -- the walk + force kernels for 1 body per lane
// (groups of up to 32 bodies), every tile and mode.
#include "tc_walk.cuh"

namespace tc {

cudaError_t prepare_walk_b1(const WalkConfig& c, int num_sms, int* grid, size_t* smem)
{
    return dispatch_b<1, PrepareF>(c, &c, num_sms, grid, smem);
}

cudaError_t launch_walk_b1(const WalkArgs& a, const WalkConfig& c, int grid, size_t smem, cudaStream_t s)
{
    return dispatch_b<1, LaunchF>(c, &a, &c, grid, smem, s);
}

}  // namespace tc
