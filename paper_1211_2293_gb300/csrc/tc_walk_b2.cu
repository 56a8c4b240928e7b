// tc_walk_b2.cu -- the walk + force kernels for 2 bodies per lane
// (groups of up to 64 bodies), every tile and mode.
#include "tc_walk.cuh"

namespace tc {

cudaError_t prepare_walk_b2(const WalkConfig& c, int num_sms, int* grid, size_t* smem)
{
    return dispatch_b<2, PrepareF>(c, &c, num_sms, grid, smem);
}

cudaError_t launch_walk_b2(const WalkArgs& a, const WalkConfig& c, int grid, size_t smem, cudaStream_t s)
{
    return dispatch_b<2, LaunchF>(c, &a, &c, grid, smem, s);
}

}  // namespace tc
