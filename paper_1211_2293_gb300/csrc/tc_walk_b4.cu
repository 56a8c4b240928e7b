// tc_walk_b4.cu -- the walk + force kernels for 4 bodies per lane
// (groups of up to 128 bodies), every tile and mode.
#include "tc_walk.cuh"

namespace tc {

cudaError_t prepare_walk_b4(const WalkConfig& c, int num_sms, int* grid, size_t* smem)
{
    return dispatch_b<4, PrepareF>(c, &c, num_sms, grid, smem);
}

cudaError_t launch_walk_b4(const WalkArgs& a, const WalkConfig& c, int grid, size_t smem, cudaStream_t s)
{
    return dispatch_b<4, LaunchF>(c, &a, &c, grid, smem, s);
}

}  // namespace tc
