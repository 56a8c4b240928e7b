// tc_walk.cu -- launchers of the walk + force kernels: the group size picks
// the translation unit holding the kernels for that many bodies per lane
// (groups of up to 32 bodies, down to the paper's one-body lists: one).
#include "tc_internal.cuh"

namespace tc {

cudaError_t prepare_walk_b1(const WalkConfig& c, int num_sms, int* grid, size_t* smem);
cudaError_t prepare_walk_b2(const WalkConfig& c, int num_sms, int* grid, size_t* smem);
cudaError_t prepare_walk_b4(const WalkConfig& c, int num_sms, int* grid, size_t* smem);
cudaError_t launch_walk_b1(const WalkArgs& a, const WalkConfig& c, int grid, size_t smem, cudaStream_t s);
cudaError_t launch_walk_b2(const WalkArgs& a, const WalkConfig& c, int grid, size_t smem, cudaStream_t s);
cudaError_t launch_walk_b4(const WalkArgs& a, const WalkConfig& c, int grid, size_t smem, cudaStream_t s);

cudaError_t prepare_walk(const WalkConfig& c, int num_sms, int* grid, size_t* smem)
{
    if (c.gmax >= 1 && c.gmax <= 32) return prepare_walk_b1(c, num_sms, grid, smem);
    switch (c.gmax) {
    case 64: return prepare_walk_b2(c, num_sms, grid, smem);
    case 128: return prepare_walk_b4(c, num_sms, grid, smem);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_walk(const WalkArgs& a, const WalkConfig& c, int grid, size_t smem, cudaStream_t s,
                        bool reset_totals)
{
    cudaMemsetAsync(&a.info->work, 0, sizeof(uint32_t), s);
    if (reset_totals && !a.list_cells)  // list export leaves the last force phase's totals alone
        cudaMemsetAsync(&a.info->interactions, 0, 3 * sizeof(unsigned long long), s);
    if (c.gmax >= 1 && c.gmax <= 32) return launch_walk_b1(a, c, grid, smem, s);
    switch (c.gmax) {
    case 64: return launch_walk_b2(a, c, grid, smem, s);
    case 128: return launch_walk_b4(a, c, grid, smem, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace tc
