// tc_walk_unit.cu -- the walk + force kernels for TC_WALK_B bodies per lane
// and list tiles of TC_WALK_TILE entries, every mode.  The build compiles this file once per
// (B, tile) in {1, 2, 4} x {64, 128, 256}, defining the two macros.
#include "tc_walk.cuh"

#if !defined(TC_WALK_B) || !defined(TC_WALK_TILE)
#error "compile with -DTC_WALK_B=<1|2|4> -DTC_WALK_TILE=<64|128|256>"
#endif

#define TC_PASTE4(a, b, c, d) a##b##c##d
#define TC_UNIT_NAME(stem, b, t) TC_PASTE4(stem, b, _t, t)

namespace tc {

cudaError_t TC_UNIT_NAME(prepare_walk_b, TC_WALK_B, TC_WALK_TILE)(const WalkConfig& c, int num_sms, int* grid,
                                                                  size_t* smem)
{
    return dispatch_modes<TC_WALK_B, TC_WALK_TILE, PrepareF>(c, &c, num_sms, grid, smem);
}

cudaError_t TC_UNIT_NAME(launch_walk_b, TC_WALK_B, TC_WALK_TILE)(const WalkArgs& a, const WalkConfig& c, int grid,
                                                                 size_t smem, cudaStream_t s)
{
    return dispatch_modes<TC_WALK_B, TC_WALK_TILE, LaunchF>(c, &a, &c, grid, smem, s);
}

}  // namespace tc
