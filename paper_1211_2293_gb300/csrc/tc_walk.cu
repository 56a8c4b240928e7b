// tc_walk.cu -- launchers of the walk + force kernels: the group size picks
// the bodies per lane (groups of up to 32 bodies, down to the paper's
// one-body lists: one; 64: two; 128: four) and the tile size the object
// (tc_walk_unit.cu, compiled once per pair) holding those kernels.
#include <cstddef>

#include "tc_internal.cuh"

namespace tc {

#define TC_WALK_DECL(B, T)                                                                                 \
    cudaError_t prepare_walk_b##B##_t##T(const WalkConfig& c, int num_sms, int* grid, size_t* smem);       \
    cudaError_t launch_walk_b##B##_t##T(const WalkArgs& a, const WalkConfig& c, int grid, size_t smem,     \
                                        cudaStream_t s);
#define TC_WALK_DECL_B(B) TC_WALK_DECL(B, 64) TC_WALK_DECL(B, 128) TC_WALK_DECL(B, 256)
TC_WALK_DECL_B(1)
TC_WALK_DECL_B(2)
TC_WALK_DECL_B(4)
#undef TC_WALK_DECL_B
#undef TC_WALK_DECL

// the walk's one memset spans the counters and the totals behind them
static_assert(offsetof(Info, interactions) == offsetof(Info, work) + sizeof(Info::work) &&
                  offsetof(Info, bodies) == offsetof(Info, interactions) + 2 * sizeof(unsigned long long),
              "work counters and interaction totals must be contiguous");

namespace {

int bodies_per_lane(int gmax)
{
    if (gmax >= 1 && gmax <= 32) return 1;
    return gmax == 64 ? 2 : (gmax == 128 ? 4 : 0);
}

}  // namespace

#define TC_WALK_PICK(fn, ...)                                                              \
    switch (bodies_per_lane(c.gmax) * 1000 + c.tile) {                                    \
    case 1064: return fn##_b1_t64(__VA_ARGS__);                                           \
    case 1128: return fn##_b1_t128(__VA_ARGS__);                                          \
    case 1256: return fn##_b1_t256(__VA_ARGS__);                                          \
    case 2064: return fn##_b2_t64(__VA_ARGS__);                                           \
    case 2128: return fn##_b2_t128(__VA_ARGS__);                                          \
    case 2256: return fn##_b2_t256(__VA_ARGS__);                                          \
    case 4064: return fn##_b4_t64(__VA_ARGS__);                                           \
    case 4128: return fn##_b4_t128(__VA_ARGS__);                                          \
    case 4256: return fn##_b4_t256(__VA_ARGS__);                                          \
    default: return cudaErrorInvalidValue;                                                \
    }

cudaError_t prepare_walk(const WalkConfig& c, int num_sms, int* grid, size_t* smem)
{
    TC_WALK_PICK(prepare_walk, c, num_sms, grid, smem)
}

cudaError_t launch_walk(const WalkArgs& a, const WalkConfig& c, int grid, size_t smem, cudaStream_t s,
                        bool reset_totals)
{
    if (bodies_per_lane(c.gmax) == 0) return cudaErrorInvalidValue;
    if (a.work_slot < 0 || a.work_slot >= 4) return cudaErrorInvalidValue;
    // the counters and the totals behind them in one memset (list export
    // leaves the last force phase's totals alone)
    if (reset_totals)
        cudaMemsetAsync(&a.info->work[0], 0,
                        a.list_cells ? sizeof(a.info->work)
                                     : sizeof(a.info->work) + 3 * sizeof(unsigned long long), s);
    TC_WALK_PICK(launch_walk, a, c, grid, smem, s)
}

#undef TC_WALK_PICK

}  // namespace tc
