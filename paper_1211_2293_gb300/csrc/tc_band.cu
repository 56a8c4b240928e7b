// tc_band.cu -- the learned far-field correction evaluated after the walk.
//
// The split walk (k_walk_ws) records every band cell of every group -- an
// accepted cell holding two bodies or more with s >= band d -- as a (node,
// group) pair, and each group's box centre.  k_band_eval then runs the
// network on all of them at once: a warp takes 32 recorded pairs, builds
// their rows (the same row k_walk builds inside its walk: d/s and s/r at the
// group's centre beside the node's precomputed features), evaluates them as
// two 16-row tiles on the tensor cores, scales each output by its factor
// G M s^2 / r^4 and adds it to its group's sum; runs of pairs of one group
// (the record keeps a group's cells together) are summed in the warp first,
// so one atomic add per run reaches memory.  k_band_apply adds each group's
// sum to the accelerations of its bodies.
#include "tc_walk.cuh"

namespace tc {

namespace {

constexpr int kEvalWarps = 4;

__global__ void __launch_bounds__(kEvalWarps * 32) k_band_eval(WalkArgs a, const MlpDev* __restrict__ model,
                                                                float* __restrict__ gcorr,
                                                                unsigned long long* __restrict__ evals)
{
    __shared__ MlpFrag m;
    __shared__ uint32_t rows_s[kEvalWarps][32 * kRowW];
    __shared__ float contrib_s[kEvalWarps][32][3];
    __shared__ int grp_s[kEvalWarps][32];
    if ((*(volatile const int32_t*)&a.info->err & kErrCapacity) != 0) return;
    for (int i = threadIdx.x; i < (int)(sizeof(MlpFrag) / 4); i += blockDim.x)
        reinterpret_cast<uint32_t*>(&m)[i] = reinterpret_cast<const uint32_t*>(&model->frag)[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t* rows = rows_s[w];
    const int64_t lim = (a.band_cap / kBandChunk) * kBandChunk;
    const int64_t total = (int64_t)(*a.band_n < (unsigned long long)lim ? *a.band_n : (unsigned long long)lim);
    const int64_t M = a.info->M, G = a.info->G;
    unsigned long long nev = 0;
    for (int64_t t0 = ((int64_t)blockIdx.x * kEvalWarps + w) * 32; t0 < total;
         t0 += (int64_t)gridDim.x * kEvalWarps * 32) {
        const int64_t e = t0 + lane;
        const int2 bv = e < total ? a.band[e] : make_int2(-1, 0);
        // every entry of a taken chunk is written (cells or -1); the range
        // checks keep a walk that gave up part-way from sending a stale
        // entry out of bounds
        const bool valid = bv.x >= 0 && bv.x < M && bv.y >= 0 && bv.y < G;
        uint32_t wr[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
        float fac = 0.f;
        if (valid) {
            const int g = bv.y;
            const int4 rc = a.nt.c[a.gref[g]];
            const SysParams& SP = a.sysp[a.sys_of[a.gfirst[g]]];
            const float xgc[3] = {a.gcentre[3 * (int64_t)g], a.gcentre[3 * (int64_t)g + 1],
                                  a.gcentre[3 * (int64_t)g + 2]};
            band_row(m, bv.x, a.nt, rc, SP.uf, SP.Lf, 1.0f / SP.Lf, xgc, a.G, wr, fac);
        }
        nev += __popc(__ballot_sync(0xffffffffu, valid));
        uint32_t* r = rows + lane * kRowW;
#pragma unroll
        for (int k = 0; k < 8; k++) r[k] = wr[k];
        r[8] = __float_as_uint(valid ? fac : 0.f);
        grp_s[w][lane] = valid ? bv.y : -1;
        __syncwarp();
        const int gq = lane >> 2, q = lane & 3;
#pragma unroll
        for (int t = 0; t < 32; t += 16) {
            const uint32_t* r0 = rows + (t + gq) * kRowW;
            const uint32_t* r1 = rows + (t + gq + 8) * kRowW;
            const uint32_t x[4] = {r0[q], r1[q], r0[q + 4], r1[q + 4]};
            float y[4];
            mlp16_infer(m, x, y, lane);
            const float f0 = __uint_as_float(r0[8]), f1 = __uint_as_float(r1[8]);
            if (q == 0) {
                contrib_s[w][t + gq][0] = y[0] * f0 * m.yscale[0];
                contrib_s[w][t + gq][1] = y[1] * f0 * m.yscale[1];
                contrib_s[w][t + gq + 8][0] = y[2] * f1 * m.yscale[0];
                contrib_s[w][t + gq + 8][1] = y[3] * f1 * m.yscale[1];
            } else if (q == 1) {
                contrib_s[w][t + gq][2] = y[0] * f0 * m.yscale[2];
                contrib_s[w][t + gq + 8][2] = y[2] * f1 * m.yscale[2];
            }
        }
        __syncwarp();
        // the first row of each run of one group sums the run and adds it
        const int g = grp_s[w][lane];
        const bool head = g >= 0 && (lane == 0 || grp_s[w][lane - 1] != g);
        if (head) {
            float c[3] = {0.f, 0.f, 0.f};
            for (int j = lane; j < 32 && grp_s[w][j] == g; j++) {
                c[0] += contrib_s[w][j][0];
                c[1] += contrib_s[w][j][1];
                c[2] += contrib_s[w][j][2];
            }
            atomicAdd(&gcorr[3 * (int64_t)g + 0], c[0]);
            atomicAdd(&gcorr[3 * (int64_t)g + 1], c[1]);
            atomicAdd(&gcorr[3 * (int64_t)g + 2], c[2]);
        }
        __syncwarp();
    }
    if (lane == 0 && evals) atomicAdd(evals, nev);
}

// every body of group g gains gcorr[g] (one warp per group)
__global__ void k_band_apply(const Info* info, const int32_t* __restrict__ gfirst, const uint32_t* __restrict__ perm,
                             const float* __restrict__ gcorr, float* __restrict__ acc)
{
    if ((*(volatile const int32_t*)&info->err & kErrCapacity) != 0) return;
    const int64_t G = info->G;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t g = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); g < G; g += warps) {
        const float c0 = gcorr[3 * g], c1 = gcorr[3 * g + 1], c2 = gcorr[3 * g + 2];
        for (int i = gfirst[g] + lane; i < gfirst[g + 1]; i += 32) {
            const int64_t o = perm[i];
            acc[3 * o + 0] += c0;
            acc[3 * o + 1] += c1;
            acc[3 * o + 2] += c2;
        }
    }
}

}  // namespace

void launch_band_eval(const WalkArgs& a, const void* model, float* gcorr, unsigned long long* evals, cudaStream_t s)
{
    // enough warps to fill the device; the kernel reads the record's length
    // on the device, so the grid is fixed and a captured step replays it
    const int blocks = 8 * sm_count();
    k_band_eval<<<blocks, kEvalWarps * 32, 0, s>>>(a, (const MlpDev*)model, gcorr, evals);
    count_launches(1);
}

void launch_band_apply(const Info* info, int64_t cap_g, const int32_t* gfirst, const uint32_t* perm,
                       const float* gcorr, float* acc, cudaStream_t s)
{
    int64_t g = (cap_g + 7) / 8;
    if (g > 8 * sm_count()) g = 8 * sm_count();
    k_band_apply<<<(unsigned)(g < 1 ? 1 : g), 256, 0, s>>>(info, gfirst, perm, gcorr, acc);
    count_launches(1);
}

}  // namespace tc
