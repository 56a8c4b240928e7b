// tc_band.cu -- the learned far-field correction evaluated after the walk.
//
// The split walk (k_walk_ws) records every band cell of every group -- an
// accepted cell holding two bodies or more with s >= band d -- with the
// cell's network row (the same row k_walk builds inside its walk: d/s and s/r
// at the group's box centre beside the node's precomputed features, as 16
// BF16 values), its factor G M s^2 / r^4 and its group.  k_band_eval then
// runs the network on all recorded rows on the fifth-generation tensor cores,
// 128 rows per tile.  A CTA holds two independent pipelines (warpgroups of
// 128 threads sharing the weights); in each:
//   * thread t copies the row of entry t of its tile into shared memory, in
//     the K-major layout of the tensor core's operands (8-row x 16-byte core
//     matrices), and loads the next tile's entry while this one runs;
//   * one thread issues the three layers as tcgen05.mma (kind::f16: BF16
//     operands, FP32 accumulators in tensor memory): 128 x 64 x 16, four
//     128 x 64 x 16 steps, four 128 x 16 x 16 steps (the three outputs padded
//     to 16 columns), each layer's completion arriving on the pipeline's
//     mbarrier (tcgen05.commit);
//   * between layers every thread reads its row of the accumulator from
//     tensor memory (tcgen05.ld; a warp reaches the lane quarter of its rank
//     in the warpgroup), adds the bias, applies the ReLU while rounding to
//     BF16 and writes the next layer's operand row back to shared memory;
//   * the output row is scaled by its factor, and runs of one group within a
//     warp's 32 rows are summed by shuffles, one atomic add per run.
// The weights are laid out once per CTA.  Tensor memory: 64 columns per
// pipeline, every layer's accumulator in the same columns once the previous
// one has been read, 128 per CTA, at most four CTAs per SM (shared memory is
// sized for it), so an allocation never waits.  Every wait on an mbarrier is
// bounded; a wait that runs out sets kErrWorkLoop and the pipeline stops; the
// CTA frees its tensor memory when both have stopped.  k_band_apply adds each
// group's sum to the accelerations of its bodies.
#include "tc_walk.cuh"

namespace tc {

namespace {

constexpr int kTcRows = 128;        // rows per tile = threads per pipeline = tensor-memory lanes
constexpr int kTcPipes = 2;         // pipelines (warpgroups) per CTA
constexpr int kTcCols = 64 * kTcPipes;  // tensor-memory columns per CTA
constexpr int kTcBlocksPerSm = 3;   // 3 x 128 of the SM's 512 columns (registers: 85 a thread)
constexpr int kTcN3 = 16;           // output layer padded to 16 columns
constexpr size_t kTcSmemBytes = 72 * 1024;  // requested per CTA: at most three CTAs per SM

struct TcSmem {
    alignas(128) uint8_t a1[kTcPipes][kTcRows * kMlpInPad * 2];  // rows: 128 x 16 BF16
    alignas(128) uint8_t a2[kTcPipes][kTcRows * kMlpHid * 2];    // hidden rows: 128 x 64 BF16
    alignas(128) uint8_t w1[kMlpHid * kMlpInPad * 2];  // [out][in], K-major
    alignas(128) uint8_t w2[kMlpHid * kMlpHid * 2];
    alignas(128) uint8_t w3[kTcN3 * kMlpHid * 2];
    float b1[kMlpHid], b2[kMlpHid], b3[kTcN3];
    float xscale[kMlpInPad], xoff[kMlpInPad], yscale[kMlpOutPad];
    uint64_t mbar[kTcPipes];
    uint32_t tmem;
};
static_assert(sizeof(TcSmem) <= kTcSmemBytes, "band-eval shared memory");

// byte offset of element (row, k) of a K-major operand with K columns: 8-row
// x 8-element core matrices of 128 bytes, the K-adjacent ones contiguous
// (leading byte offset 128), the 8-row groups K / 8 core matrices apart
// (stride byte offset K x 16)
__device__ __forceinline__ uint32_t kmaj_off(int row, int k, int K)
{
    return (uint32_t)((row >> 3) * (K * 16) + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// shared-memory matrix descriptor: start address, leading and stride byte
// offsets (each >> 4), descriptor version 1 (bits 46-47), no swizzle
__device__ __forceinline__ uint64_t umma_desc(const void* p, uint32_t lbo, uint32_t sbo)
{
    const uint32_t adr = smem_addr(p);
    return (uint64_t)((adr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16
// A and B (bits 7-9 = 1, 10-12 = 1), both K-major, N / 8 at bits 17-22,
// M / 16 at bits 24-28
__host__ __device__ constexpr uint32_t umma_idesc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// the issuing thread's MMAs so far arrive on the barrier once complete
__device__ __forceinline__ void umma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_free(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy writes to shared memory, then read by the tensor cores
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16 consecutive accumulator columns of the thread's lane (its warp's lane
// quarter), waited for in the same statement so no use can precede the load
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int k = 0; k < 16; k++) v[k] = __uint_as_float(r[k]);
}

// one layer's epilogue for the thread's row: relu(D + b) rounded to BF16,
// written as the next operand's row (K = 64), 16 columns at a time
__device__ __forceinline__ void hidden_epilogue(uint32_t taddr, const float* b, uint8_t* dst, int row)
{
#pragma unroll
    for (int c = 0; c < 4; c++) {
        float v[16];
        tmem_ld16(taddr + 16 * c, v);
        uint32_t w[8];
#pragma unroll
        for (int j = 0; j < 8; j++) w[j] = pack_relu(v[2 * j] + b[16 * c + 2 * j], v[2 * j + 1] + b[16 * c + 2 * j + 1]);
        *reinterpret_cast<uint4*>(dst + kmaj_off(row, 16 * c, kMlpHid)) = make_uint4(w[0], w[1], w[2], w[3]);
        *reinterpret_cast<uint4*>(dst + kmaj_off(row, 16 * c + 8, kMlpHid)) = make_uint4(w[4], w[5], w[6], w[7]);
    }
}

// named barrier of one warpgroup (ids 1, 2; 0 is the CTA's)
__device__ __forceinline__ void wg_sync(int id) { asm volatile("bar.sync %0, 128;" ::"r"(id) : "memory"); }

// bounded wait on the pipeline's layer barrier by its 128 threads; the
// result is the same in all of them
__device__ __forceinline__ bool layer_wait(uint64_t* bar, uint32_t parity, int id)
{
    const uint32_t mine = mbar_wait(bar, parity) ? 1u : 0u;
    uint32_t all;
    asm volatile(
        "{\n .reg .pred pi, po;\n setp.ne.b32 pi, %1, 0;\n bar.red.and.pred po, %2, 128, pi;\n"
        " selp.u32 %0, 1, 0, po;\n}"
        : "=r"(all)
        : "r"(mine), "r"(id)
        : "memory");
    return all != 0;
}

__global__ void __launch_bounds__(kTcRows * kTcPipes, kTcBlocksPerSm)
    k_band_eval(WalkArgs a, const MlpDev* __restrict__ model, float* __restrict__ gcorr,
                unsigned long long* __restrict__ evals)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    TcSmem& S = *reinterpret_cast<TcSmem*>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int pipe = tid / kTcRows, t = tid % kTcRows, bar_id = 1 + pipe;
    if ((*(volatile const int32_t*)&a.info->err & kErrCapacity) != 0) return;  // uniform: nothing allocated yet
    // the network, once per CTA: weights [out][in] in the K-major layout
    for (int i = tid; i < kMlpHid * kMlpInPad; i += blockDim.x) {
        const int n = i / kMlpInPad, k = i % kMlpInPad;
        *reinterpret_cast<__nv_bfloat16*>(S.w1 + kmaj_off(n, k, kMlpInPad)) = model->w1[k * kMlpHid + n];
    }
    for (int i = tid; i < kMlpHid * kMlpHid; i += blockDim.x) {
        const int n = i / kMlpHid, k = i % kMlpHid;
        *reinterpret_cast<__nv_bfloat16*>(S.w2 + kmaj_off(n, k, kMlpHid)) = model->w2[k * kMlpHid + n];
    }
    for (int i = tid; i < kTcN3 * kMlpHid; i += blockDim.x) {
        const int n = i / kMlpHid, k = i % kMlpHid;
        *reinterpret_cast<__nv_bfloat16*>(S.w3 + kmaj_off(n, k, kMlpHid)) =
            n < kMlpOutPad ? model->w3[k * kMlpOutPad + n] : __float2bfloat16(0.f);
    }
    for (int i = tid; i < kMlpHid; i += blockDim.x) {
        S.b1[i] = model->b1[i];
        S.b2[i] = model->b2[i];
    }
    if (tid < kTcN3) S.b3[tid] = tid < kMlpOutPad ? model->b3[tid] : 0.f;
    if (tid < kMlpInPad) {
        S.xscale[tid] = model->frag.xscale[tid];
        S.xoff[tid] = model->frag.xoff[tid];
    }
    if (tid < kMlpOutPad) S.yscale[tid] = model->frag.yscale[tid];
    if (tid < kTcPipes) mbar_init(&S.mbar[tid], 1);
    if (tid == 0) asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (warp == 0) tmem_alloc(&S.tmem, kTcCols);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t acc = S.tmem + 64 * pipe;                 // the pipeline's columns
    const uint32_t lane_row = (uint32_t)((warp & 3) * 32) << 16;  // the warp's lane quarter
    uint8_t* a1 = S.a1[pipe];
    uint8_t* a2 = S.a2[pipe];
    uint64_t* bar = &S.mbar[pipe];
    constexpr uint32_t kId64 = umma_idesc(kTcRows, kMlpHid), kId16 = umma_idesc(kTcRows, kTcN3);

    const int64_t lim = (a.band_cap / kBandChunk) * kBandChunk;
    const int64_t total = (int64_t)(*a.band_n < (unsigned long long)lim ? *a.band_n : (unsigned long long)lim);
    const int64_t G = a.info->G;
    const int64_t stride = (int64_t)gridDim.x * kTcPipes * kTcRows;
    // entry e: (node, group); node -1 (a chunk's unused tail) or out of
    // range (a walk that gave up part-way) is no cell; then the node's and
    // the group's records
    const int64_t M = a.info->M;
    struct In {
        int2 bv;
        float4 r0, r1;
        BandNode q;
    };
    auto usable = [&](int2 bv) { return bv.x >= 0 && bv.x < M && bv.y >= 0 && bv.y < G; };
    auto fetch_rest = [&](int2 bv, In& in) {
        in.bv = bv;
        if (usable(bv)) {
            in.r0 = a.grec[2 * (int64_t)bv.y];
            in.r1 = a.grec[2 * (int64_t)bv.y + 1];
            in.q = band_node_load(a.nt, bv.x);
        }
    };
    auto entry = [&](int64_t e) -> int2 { return e < total ? a.band[e] : make_int2(-1, 0); };
    unsigned long long nev = 0;
    uint32_t parity = 0;
    bool ok = true;
    int64_t base = ((int64_t)blockIdx.x * kTcPipes + pipe) * kTcRows;
    // a tile's inputs arrive one tile ahead: the entry two tiles ahead and,
    // for the next tile, its node and group records are loaded before the
    // current tile's layers run
    In cur;
    fetch_rest(entry(base + t), cur);
    int2 ahead = entry(base + stride + t);
    for (; base < total && ok; base += stride) {
        // ---- the thread's row
        const bool valid = usable(cur.bv);
        uint32_t w[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
        float fac = 0.f;
        if (valid) {
            const int4 rc = make_int4(__float_as_int(cur.r1.x), __float_as_int(cur.r1.y), __float_as_int(cur.r1.z), 0);
            const float xgc[3] = {cur.r0.x, cur.r0.y, cur.r0.z};
            band_row_from(S.xscale, S.xoff, cur.q, rc, cur.r0.w, cur.r1.w, 1.0f / cur.r1.w, xgc, a.G, w, fac);
            nev++;
        }
        const int grp = valid ? cur.bv.y : -1;
        *reinterpret_cast<uint4*>(a1 + kmaj_off(t, 0, kMlpInPad)) = make_uint4(w[0], w[1], w[2], w[3]);
        *reinterpret_cast<uint4*>(a1 + kmaj_off(t, 8, kMlpInPad)) = make_uint4(w[4], w[5], w[6], w[7]);
        // the next tile's inputs, in flight while this one runs
        fetch_rest(ahead, cur);
        ahead = entry(base + 2 * stride + t);
        fence_async_smem();
        tc_fence_before();
        wg_sync(bar_id);
        // ---- layer 1: 128 x 64, K = 16
        if (t == 0) {
            tc_fence_after();
            umma_bf16(acc, umma_desc(a1, 128, kMlpInPad * 16), umma_desc(S.w1, 128, kMlpInPad * 16), kId64, 0u);
            umma_commit(bar);
        }
        ok = layer_wait(bar, parity, bar_id);
        parity ^= 1u;
        if (!ok) break;
        tc_fence_after();
        hidden_epilogue(acc + lane_row, S.b1, a2, t);
        fence_async_smem();
        tc_fence_before();
        wg_sync(bar_id);
        // ---- layer 2: 128 x 64, K = 64 in four steps of 16 (layer 1's
        // accumulators have been read: the same columns)
        if (t == 0) {
            tc_fence_after();
#pragma unroll
            for (int k = 0; k < 4; k++)
                umma_bf16(acc, umma_desc(a2 + 256 * k, 128, kMlpHid * 16), umma_desc(S.w2 + 256 * k, 128, kMlpHid * 16),
                          kId64, k > 0 ? 1u : 0u);
            umma_commit(bar);
        }
        ok = layer_wait(bar, parity, bar_id);
        parity ^= 1u;
        if (!ok) break;
        tc_fence_after();
        hidden_epilogue(acc + lane_row, S.b2, a2, t);  // layer 2 has read a2: reuse it
        fence_async_smem();
        tc_fence_before();
        wg_sync(bar_id);
        // ---- layer 3: 128 x 16 (3 used), K = 64
        if (t == 0) {
            tc_fence_after();
#pragma unroll
            for (int k = 0; k < 4; k++)
                umma_bf16(acc, umma_desc(a2 + 256 * k, 128, kMlpHid * 16), umma_desc(S.w3 + 256 * k, 128, kMlpHid * 16),
                          kId16, k > 0 ? 1u : 0u);
            umma_commit(bar);
        }
        ok = layer_wait(bar, parity, bar_id);
        parity ^= 1u;
        if (!ok) break;
        tc_fence_after();
        float c[3];
        {
            float v[16];
            tmem_ld16(acc + lane_row, v);
#pragma unroll
            for (int i = 0; i < 3; i++) c[i] = (v[i] + S.b3[i]) * fac * S.yscale[i];
        }
        // ---- runs of one group within the warp: suffix sums inside each run
        // (a group's cells are contiguous in the record over any 32 entries),
        // the run's first row adds the run's total
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const float x0 = __shfl_down_sync(0xffffffffu, c[0], o);
            const float x1 = __shfl_down_sync(0xffffffffu, c[1], o);
            const float x2 = __shfl_down_sync(0xffffffffu, c[2], o);
            const int go = __shfl_down_sync(0xffffffffu, grp, o);
            if (lane + o < 32 && go == grp) {
                c[0] += x0;
                c[1] += x1;
                c[2] += x2;
            }
        }
        const int gprev = __shfl_up_sync(0xffffffffu, grp, 1);
        if (grp >= 0 && (lane == 0 || gprev != grp)) {
            atomicAdd(&gcorr[3 * (int64_t)grp + 0], c[0]);
            atomicAdd(&gcorr[3 * (int64_t)grp + 1], c[1]);
            atomicAdd(&gcorr[3 * (int64_t)grp + 2], c[2]);
        }
        tc_fence_before();
        wg_sync(bar_id);  // the next tile rewrites the rows and the accumulators
    }
    if (!ok && t == 0) atomicOr(&a.info->err, kErrWorkLoop);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_free(S.tmem, kTcCols);
    }
    // the evaluations, per warp
#pragma unroll
    for (int o = 16; o; o >>= 1) nev += __shfl_xor_sync(0xffffffffu, nev, o);
    if (lane == 0 && evals && nev) atomicAdd(evals, nev);
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
    // persistent CTAs, four per SM; the kernel reads the record's length on
    // the device, so the grid is fixed and a captured step replays it
    cudaFuncSetAttribute(k_band_eval, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmemBytes);
    const int blocks = kTcBlocksPerSm * sm_count();
    k_band_eval<<<blocks, kTcRows * kTcPipes, kTcSmemBytes, s>>>(a, (const MlpDev*)model, gcorr, evals);
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
