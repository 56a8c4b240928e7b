// tc_sort.cu -- device-wide exclusive scan and stable LSD radix sort.
//
// The Morton keys are sorted with ties kept in original-index order (a
// stable sort), so bodies sharing a leaf are ordered by key, then by index.
// Both primitives are written here (no CUB); they are HBM/L2-bound map and
// scatter passes.
#include "tc_internal.cuh"

namespace tc {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;  // 4096

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 16;                         // per thread
constexpr int kSortTile = kSortThreads * kSortItems;   // 4096 items per block
constexpr int kWarpItems = 32 * kSortItems;            // 512 items per warp

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// exclusive block scan of one value per thread; returns the block total
template <int THREADS>
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t x, uint32_t& total, uint32_t* sm)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t incl = warp_incl_scan(x);
    if (lane == 31) sm[w] = incl;
    __syncthreads();
    if (w == 0) {
        uint32_t v = lane < THREADS / 32 ? sm[lane] : 0;
        uint32_t vi = warp_incl_scan(v);
        if (lane < THREADS / 32) sm[lane] = vi - v;
        if (lane == THREADS / 32 - 1) sm[32] = vi;
    }
    __syncthreads();
    uint32_t r = sm[w] + incl - x;
    total = sm[32];
    __syncthreads();
    return r;
}

__global__ void k_scan_reduce(const uint32_t* __restrict__ in, int64_t n, uint32_t* __restrict__ bsum)
{
    __shared__ uint32_t sm[33];
    int64_t base = (int64_t)blockIdx.x * kScanTile;
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        int64_t k = base + (int64_t)i * kScanThreads + threadIdx.x;
        if (k < n) s += in[k];
    }
    uint32_t tot;
    block_excl_scan<kScanThreads>(s, tot, sm);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// single block: exclusive scan of nb partials, in place; total -> *total
__global__ void k_scan_top(uint32_t* __restrict__ bsum, int64_t nb, uint32_t* __restrict__ total)
{
    __shared__ uint32_t sm[33];
    uint32_t carry = 0;
    for (int64_t c = 0; c < nb; c += 1024) {
        int64_t k = c + threadIdx.x;
        uint32_t v = k < nb ? bsum[k] : 0;
        uint32_t tot;
        uint32_t e = block_excl_scan<1024>(v, tot, sm);
        if (k < nb) bsum[k] = carry + e;
        carry += tot;
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void k_scan_down(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, int64_t n,
                            const uint32_t* __restrict__ bsum)
{
    __shared__ uint32_t sm[33];
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        int64_t k = base + i;
        v[i] = k < n ? in[k] : 0;
        s += v[i];
    }
    uint32_t tot;
    uint32_t e = block_excl_scan<kScanThreads>(s, tot, sm) + bsum[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        int64_t k = base + i;
        if (k < n) out[k] = e;
        e += v[i];
    }
}

template <typename K>
__global__ void k_radix_hist(const K* __restrict__ keys, int64_t n, int shift, uint32_t* __restrict__ hist,
                             int nb)
{
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kSortTile;
#pragma unroll 4
    for (int i = 0; i < kSortItems; i++) {
        int64_t k = base + (int64_t)i * kSortThreads + threadIdx.x;
        if (k < n) atomicAdd(&h[(uint32_t)(keys[k] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nb + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: warp w of block b owns items [b*T + w*512, +512), taken in
// 16 rounds of 32 in index order.  Within a round, lanes holding equal digits
// find each other with __match_any_sync; the lowest such lane reserves their
// slots in the warp's per-digit counter.  Warp counters are then offset by
// the counts of the earlier warps and by the digit's global offset.
template <typename K>
__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(
    const K* __restrict__ kin, const uint32_t* __restrict__ vin, K* __restrict__ kout,
    uint32_t* __restrict__ vout, int64_t n, int shift, const uint32_t* __restrict__ offs, int nb)
{
    __shared__ uint32_t wh[kSortWarps][256];
    __shared__ uint32_t gb[256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kSortWarps * 256; i += kSortThreads) (&wh[0][0])[i] = 0;
    gb[threadIdx.x] = offs[(int64_t)threadIdx.x * nb + blockIdx.x];
    __syncthreads();

    const int64_t wbase = (int64_t)blockIdx.x * kSortTile + (int64_t)w * kWarpItems;
    const uint32_t lt = (1u << lane) - 1u;
    K key[kSortItems];
    uint32_t val[kSortItems];
    uint32_t rank[kSortItems];
#pragma unroll
    for (int r = 0; r < kSortItems; r++) {
        int64_t k = wbase + r * 32 + lane;
        bool ok = k < n;
        key[r] = ok ? kin[k] : K(0);
        val[r] = ok ? vin[k] : 0u;
        uint32_t d = ok ? ((uint32_t)(key[r] >> shift) & 255u) : 256u + lane;
        uint32_t peers = __match_any_sync(0xffffffffu, d);
        int leader = __ffs(peers) - 1;
        uint32_t old = 0;
        if (ok && lane == leader) {
            old = wh[w][d];
            wh[w][d] = old + __popc(peers);
        }
        old = __shfl_sync(0xffffffffu, old, leader);
        rank[r] = old + __popc(peers & lt);
        __syncwarp();
    }
    __syncthreads();
    {
        uint32_t run = 0;
        const int d = threadIdx.x;
#pragma unroll
        for (int ww = 0; ww < kSortWarps; ww++) {
            uint32_t c = wh[ww][d];
            wh[ww][d] = run + gb[d];
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortItems; r++) {
        int64_t k = wbase + r * 32 + lane;
        if (k < n) {
            uint32_t d = (uint32_t)(key[r] >> shift) & 255u;
            uint32_t p = wh[w][d] + rank[r];
            kout[p] = key[r];
            vout[p] = val[r];
        }
    }
}

}  // namespace

int64_t scan_blocksum_size(int64_t n) { return (n + kScanTile - 1) / kScanTile + 1; }

void scan_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total_dev, uint32_t* blocksum,
              cudaStream_t s)
{
    if (n <= 0) {
        if (total_dev) cudaMemsetAsync(total_dev, 0, sizeof(uint32_t), s);
        return;
    }
    int64_t nb = (n + kScanTile - 1) / kScanTile;
    k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, blocksum);
    k_scan_top<<<1, 1024, 0, s>>>(blocksum, nb, total_dev);
    k_scan_down<<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, blocksum);
    count_launches(3);
}

int64_t radix_hist_size(int64_t n) { return 256 * ((n + kSortTile - 1) / kSortTile); }

template <typename K>
static void radix_sort_impl(K* keys, uint32_t* vals, int64_t n, int nbits, SortBufs& b, K* keys_alt,
                            cudaStream_t s)
{
    if (n <= 1) return;
    int nb = (int)((n + kSortTile - 1) / kSortTile);
    int64_t nh = (int64_t)256 * nb;
    K* ka = keys;
    uint32_t* va = vals;
    K* kb = keys_alt;
    uint32_t* vb = b.vals_alt;
    int passes = 0;
    for (int shift = 0; shift < nbits; shift += 8) {
        k_radix_hist<K><<<nb, kSortThreads, 0, s>>>(ka, n, shift, b.hist, nb);
        scan_u32(b.hist, b.hist, nh, nullptr, b.blocksum, s);
        k_radix_scatter<K><<<nb, kSortThreads, 0, s>>>(ka, va, kb, vb, n, shift, b.hist, nb);
        count_launches(2);
        K* tk = ka; ka = kb; kb = tk;
        uint32_t* tv = va; va = vb; vb = tv;
        passes++;
    }
    if (passes & 1) {
        cudaMemcpyAsync(keys, ka, n * sizeof(K), cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(vals, va, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
    }
}

void radix_sort_u64(uint64_t* keys, uint32_t* vals, int64_t n, int nbits, SortBufs& b, cudaStream_t s)
{
    radix_sort_impl<uint64_t>(keys, vals, n, nbits, b, b.keys_alt, s);
}

void radix_sort_u32(uint32_t* keys, uint32_t* vals, int64_t n, int nbits, SortBufs& b,
                    uint32_t* keys_alt32, cudaStream_t s)
{
    radix_sort_impl<uint32_t>(keys, vals, n, nbits, b, keys_alt32, s);
}

}  // namespace tc
