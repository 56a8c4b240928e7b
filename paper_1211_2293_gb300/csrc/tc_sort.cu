// tc_sort.cu -- device-wide exclusive scan and stable LSD radix sort.
//
// The Morton keys are sorted with ties kept in original-index order (a
// stable sort), so bodies sharing a leaf are ordered by key, then by index.
// Both primitives are written here (no CUB); they are HBM/L2-bound map and
// scatter passes.
#include <mutex>

#include "tc_internal.cuh"

namespace tc {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;  // 4096

constexpr int kMaxDevices = 64;
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

// PREFIX: the block's offset is the sum of the raw partials of the blocks
// before it (no k_scan_top; the last block writes the total) -- for up to
// kScanFusedBlocks blocks, where that sum is cheaper than another launch
constexpr int64_t kScanFusedBlocks = 256;

template <bool PREFIX>
__global__ void k_scan_down(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, int64_t n,
                            const uint32_t* __restrict__ bsum, uint32_t* __restrict__ total)
{
    __shared__ uint32_t sm[33];
    uint32_t off = 0;
    if (PREFIX) {
        uint32_t t = 0;
        for (int64_t j = threadIdx.x; j < (int64_t)blockIdx.x; j += kScanThreads) t += bsum[j];
        block_excl_scan<kScanThreads>(t, off, sm);  // off = the block-wide sum
    } else {
        off = bsum[blockIdx.x];
    }
    // the tile through shared memory: coalesced loads and stores, each
    // thread scanning kScanItems consecutive items (padded every 32 words,
    // so the threads' strided reads hit distinct banks)
    __shared__ uint32_t tile[kScanTile + kScanTile / 32];
    auto pad = [](int p) { return p + (p >> 5); };
    const int64_t t0 = (int64_t)blockIdx.x * kScanTile;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        const int p = i * kScanThreads + threadIdx.x;
        tile[pad(p)] = t0 + p < n ? in[t0 + p] : 0u;
    }
    __syncthreads();
    uint32_t v[kScanItems];
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        v[i] = tile[pad(threadIdx.x * kScanItems + i)];
        s += v[i];
    }
    uint32_t tot;
    uint32_t e = block_excl_scan<kScanThreads>(s, tot, sm) + off;
    if (PREFIX && total && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *total = off + tot;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        tile[pad(threadIdx.x * kScanItems + i)] = e;
        e += v[i];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        const int p = i * kScanThreads + threadIdx.x;
        if (t0 + p < n) out[t0 + p] = tile[pad(p)];
    }
}

// ------------------------------------------------------------------ radix sort
// Onesweep LSD radix sort (8-bit digits): one kernel computes the global
// digit histograms of every pass, one kernel turns them into exclusive
// offsets, then each pass is a single kernel whose tiles find their place by
// decoupled look-back (Merrill & Garland's single-pass prefix scan): a tile
// publishes its per-digit count ("aggregate"), then adds up its
// predecessors' counts walking back until it meets an inclusive prefix, and
// publishes its own inclusive prefix.  Tiles take their index from an atomic
// counter in launch order, so a tile only ever waits for tiles that have
// already started and publish before they look back themselves.  Every wait
// is bounded; a tile that gives up sets the error word and writes nothing.
constexpr unsigned long long kFlagAgg = 1ull << 62;
constexpr unsigned long long kFlagPrefix = 2ull << 62;
constexpr unsigned kLookbackMaxPolls = 1u << 22;  // about a second of polling

template <typename K>
__global__ void __launch_bounds__(kSortThreads) k_sort_hist_all(const K* __restrict__ keys, int64_t n_host,
                                                                const int64_t* __restrict__ n_dev, int npass,
                                                                int shift0, uint32_t* __restrict__ ghist)
{
    __shared__ uint32_t h[8][256];
    const int64_t n = n_dev ? min(*n_dev, n_host) : n_host;  // never past the buffers
    for (int i = threadIdx.x; i < 8 * 256; i += kSortThreads) (&h[0][0])[i] = 0;
    __syncthreads();
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const K key = keys[k];
        for (int p = 0; p < npass; p++) atomicAdd(&h[p][(uint32_t)(key >> (shift0 + 8 * p)) & 255u], 1u);
    }
    __syncthreads();
    for (int p = 0; p < npass; p++) {
        const uint32_t c = h[p][threadIdx.x];
        if (c) atomicAdd(&ghist[p * 256 + threadIdx.x], c);
    }
}

// digit histograms of the system passes: the multiset of systems does not
// depend on the order, so they are counted from sys_of directly
__global__ void __launch_bounds__(kSortThreads) k_sort_hist_sys(const uint32_t* __restrict__ sys_of, int64_t n,
                                                                int npass, uint32_t* __restrict__ ghist)
{
    __shared__ uint32_t h[2][256];
    for (int i = threadIdx.x; i < 2 * 256; i += kSortThreads) (&h[0][0])[i] = 0;
    __syncthreads();
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t sy = sys_of[k];
        for (int p = 0; p < npass; p++) atomicAdd(&h[p][(sy >> (8 * p)) & 255u], 1u);
    }
    __syncthreads();
    for (int p = 0; p < npass; p++) {
        const uint32_t c = h[p][threadIdx.x];
        if (c) atomicAdd(&ghist[p * 256 + threadIdx.x], c);
    }
}

// exclusive scan of each pass's 256 digit counts, in place
__global__ void __launch_bounds__(256) k_sort_offsets(uint32_t* __restrict__ ghist, int npass)
{
    __shared__ uint32_t sm[33];
    for (int p = 0; p < npass; p++) {
        uint32_t tot;
        const uint32_t e = block_excl_scan<256>(ghist[p * 256 + threadIdx.x], tot, sm);
        ghist[p * 256 + threadIdx.x] = e;
    }
}

__device__ __forceinline__ void sort_cp16(void* smem, const void* gmem)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)), "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void sort_cp_wait() { asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory"); }

// Dynamic shared memory of one onesweep tile: the tile's items in their
// locally sorted order (keys, then values), staged so that the write to the
// output is one contiguous run per digit instead of a scatter per item.
template <typename K>
constexpr size_t onesweep_smem() { return (size_t)kSortTile * (sizeof(K) + sizeof(uint32_t)); }

// SYS: the digit is taken from the system of the value's body, sys_of[val]
// Three tiles per SM (80 registers): the build at 2^22 takes 3 % less time
// than with two, at 2^20 the same.
template <typename K, bool SYS>
__global__ void __launch_bounds__(kSortThreads, 3) k_onesweep(const K* __restrict__ kin, const uint32_t* __restrict__ vin,
                                                           K* __restrict__ kout, uint32_t* __restrict__ vout,
                                                           int64_t n_host, const int64_t* __restrict__ n_dev,
                                                           int shift, const uint32_t* __restrict__ goff,
                                                           unsigned long long* status, uint32_t* tile_counter,
                                                           int32_t* err, const uint32_t* __restrict__ sys_of)
{
    const int64_t n = n_dev ? min(*n_dev, n_host) : n_host;  // never past the buffers
    extern __shared__ __align__(16) unsigned char dsm[];
    K* skey = reinterpret_cast<K*>(dsm);
    uint32_t* sval = reinterpret_cast<uint32_t*>(dsm + (size_t)kSortTile * sizeof(K));
    __shared__ uint32_t wh[kSortWarps][256];
    __shared__ uint32_t base[256];
    __shared__ uint32_t tstart[256];
    __shared__ uint32_t wsum[kSortWarps];
    __shared__ int tile_sh;
    __shared__ int fail_sh;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kSortWarps * 256; i += kSortThreads) (&wh[0][0])[i] = 0;
    if (threadIdx.x == 0) {
        tile_sh = (int)atomicAdd(tile_counter, 1u);
        fail_sh = 0;
    }
    __syncthreads();
    const int tile = tile_sh;
    if ((int64_t)tile * kSortTile >= n) return;  // a tile past the device-side count: nothing to do
    const int tile_n = (int)min((int64_t)kSortTile, n - (int64_t)tile * kSortTile);

    // the tile's items into the staging buffer in their input order: a full
    // tile by cp.async, every 16-byte chunk in flight at once, instead of
    // one dependent round of loads per ranking round
    const int64_t tbase = (int64_t)tile * kSortTile;
    if (tile_n == kSortTile && ((reinterpret_cast<uintptr_t>(kin + tbase) | reinterpret_cast<uintptr_t>(vin + tbase)) & 15u) == 0) {
        const unsigned char* gk = reinterpret_cast<const unsigned char*>(kin + tbase);
        const unsigned char* gv = reinterpret_cast<const unsigned char*>(vin + tbase);
        unsigned char* sk = reinterpret_cast<unsigned char*>(skey);
        unsigned char* sv = reinterpret_cast<unsigned char*>(sval);
        for (int i = threadIdx.x; i < (int)(kSortTile * sizeof(K) / 16); i += kSortThreads) sort_cp16(sk + 16 * i, gk + 16 * i);
        for (int i = threadIdx.x; i < (int)(kSortTile * sizeof(uint32_t) / 16); i += kSortThreads)
            sort_cp16(sv + 16 * i, gv + 16 * i);
        sort_cp_wait();
    } else {
        for (int i = threadIdx.x; i < tile_n; i += kSortThreads) {
            skey[i] = kin[tbase + i];
            sval[i] = vin[tbase + i];
        }
    }
    __syncthreads();

    // stable ranks within the tile (warp w owns items [tile*T + w*512, +512),
    // in 16 rounds of 32; equal digits of a round find each other with
    // __match_any_sync and the lowest lane reserves their slots)
    const int64_t wbase = tbase + (int64_t)w * kWarpItems;
    const uint32_t lt = (1u << lane) - 1u;
    K key[kSortItems];
    uint32_t val[kSortItems];
    uint32_t rank[kSortItems];
#pragma unroll
    for (int r = 0; r < kSortItems; r++) {
        const int64_t k = wbase + r * 32 + lane;
        const bool ok = k < n;
        const int li = w * kWarpItems + r * 32 + lane;
        key[r] = ok ? skey[li] : K(0);
        val[r] = ok ? sval[li] : 0u;
        const uint32_t dig = SYS ? (ok ? sys_of[val[r]] >> shift : 0u) : (uint32_t)(key[r] >> shift);
        const uint32_t d = ok ? (dig & 255u) : 256u + lane;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const int leader = __ffs(peers) - 1;
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

    // per digit: offsets of the warps inside the tile and the tile's count;
    // the digits' starts inside the tile (block scan); then the decoupled
    // look-back over the preceding tiles
    const int d = threadIdx.x;
    uint32_t run = 0;
#pragma unroll
    for (int ww = 0; ww < kSortWarps; ww++) {
        const uint32_t c = wh[ww][d];
        wh[ww][d] = run;
        run += c;
    }
    {
        uint32_t x = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[w] = x;
        __syncthreads();
        uint32_t before = 0;
        for (int ww = 0; ww < w; ww++) before += wsum[ww];
        tstart[d] = before + x - run;
    }
    {
        volatile unsigned long long* st = status;
        if (tile == 0) {
            st[d] = kFlagPrefix | run;
            base[d] = goff[d];
        } else {
            st[(int64_t)tile * 256 + d] = kFlagAgg | run;
            uint32_t excl = 0;
            int64_t k = tile - 1;
            unsigned polls = 0;
            bool fail = false;
            while (k >= 0) {
                const unsigned long long v = st[k * 256 + d];
                const unsigned long long f = v & (3ull << 62);
                if (f == 0) {
                    if (++polls > kLookbackMaxPolls) {
                        fail = true;
                        break;
                    }
                    if (polls > 64) __nanosleep(32);
                    continue;
                }
                excl += (uint32_t)v;
                if (f == kFlagPrefix) break;
                k--;
            }
            st[(int64_t)tile * 256 + d] = kFlagPrefix | (uint32_t)(excl + run);
            base[d] = goff[d] + excl;
            if (fail) {
                fail_sh = 1;
                atomicOr(err, kErrWorkLoop);
            }
        }
    }
    __syncthreads();  // every item is in registers: the buffer takes the sorted order now
    // stage the tile in its sorted order (positions are inside [0, tile_n))
#pragma unroll
    for (int r = 0; r < kSortItems; r++) {
        if (wbase + r * 32 + lane < n) {
            const uint32_t dd = (SYS ? sys_of[val[r]] >> shift : (uint32_t)(key[r] >> shift)) & 255u;
            const uint32_t lp = tstart[dd] + wh[w][dd] + rank[r];
            skey[lp] = key[r];
            sval[lp] = val[r];
        }
    }
    __syncthreads();
    if (fail_sh) return;  // positions unknown: write nothing
    // write out: consecutive items of one digit go to consecutive places
    for (int i = threadIdx.x; i < tile_n; i += kSortThreads) {
        const K kk = skey[i];
        const uint32_t vv = sval[i];
        const uint32_t dd = (SYS ? sys_of[vv] >> shift : (uint32_t)(kk >> shift)) & 255u;
        const uint32_t p = base[dd] + (uint32_t)i - tstart[dd];
        kout[p] = kk;
        vout[p] = vv;
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
    if (nb <= kScanFusedBlocks) {
        k_scan_down<true><<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, blocksum, total_dev);
        count_launches(2);
        return;
    }
    k_scan_top<<<1, 1024, 0, s>>>(blocksum, nb, total_dev);
    k_scan_down<false><<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, blocksum, nullptr);
    count_launches(3);
}

// ---------------------------------------------------- per-run completion
// After passes over bits [low_bit, 63) only, items with equal top bits (and
// equal system) sit together in value order; each such run is put in
// (key, val) order -- which, the values being distinct, is the order of
// the full sort.  A run of at most kShortRun items is ranked by its own
// threads (one item each, rank = the items of the run that precede it);
// a longer run is listed and ranked by a block of its own.
constexpr int kShortRun = 32;

__device__ __forceinline__ bool same_run(const uint64_t* __restrict__ k, const uint32_t* __restrict__ v,
                                         const uint32_t* __restrict__ sys_of, int low_bit, int64_t i, int64_t j)
{
    if ((k[i] >> low_bit) != (k[j] >> low_bit)) return false;
    return !sys_of || sys_of[v[i]] == sys_of[v[j]];
}

__device__ __forceinline__ bool before(uint64_t ka, uint32_t va, uint64_t kb, uint32_t vb)
{
    return ka < kb || (ka == kb && va < vb);
}

__global__ void __launch_bounds__(256) k_sort_runs(const uint64_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                                                   uint64_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                   int64_t n, int low_bit, const uint32_t* __restrict__ sys_of,
                                                   int64_t* __restrict__ runs, unsigned long long* __restrict__ nruns,
                                                   int64_t run_cap, int32_t* __restrict__ err)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t st = i;
        while (st > 0 && i - st < kShortRun && same_run(kin, vin, sys_of, low_bit, st - 1, i)) st--;
        int64_t en = i + 1;
        while (en < n && en - st <= kShortRun && same_run(kin, vin, sys_of, low_bit, en, i)) en++;
        if (en - st > kShortRun || (st > 0 && i - st >= kShortRun && same_run(kin, vin, sys_of, low_bit, st - 1, i))) {
            // part of a long run: its first item lists it
            if (i == 0 || !same_run(kin, vin, sys_of, low_bit, i - 1, i)) {
                const unsigned long long at = atomicAdd(nruns, 1ull);
                if ((int64_t)at < run_cap) runs[at] = i;
                else atomicOr(err, kErrSortRun | kErrCapacity);
            }
            continue;
        }
        const uint64_t k = kin[i];
        const uint32_t v = vin[i];
        int64_t r = 0;
        for (int64_t j = st; j < en; j++) r += before(kin[j], vin[j], k, v) ? 1 : 0;
        kout[st + r] = k;
        vout[st + r] = v;
    }
}

__global__ void __launch_bounds__(256) k_sort_long_runs(const uint64_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                                                        uint64_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                        int64_t n, int low_bit, const uint32_t* __restrict__ sys_of,
                                                        const int64_t* __restrict__ runs,
                                                        const unsigned long long* __restrict__ nruns, int64_t run_cap,
                                                        int64_t run_max, int32_t* __restrict__ err)
{
    __shared__ long long en_sh;
    const int64_t nr = (int64_t)min(*nruns, (unsigned long long)run_cap);
    for (int64_t q = blockIdx.x; q < nr; q += gridDim.x) {
        const int64_t st = runs[q];
        // the run's end: the first item past st of another run (or n), or
        // past run_max items
        if (threadIdx.x == 0) en_sh = min(n, st + run_max + 1);
        __syncthreads();
        for (int64_t j = st + 1 + threadIdx.x; j < min(n, st + run_max + 1); j += blockDim.x) {
            if (j >= en_sh) break;
            if (!same_run(kin, vin, sys_of, low_bit, j, st)) atomicMin(&en_sh, (long long)j);
        }
        __syncthreads();
        const int64_t en = en_sh;
        __syncthreads();
        if (en - st > run_max) {
            if (threadIdx.x == 0) atomicOr(err, kErrSortRun | kErrCapacity);
            continue;
        }
        for (int64_t i = st + threadIdx.x; i < en; i += blockDim.x) {
            const uint64_t k = kin[i];
            const uint32_t v = vin[i];
            int64_t r = 0;
            for (int64_t j = st; j < en; j++) r += before(kin[j], vin[j], k, v) ? 1 : 0;
            kout[st + r] = k;
            vout[st + r] = v;
        }
    }
}

void launch_sort_runs(const uint64_t* kin, const uint32_t* vin, uint64_t* kout, uint32_t* vout, int64_t n,
                      int low_bit, const uint32_t* sys_of, SortBufs& b, cudaStream_t s, int64_t run_max)
{
    cudaMemsetAsync(b.nruns, 0, sizeof(unsigned long long), s);
    int64_t g = (n + 255) / 256;
    if (g > 16 * sm_count()) g = 16 * sm_count();
    k_sort_runs<<<(unsigned)(g < 1 ? 1 : g), 256, 0, s>>>(kin, vin, kout, vout, n, low_bit, sys_of, b.runs, b.nruns,
                                                          b.run_cap, b.err);
    k_sort_long_runs<<<(unsigned)(2 * sm_count()), 256, 0, s>>>(kin, vin, kout, vout, n, low_bit, sys_of, b.runs,
                                                                b.nruns, b.run_cap, run_max, b.err);
    count_launches(2);
}

int64_t radix_tiles(int64_t n) { return (n + kSortTile - 1) / kSortTile; }

template <typename K>
static void radix_sort_impl(K* keys, uint32_t* vals, int64_t n, const int64_t* n_dev, int nbits,
                            const uint32_t* sys_of, int sys_bits, SortBufs& b, K* keys_alt, cudaStream_t s,
                            int low_bit = 0, int64_t run_max = kSortRunMax)
{
    const int nkey = (nbits - low_bit + 7) / 8;  // 8-bit digits from bit low_bit up
    const int nsys = (sys_bits + 7) / 8;
    const int npass = nkey + nsys;
    cudaMemsetAsync(b.ghist, 0, kSortMaxPasses * 256 * sizeof(uint32_t), s);
    if (n <= 1) return;  // one item is sorted; its offsets are all zero
    const int64_t nt = radix_tiles(n);
    // zero the look-back words of every pass and the tile counters
    cudaMemsetAsync(b.status, 0, (size_t)npass * nt * 256 * sizeof(unsigned long long), s);
    cudaMemsetAsync(b.tiles, 0, kSortMaxPasses * sizeof(uint32_t), s);
    int hb = (int)((n + kSortThreads * 16 - 1) / (kSortThreads * 16));
    if (hb > 4 * sm_count()) hb = 4 * sm_count();
    k_sort_hist_all<K><<<hb, kSortThreads, 0, s>>>(keys, n, n_dev, nkey, low_bit, b.ghist);
    count_launches(1);
    if (nsys) {
        k_sort_hist_sys<<<hb, kSortThreads, 0, s>>>(sys_of, n, nsys, b.ghist + 256 * nkey);
        count_launches(1);
    }
    k_sort_offsets<<<1, 256, 0, s>>>(b.ghist, npass);
    count_launches(1);
    K* ka = keys;
    uint32_t* va = vals;
    K* kb = keys_alt;
    uint32_t* vb = b.vals_alt;
    // the staging buffer needs more than the default 48 KB of shared memory:
    // a per-device function attribute, set once per device (before any
    // stream capture: every context builds eagerly once before it captures
    // a step)
    {
        static std::mutex mu;
        static bool done[kMaxDevices] = {};
        int dev = 0;
        cudaGetDevice(&dev);
        std::lock_guard<std::mutex> lk(mu);
        if (dev >= 0 && dev < kMaxDevices && !done[dev]) {
            cudaFuncSetAttribute(k_onesweep<K, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)onesweep_smem<K>());
            cudaFuncSetAttribute(k_onesweep<K, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)onesweep_smem<K>());
            done[dev] = true;
        }
    }
    const size_t dsm = onesweep_smem<K>();
    for (int p = 0; p < npass; p++) {
        const bool sysp = p >= nkey;
        const int shift = sysp ? 8 * (p - nkey) : low_bit + 8 * p;
        if (sysp)
            k_onesweep<K, true><<<(unsigned)nt, kSortThreads, dsm, s>>>(ka, va, kb, vb, n, n_dev, shift, b.ghist + 256 * p,
                                                                      b.status + (size_t)p * nt * 256, b.tiles + p,
                                                                      b.err, sys_of);
        else
            k_onesweep<K, false><<<(unsigned)nt, kSortThreads, dsm, s>>>(ka, va, kb, vb, n, n_dev, shift,
                                                                       b.ghist + 256 * p,
                                                                       b.status + (size_t)p * nt * 256, b.tiles + p,
                                                                       b.err, sys_of);
        count_launches(1);
        K* tk = ka; ka = kb; kb = tk;
        uint32_t* tv = va; va = vb; vb = tv;
    }
    if constexpr (sizeof(K) == 8) {
        if (low_bit > 0) {
            // the runs of equal top bits into (key, val) order, from the
            // passes' result into the other buffer pair
            launch_sort_runs(ka, va, kb, vb, n, low_bit, sys_bits > 0 ? sys_of : nullptr, b, s, run_max);
            ka = kb;
            va = vb;
        }
    }
    if (ka != keys) {
        cudaMemcpyAsync(keys, ka, n * sizeof(K), cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(vals, va, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
    }
}

// Self-test of the look-back's wait limit: one block is handed tile 1 of a
// two-tile pass whose tile 0 never runs, so its look-back finds no
// predecessor, gives up after kLookbackMaxPolls polls, sets kErrWorkLoop in
// *err and writes nothing.  All buffers are the caller's device memory:
// keys/vals/kout/vout 2 * kSortTile items, status 2 * 256 words (zeroed
// here), counter 1 word.
cudaError_t sort_wait_selftest(uint64_t* keys, uint32_t* vals, uint64_t* kout, uint32_t* vout,
                               unsigned long long* status, uint32_t* counter, uint32_t* goff, int32_t* err,
                               cudaStream_t s)
{
    const int64_t n = 2 * (int64_t)kSortTile;
    cudaMemsetAsync(status, 0, 2 * 256 * sizeof(unsigned long long), s);
    cudaMemsetAsync(goff, 0, 256 * sizeof(uint32_t), s);
    const uint32_t one = 1;  // the only block launched takes tile 1
    cudaMemcpyAsync(counter, &one, sizeof(one), cudaMemcpyHostToDevice, s);
    cudaFuncSetAttribute(k_onesweep<uint64_t, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)onesweep_smem<uint64_t>());
    k_onesweep<uint64_t, false><<<1, kSortThreads, onesweep_smem<uint64_t>(), s>>>(
        keys, vals, kout, vout, n, nullptr, 0, goff, status, counter, err, nullptr);
    count_launches(1);
    return cudaGetLastError();
}
int64_t sort_selftest_items() { return 2 * (int64_t)kSortTile; }

void radix_sort_u64(uint64_t* keys, uint32_t* vals, int64_t n, int nbits, const uint32_t* sys_of, int sys_bits,
                    SortBufs& b, cudaStream_t s, int low_bit, int64_t run_max)
{
    if (low_bit < 0 || low_bit >= nbits || (low_bit > 0 && (!b.runs || !b.nruns))) low_bit = 0;
    if (run_max < 1 || run_max > kSortRunMax) run_max = kSortRunMax;
    radix_sort_impl<uint64_t>(keys, vals, n, nullptr, nbits, sys_of, sys_bits, b, b.keys_alt, s, low_bit, run_max);
}

void radix_sort_u32(uint32_t* keys, uint32_t* vals, int64_t n_cap, const int64_t* n_dev, int nbits, SortBufs& b,
                    uint32_t* keys_alt32, cudaStream_t s)
{
    radix_sort_impl<uint32_t>(keys, vals, n_cap, n_dev, nbits, nullptr, 0, b, keys_alt32, s);
}

}  // namespace tc
