// tc_api.cu -- the C ABI of libtc (declared in include/tc.h): context,
// argument checks, buffer management, the order of launches, the CUDA graph
// of a leapfrog step and the launch-configuration autotuner.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/tc.h"
#include <nvtx3/nvToolsExt.h>

#include "tc_internal.cuh"

using namespace tc;

constexpr int kMlpNParamHost = 13 * 64 + 64 + 64 * 64 + 64 + 64 * 3 + 3;

struct tc_ctx {
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;  // a stream of our own to capture step graphs on
    // the walk's smaller size classes run beside the largest on a stream of
    // their own (forked from and joined to the launching stream by events)
    cudaStream_t side_stream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int device = 0;
    int num_sms = 0;
    tc_config cfg{};
    std::string err;

    int64_t n = 0, cap_n = 0;
    int nsys = 0, cap_sys = 0;
    std::vector<int64_t> off_h;  // system offsets (host)
    int nchunks = 0, cap_chunks = 0;
    int64_t M = 0, cap_m = 0;  // nodes of the last synchronised build, node table capacity
    int leaf_max = 0;
    bool built = false, have_forces = false, forces_pot = false;
    float theta = 0.f, eps = 0.f, Gc = 0.f;

    // state, original body order
    float *pos = nullptr, *vel = nullptr, *acc = nullptr, *pot = nullptr, *mass = nullptr;
    // systems
    uint32_t* sys_of = nullptr;
    SysParams* sysp = nullptr;
    int64_t* off_dev = nullptr;
    int4* chunks = nullptr;
    // per-body build scratch
    uint64_t* keys = nullptr;
    uint32_t* perm = nullptr;
    float4* body = nullptr;
    SortBufs sb{};
    int8_t *w = nullptr, *delta = nullptr, *top = nullptr;
    uint32_t *nstart = nullptr, *prepos = nullptr;
    uint32_t *gflag = nullptr, *gscan = nullptr;
    int32_t *gref_at = nullptr, *gfirst = nullptr, *gref = nullptr;
    int32_t *ncell = nullptr, *nbody = nullptr;
    unsigned long long* hash = nullptr;
    uint32_t* totals = nullptr;  // [0] nodes, [1] groups
    int64_t* idx_dev = nullptr;
    int64_t cap_idx = 0;
    double* dir_out = nullptr;
    // per-node scratch
    uint32_t *pre_level = nullptr, *pre_first = nullptr, *iota = nullptr, *bfs_of_pre = nullptr, *lvl_alt = nullptr;
    NodeTables nt{};
    Info* info = nullptr;
    Info* info_h = nullptr;  // pinned mirror
    int64_t cap_m_h = 0;     // source of the device copy of cap_m
    size_t allocated = 0;
    std::unordered_map<void*, size_t> sizes;

    // walk launch shape for the current configuration
    bool walk_ready = false;
    int walk_grid = 0;
    size_t walk_smem = 0;
    // groups split by size (walks of up to 64 / 128 bodies): class k goes to
    // the kernel with 2^k bodies per lane
    int32_t* glists = nullptr;   // 3 x cap_n group indices
    int32_t* glist_n = nullptr;  // 3 counts, then the split's scratch
    int walk_ncls = 0;
    int depth_hint = -1;  // tree depth of the last build the host saw (-1: none)
    int64_t depth_hint_n = -1;  // its body count
    WalkConfig walk_cls[3]{};
    int walk_cls_grid[3] = {0, 0, 0};
    size_t walk_cls_smem[3] = {0, 0, 0};
    WalkConfig walk_cfg{};

    // phase timers (CUDA events on the context stream), when enabled
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_phase[3];  // build, walk, update
    long long launches_mark = 0;

    // learned far-field correction
    float* mlp_params = nullptr;  // FP32 master parameters (packed)
    float* mlp_maps = nullptr;    // feature means, feature scales, output scales
    void* mlp_dev = nullptr;      // device model (BF16 weights)
    float* mlp_m = nullptr;       // Adam moments
    float* mlp_v = nullptr;
    float* mlp_grad = nullptr;
    float* mlp_part = nullptr;    // per-warp partial gradients of a training step
    int64_t mlp_part_cap = 0;
    float* mlp_loss = nullptr;
    unsigned long long* mlp_evals = nullptr;
    float* mlp_x = nullptr;       // scratch: features / normalised rows / outputs
    float* mlp_t = nullptr;
    float* mlp_w = nullptr;       // per-pair loss weights / label factors
    int32_t* mlp_idx = nullptr;
    float* mlp_raw = nullptr;     // scratch: raw features as given (n x 13)
    double* mlp_sums = nullptr;   // FP64 sums of the training data (kMlpSums)
    float* mlp_wscale = nullptr;  // n / sum F^2 (factor weights)
    int32_t* mlp_bad = nullptr;   // a given loss weight was negative or not finite
    // learned correction evaluated after the split walk: the band-cell
    // record, its length, each group's box centre and correction
    int2* band = nullptr;
    unsigned long long* band_n = nullptr;
    float4* grec = nullptr;  // 2 per group: the rows' frame
    float* gcorr = nullptr;
    int64_t band_cap = 0;
    int64_t band_gcap = 0;
    int64_t mlp_cap = 0;
    bool have_mlp = false;
    float mlp_band = 0.5f;
    int32_t* list_buf = nullptr;    // list export scratch: cells, then leaves
    int64_t list_cap = 0;
    int64_t* list_n = nullptr;
    int32_t* pair_b = nullptr;
    int32_t* pair_v = nullptr;
    unsigned long long* pair_n = nullptr;
    int64_t pair_cap = 0;
    // the pairs' sort: keys, values and the radix sort's scratch
    uint64_t* pair_key = nullptr;
    uint32_t* pair_val = nullptr;
    SortBufs pair_sb{};
    int64_t pair_sort_cap = 0;

    // fast multipole method: parent table, local expansions, unresolved
    // source lists (per node: offset and count into the pool of its level's
    // parity), per-warp slabs, counters, level starts
    bool forces_fmm = false;
    int32_t* fmm_parent = nullptr;
    float* fmm_loc = nullptr;
    int64_t* fmm_off = nullptr;
    int32_t* fmm_cnt = nullptr;
    unsigned long long* fmm_rec = nullptr;  // 4 per node
    double* fmm_rad = nullptr;               // acceptance radii (FP64)
    int4* fmm_fnode = nullptr;               // 3 per node: the FMM's gathered cell records
    int64_t fmm_cap_m = 0;
    int32_t* fmm_pool[2] = {nullptr, nullptr};
    int64_t fmm_pool_cap = 0;
    int32_t* fmm_slab = nullptr;
    int64_t fmm_slab_cap = 0;
    int64_t fmm_slab_warps = 0;
    unsigned long long* fmm_ctr = nullptr;
    int64_t* fmm_lstart = nullptr;
    unsigned long long fmm_stats[4] = {0, 0, 0, 0};
    bool fmm_records = false;  // the last pass kept hashes and per-node records

    // the captured leapfrog step
    cudaGraphExec_t gexec = nullptr;
    std::string gkey;
    long long graph_kernels = 0;
};

namespace tc {
namespace {
std::atomic<long long> g_launches{0};
}
void count_launches(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
long long launches_total() { return g_launches.load(std::memory_order_relaxed); }

namespace {
constexpr int kSmCacheDevices = 64;
std::atomic<int> g_sm_count[kSmCacheDevices] = {};
}
int sm_count()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    if (dev >= 0 && dev < kSmCacheDevices) {
        const int c = g_sm_count[dev].load(std::memory_order_relaxed);
        if (c > 0) return c;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
        cudaGetLastError();
        return 1;
    }
    if (dev >= 0 && dev < kSmCacheDevices) g_sm_count[dev].store(sms, std::memory_order_relaxed);
    return sms;
}
}  // namespace tc

namespace {

std::mutex g_default_mu;
tc_ctx* g_default = nullptr;
thread_local std::string g_tls_err;

}  // namespace

void tc::set_thread_error(const char* msg) { g_tls_err = msg; }

namespace {

int fail(tc_ctx* c, int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    else g_tls_err = buf;
    return code;
}

#define TC_CUDA(c, call)                                                                        \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) return fail(c, TC_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

size_t alloc_cap()
{
    const char* s = getenv("TC_ALLOC_CAP_BYTES");
    if (!s || !*s) return (size_t)-1;
    return (size_t)strtoull(s, nullptr, 10);
}

void drop_graph(tc_ctx* c)
{
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
    c->gkey.clear();
}

template <typename T>
int grow(tc_ctx* c, T** p, int64_t count)
{
    drop_graph(c);  // a captured step refers to the old buffers
    if (*p) {
        auto it = c->sizes.find((void*)*p);
        if (it != c->sizes.end()) {
            c->allocated -= it->second;
            c->sizes.erase(it);
        }
        cudaFree(*p);
        *p = nullptr;
    }
    size_t bytes = (size_t)(count < 1 ? 1 : count) * sizeof(T);
    if (c->allocated + bytes > alloc_cap())
        return fail(c, TC_ENOMEM, "allocation of %zu bytes exceeds TC_ALLOC_CAP_BYTES", bytes);
    cudaError_t e = cudaMalloc((void**)p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(c, TC_ENOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    }
    c->allocated += bytes;
    c->sizes[(void*)*p] = bytes;
    return TC_OK;
}

#define TC_GROW(c, p, n)                  \
    do {                                  \
        int r_ = grow((c), &(p), (n));    \
        if (r_) return r_;                \
    } while (0)

int ensure_bodies(tc_ctx* c, int64_t n)
{
    if (n <= c->cap_n) return TC_OK;
    int64_t cap = n;
    TC_GROW(c, c->pos, 3 * cap);
    TC_GROW(c, c->vel, 3 * cap);
    TC_GROW(c, c->acc, 3 * cap);
    TC_GROW(c, c->pot, cap);
    TC_GROW(c, c->mass, cap);
    TC_GROW(c, c->sys_of, cap);
    TC_GROW(c, c->keys, cap);
    TC_GROW(c, c->perm, cap);
    TC_GROW(c, c->body, cap);
    TC_GROW(c, c->sb.keys_alt, cap);
    TC_GROW(c, c->sb.vals_alt, cap);
    TC_GROW(c, c->sb.ghist, kSortMaxPasses * 256);
    TC_GROW(c, c->sb.status, (int64_t)kSortMaxPasses * radix_tiles(cap) * 256);
    TC_GROW(c, c->sb.tiles, kSortMaxPasses);
    c->sb.err = &c->info->err;
    TC_GROW(c, c->sb.blocksum, scan_blocksum_size(cap));
    TC_GROW(c, c->sb.runs, cap / 32 + 16);  // runs of more than 32 items
    c->sb.run_cap = cap / 32 + 16;
    TC_GROW(c, c->sb.nruns, 1);
    TC_GROW(c, c->w, cap);
    TC_GROW(c, c->delta, cap);
    TC_GROW(c, c->top, cap);
    TC_GROW(c, c->nstart, cap);
    TC_GROW(c, c->prepos, cap);
    TC_GROW(c, c->gflag, cap);
    TC_GROW(c, c->gscan, cap);
    TC_GROW(c, c->gref_at, cap);
    TC_GROW(c, c->gfirst, cap + 1);
    TC_GROW(c, c->gref, cap);
    TC_GROW(c, c->ncell, cap);
    TC_GROW(c, c->nbody, cap);
    TC_GROW(c, c->hash, cap);
    TC_GROW(c, c->totals, 4);
    TC_GROW(c, c->glists, 3 * cap);
    TC_GROW(c, c->glist_n, 3 + (int64_t)group_split_scratch());
    c->cap_n = cap;
    c->cap_m = 0;  // node tables are sized with the first build at this capacity
    return TC_OK;
}

int ensure_systems(tc_ctx* c, int nsys, int nchunks)
{
    if (nsys > c->cap_sys) {
        TC_GROW(c, c->sysp, nsys);
        TC_GROW(c, c->off_dev, nsys + 1);
        c->cap_sys = nsys;
    }
    if (nchunks > c->cap_chunks) {
        TC_GROW(c, c->chunks, nchunks);
        c->cap_chunks = nchunks;
    }
    return TC_OK;
}

int ensure_nodes(tc_ctx* c, int64_t M)
{
    if (M <= c->cap_m) return TC_OK;
    const int64_t cap = M + M / 2 + 1024;  // headroom for the rebuilds of later steps
    TC_GROW(c, c->pre_level, cap);
    TC_GROW(c, c->pre_first, cap);
    TC_GROW(c, c->iota, cap);
    TC_GROW(c, c->bfs_of_pre, cap);
    TC_GROW(c, c->lvl_alt, cap);
    TC_GROW(c, c->nt.a, cap);
    TC_GROW(c, c->nt.b, cap);
    TC_GROW(c, c->nt.c, cap);
    TC_GROW(c, c->nt.d, cap);
    TC_GROW(c, c->nt.quad, 6 * cap);
    TC_GROW(c, c->nt.feat, 2 * cap);
    TC_GROW(c, c->nt.mass64, cap);
    TC_GROW(c, c->nt.dsum, 2 * cap);
    TC_GROW(c, c->nt.com64, 3 * cap);
    // the level sort reuses the body sort's value ping-pong buffer and status words
    if (cap > c->cap_n) TC_GROW(c, c->sb.vals_alt, cap);
    if (radix_tiles(cap) > (int64_t)kSortMaxPasses * radix_tiles(c->cap_n))
        TC_GROW(c, c->sb.status, radix_tiles(cap) * 256);
    c->cap_m = cap;
    c->walk_ready = false;  // the stack bound may follow the capacity
    return TC_OK;
}

// device error word -> status (synchronises); clears the word it reports
int check_device(tc_ctx* c)
{
    TC_CUDA(c, cudaStreamSynchronize(c->stream));
    TC_CUDA(c, cudaMemcpy(c->info_h, c->info, sizeof(Info), cudaMemcpyDeviceToHost));
    int32_t e = c->info_h->err;
    if (e) {
        TC_CUDA(c, cudaMemsetAsync(&c->info->err, 0, sizeof(int32_t), c->stream));
        TC_CUDA(c, cudaStreamSynchronize(c->stream));
        if (e & kErrNonFinite)
            return fail(c, TC_EINVAL, "input holds a non-finite coordinate or a non-positive/non-finite mass");
        if (e & kErrSortRun)
            return fail(c, TC_EDEVICE,
                        "a rebuild inside a step found a tree far deeper than the last synchronised build's "
                        "(a run of more than %lld bodies sharing the sorted key digits); the state holds that "
                        "step's drift -- call tc_ctx_build or tc_set_state to rebuild",
                        (long long)kSortRunMax);
        if (e & kErrCapacity)
            return fail(c, TC_EDEVICE,
                        "node table capacity exceeded by a rebuild inside a step; the state holds that step's "
                        "drift -- call tc_ctx_build or tc_set_state to resize");
        if (e & kErrStack) return fail(c, TC_EDEVICE, "walk stack overflow (raise tc_config.stack)");
        if (e & kErrWorkLoop) return fail(c, TC_EDEVICE, "a bounded device wait gave up");
        if (e & kErrFmmStack)
            return fail(c, TC_EDEVICE, "the FMM's refinement stack (2048 sources per cell) overflowed; raise theta");
        if (e & (kErrFmmPool | kErrFmmSlab))
            return fail(c, TC_EDEVICE, "the FMM's unresolved-source lists still overflowed after regrowing");
        if (e & kErrBand)
            return fail(c, TC_EDEVICE,
                        "the learned walk recorded more band cells than its buffer holds (12 per body); its "
                        "correction is incomplete -- narrow the band or use split = 0");
        return fail(c, TC_EDEVICE, "device error word 0x%x", e);
    }
    return TC_OK;
}

bool finite(float x) { return std::isfinite(x); }

cudaEvent_t take_event(tc_ctx* c)
{
    if (c->ev_used == c->ev_pool.size()) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        c->ev_pool.push_back(e);
    }
    return c->ev_pool[c->ev_used++];
}

// records the start of a timed phase; returns the event (or null).  Every
// phase is also an NVTX range on the host timeline (build, walk + force,
// update), visible to a profiler attached to the process.
const char* const kPhaseName[3] = {"tc build", "tc walk+force", "tc update"};

cudaEvent_t phase_begin(tc_ctx* c, cudaStream_t s, int phase)
{
    nvtxRangePushA(kPhaseName[phase]);
    if (!c->timing) return nullptr;
    cudaEvent_t e = take_event(c);
    if (e) cudaEventRecord(e, s);
    return e;
}

void phase_end(tc_ctx* c, int phase, cudaEvent_t start, cudaStream_t s)
{
    nvtxRangePop();
    if (!start) return;
    cudaEvent_t e = take_event(c);
    if (!e) return;
    cudaEventRecord(e, s);
    c->ev_phase[phase].push_back({start, e});
}

int sys_bits(int nsys)
{
    int b = 0;
    while ((1 << b) < nsys) b++;
    return b;
}

// system offsets -> per-body system ids, bounding-box chunks
int setup_systems(tc_ctx* c, const int64_t* off, int nsys)
{
    std::vector<int4> ch;
    for (int s = 0; s < nsys; s++)
        for (int64_t a = off[s]; a < off[s + 1]; a += kBboxChunk)
            ch.push_back(make_int4(s, (int)a, (int)std::min(off[s + 1], a + (int64_t)kBboxChunk), 0));
    int r = ensure_systems(c, nsys, (int)ch.size());
    if (r) return r;
    c->off_h.assign(off, off + nsys + 1);
    c->nsys = nsys;
    c->nchunks = (int)ch.size();
    TC_CUDA(c, cudaMemcpyAsync(c->off_dev, c->off_h.data(), (nsys + 1) * sizeof(int64_t), cudaMemcpyHostToDevice,
                               c->stream));
    TC_CUDA(c, cudaMemcpyAsync(c->chunks, ch.data(), ch.size() * sizeof(int4), cudaMemcpyHostToDevice, c->stream));
    launch_sys_ids(c->off_dev, nsys, c->n, c->sys_of, c->sysp, c->stream);
    // the host vectors above may be copied from pageable memory: wait before they go
    TC_CUDA(c, cudaStreamSynchronize(c->stream));
    return TC_OK;
}

// The build from c->pos / c->mass (already on the device), on stream s.
// synced: validate the input and size the node table (one synchronisation);
// otherwise no host interaction at all (the form captured in a step graph),
// with the node count checked against the capacity on the device.
int build_tree(tc_ctx* c, bool synced, cudaStream_t s, bool all_digits = false)
{
    const int64_t n = c->n;
    cudaEvent_t t0 = phase_begin(c, s, 0);
    if (synced) TC_CUDA(c, cudaMemsetAsync(&c->info->err, 0, sizeof(int32_t), s));
    launch_bbox(c->pos, c->chunks, c->nchunks, c->sysp, c->nsys, &c->info->err, s);
    launch_keys(c->pos, c->mass, n, c->sys_of, c->sysp, c->keys, c->perm, &c->info->err, s);
    // The passes sort only the key digits of the levels down to the last
    // synchronised build's depth + kSortMarginLevels; runs of equal top
    // digits, a leaf's bodies as long as the tree is no deeper than that,
    // are then completed one by one, which gives the full sort's order (a
    // deeper tree gives longer runs, which the completion still orders: up
    // to kSortRunMax bodies a run inside a step; in a synchronised build up
    // to kSortRunMaxSynced, past which the build is redone sorting every
    // digit).  With no earlier depth every digit is sorted.
    int low_bit = 0;
    if (!all_digits && c->depth_hint >= 0 && (!synced || n == c->depth_hint_n)) {
        const int levels = std::min(kMaxLevel, c->depth_hint + kSortMarginLevels);
        low_bit = 63 - 3 * levels;
    }
    radix_sort_u64(c->keys, c->perm, n, 63, c->sys_of, c->nsys > 1 ? sys_bits(c->nsys) : 0, c->sb, s, low_bit,
                   synced ? kSortRunMaxSynced : kSortRunMax);
    launch_gather(c->pos, c->mass, c->perm, n, c->body, s);
    TC_CUDA(c, cudaMemsetAsync(&c->info->depth, 0, sizeof(int32_t), s));
    launch_node_counts(c->keys, c->sys_of, n, c->leaf_max, c->w, c->delta, c->top, c->nstart, &c->info->depth, s);
    scan_u32(c->nstart, c->prepos, n, &c->totals[0], c->sb.blocksum, s);
    int depth = -1;
    if (synced) {
        TC_CUDA(c, cudaGetLastError());
        if (low_bit > 0) {
            // a run too long for the completion: build again, sorting every digit
            TC_CUDA(c, cudaStreamSynchronize(s));
            int32_t err = 0;
            TC_CUDA(c, cudaMemcpy(&err, &c->info->err, sizeof(err), cudaMemcpyDeviceToHost));
            if (err & kErrSortRun) {
                TC_CUDA(c, cudaMemsetAsync(&c->info->err, 0, sizeof(int32_t), s));
                phase_end(c, 0, t0, s);
                return build_tree(c, true, s, true);
            }
        }
        int r = check_device(c);  // synchronises; reports invalid input
        if (r) return r;
        uint32_t M32 = 0;
        TC_CUDA(c, cudaMemcpy(&M32, &c->totals[0], sizeof(uint32_t), cudaMemcpyDeviceToHost));
        if (M32 < 1) return fail(c, TC_EDEVICE, "empty node table");
        r = ensure_nodes(c, M32);
        if (r) return r;
        c->M = M32;
        c->cap_m_h = c->cap_m;
        TC_CUDA(c, cudaMemcpyAsync(&c->info->cap_m, &c->cap_m_h, sizeof(int64_t), cudaMemcpyHostToDevice, s));
        depth = c->info_h->depth;
        c->depth_hint = depth;
        c->depth_hint_n = n;
    }
    launch_check_capacity(&c->totals[0], c->info, s);
    launch_emit_preorder(c->delta, c->nstart, c->prepos, n, c->info, c->pre_level, c->pre_first, c->iota, s);
    // breadth-first order: stable sort of the pre-order nodes by level
    SortBufs lb = c->sb;
    radix_sort_u32(c->pre_level, c->iota, c->cap_m, &c->info->M, 8, lb, c->lvl_alt, s);
    launch_inverse_perm(c->iota, c->cap_m, c->info, c->bfs_of_pre, s);
    launch_node_finalize(c->keys, c->top, c->sys_of, c->sysp, n, c->pre_level, c->iota, c->pre_first, c->bfs_of_pre,
                         c->cap_m, c->info, c->nt, s);
    // after the level sort, ghist[l] is the first breadth-first index of level l
    launch_moments(c->body, c->cap_m, depth, c->depth_hint, c->sb.ghist, c->sys_of, c->sysp, c->info, c->nt, c->cfg.quad != 0, s);
    launch_sys_mass(c->sysp, c->nsys, c->nt, c->info, s);
    launch_group_marks(c->cap_m, c->info, c->nt, c->cfg.gmax, n, c->gflag, c->gref_at, s);
    scan_u32(c->gflag, c->gscan, n, &c->totals[1], c->sb.blocksum, s);
    launch_group_table(c->gflag, c->gscan, c->gref_at, n, &c->totals[1], c->gfirst, c->gref, c->info, s);
    if (c->cfg.gmax > 32) launch_group_split(c->gfirst, c->info, c->cap_n, c->glists, c->glist_n, c->glist_n + 3, s);
    TC_CUDA(c, cudaGetLastError());
    phase_end(c, 0, t0, s);
    c->built = true;
    c->have_forces = false;
    return TC_OK;
}

int prepare_forces(tc_ctx* c)
{
    WalkConfig wc{};
    wc.gmax = c->cfg.gmax;
    wc.warps = c->cfg.warps;
    wc.precise = c->cfg.precise;
    wc.want_pot = c->cfg.want_pot;
    wc.verify = c->cfg.verify;
    wc.blocks_per_sm = c->cfg.blocks_per_sm;
    wc.tile = c->cfg.tile;
    wc.learned = c->cfg.learned && c->have_mlp;
    wc.quadw = c->cfg.quadrupole;
    wc.classes = c->cfg.gmax > 32 ? c->cfg.classes : 0;
    // split 1: producer/consumer walks for the monopole walks, the learned
    // walk keeps the network inside the one-warp walk; 2: the learned walk
    // too, the network then evaluated after the walk
    wc.split = (!wc.quadw && (c->cfg.split == 2 || (c->cfg.split == 1 && !wc.learned))) ? 1 : 0;
    int64_t st = c->cfg.stack;
    if (c->cap_m < st) st = c->cap_m < 32 ? 32 : c->cap_m;  // a stack of M entries cannot overflow
    st = (st + 3) & ~(int64_t)3;                            // keeps every warp's tiles 16-byte aligned
    wc.stack = (int)st;
    if (wc.learned && wc.split) {
        // the band-cell record: 12 cells per body (the learned workloads
        // record 2 to 7) plus a chunk per producer warp of every size-class
        // launch (each keeps a partly filled chunk); a walk that records
        // more stops with an error (TC_EDEVICE) instead of writing past it.
        // TC_BAND_CAP (entries) overrides the size, to exercise that error.
        int64_t want = 12 * c->cap_n + (int64_t)3 * c->num_sms * 2 * 4 * kBandChunk + 65536;
        if (const char* env = getenv("TC_BAND_CAP")) {
            const long long v = atoll(env);
            if (v > 0) want = v;
        }
        if (want != c->band_cap) {
            if (want > c->band_cap) TC_GROW(c, c->band, want);
            c->band_cap = want;
            c->walk_ready = false;
            drop_graph(c);
        }
        if (!c->band_n) TC_GROW(c, c->band_n, 1);
        if (c->cap_n + 1 > c->band_gcap) {
            TC_GROW(c, c->grec, 2 * (c->cap_n + 1));
            TC_GROW(c, c->gcorr, 3 * (c->cap_n + 1));
            c->band_gcap = c->cap_n + 1;
            drop_graph(c);
        }
    }
    if (c->walk_ready && memcmp(&wc, &c->walk_cfg, sizeof(wc)) == 0) return TC_OK;
    cudaError_t e = prepare_walk(wc, c->num_sms, &c->walk_grid, &c->walk_smem);
    if (e != cudaSuccess) return fail(c, TC_ECUDA, "walk kernel set-up: %s", cudaGetErrorString(e));
    // one launch per size class: groups of up to 32 bodies one per lane, up
    // to 64 two per lane, more four per lane (the launch for the context's
    // gmax walks every group, or single groups)
    c->walk_ncls = wc.classes ? (wc.gmax == 64 ? 2 : 3) : 0;
    for (int k = 0; k < c->walk_ncls; k++) {
        c->walk_cls[k] = wc;
        c->walk_cls[k].gmax = 32 << k;
        e = prepare_walk(c->walk_cls[k], c->num_sms, &c->walk_cls_grid[k], &c->walk_cls_smem[k]);
        if (e != cudaSuccess) return fail(c, TC_ECUDA, "walk kernel set-up: %s", cudaGetErrorString(e));
    }
    c->walk_cfg = wc;
    c->walk_ready = true;
    return TC_OK;
}

int run_forces(tc_ctx* c, float theta, float eps, float G, cudaStream_t s)
{
    WalkArgs a{};
    a.body = c->body;
    a.perm = c->perm;
    a.sys_of = c->sys_of;
    a.sysp = c->sysp;
    a.nt = c->nt;
    a.gfirst = c->gfirst;
    a.gref = c->gref;
    a.info = c->info;
    a.acc = c->acc;
    a.pot = c->cfg.want_pot ? c->pot : nullptr;
    a.ncell = c->cfg.verify ? c->ncell : nullptr;
    a.nbody = c->cfg.verify ? c->nbody : nullptr;
    a.hash = c->cfg.verify ? c->hash : nullptr;
    a.theta2 = theta * theta;
    a.eps2 = eps * eps;
    a.G = G;
    a.inv_eps = 1.0f / eps;
    a.eps = eps;
    const bool deferred = c->walk_cfg.learned && c->walk_cfg.split;
    if (c->walk_cfg.learned) {
        a.mlp = c->mlp_dev;
        a.band2 = c->mlp_band * c->mlp_band;
        a.mlp_evals = c->mlp_evals;
    }
    if (deferred) {
        a.band = c->band;
        a.band_n = c->band_n;
        a.band_cap = c->band_cap;
        a.grec = c->grec;
    }
    cudaEvent_t t0 = phase_begin(c, s, 1);
    cudaError_t e = cudaSuccess;
    if (c->walk_cfg.learned) launch_node_features(c->info, c->cap_m, c->sysp, c->nt, eps, c->mlp_dev, s);
    if (deferred) {
        cudaMemsetAsync(c->band_n, 0, sizeof(unsigned long long), s);
        cudaMemsetAsync(c->gcorr, 0, 3 * c->band_gcap * sizeof(float), s);
    }
    if (c->walk_ncls == 0) {
        e = launch_walk(a, c->walk_cfg, c->walk_grid, c->walk_smem, s);
    } else {
        // the largest class on s, the others after it on the side stream:
        // their blocks take the SMs that the largest class's blocks leave
        // when its groups run out, instead of waiting for its last block
        if (!c->side_stream) TC_CUDA(c, cudaStreamCreateWithFlags(&c->side_stream, cudaStreamNonBlocking));
        if (!c->ev_fork) TC_CUDA(c, cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
        if (!c->ev_join) TC_CUDA(c, cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
        // the work counters and the totals behind them, before either stream starts
        TC_CUDA(c, cudaMemsetAsync(&c->info->work[0], 0, sizeof(c->info->work) + 3 * sizeof(unsigned long long), s));
        TC_CUDA(c, cudaEventRecord(c->ev_fork, s));
        TC_CUDA(c, cudaStreamWaitEvent(c->side_stream, c->ev_fork, 0));
        for (int k = c->walk_ncls - 1; k >= 0 && e == cudaSuccess; k--) {
            a.glist = c->glists + (int64_t)k * c->cap_n;
            a.glist_n = c->glist_n + k;
            a.work_slot = k;
            e = launch_walk(a, c->walk_cls[k], c->walk_cls_grid[k], c->walk_cls_smem[k],
                            k == c->walk_ncls - 1 ? s : c->side_stream, false);
        }
        TC_CUDA(c, cudaEventRecord(c->ev_join, c->side_stream));
        TC_CUDA(c, cudaStreamWaitEvent(s, c->ev_join, 0));
    }
    if (e == cudaSuccess && deferred) {
        launch_band_eval(a, c->mlp_dev, c->gcorr, c->mlp_evals, s);
        launch_band_apply(c->info, c->band_gcap - 1, c->gfirst, c->perm, c->gcorr, c->acc, s);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return fail(c, TC_ECUDA, "walk launch: %s", cudaGetErrorString(e));
    phase_end(c, 1, t0, s);
    c->have_forces = true;
    c->forces_fmm = false;
    c->forces_pot = c->cfg.want_pot != 0;
    c->theta = theta;
    c->eps = eps;
    c->Gc = G;
    return TC_OK;
}

// kick + drift, sync-free rebuild, walk, kick -- eagerly on the context stream
int step_eager(tc_ctx* c, float dt)
{
    cudaStream_t s = c->stream;
    int r = prepare_forces(c);
    if (r) return r;
    cudaEvent_t t0 = phase_begin(c, s, 2);
    launch_kick_drift(c->pos, c->vel, c->acc, c->n, 0.5f * dt, dt, c->info, s);
    phase_end(c, 2, t0, s);
    r = build_tree(c, false, s);
    if (r) return r;
    r = run_forces(c, c->theta, c->eps, c->Gc, s);
    if (r) return r;
    t0 = phase_begin(c, s, 2);
    launch_kick(c->vel, c->acc, c->n, 0.5f * dt, c->info, s);
    phase_end(c, 2, t0, s);
    TC_CUDA(c, cudaGetLastError());
    return TC_OK;
}

std::string graph_key(tc_ctx* c, float dt)
{
    char b[512];
    snprintf(b, sizeof(b), "%lld/%lld/%d/%d/%a/%a/%a/%a/%d/%d/%d/%d/%d/%d/%d/%d/%d/%d/%a/%d/%d", (long long)c->n,
             (long long)c->cap_m, c->nsys, c->leaf_max, (double)dt, (double)c->theta, (double)c->eps, (double)c->Gc,
             c->cfg.gmax, c->cfg.warps, c->cfg.precise, c->cfg.want_pot, c->cfg.verify, c->cfg.stack,
             c->cfg.blocks_per_sm, c->cfg.quad, c->cfg.tile, c->cfg.learned && c->have_mlp, (double)c->mlp_band,
             c->cfg.quadrupole, c->cfg.classes);
    return b;
}

// One step as a captured CUDA graph, captured once per configuration on a
// stream of our own and replayed on the context stream.  Without phase
// timing the graph holds the whole step (kick, drift, rebuild, walk, kick).
// With phase timing it holds kick + drift + rebuild, and the walk and the
// closing kick follow as direct launches bracketed by CUDA events on the
// context stream (events recorded inside a graph cannot be timed).
int step_graph(tc_ctx* c, float dt)
{
    const bool timing = c->timing;
    const std::string key = graph_key(c, dt) + (timing ? "/timed" : "");
    if (!c->gexec || key != c->gkey) {
        drop_graph(c);
        if (!c->cap_stream) TC_CUDA(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
        int r = prepare_forces(c);
        if (r) return r;
        c->timing = false;
        const long long k0 = launches_total();
        cudaStream_t s = c->cap_stream;
        TC_CUDA(c, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        launch_kick_drift(c->pos, c->vel, c->acc, c->n, 0.5f * dt, dt, c->info, s);
        r = build_tree(c, false, s);
        if (!timing) {
            if (!r) r = run_forces(c, c->theta, c->eps, c->Gc, s);
            launch_kick(c->vel, c->acc, c->n, 0.5f * dt, c->info, s);
        }
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(s, &g);
        c->timing = timing;
        c->graph_kernels = launches_total() - k0;
        count_launches((int)-c->graph_kernels);  // counted when the graph runs
        if (r) {
            if (g) cudaGraphDestroy(g);
            return r;
        }
        if (e != cudaSuccess) return fail(c, TC_ECUDA, "step capture: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&c->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            c->gexec = nullptr;
            return fail(c, TC_ECUDA, "step graph instantiation: %s", cudaGetErrorString(e));
        }
        c->gkey = key;
    }
    cudaEvent_t t0 = phase_begin(c, c->stream, 0);
    TC_CUDA(c, cudaGraphLaunch(c->gexec, c->stream));
    count_launches((int)c->graph_kernels);
    phase_end(c, 0, t0, c->stream);  // (timing mode: kick + drift + rebuild)
    if (timing) {
        int r = run_forces(c, c->theta, c->eps, c->Gc, c->stream);
        if (r) return r;
        t0 = phase_begin(c, c->stream, 2);
        launch_kick(c->vel, c->acc, c->n, 0.5f * dt, c->info, c->stream);
        phase_end(c, 2, t0, c->stream);
        TC_CUDA(c, cudaGetLastError());
    }
    c->have_forces = true;
    return TC_OK;
}

}  // namespace

extern "C" {

int tc_create(tc_ctx** out, void* stream)
{
    if (!out) return fail(nullptr, TC_EINVAL, "tc_create: null output pointer");
    *out = nullptr;
    tc_ctx* c = new (std::nothrow) tc_ctx();
    if (!c) return fail(nullptr, TC_ENOMEM, "tc_create: out of host memory");
    c->stream = (cudaStream_t)stream;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e == cudaSuccess) e = cudaMalloc((void**)&c->info, sizeof(Info));
    if (e == cudaSuccess) e = cudaMemset(c->info, 0, sizeof(Info));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&c->info_h, sizeof(Info));
    if (e != cudaSuccess) {
        int r = fail(nullptr, TC_ECUDA, "tc_create: %s", cudaGetErrorString(e));
        cudaGetLastError();
        tc_destroy(c);
        return r;
    }
    c->cfg.gmax = 64;
    c->cfg.warps = 4;
    c->cfg.precise = 1;
    c->cfg.want_pot = 0;
    c->cfg.verify = 0;
    c->cfg.stack = 1024;
    c->cfg.blocks_per_sm = 0;
    c->cfg.quad = 0;
    c->cfg.tile = 128;
    c->cfg.graph = 1;
    c->cfg.learned = 0;
    c->cfg.quadrupole = 0;
    c->cfg.classes = 1;
    c->cfg.split = 1;
    *out = c;
    return TC_OK;
}

void tc_destroy(tc_ctx* c)
{
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    drop_graph(c);
    // every device buffer but the Info word was made by grow(), which records it
    for (auto& kv : c->sizes) cudaFree(kv.first);
    c->sizes.clear();
    if (c->info) cudaFree(c->info);
    if (c->info_h) cudaFreeHost(c->info_h);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->side_stream) cudaStreamDestroy(c->side_stream);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    delete c;
}

int tc_set_config(tc_ctx* c, const tc_config* cfg)
{
    if (!c || !cfg) return fail(c, TC_EINVAL, "tc_set_config: null argument");
    if (!((cfg->gmax >= 1 && cfg->gmax <= 32) || cfg->gmax == 64 || cfg->gmax == 128))
        return fail(c, TC_EINVAL, "gmax must be 1..32, 64 or 128 (got %d)", cfg->gmax);
    if (cfg->warps < 1 || cfg->warps > 4) return fail(c, TC_EINVAL, "warps must be 1..4 (got %d)", cfg->warps);
    if (cfg->stack < 64 || cfg->stack > 8192) return fail(c, TC_EINVAL, "stack must be 64..8192 (got %d)", cfg->stack);
    if (cfg->blocks_per_sm < 0) return fail(c, TC_EINVAL, "blocks_per_sm must be >= 0");
    if (cfg->tile != 64 && cfg->tile != 128 && cfg->tile != 256)
        return fail(c, TC_EINVAL, "tile must be 64, 128 or 256 (got %d)", cfg->tile);
    if (cfg->learned && (!cfg->precise || cfg->want_pot || !cfg->quad || cfg->quadrupole))
        return fail(c, TC_EINVAL, "learned = 1 needs precise = 1, want_pot = 0, quad = 1 and quadrupole = 0");
    if (cfg->quadrupole && (!cfg->precise || !cfg->quad))
        return fail(c, TC_EINVAL, "quadrupole = 1 needs precise = 1 and quad = 1");
    if (cfg->classes < 0 || cfg->classes > 1) return fail(c, TC_EINVAL, "classes must be 0 or 1 (got %d)", cfg->classes);
    if (cfg->split < 0 || cfg->split > 2) return fail(c, TC_EINVAL, "split must be 0, 1 or 2 (got %d)", cfg->split);
    bool rebuild = c->built && (cfg->gmax != c->cfg.gmax || (cfg->quad != 0) != (c->cfg.quad != 0));
    c->cfg = *cfg;
    c->cfg.precise = cfg->precise ? 1 : 0;
    c->cfg.want_pot = cfg->want_pot ? 1 : 0;
    c->cfg.verify = cfg->verify ? 1 : 0;
    c->cfg.quad = cfg->quad ? 1 : 0;
    c->cfg.graph = cfg->graph ? 1 : 0;
    c->cfg.learned = cfg->learned ? 1 : 0;
    c->cfg.quadrupole = cfg->quadrupole ? 1 : 0;
    c->walk_ready = false;
    if (rebuild) return build_tree(c, true, c->stream);  // groups depend on gmax, moments on quad
    return TC_OK;
}

int tc_get_config(tc_ctx* c, tc_config* cfg)
{
    if (!c || !cfg) return fail(c, TC_EINVAL, "tc_get_config: null argument");
    *cfg = c->cfg;
    return TC_OK;
}

int tc_set_stream(tc_ctx* c, void* stream)
{
    if (!c) return fail(c, TC_EINVAL, "tc_set_stream: null context");
    TC_CUDA(c, cudaStreamSynchronize(c->stream));
    c->stream = (cudaStream_t)stream;
    return TC_OK;
}

int tc_ctx_build_batch(tc_ctx* c, const float* pos, const float* mass, const int64_t* offsets, int64_t nsys,
                       int leaf_max)
{
    if (!c) return fail(c, TC_EINVAL, "tc_build: null context");
    if (!pos || !mass || !offsets) return fail(c, TC_EINVAL, "tc_build: null pos, mass or offsets");
    if (nsys < 1 || nsys > (1 << 16)) return fail(c, TC_EINVAL, "tc_build: nsys must be in [1, 65536]");
    if (leaf_max < 1 || leaf_max > kLeafMaxLimit)
        return fail(c, TC_EINVAL, "tc_build: leaf_max must be in [1, %d] (got %d)", kLeafMaxLimit, leaf_max);
    std::vector<int64_t> off(nsys + 1);
    TC_CUDA(c, cudaMemcpy(off.data(), offsets, (nsys + 1) * sizeof(int64_t), cudaMemcpyDefault));
    if (off[0] != 0) return fail(c, TC_EINVAL, "tc_build: offsets[0] must be 0");
    for (int64_t s = 0; s < nsys; s++)
        if (off[s + 1] <= off[s]) return fail(c, TC_EINVAL, "tc_build: system %lld holds no body", (long long)s);
    const int64_t n = off[nsys];
    if (n >= (int64_t)1 << 31) return fail(c, TC_EINVAL, "tc_build: n must be below 2^31 (got %lld)", (long long)n);
    int r = ensure_bodies(c, n);
    if (r) return r;
    if (n != c->n) TC_CUDA(c, cudaMemsetAsync(c->vel, 0, 3 * n * sizeof(float), c->stream));
    c->n = n;
    c->leaf_max = leaf_max;
    if ((int)nsys != c->nsys || off != c->off_h) {
        r = setup_systems(c, off.data(), (int)nsys);
        if (r) return r;
    }
    TC_CUDA(c, cudaMemcpyAsync(c->pos, pos, 3 * n * sizeof(float), cudaMemcpyDefault, c->stream));
    TC_CUDA(c, cudaMemcpyAsync(c->mass, mass, n * sizeof(float), cudaMemcpyDefault, c->stream));
    c->built = false;
    return build_tree(c, true, c->stream);
}

int tc_ctx_build(tc_ctx* c, const float* pos, const float* mass, int64_t n, int leaf_max)
{
    if (!c) return fail(c, TC_EINVAL, "tc_build: null context");
    if (n < 1 || n >= (int64_t)1 << 31) return fail(c, TC_EINVAL, "tc_build: n must be in [1, 2^31) (got %lld)", (long long)n);
    const int64_t off[2] = {0, n};
    return tc_ctx_build_batch(c, pos, mass, off, 1, leaf_max);
}

int tc_ctx_set_velocity(tc_ctx* c, const float* vel)
{
    if (!c || !vel) return fail(c, TC_EINVAL, "tc_set_velocity: null argument");
    if (!c->built) return fail(c, TC_ESTATE, "tc_set_velocity: build first");
    TC_CUDA(c, cudaMemcpyAsync(c->vel, vel, 3 * c->n * sizeof(float), cudaMemcpyDefault, c->stream));
    return TC_OK;
}

int tc_ctx_forces(tc_ctx* c, float theta, float eps, float G)
{
    if (!c) return fail(c, TC_EINVAL, "tc_forces: null context");
    if (!c->built) return fail(c, TC_ESTATE, "tc_forces: build the tree first");
    if (!finite(theta) || theta < 0.f) return fail(c, TC_EINVAL, "tc_forces: theta must be finite and >= 0");
    if (!finite(eps) || eps <= 0.f) return fail(c, TC_EINVAL, "tc_forces: eps must be finite and > 0");
    if (!finite(G)) return fail(c, TC_EINVAL, "tc_forces: G must be finite");
    if (c->cfg.learned && !c->have_mlp) return fail(c, TC_ESTATE, "tc_forces: learned = 1 but no model is set");
    int r = prepare_forces(c);
    if (r) return r;
    return run_forces(c, theta, eps, G, c->stream);
}

int tc_ctx_step(tc_ctx* c, float dt)
{
    if (!c) return fail(c, TC_EINVAL, "tc_step: null context");
    if (!finite(dt)) return fail(c, TC_EINVAL, "tc_step: dt must be finite");
    if (!c->have_forces) return fail(c, TC_ESTATE, "tc_step: compute forces on the current positions first");
    if (c->forces_fmm)
        return fail(c, TC_ESTATE, "tc_step: the step integrates with the treecode; call tc_ctx_forces first");
    if (c->cfg.graph) return step_graph(c, dt);
    return step_eager(c, dt);
}

int tc_sync(tc_ctx* c)
{
    if (!c) return fail(c, TC_EINVAL, "tc_sync: null context");
    return check_device(c);
}

int tc_get_acc(tc_ctx* c, float* acc, float* pot)
{
    if (!c) return fail(c, TC_EINVAL, "tc_get_acc: null context");
    if (!c->have_forces) return fail(c, TC_ESTATE, "tc_get_acc: no forces computed");
    if (pot && !c->forces_pot) return fail(c, TC_ESTATE, "tc_get_acc: potential not computed (want_pot = 0)");
    int r = check_device(c);
    if (r) return r;
    if (acc) TC_CUDA(c, cudaMemcpyAsync(acc, c->acc, 3 * c->n * sizeof(float), cudaMemcpyDefault, c->stream));
    if (pot) TC_CUDA(c, cudaMemcpyAsync(pot, c->pot, c->n * sizeof(float), cudaMemcpyDefault, c->stream));
    TC_CUDA(c, cudaStreamSynchronize(c->stream));
    return TC_OK;
}

int tc_get_state(tc_ctx* c, float* pos, float* vel)
{
    if (!c) return fail(c, TC_EINVAL, "tc_get_state: null context");
    if (!c->built) return fail(c, TC_ESTATE, "tc_get_state: build first");
    if (pos) TC_CUDA(c, cudaMemcpyAsync(pos, c->pos, 3 * c->n * sizeof(float), cudaMemcpyDefault, c->stream));
    if (vel) TC_CUDA(c, cudaMemcpyAsync(vel, c->vel, 3 * c->n * sizeof(float), cudaMemcpyDefault, c->stream));
    return check_device(c);
}

int tc_set_state(tc_ctx* c, const float* pos, const float* vel)
{
    if (!c || !pos || !vel) return fail(c, TC_EINVAL, "tc_set_state: null argument");
    if (!c->built) return fail(c, TC_ESTATE, "tc_set_state: build first");
    TC_CUDA(c, cudaMemcpyAsync(c->pos, pos, 3 * c->n * sizeof(float), cudaMemcpyDefault, c->stream));
    TC_CUDA(c, cudaMemcpyAsync(c->vel, vel, 3 * c->n * sizeof(float), cudaMemcpyDefault, c->stream));
    return build_tree(c, true, c->stream);
}

int tc_get_sizes(tc_ctx* c, int64_t* n, int64_t* nnodes, int64_t* ngroups)
{
    if (!c) return fail(c, TC_EINVAL, "tc_get_sizes: null context");
    if (!c->built) return fail(c, TC_ESTATE, "tc_get_sizes: build first");
    int r = check_device(c);
    if (r) return r;
    if (n) *n = c->n;
    if (nnodes) *nnodes = c->info_h->M;
    if (ngroups) *ngroups = c->info_h->G;
    return TC_OK;
}

int tc_get_systems(tc_ctx* c, int64_t* nsys, double* cubes)
{
    if (!c) return fail(c, TC_EINVAL, "tc_get_systems: null context");
    if (!c->built) return fail(c, TC_ESTATE, "tc_get_systems: build first");
    int r = check_device(c);
    if (r) return r;
    if (nsys) *nsys = c->nsys;
    if (cubes) {
        std::vector<SysParams> sp(c->nsys);
        TC_CUDA(c, cudaMemcpy(sp.data(), c->sysp, c->nsys * sizeof(SysParams), cudaMemcpyDeviceToHost));
        for (int s = 0; s < c->nsys; s++) {
            for (int a = 0; a < 3; a++) cubes[5 * s + a] = sp[s].c0[a];
            cubes[5 * s + 3] = sp[s].L;
            cubes[5 * s + 4] = sp[s].h;
        }
    }
    return TC_OK;
}

int tc_get_cube(tc_ctx* c, double* out5)
{
    if (!c || !out5) return fail(c, TC_EINVAL, "tc_get_cube: null argument");
    if (!c->built) return fail(c, TC_ESTATE, "tc_get_cube: build first");
    std::vector<double> all(5 * (size_t)c->nsys);
    int r = tc_get_systems(c, nullptr, all.data());
    if (r) return r;
    for (int k = 0; k < 5; k++) out5[k] = all[k];
    return TC_OK;
}

int tc_get_tree(tc_ctx* c, uint32_t* perm, uint64_t* keys)
{
    if (!c) return fail(c, TC_EINVAL, "tc_get_tree: null context");
    if (!c->built) return fail(c, TC_ESTATE, "tc_get_tree: build first");
    if (perm) TC_CUDA(c, cudaMemcpyAsync(perm, c->perm, c->n * sizeof(uint32_t), cudaMemcpyDefault, c->stream));
    if (keys) TC_CUDA(c, cudaMemcpyAsync(keys, c->keys, c->n * sizeof(uint64_t), cudaMemcpyDefault, c->stream));
    return check_device(c);
}

int tc_get_nodes(tc_ctx* c, int32_t* level, uint64_t* prefix, int32_t* first, int32_t* count, int32_t* child_first,
                 int32_t* nchild, double* mass, double* com, double* quad)
{
    if (!c) return fail(c, TC_EINVAL, "tc_get_nodes: null context");
    if (!c->built) return fail(c, TC_ESTATE, "tc_get_nodes: build first");
    if (quad && !c->cfg.quad) return fail(c, TC_ESTATE, "tc_get_nodes: second moments not computed (quad = 0)");
    int r = check_device(c);
    if (r) return r;
    const int64_t M = c->info_h->M;
    std::vector<int4> b(M);
    TC_CUDA(c, cudaMemcpy(b.data(), c->nt.b, M * sizeof(int4), cudaMemcpyDeviceToHost));
    std::vector<uint64_t> keys;
    if (prefix) {
        keys.resize(c->n);
        TC_CUDA(c, cudaMemcpy(keys.data(), c->keys, c->n * sizeof(uint64_t), cudaMemcpyDeviceToHost));
    }
    for (int64_t v = 0; v < M; v++) {
        int l = b[v].w & 255;
        if (level) level[v] = l;
        if (first) first[v] = b[v].x;
        if (count) count[v] = b[v].y;
        if (child_first) child_first[v] = b[v].z;
        if (nchild) nchild[v] = b[v].w >> 8;
        if (prefix) prefix[v] = l == 0 ? 0ull : (keys[b[v].x] >> (3 * (kMaxLevel - l)));
    }
    if (mass) TC_CUDA(c, cudaMemcpy(mass, c->nt.mass64, M * sizeof(double), cudaMemcpyDefault));
    if (com) TC_CUDA(c, cudaMemcpy(com, c->nt.com64, 3 * M * sizeof(double), cudaMemcpyDefault));
    if (quad) {
        std::vector<float> qf((size_t)6 * M);
        TC_CUDA(c, cudaMemcpy(qf.data(), c->nt.quad, 6 * M * sizeof(float), cudaMemcpyDeviceToHost));
        std::vector<double> qd(qf.begin(), qf.end());
        TC_CUDA(c, cudaMemcpy(quad, qd.data(), 6 * M * sizeof(double), cudaMemcpyDefault));
    }
    return TC_OK;
}

int tc_get_groups(tc_ctx* c, int32_t* gfirst, int32_t* gcount, int32_t* gref)
{
    if (!c) return fail(c, TC_EINVAL, "tc_get_groups: null context");
    if (!c->built) return fail(c, TC_ESTATE, "tc_get_groups: build first");
    int r = check_device(c);
    if (r) return r;
    const int64_t G = c->info_h->G;
    std::vector<int32_t> f(G + 1);
    TC_CUDA(c, cudaMemcpy(f.data(), c->gfirst, (G + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost));
    if (gref) TC_CUDA(c, cudaMemcpy(gref, c->gref, G * sizeof(int32_t), cudaMemcpyDefault));
    for (int64_t g = 0; g < G; g++) {
        if (gfirst) gfirst[g] = f[g];
        if (gcount) gcount[g] = f[g + 1] - f[g];
    }
    return TC_OK;
}

int tc_get_lists(tc_ctx* c, int32_t* ncell, int32_t* nbody, uint64_t* hash, int64_t* inter, int64_t* cells,
                 int64_t* bodies)
{
    if (!c) return fail(c, TC_EINVAL, "tc_get_lists: null context");
    if (!c->have_forces) return fail(c, TC_ESTATE, "tc_get_lists: no forces computed");
    if ((ncell || nbody || hash) && !c->cfg.verify)
        return fail(c, TC_ESTATE, "tc_get_lists: per-group lists need verify = 1");
    int r = check_device(c);
    if (r) return r;
    const int64_t G = c->info_h->G;
    if (ncell) TC_CUDA(c, cudaMemcpy(ncell, c->ncell, G * sizeof(int32_t), cudaMemcpyDefault));
    if (nbody) TC_CUDA(c, cudaMemcpy(nbody, c->nbody, G * sizeof(int32_t), cudaMemcpyDefault));
    if (hash) TC_CUDA(c, cudaMemcpy(hash, c->hash, G * sizeof(uint64_t), cudaMemcpyDefault));
    if (inter) *inter = (int64_t)c->info_h->interactions;
    if (cells) *cells = (int64_t)c->info_h->cells;
    if (bodies) *bodies = (int64_t)c->info_h->bodies;
    return TC_OK;
}

int tc_diag(tc_ctx* c, double* out8)
{
    if (!c || !out8) return fail(c, TC_EINVAL, "tc_diag: null argument");
    if (!c->built) return fail(c, TC_ESTATE, "tc_diag: build first");
    const float* pot = (c->have_forces && c->forces_pot) ? c->pot : nullptr;
    launch_diag(c->pos, c->vel, c->mass, pot, c->n, c->info, c->stream);
    TC_CUDA(c, cudaGetLastError());
    int r = check_device(c);
    if (r) return r;
    for (int k = 0; k < 8; k++) out8[k] = c->info_h->diag[k];
    if (!pot) out8[1] = NAN;
    return TC_OK;
}

int tc_ctx_fmm(tc_ctx* c, float theta, float eps, float G)
{
    if (!c) return fail(c, TC_EINVAL, "tc_fmm: null context");
    if (!c->built) return fail(c, TC_ESTATE, "tc_fmm: build the tree first");
    if (!finite(theta) || theta < 0.f) return fail(c, TC_EINVAL, "tc_fmm: theta must be finite and >= 0");
    if (!finite(eps) || eps <= 0.f) return fail(c, TC_EINVAL, "tc_fmm: eps must be finite and > 0");
    if (!finite(G)) return fail(c, TC_EINVAL, "tc_fmm: G must be finite");
    int r = check_device(c);  // synchronises: the last build's node count, no pending error
    if (r) return r;
    const int64_t M = c->info_h->M;
    cudaStream_t s = c->stream;
    if (c->fmm_cap_m < c->cap_m) {
        TC_GROW(c, c->fmm_parent, c->cap_m);
        TC_GROW(c, c->fmm_loc, c->cap_m * fmm_loc_width());
        TC_GROW(c, c->fmm_off, c->cap_m);
        TC_GROW(c, c->fmm_cnt, c->cap_m);
        TC_GROW(c, c->fmm_rec, 4 * c->cap_m);
        TC_GROW(c, c->fmm_rad, c->cap_m);
        TC_GROW(c, c->fmm_fnode, 3 * c->cap_m);
        c->fmm_cap_m = c->cap_m;
    }
    if (!c->fmm_ctr) TC_GROW(c, c->fmm_ctr, 8);
    if (!c->fmm_lstart) TC_GROW(c, c->fmm_lstart, kFmmLevelSlots);
    launch_fmm_level_starts(c->info, c->cap_m, c->nt, c->fmm_lstart, s);
    TC_CUDA(c, cudaGetLastError());
    int64_t ls[kFmmLevelSlots];
    TC_CUDA(c, cudaMemcpyAsync(ls, c->fmm_lstart, sizeof(ls), cudaMemcpyDeviceToHost, s));
    TC_CUDA(c, cudaStreamSynchronize(s));
    int depth = 0;
    while (depth < kMaxLevel && ls[depth + 1] < M) depth++;
    // the pools and slabs start at an estimate and grow to what an attempt
    // that overflowed them counted; the overflowing attempt is discarded
    // (TC_FMM_POOL / TC_FMM_SLAB, in entries, override the first estimate
    // of a context, to exercise the regrowth)
    int64_t want_pool = std::max<int64_t>(c->fmm_pool_cap, 32 * c->cap_m + 65536);
    int64_t want_slab = std::max<int64_t>(c->fmm_slab_cap, 4096);
    if (c->fmm_pool_cap == 0)
        if (const char* env = getenv("TC_FMM_POOL")) want_pool = std::max<long long>(1, atoll(env));
    if (c->fmm_slab_cap == 0)
        if (const char* env = getenv("TC_FMM_SLAB")) want_slab = std::max<long long>(1, atoll(env));
    cudaEvent_t t0 = phase_begin(c, s, 1);
    unsigned long long ctr[8];
    for (int attempt = 0;; attempt++) {
        if (want_pool > c->fmm_pool_cap) {
            TC_GROW(c, c->fmm_pool[0], want_pool);
            TC_GROW(c, c->fmm_pool[1], want_pool);
            c->fmm_pool_cap = want_pool;
        }
        const int64_t warps = fmm_slab_warps();
        if (want_slab > c->fmm_slab_cap || warps != c->fmm_slab_warps) {
            TC_GROW(c, c->fmm_slab, want_slab * warps);
            c->fmm_slab_cap = want_slab;
            c->fmm_slab_warps = warps;
        }
        TC_CUDA(c, cudaMemsetAsync(c->fmm_ctr, 0, 8 * sizeof(unsigned long long), s));
        TC_CUDA(c, cudaMemsetAsync(c->fmm_cnt, 0, c->cap_m * sizeof(int32_t), s));
        TC_CUDA(c, cudaMemsetAsync(c->fmm_off, 0, c->cap_m * sizeof(int64_t), s));
        FmmLaunch p{};
        p.body = c->body;
        p.perm = c->perm;
        p.sysp = c->sysp;
        p.nt = c->nt;
        p.info = c->info;
        p.err = &c->info->err;
        p.cap_m = c->cap_m;
        p.parent = c->fmm_parent;
        p.loc = c->fmm_loc;
        p.pool[0] = c->fmm_pool[0];
        p.pool[1] = c->fmm_pool[1];
        p.pool_cap = c->fmm_pool_cap;
        p.slab = c->fmm_slab;
        p.slab_cap = c->fmm_slab_cap;
        p.near_off = c->fmm_off;
        p.near_cnt = c->fmm_cnt;
        p.ctr = c->fmm_ctr;
        p.rec = c->fmm_rec;
        p.rad = c->fmm_rad;
        p.fnode = c->fmm_fnode;
        p.records = c->cfg.verify;
        p.acc = c->acc;
        p.theta = theta;
        p.eps = eps;
        p.G = G;
        cudaError_t e = launch_fmm(p, ls, depth, s);
        if (e != cudaSuccess) return fail(c, TC_ECUDA, "fmm launch: %s", cudaGetErrorString(e));
        TC_CUDA(c, cudaMemcpyAsync(ctr, c->fmm_ctr, sizeof(ctr), cudaMemcpyDeviceToHost, s));
        TC_CUDA(c, cudaStreamSynchronize(s));
        TC_CUDA(c, cudaMemcpy(c->info_h, c->info, sizeof(Info), cudaMemcpyDeviceToHost));
        const int32_t err = c->info_h->err;
        const int32_t grow_bits = kErrFmmPool | kErrFmmSlab;
        // a level that overflowed handed its children short lists, so deeper
        // levels may need more than this pass counted: grow at least 2x
        if ((err & grow_bits) && !(err & ~grow_bits) && attempt < 16) {
            TC_CUDA(c, cudaMemsetAsync(&c->info->err, 0, sizeof(int32_t), s));
            if (err & kErrFmmPool)
                want_pool = std::max<int64_t>((int64_t)(ctr[2] + ctr[2] / 4 + 4096), 2 * c->fmm_pool_cap);
            if (err & kErrFmmSlab)
                want_slab = std::max<int64_t>((int64_t)(ctr[3] + ctr[3] / 4 + 256), 2 * c->fmm_slab_cap);
            continue;
        }
        if (err) {
            c->have_forces = false;
            return check_device(c);  // reports and clears the error word
        }
        break;
    }
    phase_end(c, 1, t0, s);
    for (int k = 0; k < 4; k++) c->fmm_stats[k] = ctr[4 + k];
    c->fmm_records = c->cfg.verify != 0;
    c->have_forces = true;
    c->forces_fmm = true;
    c->forces_pot = false;
    return TC_OK;
}

int tc_get_fmm_pairs(tc_ctx* c, int64_t* nm2l, int64_t* np2p, uint64_t* hm2l, uint64_t* hp2p)
{
    if (!c) return fail(c, TC_EINVAL, "tc_get_fmm_pairs: null context");
    if (!c->have_forces || !c->forces_fmm) return fail(c, TC_ESTATE, "tc_get_fmm_pairs: the last forces were not tc_ctx_fmm's");
    if (!c->fmm_records) return fail(c, TC_ESTATE, "tc_get_fmm_pairs: per-cell records need verify = 1");
    const int64_t M = c->info_h->M;
    std::vector<unsigned long long> rec(4 * M);
    TC_CUDA(c, cudaMemcpy(rec.data(), c->fmm_rec, rec.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
    for (int64_t v = 0; v < M; v++) {
        if (nm2l) nm2l[v] = (int64_t)rec[4 * v];
        if (np2p) np2p[v] = (int64_t)rec[4 * v + 1];
        if (hm2l) hm2l[v] = rec[4 * v + 2];
        if (hp2p) hp2p[v] = rec[4 * v + 3];
    }
    return TC_OK;
}

int tc_get_fmm_stats(tc_ctx* c, int64_t* m2l, int64_t* p2p, uint64_t* hash2)
{
    if (!c) return fail(c, TC_EINVAL, "tc_get_fmm_stats: null context");
    if (!c->have_forces || !c->forces_fmm) return fail(c, TC_ESTATE, "tc_get_fmm_stats: the last forces were not tc_ctx_fmm's");
    if (hash2 && !c->fmm_records) return fail(c, TC_ESTATE, "tc_get_fmm_stats: pair-set hashes need verify = 1");
    if (m2l) *m2l = (int64_t)c->fmm_stats[0];
    if (p2p) *p2p = (int64_t)c->fmm_stats[1];
    if (hash2) {
        hash2[0] = c->fmm_stats[2];
        hash2[1] = c->fmm_stats[3];
    }
    return TC_OK;
}

int tc_direct(tc_ctx* c, const int64_t* idx, int64_t ns, float eps, float G, double* acc, double* pot)
{
    if (!c || !idx || !acc) return fail(c, TC_EINVAL, "tc_direct: null argument");
    if (!c->built) return fail(c, TC_ESTATE, "tc_direct: build first");
    if (ns < 1) return fail(c, TC_EINVAL, "tc_direct: ns must be >= 1");
    if (!finite(eps) || eps <= 0.f || !finite(G)) return fail(c, TC_EINVAL, "tc_direct: eps > 0 and finite G required");
    std::vector<int64_t> hidx(ns);
    TC_CUDA(c, cudaMemcpy(hidx.data(), idx, ns * sizeof(int64_t), cudaMemcpyDefault));
    for (int64_t k = 0; k < ns; k++)
        if (hidx[k] < 0 || hidx[k] >= c->n)
            return fail(c, TC_EINVAL, "tc_direct: index %lld out of range", (long long)hidx[k]);
    if (ns > c->cap_idx) {
        TC_GROW(c, c->idx_dev, ns);
        TC_GROW(c, c->dir_out, 4 * ns);
        c->cap_idx = ns;
    }
    TC_CUDA(c, cudaMemcpyAsync(c->idx_dev, hidx.data(), ns * sizeof(int64_t), cudaMemcpyHostToDevice, c->stream));
    launch_direct(c->pos, c->mass, c->sys_of, c->sysp, c->idx_dev, ns, eps * eps, G, c->dir_out, c->dir_out + 3 * ns,
                  c->stream);
    TC_CUDA(c, cudaGetLastError());
    TC_CUDA(c, cudaMemcpyAsync(acc, c->dir_out, 3 * ns * sizeof(double), cudaMemcpyDefault, c->stream));
    if (pot) TC_CUDA(c, cudaMemcpyAsync(pot, c->dir_out + 3 * ns, ns * sizeof(double), cudaMemcpyDefault, c->stream));
    return check_device(c);
}

int tc_set_timing(tc_ctx* c, int on)
{
    if (!c) return fail(c, TC_EINVAL, "tc_set_timing: null context");
    TC_CUDA(c, cudaStreamSynchronize(c->stream));
    c->timing = on != 0;
    for (auto& v : c->ev_phase) v.clear();
    c->ev_used = 0;
    c->launches_mark = launches_total();
    return TC_OK;
}

int tc_get_timings(tc_ctx* c, double* out6)
{
    if (!c || !out6) return fail(c, TC_EINVAL, "tc_get_timings: null argument");
    int r = check_device(c);
    if (r) return r;
    for (int p = 0; p < 3; p++) {
        double ms = 0.0;
        for (auto& pr : c->ev_phase[p]) {
            float t = 0.f;
            TC_CUDA(c, cudaEventElapsedTime(&t, pr.first, pr.second));
            ms += t;
        }
        out6[p] = ms;
        c->ev_phase[p].clear();
    }
    long long now = launches_total();
    out6[3] = (double)(now - c->launches_mark);
    c->launches_mark = now;
    c->ev_used = 0;
    out6[4] = (double)launches_total();
    out6[5] = (double)c->graph_kernels;
    return TC_OK;
}
}  // extern "C"

// ---------------------------------------------------------------- learned correction
namespace {

// copies of the learned-correction calls run on the context's stream and are
// waited for (host staging buffers are locals)
#define TC_COPY(c, dst, src, bytes)                                                              \
    do {                                                                                         \
        TC_CUDA(c, cudaMemcpyAsync((dst), (src), (bytes), cudaMemcpyDefault, (c)->stream));       \
        TC_CUDA(c, cudaStreamSynchronize((c)->stream));                                          \
    } while (0)

constexpr int kMlpNModel = kMlpNParamHost + 2 * 13 + 3;  // parameters + feature means, scales + output scales



int mlp_alloc(tc_ctx* c)
{
    if (c->mlp_params) return TC_OK;
    TC_GROW(c, c->mlp_params, kMlpNParamHost);
    TC_GROW(c, c->mlp_maps, 32);
    TC_GROW(c, *(char**)&c->mlp_dev, (int64_t)mlp_dev_size());
    TC_GROW(c, c->mlp_m, kMlpNParamHost);
    TC_GROW(c, c->mlp_v, kMlpNParamHost);
    TC_GROW(c, c->mlp_grad, kMlpNParamHost);
    TC_GROW(c, c->mlp_loss, 4);
    TC_GROW(c, c->mlp_evals, 1);
    TC_GROW(c, c->mlp_sums, kMlpSums);
    TC_GROW(c, c->mlp_wscale, 1);
    TC_GROW(c, c->mlp_bad, 1);
    TC_CUDA(c, cudaMemsetAsync(c->mlp_evals, 0, sizeof(*c->mlp_evals), c->stream));
    return TC_OK;
}

int mlp_scratch(tc_ctx* c, int64_t n)
{
    if (n <= c->mlp_cap) return TC_OK;
    TC_GROW(c, c->mlp_x, n * 16);
    TC_GROW(c, c->mlp_t, n * 3);
    TC_GROW(c, c->mlp_w, n);
    TC_GROW(c, c->mlp_idx, n);
    TC_GROW(c, c->mlp_raw, n * 13);
    c->mlp_cap = n;
    return TC_OK;
}

// raw features X (n x 13) and targets T (n x 3, nullable), host or device
// memory, -> normalised padded rows in mlp_x and scaled targets in mlp_t
// (kernels; the inputs are first copied as they are)
int mlp_rows(tc_ctx* c, const float* X, const float* T, int64_t n)
{
    TC_CUDA(c, cudaMemcpyAsync(c->mlp_raw, X, n * 13 * sizeof(float), cudaMemcpyDefault, c->stream));
    if (T) TC_CUDA(c, cudaMemcpyAsync(c->mlp_t, T, n * 3 * sizeof(float), cudaMemcpyDefault, c->stream));
    // the scaled targets are written in place of the raw ones
    launch_mlp_rows(c->mlp_raw, T ? c->mlp_t : nullptr, n, c->mlp_maps, c->mlp_x, c->mlp_t, c->stream);
    TC_CUDA(c, cudaGetLastError());
    return TC_OK;
}

// per-pair loss weights (n, host or device; nullable) -> c->mlp_w: mode 0
// the given weights (checked: finite, >= 0), mode 1 W holds the pairs' label
// factors F and the weights become F^2 / mean(F^2) (needs mlp_wscale from
// the training data's sums); *wdev = the device pointer to pass to the
// training kernel (null without weights)
int mlp_weights(tc_ctx* c, const float* W, int mode, int64_t n, const float** wdev)
{
    *wdev = nullptr;
    if (!W) return TC_OK;
    TC_CUDA(c, cudaMemcpyAsync(c->mlp_w, W, n * sizeof(float), cudaMemcpyDefault, c->stream));
    TC_CUDA(c, cudaMemsetAsync(c->mlp_bad, 0, sizeof(int32_t), c->stream));
    launch_mlp_weights(c->mlp_w, n, mode, c->mlp_wscale, c->mlp_bad, c->stream);
    TC_CUDA(c, cudaGetLastError());
    int32_t bad = 0;
    TC_COPY(c, &bad, c->mlp_bad, sizeof(int32_t));
    if (bad)
        return fail(c, TC_EINVAL, mode ? "mlp label factors must be finite" : "mlp weights must be finite and >= 0");
    *wdev = c->mlp_w;
    return TC_OK;
}

int mlp_upload(tc_ctx* c, const float* model)
{
    int r = mlp_alloc(c);
    if (r) return r;
    std::vector<float> h(kMlpNModel);
    TC_COPY(c, h.data(), model, kMlpNModel * sizeof(float));
    for (float v : h)
        if (!std::isfinite(v)) return fail(c, TC_EINVAL, "tc_mlp_set: non-finite model value");
    TC_COPY(c, c->mlp_params, h.data(), kMlpNParamHost * sizeof(float));
    TC_COPY(c, c->mlp_maps, h.data() + kMlpNParamHost, 29 * sizeof(float));
    launch_mlp_pack(c->mlp_params, c->mlp_maps, c->mlp_dev, c->stream);
    TC_CUDA(c, cudaGetLastError());
    c->have_mlp = true;
    c->walk_ready = false;
    drop_graph(c);
    return TC_OK;
}

}  // namespace

extern "C" {

int tc_mlp_set(tc_ctx* c, const float* model, float band)
{
    if (!c || !model) return fail(c, TC_EINVAL, "tc_mlp_set: null argument");
    if (!finite(band) || band < 0.f) return fail(c, TC_EINVAL, "tc_mlp_set: band must be finite and >= 0");
    c->mlp_band = band;
    return mlp_upload(c, model);
}

int tc_mlp_get(tc_ctx* c, float* model, float* band)
{
    if (!c) return fail(c, TC_EINVAL, "tc_mlp_get: null context");
    if (!c->have_mlp) return fail(c, TC_ESTATE, "tc_mlp_get: no model");
    if (model) {
        TC_COPY(c, model, c->mlp_params, kMlpNParamHost * sizeof(float));
        TC_COPY(c, model + kMlpNParamHost, c->mlp_maps, 29 * sizeof(float));
    }
    if (band) *band = c->mlp_band;
    return TC_OK;
}

int tc_mlp_forward(tc_ctx* c, const float* X, int64_t n, float* Y)
{
    if (!c || !X || !Y) return fail(c, TC_EINVAL, "tc_mlp_forward: null argument");
    if (!c->have_mlp) return fail(c, TC_ESTATE, "tc_mlp_forward: no model");
    if (n < 1) return fail(c, TC_EINVAL, "tc_mlp_forward: n must be >= 1");
    int r = mlp_scratch(c, n);
    if (r) return r;
    if ((r = mlp_rows(c, X, nullptr, n))) return r;
    launch_mlp_infer(c->mlp_x, n, c->mlp_dev, c->mlp_t, c->stream);
    TC_CUDA(c, cudaGetLastError());
    TC_CUDA(c, cudaMemcpyAsync(Y, c->mlp_t, n * 3 * sizeof(float), cudaMemcpyDefault, c->stream));
    return check_device(c);
}

// scratch of a training step's per-warp partial gradients
static int mlp_part(tc_ctx* c, int blocks)
{
    const int64_t want = mlp_train_part_floats(blocks);
    if (want > c->mlp_part_cap) {
        TC_GROW(c, c->mlp_part, want);
        c->mlp_part_cap = want;
    }
    return TC_OK;
}

int tc_mlp_loss_grad(tc_ctx* c, const float* X, const float* T, const float* W, int64_t n, float* grad, float* loss)
{
    if (!c || !X || !T) return fail(c, TC_EINVAL, "tc_mlp_loss_grad: null argument");
    if (!c->have_mlp) return fail(c, TC_ESTATE, "tc_mlp_loss_grad: no model");
    if (n < 1 || n >= (int64_t)1 << 31) return fail(c, TC_EINVAL, "tc_mlp_loss_grad: bad n");
    int r = mlp_scratch(c, n);
    if (r) return r;
    if ((r = mlp_rows(c, X, T, n))) return r;
    launch_mlp_shuffle(n, 0, c->mlp_idx, c->stream);  // key 0: the rows in order
    const float* wdev = nullptr;
    if ((r = mlp_weights(c, W, 0, n, &wdev))) return r;
    TC_CUDA(c, cudaMemsetAsync(c->mlp_loss, 0, sizeof(float), c->stream));
    int64_t blocks = (n + 63) / 64;
    if (blocks > 2 * c->num_sms) blocks = 2 * c->num_sms;
    if ((r = mlp_part(c, (int)blocks))) return r;
    cudaError_t e = launch_mlp_train(c->mlp_x, c->mlp_t, wdev, c->mlp_idx, (int)n, c->mlp_dev, c->mlp_grad,
                                     c->mlp_loss, c->mlp_part, (int)blocks, c->stream);
    if (e != cudaSuccess) return fail(c, TC_ECUDA, "mlp training kernel: %s", cudaGetErrorString(e));
    if (grad) TC_CUDA(c, cudaMemcpyAsync(grad, c->mlp_grad, kMlpNParamHost * sizeof(float), cudaMemcpyDefault, c->stream));
    if (loss) TC_CUDA(c, cudaMemcpyAsync(loss, c->mlp_loss, sizeof(float), cudaMemcpyDefault, c->stream));
    return check_device(c);
}

int tc_mlp_train(tc_ctx* c, const float* X, const float* T, const float* W, int32_t weight_mode, int64_t n,
                 int epochs, int batch, float lr, uint64_t seed, float band, float* losses)
{
    if (!c || !X || !T) return fail(c, TC_EINVAL, "tc_mlp_train: null argument");
    if (n < 16 || n >= (int64_t)1 << 31) return fail(c, TC_EINVAL, "tc_mlp_train: need 16 <= n < 2^31 pairs");
    if (epochs < 1 || batch < 16 || !finite(lr) || lr <= 0.f || !finite(band) || band < 0.f)
        return fail(c, TC_EINVAL, "tc_mlp_train: epochs >= 1, batch >= 16, lr > 0, band >= 0 required");
    if (weight_mode != TC_MLP_WEIGHTS && weight_mode != TC_MLP_FACTORS)
        return fail(c, TC_EINVAL, "tc_mlp_train: weight_mode must be TC_MLP_WEIGHTS or TC_MLP_FACTORS");
    if (weight_mode == TC_MLP_FACTORS && !W) return fail(c, TC_EINVAL, "tc_mlp_train: TC_MLP_FACTORS needs W");
    int r = mlp_alloc(c);
    if (r) return r;
    if ((r = mlp_scratch(c, n))) return r;
    // the data as given, then (kernels) its sums, the model's maps (feature
    // means and scales, output RMS), fresh parameters, normalised rows and
    // scaled targets, loss weights
    TC_CUDA(c, cudaMemcpyAsync(c->mlp_raw, X, n * 13 * sizeof(float), cudaMemcpyDefault, c->stream));
    TC_CUDA(c, cudaMemcpyAsync(c->mlp_t, T, n * 3 * sizeof(float), cudaMemcpyDefault, c->stream));
    if (W) TC_CUDA(c, cudaMemcpyAsync(c->mlp_w, W, n * sizeof(float), cudaMemcpyDefault, c->stream));
    launch_mlp_sums(c->mlp_raw, c->mlp_t, weight_mode == TC_MLP_FACTORS ? c->mlp_w : nullptr, n, c->mlp_sums,
                    c->stream);
    launch_mlp_maps(c->mlp_sums, n, c->mlp_maps, c->mlp_wscale, c->stream);
    launch_mlp_init(c->mlp_params, seed, c->stream);
    launch_mlp_pack(c->mlp_params, c->mlp_maps, c->mlp_dev, c->stream);
    launch_mlp_rows(c->mlp_raw, c->mlp_t, n, c->mlp_maps, c->mlp_x, c->mlp_t, c->stream);
    TC_CUDA(c, cudaGetLastError());
    c->mlp_band = band;
    c->have_mlp = true;
    c->walk_ready = false;
    drop_graph(c);
    const float* wdev = nullptr;
    if (W) {
        TC_CUDA(c, cudaMemsetAsync(c->mlp_bad, 0, sizeof(int32_t), c->stream));
        launch_mlp_weights(c->mlp_w, n, weight_mode == TC_MLP_FACTORS ? 1 : 0, c->mlp_wscale, c->mlp_bad, c->stream);
        TC_CUDA(c, cudaGetLastError());
        int32_t bad = 0;
        TC_COPY(c, &bad, c->mlp_bad, sizeof(int32_t));
        if (bad) {
            c->have_mlp = false;
            return fail(c, TC_EINVAL, weight_mode == TC_MLP_FACTORS ? "tc_mlp_train: label factors must be finite"
                                                                    : "tc_mlp_train: weights must be finite and >= 0");
        }
        wdev = c->mlp_w;
    }
    TC_CUDA(c, cudaMemsetAsync(c->mlp_m, 0, kMlpNParamHost * sizeof(float), c->stream));
    TC_CUDA(c, cudaMemsetAsync(c->mlp_v, 0, kMlpNParamHost * sizeof(float), c->stream));
    int step = 0;
    const int64_t total_steps = (int64_t)epochs * ((n + batch - 1) / batch);
    uint64_t key = seed;
    for (int ep = 0; ep < epochs; ep++) {
        // a fresh seeded permutation of the pairs each pass (on the device)
        key = key * 6364136223846793005ull + 1442695040888963407ull;
        launch_mlp_shuffle(n, key, c->mlp_idx, c->stream);
        TC_CUDA(c, cudaMemsetAsync(c->mlp_loss, 0, sizeof(float), c->stream));
        int nb = 0;
        for (int64_t b0 = 0; b0 < n; b0 += batch) {
            const int B = (int)std::min<int64_t>(batch, n - b0);
            int64_t blocks = (B + 63) / 64;
            if (blocks > 2 * c->num_sms) blocks = 2 * c->num_sms;
            if ((r = mlp_part(c, (int)blocks))) return r;
            cudaError_t e = launch_mlp_train(c->mlp_x, c->mlp_t, wdev, c->mlp_idx + b0, B, c->mlp_dev,
                                             c->mlp_grad, c->mlp_loss, c->mlp_part, (int)blocks, c->stream);
            if (e != cudaSuccess) return fail(c, TC_ECUDA, "mlp training kernel: %s", cudaGetErrorString(e));
            // cosine decay of the learning rate over all steps
            const float lr_t = (float)(0.5 * lr * (1.0 + std::cos(3.141592653589793 * step / (double)total_steps)));
            launch_adam(c->mlp_params, c->mlp_m, c->mlp_v, c->mlp_grad, kMlpNParamHost, lr_t, ++step, c->stream);
            launch_mlp_pack(c->mlp_params, c->mlp_maps, c->mlp_dev, c->stream);
            nb++;
        }
        if (losses) {
            float l = 0.f;
            TC_COPY(c, &l, c->mlp_loss, sizeof(float));
            losses[ep] = l / (float)nb;
        }
    }
    return check_device(c);
}

int tc_mlp_pairs(tc_ctx* c, float theta, float eps, float band, float prob, uint64_t seed, int64_t max_pairs, float* X,
                 float* T, float* F, int64_t* body, int64_t* node, int64_t* npairs)
{
    if (!c || !npairs) return fail(c, TC_EINVAL, "tc_mlp_pairs: null argument");
    if (!c->built) return fail(c, TC_ESTATE, "tc_mlp_pairs: build first");
    if (!c->cfg.quad) return fail(c, TC_ESTATE, "tc_mlp_pairs: the features need quad = 1");
    if (!finite(theta) || theta < 0.f || !finite(eps) || eps <= 0.f || !finite(band) || band < 0.f ||
        !(prob > 0.f && prob <= 1.f) || max_pairs < 1)
        return fail(c, TC_EINVAL, "tc_mlp_pairs: theta >= 0, eps > 0, band >= 0, 0 < prob <= 1, max_pairs >= 1");
    if (max_pairs > c->pair_cap) {
        TC_GROW(c, c->pair_b, max_pairs);
        TC_GROW(c, c->pair_v, max_pairs);
        TC_GROW(c, c->pair_n, 1);
        c->pair_cap = max_pairs;
    }
    if (max_pairs > c->pair_sort_cap) {
        const int64_t cap = max_pairs;
        TC_GROW(c, c->pair_key, cap);
        TC_GROW(c, c->pair_val, cap);
        TC_GROW(c, c->pair_sb.keys_alt, cap);
        TC_GROW(c, c->pair_sb.vals_alt, cap);
        TC_GROW(c, c->pair_sb.ghist, kSortMaxPasses * 256);
        TC_GROW(c, c->pair_sb.status, (int64_t)kSortMaxPasses * radix_tiles(cap) * 256);
        TC_GROW(c, c->pair_sb.tiles, kSortMaxPasses);
        TC_GROW(c, c->pair_sb.blocksum, scan_blocksum_size(cap));
        c->pair_sb.err = &c->info->err;
        c->pair_sort_cap = cap;
    }
    int r = mlp_scratch(c, max_pairs);
    if (r) return r;
    // a plain walk at theta that also emits pairs
    tc_config keep = c->cfg;
    c->cfg.learned = 0;
    c->cfg.quadrupole = 0;
    c->cfg.split = 0;  // list export and pair emission live in k_walk
    c->walk_ready = false;
    r = prepare_forces(c);
    c->cfg = keep;
    if (r) return r;
    WalkArgs a{};
    a.body = c->body;
    a.perm = c->perm;
    a.sys_of = c->sys_of;
    a.sysp = c->sysp;
    a.nt = c->nt;
    a.gfirst = c->gfirst;
    a.gref = c->gref;
    a.info = c->info;
    a.acc = c->acc;
    a.theta2 = theta * theta;
    a.eps2 = eps * eps;
    a.G = 1.f;
    a.inv_eps = 1.f / eps;
    a.eps = eps;
    a.band2 = band * band;
    a.pair_body = c->pair_b;
    a.pair_node = c->pair_v;
    a.pair_count = c->pair_n;
    a.pair_cap = max_pairs;
    a.pair_prob = prob;
    a.pair_seed = seed;
    TC_CUDA(c, cudaMemsetAsync(c->pair_n, 0, sizeof(unsigned long long), c->stream));
    cudaError_t e = launch_walk(a, c->walk_cfg, c->walk_grid, c->walk_smem, c->stream);
    c->walk_ready = false;
    if (e != cudaSuccess) return fail(c, TC_ECUDA, "pair walk: %s", cudaGetErrorString(e));
    c->have_forces = false;  // the accelerations of that walk use G = 1
    unsigned long long cnt = 0;
    r = check_device(c);
    if (r) return r;
    TC_COPY(c, &cnt, c->pair_n, sizeof(cnt));
    const int64_t np = (int64_t)std::min<unsigned long long>(cnt, (unsigned long long)max_pairs);
    *npairs = np;
    if (np == 0) return TC_OK;
    // one order whatever the order the walk's warps emitted them in
    launch_pair_order(c->pair_b, c->pair_v, np, c->pair_key, c->pair_val, c->pair_sb, c->stream);
    launch_pair_labels(c->pair_b, c->pair_v, np, c->body, c->sys_of, c->sysp, c->nt, eps, 1.f, c->mlp_x, c->mlp_t,
                       c->mlp_w, c->stream);
    TC_CUDA(c, cudaGetLastError());
    r = check_device(c);
    if (r) return r;
    if (X) TC_COPY(c, X, c->mlp_x, np * 13 * sizeof(float));
    if (T) TC_COPY(c, T, c->mlp_t, np * 3 * sizeof(float));
    if (F) TC_COPY(c, F, c->mlp_w, np * sizeof(float));
    if (body || node) {
        std::vector<int32_t> pb(np), pv(np);
        std::vector<uint32_t> perm(c->n);
        TC_COPY(c, pb.data(), c->pair_b, np * sizeof(int32_t));
        TC_COPY(c, pv.data(), c->pair_v, np * sizeof(int32_t));
        TC_COPY(c, perm.data(), c->perm, c->n * sizeof(uint32_t));
        std::vector<int64_t> ob(np), ov(np);
        for (int64_t k = 0; k < np; k++) {
            ob[k] = perm[pb[k]];
            ov[k] = pv[k];
        }
        if (body) TC_COPY(c, body, ob.data(), np * sizeof(int64_t));
        if (node) TC_COPY(c, node, ov.data(), np * sizeof(int64_t));
    }
    return TC_OK;
}

int tc_mlp_evals(tc_ctx* c, int64_t* evals)
{
    if (!c || !evals) return fail(c, TC_EINVAL, "tc_mlp_evals: null argument");
    int r = mlp_alloc(c);
    if (r) return r;
    r = check_device(c);
    if (r) return r;
    unsigned long long v = 0;
    TC_COPY(c, &v, c->mlp_evals, sizeof(v));
    TC_CUDA(c, cudaMemsetAsync(c->mlp_evals, 0, sizeof(v), c->stream));
    TC_CUDA(c, cudaStreamSynchronize(c->stream));
    *evals = (int64_t)v;
    return TC_OK;
}

}  // extern "C"

extern "C" {


// The interaction list of one group (list-export mode): a walk of that group
// alone that writes its accepted cells and opened leaves instead of forces.
int tc_get_group_list(tc_ctx* c, int64_t group, float theta, int32_t* cells, int32_t* leaves, int64_t cap,
                      int64_t* ncells, int64_t* nleaves)
{
    if (!c || !ncells || !nleaves) return fail(c, TC_EINVAL, "tc_get_group_list: null argument");
    if (!c->built) return fail(c, TC_ESTATE, "tc_get_group_list: build first");
    if (!finite(theta) || theta < 0.f || cap < 0) return fail(c, TC_EINVAL, "tc_get_group_list: theta >= 0, cap >= 0");
    int r = check_device(c);
    if (r) return r;
    if (group < 0 || group >= c->info_h->G) return fail(c, TC_EINVAL, "tc_get_group_list: no group %lld", (long long)group);
    const int64_t want = cap < 1 ? 1 : cap;
    if (want > c->list_cap) {
        TC_GROW(c, c->list_buf, 2 * want);
        c->list_cap = want;
    }
    if (!c->list_n) TC_GROW(c, c->list_n, 2);
    // the plain walk defines the lists (the learned and quadrupole variants
    // walk the same way)
    tc_config keep = c->cfg;
    c->cfg.learned = 0;
    c->cfg.quadrupole = 0;
    c->cfg.split = 0;  // list export and pair emission live in k_walk
    c->walk_ready = false;
    r = prepare_forces(c);
    c->cfg = keep;
    if (r) return r;
    WalkArgs a{};
    a.body = c->body;
    a.perm = c->perm;
    a.sys_of = c->sys_of;
    a.sysp = c->sysp;
    a.nt = c->nt;
    a.gfirst = c->gfirst;
    a.gref = c->gref;
    a.info = c->info;
    a.acc = c->acc;  // not written in list mode
    a.theta2 = theta * theta;
    a.eps2 = 1.f;
    a.G = 1.f;
    a.inv_eps = 1.f;
    a.eps = 1.f;
    a.list_cells = c->list_buf;
    a.list_leaves = c->list_buf + c->list_cap;
    a.list_cap = cap;
    a.list_n = c->list_n;
    a.list_group = (int32_t)group;
    TC_CUDA(c, cudaMemsetAsync(c->list_n, 0, 2 * sizeof(int64_t), c->stream));
    cudaError_t e = launch_walk(a, c->walk_cfg, c->walk_grid, c->walk_smem, c->stream);
    c->walk_ready = false;
    if (e != cudaSuccess) return fail(c, TC_ECUDA, "list walk: %s", cudaGetErrorString(e));
    r = check_device(c);
    if (r) return r;
    int64_t nn[2] = {0, 0};
    TC_CUDA(c, cudaMemcpy(nn, c->list_n, sizeof(nn), cudaMemcpyDeviceToHost));
    *ncells = nn[0];
    *nleaves = nn[1];
    const int64_t kc = std::min<int64_t>(nn[0], cap), kl = std::min<int64_t>(nn[1], cap);
    if (cells && kc > 0) TC_CUDA(c, cudaMemcpy(cells, c->list_buf, kc * sizeof(int32_t), cudaMemcpyDefault));
    if (leaves && kl > 0)
        TC_CUDA(c, cudaMemcpy(leaves, c->list_buf + c->list_cap, kl * sizeof(int32_t), cudaMemcpyDefault));
    return TC_OK;
}

// Launch-configuration autotuner: times the walk + force kernel for every
// (group size, list tile, warps per block) on the context's current bodies
// and keeps the fastest.  Results are cached in the text file named by the
// TC_AUTOTUNE_CACHE environment variable (one "key gmax tile warps ms" line
// per workload) when it is set.
int tc_autotune(tc_ctx* c, float theta, float eps, float G, int reps, tc_config* best_out, double* best_ms_out)
{
    if (!c) return fail(c, TC_EINVAL, "tc_autotune: null context");
    if (!c->built) return fail(c, TC_ESTATE, "tc_autotune: build first");
    if (!finite(theta) || theta < 0.f || !finite(eps) || eps <= 0.f || !finite(G))
        return fail(c, TC_EINVAL, "tc_autotune: theta >= 0, eps > 0, finite G required");
    if (reps < 1) reps = 1;
    char key[256];
    snprintf(key, sizeof(key), "n=%lld,nsys=%d,leaf=%d,theta=%a,eps=%a,precise=%d,pot=%d,quad=%d", (long long)c->n,
             c->nsys, c->leaf_max, (double)theta, (double)eps, c->cfg.precise, c->cfg.want_pot, c->cfg.quad);
    const char* cache = getenv("TC_AUTOTUNE_CACHE");
    tc_config best = c->cfg;
    double best_ms = -1.0;
    if (cache && *cache) {
        FILE* f = fopen(cache, "r");
        if (f) {
            char k[256];
            int gm, ti, wa;
            double ms;
            while (fscanf(f, "%255s %d %d %d %lf", k, &gm, &ti, &wa, &ms) == 5)
                if (strcmp(k, key) == 0) {
                    best.gmax = gm;
                    best.tile = ti;
                    best.warps = wa;
                    best_ms = ms;
                }
            fclose(f);
        }
    }
    if (best_ms < 0.0) {
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        TC_CUDA(c, cudaEventCreate(&e0));
        TC_CUDA(c, cudaEventCreate(&e1));
        const int gmaxes[3] = {32, 64, 128}, tiles[3] = {64, 128, 256}, warps[2] = {2, 4};
        int rc = TC_OK;
        for (int gi = 0; gi < 3 && !rc; gi++) {
            tc_config t = c->cfg;
            t.gmax = gmaxes[gi];
            rc = tc_set_config(c, &t);  // regroups the bodies for the group size
            for (int ti = 0; ti < 3 && !rc; ti++)
                for (int wi = 0; wi < 2 && !rc; wi++) {
                    t.tile = tiles[ti];
                    t.warps = warps[wi];
                    rc = tc_set_config(c, &t);
                    if (!rc) rc = prepare_forces(c);
                    if (!rc) rc = run_forces(c, theta, eps, G, c->stream);  // warm-up
                    double tmin = 1e30;
                    for (int k = 0; k < reps && !rc; k++) {
                        cudaEventRecord(e0, c->stream);
                        rc = run_forces(c, theta, eps, G, c->stream);
                        cudaEventRecord(e1, c->stream);
                        if (!rc) rc = check_device(c);
                        float ms = 0.f;
                        if (!rc && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms < tmin) tmin = ms;
                    }
                    if (!rc && (best_ms < 0.0 || tmin < best_ms)) {
                        best = t;
                        best_ms = tmin;
                    }
                }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (rc) return rc;
        if (cache && *cache) {
            FILE* f = fopen(cache, "a");
            if (f) {
                fprintf(f, "%s %d %d %d %.6f\n", key, best.gmax, best.tile, best.warps, best_ms);
                fclose(f);
            }
        }
    }
    int rc = tc_set_config(c, &best);
    if (rc) return rc;
    if (best_out) *best_out = best;
    if (best_ms_out) *best_ms_out = best_ms;
    return TC_OK;
}

// Measured FP32 throughput of the current device: 8 resident blocks of 256
// threads per SM, each thread 8 independent chains of fused multiply-adds;
// the best of three timed launches.
int tc_probe_fp32(int paired, double* tflops)
{
    if (!tflops) {
        set_thread_error("tc_probe_fp32: null argument");
        return TC_EINVAL;
    }
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    float* out = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&out, sizeof(float));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const int blocks = 8 * sms, iters = 1 << 14;
    double best = 0.0;
    for (int rep = 0; rep < 4 && e == cudaSuccess; rep++) {
        cudaEventRecord(e0, s);
        launch_fp32_probe(paired != 0, blocks, iters, out, s);
        cudaEventRecord(e1, s);
        e = cudaStreamSynchronize(s);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        // flops: threads x 8 chains x iters x 2 (a paired instruction does two)
        const double flops = (double)blocks * 256 * 8 * iters * 2.0;
        if (e == cudaSuccess && rep > 0 && ms > 0.f) best = std::max(best, flops / (ms * 1e-3) / 1e12);
    }
    if (out) cudaFree(out);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    if (e != cudaSuccess) {
        set_thread_error("tc_probe_fp32: CUDA error");
        return TC_ECUDA;
    }
    *tflops = best;
    return TC_OK;
}

int tc_probe_force(double* tflops)
{
    if (!tflops) {
        set_thread_error("tc_probe_force: null argument");
        return TC_EINVAL;
    }
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    float* out = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&out, sizeof(float));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const int blocks = 4 * sms, reps = 4096;
    double best = 0.0;
    for (int rep = 0; rep < 4 && e == cudaSuccess; rep++) {
        cudaEventRecord(e0, s);
        const double inter = launch_force_probe(blocks, reps, out, s);
        cudaEventRecord(e1, s);
        e = cudaStreamSynchronize(s);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0 && ms > 0.f) best = std::max(best, 20.0 * inter / (ms * 1e-3) / 1e12);
    }
    if (out) cudaFree(out);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    if (e != cudaSuccess) {
        set_thread_error("tc_probe_force: CUDA error");
        return TC_ECUDA;
    }
    *tflops = best;
    return TC_OK;
}

// Failure-path self-test: a device wait that can never be satisfied must
// give up within its limit, report itself in the error word and leave the
// device usable.
int tc_selftest_bounded_wait(int32_t* err_bits, double* elapsed_ms)
{
    if (!err_bits) {
        set_thread_error("tc_selftest_bounded_wait: null argument");
        return TC_EINVAL;
    }
    const int64_t n = sort_selftest_items();
    uint64_t* keys = nullptr;
    uint64_t* kout = nullptr;
    uint32_t *vals = nullptr, *vout = nullptr, *counter = nullptr, *goff = nullptr;
    unsigned long long* status = nullptr;
    int32_t* err = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = TC_OK;
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t x) {
        if (x != cudaSuccess && e == cudaSuccess) e = x;
    };
    chk(cudaMalloc(&keys, n * sizeof(uint64_t)));
    chk(cudaMalloc(&kout, n * sizeof(uint64_t)));
    chk(cudaMalloc(&vals, n * sizeof(uint32_t)));
    chk(cudaMalloc(&vout, n * sizeof(uint32_t)));
    chk(cudaMalloc(&status, 2 * 256 * sizeof(unsigned long long)));
    chk(cudaMalloc(&counter, sizeof(uint32_t)));
    chk(cudaMalloc(&goff, 256 * sizeof(uint32_t)));
    chk(cudaMalloc(&err, sizeof(int32_t)));
    chk(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    chk(cudaEventCreate(&e0));
    chk(cudaEventCreate(&e1));
    if (e == cudaSuccess) {
        chk(cudaMemsetAsync(keys, 0, n * sizeof(uint64_t), s));
        chk(cudaMemsetAsync(vals, 0, n * sizeof(uint32_t), s));
        chk(cudaMemsetAsync(err, 0, sizeof(int32_t), s));
        chk(cudaEventRecord(e0, s));
        chk(sort_wait_selftest(keys, vals, kout, vout, status, counter, goff, err, s));
        chk(cudaEventRecord(e1, s));
        chk(cudaStreamSynchronize(s));
        int32_t bits = 0;
        chk(cudaMemcpy(&bits, err, sizeof(bits), cudaMemcpyDeviceToHost));
        float ms = 0.f;
        chk(cudaEventElapsedTime(&ms, e0, e1));
        *err_bits = bits;
        if (elapsed_ms) *elapsed_ms = ms;
    }
    if (e != cudaSuccess) {
        set_thread_error("tc_selftest_bounded_wait: CUDA error");
        rc = TC_ECUDA;
    }
    cudaFree(keys);
    cudaFree(kout);
    cudaFree(vals);
    cudaFree(vout);
    cudaFree(status);
    cudaFree(counter);
    cudaFree(goff);
    cudaFree(err);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    return rc;
}

const char* tc_last_error(tc_ctx* c)
{
    if (!c) {
        std::lock_guard<std::mutex> lk(g_default_mu);
        if (g_default && !g_default->err.empty()) return g_default->err.c_str();
        return g_tls_err.c_str();
    }
    return c->err.c_str();
}

tc_ctx* tc_default(void)
{
    std::lock_guard<std::mutex> lk(g_default_mu);
    if (!g_default) {
        tc_ctx* c = nullptr;
        if (tc_create(&c, nullptr) == TC_OK) g_default = c;
    }
    return g_default;
}

int tc_build(const float* pos, const float* mass, int64_t n, int leaf_max)
{
    tc_ctx* c = tc_default();
    if (!c) return TC_ECUDA;
    return tc_ctx_build(c, pos, mass, n, leaf_max);
}

int tc_forces(float theta, float eps, float G)
{
    tc_ctx* c = tc_default();
    if (!c) return TC_ECUDA;
    return tc_ctx_forces(c, theta, eps, G);
}

int tc_step(float dt)
{
    tc_ctx* c = tc_default();
    if (!c) return TC_ECUDA;
    return tc_ctx_step(c, dt);
}

}  // extern "C"
