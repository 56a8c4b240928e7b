// tc_api.cu -- the C ABI of libtc (declared in include/tc.h): context,
// argument checks, buffer management and the order of launches.
#include <cuda_runtime.h>

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
#include "tc_internal.cuh"

using namespace tc;

struct tc_ctx {
    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = 0;
    tc_config cfg{};
    std::string err;

    int64_t n = 0, cap_n = 0;
    int64_t M = 0, cap_m = 0;
    int leaf_max = 0;
    bool built = false, have_forces = false, forces_pot = false;
    float theta = 0.f, eps = 0.f, Gc = 0.f;

    // state, original body order
    float *pos = nullptr, *vel = nullptr, *acc = nullptr, *pot = nullptr, *mass = nullptr;
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
    float* bbox_partial = nullptr;
    uint32_t* totals = nullptr;  // [0] nodes, [1] groups
    int64_t* idx_dev = nullptr;
    int64_t cap_idx = 0;
    double* dir_out = nullptr;
    // per-node scratch
    uint32_t *pre_level = nullptr, *pre_first = nullptr, *iota = nullptr, *bfs_of_pre = nullptr, *lvl_alt = nullptr;
    NodeTables nt{};
    Info* info = nullptr;
    Info* info_h = nullptr;  // pinned mirror
    size_t allocated = 0;
    std::unordered_map<void*, size_t> sizes;

    // phase timers (CUDA events on the context stream), when enabled
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_phase[3];  // build, walk, update
    long long launches_mark = 0;
};

namespace tc {
namespace {
std::atomic<long long> g_launches{0};
}
void count_launches(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
long long launches_total() { return g_launches.load(std::memory_order_relaxed); }
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

template <typename T>
int grow(tc_ctx* c, T** p, int64_t count)
{
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
    TC_GROW(c, c->keys, cap);
    TC_GROW(c, c->perm, cap);
    TC_GROW(c, c->body, cap);
    TC_GROW(c, c->sb.keys_alt, cap);
    TC_GROW(c, c->sb.vals_alt, cap);
    TC_GROW(c, c->sb.ghist, 8 * 256);
    TC_GROW(c, c->sb.status, 8 * radix_tiles(cap) * 256);  // look-back words of the 8 key passes
    TC_GROW(c, c->sb.tiles, 8);
    c->sb.err = &c->info->err;
    TC_GROW(c, c->sb.blocksum, scan_blocksum_size(cap));
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
    TC_GROW(c, c->bbox_partial, 6 * 1024);
    TC_GROW(c, c->totals, 4);
    c->cap_n = cap;
    c->cap_m = 0;  // node tables are sized with the first build at this capacity
    return TC_OK;
}

int ensure_nodes(tc_ctx* c, int64_t M)
{
    if (M <= c->cap_m) return TC_OK;
    int64_t cap = M + M / 4 + 64;
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
    TC_GROW(c, c->nt.mass64, cap);
    TC_GROW(c, c->nt.com64, 3 * cap);
    TC_GROW(c, c->nt.quad64, 6 * cap);
    // the level sort reuses the body sort's value ping-pong buffer
    if (cap > c->cap_n) TC_GROW(c, c->sb.vals_alt, cap);
    if (radix_tiles(cap) > 8 * radix_tiles(c->cap_n))  // the level sort's single pass
        TC_GROW(c, c->sb.status, radix_tiles(cap) * 256);
    c->cap_m = cap;
    return TC_OK;
}

// device error word -> status (synchronises)
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
        if (e & kErrStack)
            return fail(c, TC_EDEVICE, "walk stack overflow (raise tc_config.stack)");
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

// records the start of a timed phase; returns the event (or null)
cudaEvent_t phase_begin(tc_ctx* c)
{
    if (!c->timing) return nullptr;
    cudaEvent_t e = take_event(c);
    if (e) cudaEventRecord(e, c->stream);
    return e;
}

void phase_end(tc_ctx* c, int phase, cudaEvent_t start)
{
    if (!start) return;
    cudaEvent_t e = take_event(c);
    if (!e) return;
    cudaEventRecord(e, c->stream);
    c->ev_phase[phase].push_back({start, e});
}

// The whole build from c->pos / c->mass (already on the device).
int build_tree(tc_ctx* c)
{
    cudaStream_t s = c->stream;
    const int64_t n = c->n;
    cudaEvent_t t0 = phase_begin(c);
    TC_CUDA(c, cudaMemsetAsync(&c->info->err, 0, sizeof(int32_t), s));
    int nb = bbox_blocks(n);
    launch_bbox(c->pos, n, c->bbox_partial, nb, c->info, s);
    launch_keys(c->pos, c->mass, n, c->info, c->keys, c->perm, s);
    radix_sort_u64(c->keys, c->perm, n, 63, c->sb, s);
    launch_gather(c->pos, c->mass, c->perm, n, c->body, s);
    TC_CUDA(c, cudaMemsetAsync(&c->info->depth, 0, sizeof(int32_t), s));
    launch_node_counts(c->keys, n, c->leaf_max, c->w, c->delta, c->top, c->nstart, &c->info->depth, s);
    scan_u32(c->nstart, c->prepos, n, &c->totals[0], c->sb.blocksum, s);
    TC_CUDA(c, cudaGetLastError());
    uint32_t M32 = 0;
    TC_CUDA(c, cudaMemcpyAsync(&M32, &c->totals[0], sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    int r = check_device(c);  // synchronises: M32 valid afterwards
    if (r) return r;
    const int64_t M = M32;
    if (M < 1) return fail(c, TC_EDEVICE, "empty node table");
    r = ensure_nodes(c, M);
    if (r) return r;
    c->M = M;
    launch_emit_preorder(c->delta, c->nstart, c->prepos, n, c->pre_level, c->pre_first, c->iota, s);
    // breadth-first order: stable sort of the pre-order nodes by level
    SortBufs lb = c->sb;
    radix_sort_u32(c->pre_level, c->iota, M, 8, lb, c->lvl_alt, s);
    launch_inverse_perm(c->iota, M, c->bfs_of_pre, s);
    launch_node_finalize(c->keys, c->top, n, c->pre_level, c->iota, c->pre_first, c->bfs_of_pre, M, c->nt, s);
    // after the level sort, ghist[l] is the first breadth-first index of level l
    launch_moments(c->body, M, c->info_h->depth, c->sb.ghist, c->info, c->nt, c->cfg.quad != 0, s);
    launch_group_marks(M, c->nt, c->cfg.gmax, n, c->gflag, c->gref_at, s);
    scan_u32(c->gflag, c->gscan, n, &c->totals[1], c->sb.blocksum, s);
    launch_group_table(c->gflag, c->gscan, c->gref_at, n, &c->totals[1], c->gfirst, c->gref, c->info, s);
    TC_CUDA(c, cudaGetLastError());
    phase_end(c, 0, t0);
    c->built = true;
    c->have_forces = false;
    return TC_OK;
}

int run_forces(tc_ctx* c, float theta, float eps, float G)
{
    WalkArgs a{};
    a.body = c->body;
    a.perm = c->perm;
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
    WalkConfig wc{};
    wc.gmax = c->cfg.gmax;
    wc.warps = c->cfg.warps;
    wc.precise = c->cfg.precise;
    wc.want_pot = c->cfg.want_pot;
    wc.verify = c->cfg.verify;
    wc.blocks_per_sm = c->cfg.blocks_per_sm;
    int64_t st = c->cfg.stack;
    if (c->M < st) st = c->M < 32 ? 32 : c->M;  // a stack of M entries cannot overflow
    st = (st + 3) & ~(int64_t)3;                // keeps every warp's tiles 16-byte aligned
    wc.stack = (int)st;
    cudaEvent_t t0 = phase_begin(c);
    cudaError_t e = launch_walk(a, wc, c->num_sms, c->stream);
    if (e != cudaSuccess) return fail(c, TC_ECUDA, "walk launch: %s", cudaGetErrorString(e));
    phase_end(c, 1, t0);
    c->have_forces = true;
    c->forces_pot = c->cfg.want_pot != 0;
    c->theta = theta;
    c->eps = eps;
    c->Gc = G;
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
    *out = c;
    return TC_OK;
}

void tc_destroy(tc_ctx* c)
{
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    void* bufs[] = {c->pos, c->vel, c->acc, c->pot, c->mass, c->keys, c->perm, c->body, c->sb.keys_alt,
                    c->sb.vals_alt, c->sb.ghist, c->sb.status, c->sb.tiles, c->sb.blocksum, c->w, c->delta, c->top, c->nstart, c->prepos,
                    c->gflag, c->gscan, c->gref_at, c->gfirst, c->gref, c->ncell, c->nbody, c->hash,
                    c->bbox_partial, c->totals, c->idx_dev, c->dir_out, c->pre_level, c->pre_first, c->iota,
                    c->bfs_of_pre, c->lvl_alt, c->nt.a, c->nt.b, c->nt.c, c->nt.d, c->nt.quad, c->nt.mass64,
                    c->nt.com64, c->nt.quad64, c->info};
    for (void* p : bufs)
        if (p) cudaFree(p);
    if (c->info_h) cudaFreeHost(c->info_h);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    delete c;
}

int tc_set_config(tc_ctx* c, const tc_config* cfg)
{
    if (!c || !cfg) return fail(c, TC_EINVAL, "tc_set_config: null argument");
    if (cfg->gmax != 32 && cfg->gmax != 64 && cfg->gmax != 128)
        return fail(c, TC_EINVAL, "gmax must be 32, 64 or 128 (got %d)", cfg->gmax);
    if (cfg->warps < 1 || cfg->warps > 4) return fail(c, TC_EINVAL, "warps must be 1..4 (got %d)", cfg->warps);
    if (cfg->stack < 64 || cfg->stack > 8192) return fail(c, TC_EINVAL, "stack must be 64..8192 (got %d)", cfg->stack);
    if (cfg->blocks_per_sm < 0) return fail(c, TC_EINVAL, "blocks_per_sm must be >= 0");
    bool regroup = c->built && (cfg->gmax != c->cfg.gmax || (cfg->quad != 0) != (c->cfg.quad != 0));
    c->cfg = *cfg;
    c->cfg.precise = cfg->precise ? 1 : 0;
    c->cfg.want_pot = cfg->want_pot ? 1 : 0;
    c->cfg.verify = cfg->verify ? 1 : 0;
    c->cfg.quad = cfg->quad ? 1 : 0;
    if (regroup) return build_tree(c);  // groups depend on gmax
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

int tc_ctx_build(tc_ctx* c, const float* pos, const float* mass, int64_t n, int leaf_max)
{
    if (!c) return fail(c, TC_EINVAL, "tc_build: null context");
    if (!pos || !mass) return fail(c, TC_EINVAL, "tc_build: null pos or mass");
    if (n < 1 || n >= (int64_t)1 << 31) return fail(c, TC_EINVAL, "tc_build: n must be in [1, 2^31) (got %lld)", (long long)n);
    if (leaf_max < 1 || leaf_max > kLeafMaxLimit)
        return fail(c, TC_EINVAL, "tc_build: leaf_max must be in [1, %d] (got %d)", kLeafMaxLimit, leaf_max);
    int r = ensure_bodies(c, n);
    if (r) return r;
    if (n != c->n) TC_CUDA(c, cudaMemsetAsync(c->vel, 0, 3 * n * sizeof(float), c->stream));
    c->n = n;
    c->leaf_max = leaf_max;
    TC_CUDA(c, cudaMemcpyAsync(c->pos, pos, 3 * n * sizeof(float), cudaMemcpyDefault, c->stream));
    TC_CUDA(c, cudaMemcpyAsync(c->mass, mass, n * sizeof(float), cudaMemcpyDefault, c->stream));
    c->built = false;
    return build_tree(c);
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
    return run_forces(c, theta, eps, G);
}

int tc_ctx_step(tc_ctx* c, float dt)
{
    if (!c) return fail(c, TC_EINVAL, "tc_step: null context");
    if (!finite(dt)) return fail(c, TC_EINVAL, "tc_step: dt must be finite");
    if (!c->have_forces) return fail(c, TC_ESTATE, "tc_step: compute forces on the current positions first");
    cudaEvent_t t0 = phase_begin(c);
    launch_kick_drift(c->pos, c->vel, c->acc, c->n, 0.5f * dt, dt, c->stream);
    phase_end(c, 2, t0);
    int r = build_tree(c);
    if (r) return r;
    r = run_forces(c, c->theta, c->eps, c->Gc);
    if (r) return r;
    t0 = phase_begin(c);
    launch_kick(c->vel, c->acc, c->n, 0.5f * dt, c->stream);
    phase_end(c, 2, t0);
    TC_CUDA(c, cudaGetLastError());
    return TC_OK;
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
    return build_tree(c);
}

int tc_get_sizes(tc_ctx* c, int64_t* n, int64_t* nnodes, int64_t* ngroups)
{
    if (!c) return fail(c, TC_EINVAL, "tc_get_sizes: null context");
    if (!c->built) return fail(c, TC_ESTATE, "tc_get_sizes: build first");
    int r = check_device(c);
    if (r) return r;
    if (n) *n = c->n;
    if (nnodes) *nnodes = c->M;
    if (ngroups) *ngroups = c->info_h->G;
    return TC_OK;
}

int tc_get_cube(tc_ctx* c, double* out5)
{
    if (!c || !out5) return fail(c, TC_EINVAL, "tc_get_cube: null argument");
    if (!c->built) return fail(c, TC_ESTATE, "tc_get_cube: build first");
    int r = check_device(c);
    if (r) return r;
    for (int a = 0; a < 3; a++) out5[a] = c->info_h->c0[a];
    out5[3] = c->info_h->L;
    out5[4] = c->info_h->h;
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
    const int64_t M = c->M;
    int4* b = (int4*)malloc(M * sizeof(int4));
    if (!b) return fail(c, TC_ENOMEM, "tc_get_nodes: host memory");
    cudaError_t e = cudaMemcpy(b, c->nt.b, M * sizeof(int4), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        free(b);
        return fail(c, TC_ECUDA, "tc_get_nodes: %s", cudaGetErrorString(e));
    }
    uint64_t* keys = nullptr;
    if (prefix) {
        keys = (uint64_t*)malloc(c->n * sizeof(uint64_t));
        if (!keys || cudaMemcpy(keys, c->keys, c->n * sizeof(uint64_t), cudaMemcpyDeviceToHost) != cudaSuccess) {
            free(b);
            free(keys);
            return fail(c, TC_ECUDA, "tc_get_nodes: key copy failed");
        }
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
    free(b);
    free(keys);
    if (mass) TC_CUDA(c, cudaMemcpy(mass, c->nt.mass64, M * sizeof(double), cudaMemcpyDefault));
    if (com) TC_CUDA(c, cudaMemcpy(com, c->nt.com64, 3 * M * sizeof(double), cudaMemcpyDefault));
    if (quad) TC_CUDA(c, cudaMemcpy(quad, c->nt.quad64, 6 * M * sizeof(double), cudaMemcpyDefault));
    return TC_OK;
}

int tc_get_groups(tc_ctx* c, int32_t* gfirst, int32_t* gcount, int32_t* gref)
{
    if (!c) return fail(c, TC_EINVAL, "tc_get_groups: null context");
    if (!c->built) return fail(c, TC_ESTATE, "tc_get_groups: build first");
    int r = check_device(c);
    if (r) return r;
    const int64_t G = c->info_h->G;
    int32_t* f = (int32_t*)malloc((G + 1) * sizeof(int32_t));
    if (!f) return fail(c, TC_ENOMEM, "tc_get_groups: host memory");
    cudaError_t e = cudaMemcpy(f, c->gfirst, (G + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && gref) e = cudaMemcpy(gref, c->gref, G * sizeof(int32_t), cudaMemcpyDefault);
    if (e != cudaSuccess) {
        free(f);
        return fail(c, TC_ECUDA, "tc_get_groups: %s", cudaGetErrorString(e));
    }
    for (int64_t g = 0; g < G; g++) {
        if (gfirst) gfirst[g] = f[g];
        if (gcount) gcount[g] = f[g + 1] - f[g];
    }
    free(f);
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

int tc_direct(tc_ctx* c, const int64_t* idx, int64_t ns, float eps, float G, double* acc, double* pot)
{
    if (!c || !idx || !acc) return fail(c, TC_EINVAL, "tc_direct: null argument");
    if (!c->built) return fail(c, TC_ESTATE, "tc_direct: build first");
    if (ns < 1) return fail(c, TC_EINVAL, "tc_direct: ns must be >= 1");
    if (!finite(eps) || eps <= 0.f || !finite(G)) return fail(c, TC_EINVAL, "tc_direct: eps > 0 and finite G required");
    if (ns > c->cap_idx) {
        TC_GROW(c, c->idx_dev, ns);
        TC_GROW(c, c->dir_out, 4 * ns);
        c->cap_idx = ns;
    }
    TC_CUDA(c, cudaMemcpyAsync(c->idx_dev, idx, ns * sizeof(int64_t), cudaMemcpyDefault, c->stream));
    // indices must address bodies: checked on the host copy
    int64_t* hidx = (int64_t*)malloc(ns * sizeof(int64_t));
    if (!hidx) return fail(c, TC_ENOMEM, "tc_direct: host memory");
    TC_CUDA(c, cudaMemcpyAsync(hidx, c->idx_dev, ns * sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
    TC_CUDA(c, cudaStreamSynchronize(c->stream));
    for (int64_t k = 0; k < ns; k++)
        if (hidx[k] < 0 || hidx[k] >= c->n) {
            long long bad = (long long)hidx[k];
            free(hidx);
            return fail(c, TC_EINVAL, "tc_direct: index %lld out of range", bad);
        }
    free(hidx);
    launch_direct(c->pos, c->mass, c->n, c->idx_dev, ns, eps * eps, G, c->dir_out, c->dir_out + 3 * ns, c->stream);
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
    out6[5] = 0.0;
    return TC_OK;
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
