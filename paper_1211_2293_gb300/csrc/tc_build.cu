// tc_build.cu -- oct-tree construction on the GPU (Sec. 3.1 of the paper:
// the space is divided recursively into 8 sub-cubes until a cube holds no
// more than a threshold of bodies; every cell carries its total mass and
// centre of mass).
//
// Pipeline (all on one stream):
//   1. k_bbox      FP64 bounding box -> power-of-two root cube on a 2^21 grid
//   2. k_keys      63-bit Morton keys (exact FP64 quantisation)
//   3. radix sort  stable (key, index) sort            [tc_sort.cu]
//   4. k_gather    bodies in Morton order as float4 (x, y, z, m)
//   5. k_window / k_node_counts
//                  which cubes of the recursive subdivision start at each
//                  sorted body (a sliding-window test, below)
//   6. scan + k_emit_preorder      node table in pre-order
//   7. one stable radix pass by level  -> breadth-first order
//   8. k_node_finalize  counts, children, integer centres
//   9. k_leaf_moments, then k_level_moments level by level from the deepest
//                  FP64 mass / centre of mass / second moments, bottom-up
//  10. k_group_marks + scan + k_group_table   body groups for the walk
//
// Which cubes exist.  Let cd(a, b) be the number of leading octal digits two
// keys share.  The level-l run of equal l-digit prefixes that contains sorted
// body s holds more than leaf_max bodies iff some window of leaf_max + 1
// consecutive bodies containing s lies inside it, i.e. iff
//     W_s = max_{j in [s - leaf_max, s]} cd(key_j, key_{j + leaf_max}) >= l.
// A cube at level l is created by the subdivision iff its parent cube holds
// more than leaf_max bodies (and the parent is above level 21).  So the cubes
// whose first body is s are the levels l with
//     delta_s < l <= min(W_s + 1, 21),   delta_s = cd(key_{s-1}, key_s)
// (delta_0 = -1), and the deepest of them is a leaf.  Pre-order of the tree
// is the order of (first body, level), so one scan over the per-body counts
// places every node.
#include "tc_internal.cuh"

namespace tc {

namespace {

__device__ __forceinline__ int common_digits(uint64_t a, uint64_t b)
{
    uint64_t x = a ^ b;
    if (x == 0) return kMaxLevel;
    return (__clzll((long long)x) - 1) / 3;  // keys use bits 0..62
}

__device__ __forceinline__ uint64_t spread3(uint64_t v)
{
    v &= 0x1fffffull;
    v = (v | (v << 32)) & 0x1f00000000ffffull;
    v = (v | (v << 16)) & 0x1f0000ff0000ffull;
    v = (v | (v << 8)) & 0x100f00f00f00f00full;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

__device__ __forceinline__ uint32_t compact3(uint64_t v)
{
    v &= 0x1249249249249249ull;
    v = (v ^ (v >> 2)) & 0x10c30c30c30c30c3ull;
    v = (v ^ (v >> 4)) & 0x100f00f00f00f00full;
    v = (v ^ (v >> 8)) & 0x1f0000ff0000ffull;
    v = (v ^ (v >> 16)) & 0x1f00000000ffffull;
    v = (v ^ (v >> 32)) & 0x1fffffull;
    return (uint32_t)v;
}

// ------------------------------------------------------------------ bbox
constexpr int kBboxThreads = 256;

__device__ __forceinline__ float warp_min(float x)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) x = fminf(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}
__device__ __forceinline__ float warp_max(float x)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}

// Root cube (power-of-two side L >= extent * (1 + 2^-20), grid step h =
// L / 2^21, corner c0 = floor(min / h) * h), computed by the last block.
__global__ void __launch_bounds__(kBboxThreads) k_bbox(const float* __restrict__ pos, int64_t n,
                                                       float* __restrict__ partial, Info* info)
{
    __shared__ float sm[6][kBboxThreads / 32];
    __shared__ bool last;
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int a = 0; a < 3; a++) {
            float x = pos[3 * i + a];
            bad |= !isfinite(x);
            lo[a] = fminf(lo[a], x);
            hi[a] = fmaxf(hi[a], x);
        }
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&info->err, kErrNonFinite);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        float l = warp_min(lo[a]), h = warp_max(hi[a]);
        if (lane == 0) {
            sm[a][w] = l;
            sm[3 + a][w] = h;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float r[6];
        for (int a = 0; a < 3; a++) {
            r[a] = INFINITY;
            r[3 + a] = -INFINITY;
            for (int k = 0; k < kBboxThreads / 32; k++) {
                r[a] = fminf(r[a], sm[a][k]);
                r[3 + a] = fmaxf(r[3 + a], sm[3 + a][k]);
            }
        }
        for (int k = 0; k < 6; k++) partial[6 * blockIdx.x + k] = r[k];
        __threadfence();
        unsigned t = atomicAdd(&info->ticket, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // the last block reduces the partials with all its threads
    float r[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
        for (int a = 0; a < 3; a++) {
            r[a] = fminf(r[a], __ldcg(&partial[6 * b + a]));
            r[3 + a] = fmaxf(r[3 + a], __ldcg(&partial[6 * b + 3 + a]));
        }
    }
    for (int a = 0; a < 3; a++) {
        r[a] = warp_min(r[a]);
        r[3 + a] = warp_max(r[3 + a]);
    }
    __syncthreads();
    if (lane == 0)
        for (int a = 0; a < 6; a++) sm[a][w] = r[a];
    __syncthreads();
    if (threadIdx.x != 0) return;
    double dlo[3], dhi[3];
    for (int a = 0; a < 3; a++) {
        float l = INFINITY, h = -INFINITY;
        for (int k = 0; k < kBboxThreads / 32; k++) {
            l = fminf(l, sm[a][k]);
            h = fmaxf(h, sm[3 + a][k]);
        }
        dlo[a] = (double)l;
        dhi[a] = (double)h;
    }
    double extent = 0.0;
    for (int a = 0; a < 3; a++) {
        double e = dhi[a] - dlo[a];
        if (e > extent) extent = e;
    }
    double target = extent * (1.0 + 0x1p-20);
    double L = 1.0;  // all bodies coincide: unit cube
    if (target > 0.0) {
        int e;
        double m = frexp(target, &e);
        L = (m == 0.5) ? target : ldexp(1.0, e);
    }
    double h = L / 2097152.0;
    int eh;
    frexp(h, &eh);  // h = 2^(eh - 1)
    info->qexp = 1 - eh;  // 1/h = 2^qexp
    for (int a = 0; a < 3; a++) {
        const double K0 = floor(dlo[a] / h);
        info->c0[a] = K0 * h;
        info->qoff[a] = (long long)K0;
    }
    info->L = L;
    info->h = h;
    info->inv_h = 1.0 / h;
    info->Lf = (float)L;
    info->uf = (float)(h * 0.5);
    info->ticket = 0;
}

// ------------------------------------------------------------------ keys
// q = floor((x - c0) / h) clamped to [0, 2^21 - 1], evaluated exactly: h is
// a power of two and c0 = K0 h with K0 an integer, so q = floor(x * 2^k) - K0
// with 2^k = 1/h -- an exact float scaling, an exact floor and an integer
// subtraction.  Key digit l holds the level-l bits of (qx, qy, qz), x highest.
__device__ __forceinline__ uint64_t quantise(float x, int k, long long K0)
{
    float t = floorf(scalbnf(x, k));
    if (x < 0.0f && t == 0.0f) t = -1.0f;  // a negative value scaled below the float range
    long long q = __float2ll_rz(t) - K0;    // the conversion saturates out-of-range values
    q = q < 0 ? 0 : (q > 2097151 ? 2097151 : q);
    return (uint64_t)q;
}

__global__ void k_keys(const float* __restrict__ pos, const float* __restrict__ mass, int64_t n,
                       const Info* __restrict__ info, uint64_t* __restrict__ keys,
                       uint32_t* __restrict__ idx, int32_t* err)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int k = info->qexp;
    const uint64_t qx = quantise(pos[3 * i], k, info->qoff[0]);
    const uint64_t qy = quantise(pos[3 * i + 1], k, info->qoff[1]);
    const uint64_t qz = quantise(pos[3 * i + 2], k, info->qoff[2]);
    keys[i] = (spread3(qx) << 2) | (spread3(qy) << 1) | spread3(qz);
    idx[i] = (uint32_t)i;
    float m = mass[i];
    if (!(isfinite(m) && m > 0.0f)) atomicOr(err, kErrNonFinite);
}

__global__ void k_gather(const float* __restrict__ pos, const float* __restrict__ mass,
                         const uint32_t* __restrict__ perm, int64_t n, float4* __restrict__ body)
{
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int64_t i = perm[k];
    body[k] = make_float4(pos[3 * i], pos[3 * i + 1], pos[3 * i + 2], mass[i]);
}

// ------------------------------------------------------------------ nodes
__global__ void k_window(const uint64_t* __restrict__ keys, int64_t n, int leaf_max, int8_t* __restrict__ w)
{
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    w[j] = (j + leaf_max < n) ? (int8_t)common_digits(keys[j], keys[j + leaf_max]) : (int8_t)-1;
}

__global__ void k_node_counts(const uint64_t* __restrict__ keys, const int8_t* __restrict__ w, int64_t n,
                              int leaf_max, int8_t* __restrict__ delta, int8_t* __restrict__ top,
                              uint32_t* __restrict__ nstart, int32_t* __restrict__ depth)
{
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int t = 0;
    if (s < n) {
        int d = (s == 0) ? -1 : common_digits(keys[s - 1], keys[s]);
        int W = -1;
        int64_t j0 = s - leaf_max < 0 ? 0 : s - leaf_max;
        for (int64_t j = j0; j <= s; j++) W = max(W, (int)w[j]);
        t = min(W + 1, kMaxLevel);
        delta[s] = (int8_t)d;
        top[s] = (int8_t)t;
        nstart[s] = (uint32_t)max(0, t - d);
    }
    // deepest level of the tree: a warp maximum (every lane of the launch's
    // full warps takes part), then one atomic per warp
#pragma unroll
    for (int o = 16; o; o >>= 1) t = max(t, __shfl_xor_sync(0xffffffffu, t, o));
    if ((threadIdx.x & 31) == 0) atomicMax(depth, t);
}

__global__ void k_emit_preorder(const int8_t* __restrict__ delta, const uint32_t* __restrict__ nstart,
                                const uint32_t* __restrict__ prepos, int64_t n,
                                uint32_t* __restrict__ pre_level, uint32_t* __restrict__ pre_first,
                                uint32_t* __restrict__ iota)
{
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    uint32_t c = nstart[s], p = prepos[s];
    int l0 = delta[s] + 1;
    for (uint32_t k = 0; k < c; k++) {
        pre_level[p + k] = (uint32_t)(l0 + (int)k);
        pre_first[p + k] = (uint32_t)s;
        iota[p + k] = p + k;
    }
}

__global__ void k_inverse_perm(const uint32_t* __restrict__ perm, int64_t M, uint32_t* __restrict__ inv)
{
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b < M) inv[perm[b]] = (uint32_t)b;
}

// first index e in [lo, hi) with (keys[e] >> sh) > pfx, or hi
__device__ __forceinline__ int64_t run_end(const uint64_t* __restrict__ keys, int64_t lo, int64_t hi,
                                           int sh, uint64_t pfx)
{
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if ((keys[mid] >> sh) > pfx) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

__global__ void k_node_finalize(const uint64_t* __restrict__ keys, const int8_t* __restrict__ top, int64_t n,
                                const uint32_t* __restrict__ bfs_level, const uint32_t* __restrict__ bfs_pre,
                                const uint32_t* __restrict__ pre_first, const uint32_t* __restrict__ bfs_of_pre,
                                int64_t M, NodeTables nt)
{
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= M) return;
    uint32_t p = bfs_pre[b];
    int l = (int)bfs_level[b];
    int64_t s = pre_first[p];
    int sh = 3 * (kMaxLevel - l);
    uint64_t pfx = (l == 0) ? 0ull : (keys[s] >> sh);
    int64_t e = (l == 0) ? n : run_end(keys, s + 1, n, sh, pfx);
    int nch = 0;
    int32_t cf = -1;
    if (l < (int)top[s]) {
        cf = (int32_t)bfs_of_pre[p + 1];
        int shc = sh - 3;
        int64_t c = s;
        while (c < e) {
            uint64_t cp = keys[c] >> shc;
            c = run_end(keys, c + 1, e, shc, cp);
            nch++;
        }
    }
    nt.b[b] = make_int4((int)s, (int)(e - s), cf, l | (nch << 8));
    uint32_t ix = compact3(pfx >> 2), iy = compact3(pfx >> 1), iz = compact3(pfx);
    int c1 = 1 << (kMaxLevel - l);
    nt.c[b] = make_int4((int)(2 * ix + 1) * c1, (int)(2 * iy + 1) * c1, (int)(2 * iz + 1) * c1, 0);
}

// ------------------------------------------------------------------ moments
// Mass, centre of mass and second moments about the centre of mass, FP64.
// Leaves sum their bodies (positions taken relative to the cube centre);
// an internal cell combines its children: M = sum M_c,
// com = sum M_c com_c / M, Q = sum Q_c + M_c dc dc^T with dc = com_c - com.
// Leaves are done in one launch; internal cells level by level from the
// deepest, one thread per cell of the level (cells of a level are contiguous
// in breadth-first order), so every lane of a warp has a cell to do.
template <bool QUAD>
__device__ void store_node(NodeTables& nt, int64_t v, double M, const double* com, const double* Q,
                           const Info* info, int4 c)
{
    nt.mass64[v] = M;
    for (int a = 0; a < 3; a++) nt.com64[3 * v + a] = com[a];
    const double u = 0.5 * info->h;
    double C[3] = {info->c0[0] + (double)c.x * u, info->c0[1] + (double)c.y * u, info->c0[2] + (double)c.z * u};
    nt.a[v] = make_float4((float)(com[0] - C[0]), (float)(com[1] - C[1]), (float)(com[2] - C[2]), (float)M);
    nt.d[v] = make_float4((float)com[0], (float)com[1], (float)com[2], (float)M);
    if (QUAD) {
        for (int a = 0; a < 6; a++) nt.quad64[6 * v + a] = Q[a];
        for (int a = 0; a < 6; a++) nt.quad[6 * v + a] = (float)Q[a];
    }
}

template <bool QUAD>
__global__ void k_leaf_moments(const float4* __restrict__ body, int64_t M, const Info* __restrict__ info,
                               NodeTables nt)
{
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= M) return;
    const int4 b = nt.b[v];
    if ((b.w >> 8) != 0) return;  // internal
    const int4 c = nt.c[v];
    const double u = 0.5 * info->h;
    const double C[3] = {info->c0[0] + (double)c.x * u, info->c0[1] + (double)c.y * u,
                         info->c0[2] + (double)c.z * u};
    double m = 0.0, S[3] = {0, 0, 0};
    for (int j = b.x; j < b.x + b.y; j++) {
        const float4 q = body[j];
        m += (double)q.w;
        S[0] += (double)q.w * ((double)q.x - C[0]);
        S[1] += (double)q.w * ((double)q.y - C[1]);
        S[2] += (double)q.w * ((double)q.z - C[2]);
    }
    const double inv = 1.0 / m;
    const double off[3] = {S[0] * inv, S[1] * inv, S[2] * inv};
    double Q[6] = {0, 0, 0, 0, 0, 0};
    for (int j = b.x; QUAD && j < b.x + b.y; j++) {
        const float4 q = body[j];
        const double dx = ((double)q.x - C[0]) - off[0];
        const double dy = ((double)q.y - C[1]) - off[1];
        const double dz = ((double)q.z - C[2]) - off[2];
        const double mj = (double)q.w;
        Q[0] += mj * dx * dx;
        Q[1] += mj * dx * dy;
        Q[2] += mj * dx * dz;
        Q[3] += mj * dy * dy;
        Q[4] += mj * dy * dz;
        Q[5] += mj * dz * dz;
    }
    const double com[3] = {C[0] + off[0], C[1] + off[1], C[2] + off[2]};
    store_node<QUAD>(nt, v, m, com, Q, info, c);
}

// internal cells of level `lev`: [level_start[lev], level_start[lev + 1])
template <bool QUAD>
__global__ void k_level_moments(int lev, const uint32_t* __restrict__ level_start, const Info* __restrict__ info,
                                NodeTables nt)
{
    const int64_t start = level_start[lev];
    const int64_t end = level_start[lev + 1];
    for (int64_t v = start + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < end;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int4 pb = nt.b[v];
        const int nch = pb.w >> 8;
        if (nch == 0) continue;  // leaf: done by k_leaf_moments
        double m = 0.0, S[3] = {0, 0, 0};
        for (int k = 0; k < nch; k++) {
            const int64_t c = pb.z + k;
            const double mc = nt.mass64[c];
            m += mc;
            for (int a = 0; a < 3; a++) S[a] += mc * nt.com64[3 * c + a];
        }
        const double inv = 1.0 / m;
        const double com[3] = {S[0] * inv, S[1] * inv, S[2] * inv};
        double Q[6] = {0, 0, 0, 0, 0, 0};
        for (int k = 0; QUAD && k < nch; k++) {
            const int64_t c = pb.z + k;
            const double mc = nt.mass64[c];
            double d[3];
            for (int a = 0; a < 3; a++) d[a] = nt.com64[3 * c + a] - com[a];
            Q[0] += nt.quad64[6 * c + 0] + mc * d[0] * d[0];
            Q[1] += nt.quad64[6 * c + 1] + mc * d[0] * d[1];
            Q[2] += nt.quad64[6 * c + 2] + mc * d[0] * d[2];
            Q[3] += nt.quad64[6 * c + 3] + mc * d[1] * d[1];
            Q[4] += nt.quad64[6 * c + 4] + mc * d[1] * d[2];
            Q[5] += nt.quad64[6 * c + 5] + mc * d[2] * d[2];
        }
        store_node<QUAD>(nt, v, m, com, Q, info, nt.c[v]);
    }
}

// ------------------------------------------------------------------ groups
// Bodies are walked in groups of at most gmax consecutive Morton-ordered
// bodies.  A cube holding more than gmax bodies is split into groups: a leaf
// into consecutive chunks of gmax; an internal cube by packing runs of its
// consecutive children that hold at most gmax each, greedily left to right
// (children holding more than gmax are split in turn by their own thread).
// A root holding at most gmax is one group.  Each group records a reference
// cube (itself, the leaf it was cut from, or the common parent of the packed
// children); the walk measures positions from that cube's centre.
__global__ void k_group_marks(int64_t M, const NodeTables nt, int gmax, uint32_t* __restrict__ gflag,
                              int32_t* __restrict__ gref_at)
{
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= M) return;
    int4 b = nt.b[v];
    int nch = b.w >> 8;
    if (b.y <= gmax) {
        if (v == 0) {
            gflag[0] = 1;
            gref_at[0] = 0;
        }
        return;
    }
    if (nch == 0) {
        for (int s = 0; s < b.y; s += gmax) {
            gflag[b.x + s] = 1;
            gref_at[b.x + s] = (int32_t)v;
        }
        return;
    }
    int run_first = -1, run_count = 0, run_len = 0, run_only = -1;
    for (int k = 0; k < nch; k++) {
        int c = b.z + k;
        int4 cb = nt.b[c];
        if (cb.y > gmax || run_count + cb.y > gmax) {
            if (run_len > 0) {
                gflag[run_first] = 1;
                gref_at[run_first] = run_len == 1 ? run_only : (int32_t)v;
            }
            run_len = 0;
            run_count = 0;
        }
        if (cb.y > gmax) continue;
        if (run_len == 0) {
            run_first = cb.x;
            run_only = c;
        }
        run_count += cb.y;
        run_len++;
    }
    if (run_len > 0) {
        gflag[run_first] = 1;
        gref_at[run_first] = run_len == 1 ? run_only : (int32_t)v;
    }
}

__global__ void k_group_table(const uint32_t* __restrict__ gflag, const uint32_t* __restrict__ gscan,
                              const int32_t* __restrict__ gref_at, int64_t n, const uint32_t* __restrict__ total,
                              int32_t* __restrict__ gfirst, int32_t* __restrict__ gref, Info* info)
{
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s == 0) {
        gfirst[*total] = (int32_t)n;
        info->G = *total;
    }
    if (s >= n || !gflag[s]) return;
    uint32_t g = gscan[s];
    gfirst[g] = (int32_t)s;
    gref[g] = gref_at[s];
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

int bbox_blocks(int64_t n)
{
    int64_t b = (n + kBboxThreads * 8 - 1) / (kBboxThreads * 8);
    return (int)(b < 1 ? 1 : (b > 1024 ? 1024 : b));
}

void launch_bbox(const float* pos, int64_t n, float* partial, int nblocks, Info* info, cudaStream_t s)
{
    k_bbox<<<nblocks, kBboxThreads, 0, s>>>(pos, n, partial, info);
    count_launches(1);
}

void launch_keys(const float* pos, const float* mass, int64_t n, const Info* info, uint64_t* keys,
                 uint32_t* idx, cudaStream_t s)
{
    k_keys<<<nblk(n, 256), 256, 0, s>>>(pos, mass, n, info, keys, idx,
                                         const_cast<int32_t*>(&info->err));
    count_launches(1);
}

void launch_gather(const float* pos, const float* mass, const uint32_t* perm, int64_t n, float4* body,
                   cudaStream_t s)
{
    k_gather<<<nblk(n, 256), 256, 0, s>>>(pos, mass, perm, n, body);
    count_launches(1);
}

void launch_node_counts(const uint64_t* keys, int64_t n, int leaf_max, int8_t* w, int8_t* delta, int8_t* top,
                        uint32_t* nstart, int32_t* depth, cudaStream_t s)
{
    k_window<<<nblk(n, 256), 256, 0, s>>>(keys, n, leaf_max, w);
    k_node_counts<<<nblk(n, 256), 256, 0, s>>>(keys, w, n, leaf_max, delta, top, nstart, depth);
    count_launches(2);
}

void launch_emit_preorder(const int8_t* delta, const uint32_t* nstart, const uint32_t* prepos, int64_t n,
                          uint32_t* pre_level, uint32_t* pre_first, uint32_t* iota, cudaStream_t s)
{
    k_emit_preorder<<<nblk(n, 256), 256, 0, s>>>(delta, nstart, prepos, n, pre_level, pre_first, iota);
    count_launches(1);
}

void launch_inverse_perm(const uint32_t* perm, int64_t M, uint32_t* inv, cudaStream_t s)
{
    k_inverse_perm<<<nblk(M, 256), 256, 0, s>>>(perm, M, inv);
    count_launches(1);
}

void launch_node_finalize(const uint64_t* keys, const int8_t* top, int64_t n, const uint32_t* bfs_level,
                          const uint32_t* bfs_pre, const uint32_t* pre_first, const uint32_t* bfs_of_pre,
                          int64_t M, NodeTables nt, cudaStream_t s)
{
    k_node_finalize<<<nblk(M, 128), 128, 0, s>>>(keys, top, n, bfs_level, bfs_pre, pre_first, bfs_of_pre, M, nt);
    count_launches(1);
}

void launch_moments(const float4* body, int64_t M, int depth, const uint32_t* level_start, const Info* info,
                    NodeTables nt, bool quad, cudaStream_t s)
{
    if (quad) k_leaf_moments<true><<<nblk(M, 128), 128, 0, s>>>(body, M, info, nt);
    else k_leaf_moments<false><<<nblk(M, 128), 128, 0, s>>>(body, M, info, nt);
    count_launches(1);
    int64_t g = nblk(M, 128);
    if (g > 8 * 152) g = 8 * 152;
    for (int lev = depth - 1; lev >= 0; lev--) {
        if (quad) k_level_moments<true><<<(unsigned)g, 128, 0, s>>>(lev, level_start, info, nt);
        else k_level_moments<false><<<(unsigned)g, 128, 0, s>>>(lev, level_start, info, nt);
        count_launches(1);
    }
}

void launch_group_marks(int64_t M, const NodeTables nt, int gmax, int64_t n, uint32_t* gflag, int32_t* gref_at,
                        cudaStream_t s)
{
    cudaMemsetAsync(gflag, 0, n * sizeof(uint32_t), s);
    k_group_marks<<<nblk(M, 128), 128, 0, s>>>(M, nt, gmax, gflag, gref_at);
    count_launches(1);
}

void launch_group_table(const uint32_t* gflag, const uint32_t* gscan, const int32_t* gref_at, int64_t n,
                        const uint32_t* total, int32_t* gfirst, int32_t* gref, Info* info, cudaStream_t s)
{
    k_group_table<<<nblk(n, 256), 256, 0, s>>>(gflag, gscan, gref_at, n, total, gfirst, gref, info);
    count_launches(1);
}

}  // namespace tc
