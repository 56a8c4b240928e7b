// tc_build.cu -- oct-tree construction on the GPU (Sec. 3.1 of the paper:
// the space is divided recursively into 8 sub-cubes until a cube holds no
// more than a threshold of bodies; every cell carries its total mass and
// centre of mass).
//
// The bodies of a batch of independent systems are processed together: each
// system gets its own root cube and tree, and a system boundary acts like a
// difference in the first digit of two keys.
//
// Pipeline (all on one stream):
//   1. k_bbox, k_sys_cube  per-system bounding box -> power-of-two root cube
//                  on a 2^21 grid (FP64)
//   2. k_keys      63-bit Morton keys (exact FP64 quantisation)
//   3. radix sort  stable sort by (system, key, index)    [tc_sort.cu]
//   4. k_gather    bodies in Morton order as float4 (x, y, z, m)
//   5. k_window / k_node_counts
//                  which cubes of the recursive subdivision start at each
//                  sorted body (a sliding-window test, below)
//   6. scan + k_emit_preorder      node table in pre-order
//   7. one stable radix pass by level  -> breadth-first order
//   8. k_node_finalize  counts, children, integer centres
//   9. k_leaf_moments, then k_level_moments level by level from the deepest
//                  mass / centre of mass (float-pair sums, FP64-class, stored
//                  in FP64) / second moments (FP32), bottom-up
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

// With several systems, cd() of two bodies of different systems is taken as
// -1 (no common cube), so delta_s = -1 at the first body of every system and
// each system's root is a node of level 0.  The node table is sized by the
// host from an earlier build; a device-side check stops the build (error word
// kErrCapacity) if a later tree needs more, so no kernel writes past it.

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

__device__ __forceinline__ bool capacity_failed(const Info* info)
{
    return (*(volatile const int32_t*)&info->err & kErrCapacity) != 0;
}

// ------------------------------------------------------------------ systems
__global__ void k_sys_ids(const int64_t* __restrict__ off, int nsys, int64_t n, uint32_t* __restrict__ sys_of,
                          SysParams* __restrict__ sysp)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nsys) {
        sysp[i].first = (int32_t)off[i];
        sysp[i].end = (int32_t)off[i + 1];
    }
    if (i >= n) return;
    int lo = 0, hi = nsys - 1;  // last system whose offset is <= i
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= i) lo = mid;
        else hi = mid - 1;
    }
    sys_of[i] = (uint32_t)lo;
}

// ------------------------------------------------------------------ bbox
constexpr int kBboxThreads = 256;

// floats as ints with the same order (no NaN): min/max by integer atomics
__device__ __forceinline__ int f2o(float x)
{
    const int i = __float_as_int(x);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float o2f(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

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

__global__ void k_bbox_init(SysParams* __restrict__ sysp, int nsys)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys) return;
    for (int a = 0; a < 3; a++) {
        sysp[s].bb[a] = f2o(INFINITY);
        sysp[s].bb[3 + a] = f2o(-INFINITY);
    }
}

// one block per chunk (system, start, end) of at most kBboxChunk bodies
__global__ void __launch_bounds__(kBboxThreads) k_bbox(const float* __restrict__ pos, const int4* __restrict__ chunks,
                                                       SysParams* __restrict__ sysp, int32_t* __restrict__ err)
{
    __shared__ float sm[6][kBboxThreads / 32];
    const int4 ch = chunks[blockIdx.x];
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    bool bad = false;
    for (int64_t i = ch.y + threadIdx.x; i < ch.z; i += kBboxThreads) {
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const float x = pos[3 * i + a];
            bad |= !isfinite(x);
            lo[a] = fminf(lo[a], x);
            hi[a] = fmaxf(hi[a], x);
        }
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(err, kErrNonFinite);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const float l = warp_min(lo[a]), h = warp_max(hi[a]);
        if (lane == 0) {
            sm[a][w] = l;
            sm[3 + a][w] = h;
        }
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        const int a = threadIdx.x;
        float r = a < 3 ? INFINITY : -INFINITY;
        for (int k = 0; k < kBboxThreads / 32; k++) r = a < 3 ? fminf(r, sm[a][k]) : fmaxf(r, sm[a][k]);
        if (a < 3) atomicMin(&sysp[ch.x].bb[a], f2o(r));
        else atomicMax(&sysp[ch.x].bb[a], f2o(r));
    }
}

// Root cube of each system: side L = smallest power of two with
// L >= extent * (1 + 2^-20), grid step h = L / 2^21, corner c0 = floor(min/h) h.
__global__ void k_sys_cube(SysParams* __restrict__ sysp, int nsys)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys) return;
    SysParams& P = sysp[s];
    double dlo[3], dhi[3];
    for (int a = 0; a < 3; a++) {
        dlo[a] = (double)o2f(P.bb[a]);
        dhi[a] = (double)o2f(P.bb[3 + a]);
    }
    double extent = 0.0;
    for (int a = 0; a < 3; a++) {
        const double e = dhi[a] - dlo[a];
        if (e > extent) extent = e;
    }
    const double target = extent * (1.0 + 0x1p-20);
    double L = 1.0;  // all bodies coincide (or a non-finite input): unit cube
    if (target > 0.0 && target < INFINITY) {
        int e;
        const double m = frexp(target, &e);
        L = (m == 0.5) ? target : ldexp(1.0, e);
    }
    const double h = L / 2097152.0;
    int eh;
    frexp(h, &eh);        // h = 2^(eh - 1)
    P.qexp = 1 - eh;      // 1/h = 2^qexp
    for (int a = 0; a < 3; a++) {
        double K0 = floor(dlo[a] / h);
        if (!(K0 == K0) || K0 > 9e15 || K0 < -9e15) K0 = 0.0;  // non-finite input: keys are reported, not used
        P.c0[a] = K0 * h;
        P.qoff[a] = (long long)K0;
    }
    P.L = L;
    P.h = h;
    P.Lf = (float)L;
    P.uf = (float)(h * 0.5);
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
                       const uint32_t* __restrict__ sys_of, const SysParams* __restrict__ sysp,
                       uint64_t* __restrict__ keys, uint32_t* __restrict__ idx, int32_t* err)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const SysParams& P = sysp[sys_of[i]];
    const int k = P.qexp;
    const uint64_t qx = quantise(pos[3 * i], k, P.qoff[0]);
    const uint64_t qy = quantise(pos[3 * i + 1], k, P.qoff[1]);
    const uint64_t qz = quantise(pos[3 * i + 2], k, P.qoff[2]);
    keys[i] = (spread3(qx) << 2) | (spread3(qy) << 1) | spread3(qz);
    idx[i] = (uint32_t)i;
    const float m = mass[i];
    if (!(isfinite(m) && m > 0.0f)) atomicOr(err, kErrNonFinite);
}

__global__ void k_gather(const float* __restrict__ pos, const float* __restrict__ mass,
                         const uint32_t* __restrict__ perm, int64_t n, float4* __restrict__ body)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t i = perm[k];
    body[k] = make_float4(pos[3 * i], pos[3 * i + 1], pos[3 * i + 2], mass[i]);
}

// ------------------------------------------------------------------ nodes
__global__ void k_window(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ sys_of, int64_t n,
                         int leaf_max, int8_t* __restrict__ w)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    w[j] = (j + leaf_max < n && sys_of[j] == sys_of[j + leaf_max])
               ? (int8_t)common_digits(keys[j], keys[j + leaf_max])
               : (int8_t)-1;
}

__global__ void k_node_counts(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ sys_of,
                              const int8_t* __restrict__ w, int64_t n, int leaf_max, int8_t* __restrict__ delta,
                              int8_t* __restrict__ top, uint32_t* __restrict__ nstart, int32_t* __restrict__ depth)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int t = 0;
    if (s < n) {
        const int d = (s == 0 || sys_of[s] != sys_of[s - 1]) ? -1 : common_digits(keys[s - 1], keys[s]);
        int W = -1;
        const int64_t j0 = s - leaf_max < 0 ? 0 : s - leaf_max;
        for (int64_t j = j0; j <= s; j++) W = max(W, (int)w[j]);
        t = min(W + 1, kMaxLevel);
        delta[s] = (int8_t)d;
        top[s] = (int8_t)t;
        nstart[s] = (uint32_t)max(0, t - d);
    }
    // deepest level of the forest: a block maximum, then one atomic per
    // block (blocks of 256)
    __shared__ int wmax[8];
#pragma unroll
    for (int o = 16; o; o >>= 1) t = max(t, __shfl_xor_sync(0xffffffffu, t, o));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); k++) t = max(t, wmax[k]);
        atomicMax(depth, t);
    }
}

// The same two steps in one kernel for leaf_max <= kTileWindow: a block of
// kCountThreads sorted bodies stages the keys and systems of
// [b0 - leaf_max, b0 + kCountThreads + leaf_max) in shared memory, forms the
// window digits cd(key_j, key_j+leaf_max) of [b0 - leaf_max, b0 + kCountThreads)
// there, and takes each body's window maximum from them.
constexpr int kCountThreads = 256;
constexpr int kTileWindow = 256;

__global__ void __launch_bounds__(kCountThreads) k_node_counts_tiled(const uint64_t* __restrict__ keys,
                                                                     const uint32_t* __restrict__ sys_of, int64_t n,
                                                                     int leaf_max, int8_t* __restrict__ delta,
                                                                     int8_t* __restrict__ top,
                                                                     uint32_t* __restrict__ nstart,
                                                                     int32_t* __restrict__ depth)
{
    __shared__ uint64_t sk[kCountThreads + 2 * kTileWindow];
    __shared__ uint32_t ss[kCountThreads + 2 * kTileWindow];
    __shared__ int8_t sw[kCountThreads + kTileWindow];
    const int64_t b0 = (int64_t)blockIdx.x * kCountThreads;
    const int64_t base = b0 - leaf_max;  // smem index 0 holds body base
    const int nk = kCountThreads + 2 * leaf_max;
    for (int i = threadIdx.x; i < nk; i += kCountThreads) {
        const int64_t j = base + i;
        const bool in = j >= 0 && j < n;
        sk[i] = in ? keys[j] : 0ull;
        ss[i] = in ? sys_of[j] : 0xffffffffu;
    }
    __syncthreads();
    // window digits of bodies base .. b0 + kCountThreads - 1
    const int nw = kCountThreads + leaf_max;
    for (int i = threadIdx.x; i < nw; i += kCountThreads) {
        const int64_t j = base + i;
        int8_t v = -1;
        if (j >= 0 && j + leaf_max < n && ss[i] == ss[i + leaf_max]) v = (int8_t)common_digits(sk[i], sk[i + leaf_max]);
        sw[i] = v;
    }
    __syncthreads();
    const int64_t s = b0 + threadIdx.x;
    int t = 0;
    if (s < n) {
        const int i = threadIdx.x + leaf_max;  // smem index of body s
        const int d = (s == 0 || ss[i] != ss[i - 1]) ? -1 : common_digits(sk[i - 1], sk[i]);
        int W = -1;
        const int i0 = s - leaf_max < 0 ? (int)(leaf_max - s) : 0;  // window clipped at body 0
        for (int k = i0; k <= leaf_max; k++) W = max(W, (int)sw[threadIdx.x + k]);
        t = min(W + 1, kMaxLevel);
        delta[s] = (int8_t)d;
        top[s] = (int8_t)t;
        nstart[s] = (uint32_t)max(0, t - d);
    }
    // deepest level: a block maximum, then one atomic per block (one per
    // warp made the atomics on the single word the kernel's bottleneck)
    __shared__ int wmax[kCountThreads / 32];
#pragma unroll
    for (int o = 16; o; o >>= 1) t = max(t, __shfl_xor_sync(0xffffffffu, t, o));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < kCountThreads / 32; k++) t = max(t, wmax[k]);
        atomicMax(depth, t);
    }
}

__global__ void k_check_capacity(const uint32_t* __restrict__ m_total, Info* info)
{
    const int64_t M = *m_total;
    info->M = M;
    if (M > info->cap_m) atomicOr(&info->err, kErrCapacity);
}

__global__ void k_emit_preorder(const int8_t* __restrict__ delta, const uint32_t* __restrict__ nstart,
                                const uint32_t* __restrict__ prepos, int64_t n, const Info* info,
                                uint32_t* __restrict__ pre_level, uint32_t* __restrict__ pre_first,
                                uint32_t* __restrict__ iota)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n || capacity_failed(info)) return;
    const uint32_t c = nstart[s], p = prepos[s];
    const int l0 = delta[s] + 1;
    for (uint32_t k = 0; k < c; k++) {
        pre_level[p + k] = (uint32_t)(l0 + (int)k);
        pre_first[p + k] = (uint32_t)s;
        iota[p + k] = p + k;
    }
}

__global__ void k_inverse_perm(const uint32_t* __restrict__ perm, const Info* info, uint32_t* __restrict__ inv)
{
    if (capacity_failed(info)) return;
    const int64_t M = info->M;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < M; b += (int64_t)gridDim.x * blockDim.x)
        inv[perm[b]] = (uint32_t)b;
}

// first index e in [lo, hi) with (keys[e] >> sh) > pfx, or hi
__device__ __forceinline__ int64_t run_end(const uint64_t* __restrict__ keys, int64_t lo, int64_t hi,
                                           int sh, uint64_t pfx)
{
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if ((keys[mid] >> sh) > pfx) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

__global__ void k_node_finalize(const uint64_t* __restrict__ keys, const int8_t* __restrict__ top,
                                const uint32_t* __restrict__ sys_of, const SysParams* __restrict__ sysp,
                                const uint32_t* __restrict__ bfs_level, const uint32_t* __restrict__ bfs_pre,
                                const uint32_t* __restrict__ pre_first, const uint32_t* __restrict__ bfs_of_pre,
                                const Info* info, NodeTables nt)
{
    if (capacity_failed(info)) return;
    const int64_t M = info->M;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < M; b += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t p = bfs_pre[b];
        const int l = (int)bfs_level[b];
        const int64_t s = pre_first[p];
        const uint32_t sy = sys_of[s];
        const int64_t send = sysp[sy].end;
        const int sh = 3 * (kMaxLevel - l);
        const uint64_t pfx = (l == 0) ? 0ull : (keys[s] >> sh);
        const int64_t e = (l == 0) ? send : run_end(keys, s + 1, send, sh, pfx);
        int nch = 0;
        int32_t cf = -1;
        if (l < (int)top[s]) {
            cf = (int32_t)bfs_of_pre[p + 1];
            const int shc = sh - 3;
            int64_t c = s;
            while (c < e) {
                const uint64_t cp = keys[c] >> shc;
                c = run_end(keys, c + 1, e, shc, cp);
                nch++;
            }
        }
        nt.b[b] = make_int4((int)s, (int)(e - s), cf, l | (nch << 8));
        const uint32_t ix = compact3(pfx >> 2), iy = compact3(pfx >> 1), iz = compact3(pfx);
        const int c1 = 1 << (kMaxLevel - l);
        nt.c[b] = make_int4((int)(2 * ix + 1) * c1, (int)(2 * iy + 1) * c1, (int)(2 * iz + 1) * c1, (int)sy);
    }
}

// ------------------------------------------------------------------ moments
// Mass, centre of mass and second moments about the centre of mass.  The
// sums of m and m x are kept as unevaluated pairs of floats (hi + lo, about
// 48 significant bits) on the FP32 pipe and stored in FP64 as well; GB300's
// FP64 pipe, a small fraction of its FP32 rate, bound these kernels when
// they summed in FP64.  Leaves sum their bodies;
// an internal cell combines its children: M = sum M_c,
// com = sum M_c com_c / M, Q = sum Q_c + M_c dc dc^T with dc = com_c - com.
// Leaves are done in one launch; internal cells level by level from the
// deepest, one thread per cell of the level (cells of a level are contiguous
// in breadth-first order), so every lane of a warp has a cell to do.
__device__ __forceinline__ void cube_centre(const SysParams& P, int4 c, double* C)
{
    const double u = 0.5 * P.h;
    C[0] = P.c0[0] + (double)c.x * u;
    C[1] = P.c0[1] + (double)c.y * u;
    C[2] = P.c0[2] + (double)c.z * u;
}

// The exact FP64 value of a float, formed on the integer pipe from the
// IEEE-754 fields (sign, exponent rebased from 127 to 1023, the 23 mantissa
// bits moved to the top of the 52): GB300's FP64 pipe, which the leaf
// moments saturate, then only adds and multiplies.  Zero, subnormal and
// non-finite values take the conversion instruction.
__device__ __forceinline__ double widen(float f)
{
    const uint32_t u = __float_as_uint(f);
    const uint32_t e = (u >> 23) & 0xffu;
    if (e == 0u || e == 0xffu) return (double)f;
    const uint64_t d = ((uint64_t)(u >> 31) << 63) | ((uint64_t)(e + 896u) << 52) | ((uint64_t)(u & 0x7fffffu) << 29);
    return __longlong_as_double((long long)d);
}

// (hi, lo) += p + e for a normalised pair (|lo| <= ulp(hi) / 2): hi + p by
// Knuth's TwoSum (s + t = hi + p exactly), the error t, lo and e added in
// FP32, then renormalised by Dekker's FastTwoSum (exact: |t| is a few ulps
// of s at most, or s = 0).  One call errs by at most about 2^-46 |s|.
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float p, float e)
{
    const float s = hi + p;
    const float bp = s - hi;
    const float t = ((hi - (s - bp)) + (p - bp)) + (lo + e);
    hi = s + t;
    lo = t - (hi - s);
}

// the centre of mass S / m of float pairs as a pair of floats: q1 = Sh / mh,
// the remainder S - q1 m (Sh - q1 mh exact by one FMA: the residual of a
// correctly rounded quotient is a float), q2 = remainder / mh; q1 + q2 is
// S / m within about 2^-44 of it, taken exactly into FP64 (com) and rounded
// once to float (comf); the FP64 pipe is spared the division
__device__ __forceinline__ void pair_quotient(const float (&Sh)[3], const float (&Sl)[3], float mh, float ml,
                                              double (&com)[3], float (&comf)[3])
{
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const float q1 = Sh[a] / mh;
        const float r = fmaf(-q1, mh, Sh[a]) + fmaf(-q1, ml, Sl[a]);
        const float q2 = r / mh;
        com[a] = widen(q1) + widen(q2);
        comf[a] = q1 + q2;
    }
}

// comf / Mf: the float roundings of com and M when the caller has
// them (the same values, without the FP64 pipe's conversions)
template <bool QUAD>
__device__ void store_node(NodeTables& nt, int64_t v, double M, const double* com, const float* Q, const double* C,
                           const float* comf = nullptr, float Mf = 0.f)
{
    nt.mass64[v] = M;
    for (int a = 0; a < 3; a++) nt.com64[3 * v + a] = com[a];
    const float mf = comf ? Mf : (float)M;
    nt.a[v] = make_float4((float)(com[0] - C[0]), (float)(com[1] - C[1]), (float)(com[2] - C[2]), mf);
    if (comf) nt.d[v] = make_float4(comf[0], comf[1], comf[2], mf);
    else nt.d[v] = make_float4((float)com[0], (float)com[1], (float)com[2], mf);
    if (QUAD) {
        for (int a = 0; a < 6; a++) nt.quad[6 * v + a] = Q[a];
    }
}

// Mass and centre of mass as float pairs (FP64-class); second moments in
// FP32.  The second moments only feed the learned correction's BF16
// features and the quadrupole terms, small corrections to the monopole, so
// FP32 serves them (their error stays a few hundred FP32 ulps of M s^2).
// Per leaf: Q about the cube centre C from the bodies'
// offsets x - C, then moved to the centre of mass by the parallel-axis rule
// Q_com = Q_C - M (com - C)(com - C)^T.  The offsets are formed in FP32
// against C split into C_hi = fl(C) and C_lo = fl(C - C_hi): (x - C_hi) -
// C_lo, within 2 FP32 roundings of x - C (the first subtraction is exact
// unless |C| < 2 s, where its rounding is one of a number below 2 s).
template <bool QUAD>
__global__ void k_leaf_moments(const float4* __restrict__ body, const SysParams* __restrict__ sysp,
                               const Info* info, NodeTables nt)
{
    if (capacity_failed(info)) return;
    const int64_t M = info->M;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < M; v += (int64_t)gridDim.x * blockDim.x) {
        const int4 b = nt.b[v];
        if ((b.w >> 8) != 0) continue;  // internal
        const int4 c = nt.c[v];
        double C[3];
        cube_centre(sysp[c.w], c, C);
        float Chi[3] = {0.f, 0.f, 0.f}, Clo[3] = {0.f, 0.f, 0.f};
        if (QUAD)
            for (int a = 0; a < 3; a++) {
                Chi[a] = (float)C[a];
                Clo[a] = (float)(C[a] - (double)Chi[a]);
            }
        // m and sum m x in absolute coordinates as unevaluated sums of two
        // floats (hi + lo): each product m x split exactly into p + e by
        // one FMA and added by two_sum_acc.  Over a leaf's c bodies the error
        // stays below about c 2^-46 of the largest partial sum of |terms|
        // (2.3e-13 of it for c = 16): FP64-class accuracy on the FP32 pipe,
        // which GB300 runs 64 times faster than its FP64 pipe; the pair goes
        // to the levels above, and hi + lo exactly into FP64.  Q about C in
        // FP32 alongside.
        float mh = 0.f, ml = 0.f, Sh[3] = {0.f, 0.f, 0.f}, Sl[3] = {0.f, 0.f, 0.f};
        float QC[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int j = b.x; j < b.x + b.y; j++) {
            const float4 q = body[j];
            two_sum_acc(mh, ml, q.w, 0.f);
            const float xs[3] = {q.x, q.y, q.z};
#pragma unroll
            for (int a = 0; a < 3; a++) {
                const float p = q.w * xs[a];
                const float e = fmaf(q.w, xs[a], -p);  // q.w x = p + e exactly
                two_sum_acc(Sh[a], Sl[a], p, e);
            }
            if (QUAD) {
                const float dx = (q.x - Chi[0]) - Clo[0], dy = (q.y - Chi[1]) - Clo[1], dz = (q.z - Chi[2]) - Clo[2];
                const float wx = q.w * dx, wy = q.w * dy, wz = q.w * dz;
                QC[0] = fmaf(wx, dx, QC[0]);
                QC[1] = fmaf(wx, dy, QC[1]);
                QC[2] = fmaf(wx, dz, QC[2]);
                QC[3] = fmaf(wy, dy, QC[3]);
                QC[4] = fmaf(wy, dz, QC[4]);
                QC[5] = fmaf(wz, dz, QC[5]);
            }
        }
        const double m = widen(mh) + widen(ml);
        double com[3];
        float comf[3];
        pair_quotient(Sh, Sl, mh, ml, com, comf);
        float Q[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (QUAD) {
            const float ex = (float)(com[0] - C[0]), ey = (float)(com[1] - C[1]), ez = (float)(com[2] - C[2]);
            const float mf = (float)m;
            Q[0] = fmaf(-mf * ex, ex, QC[0]);
            Q[1] = fmaf(-mf * ex, ey, QC[1]);
            Q[2] = fmaf(-mf * ex, ez, QC[2]);
            Q[3] = fmaf(-mf * ey, ey, QC[3]);
            Q[4] = fmaf(-mf * ey, ez, QC[4]);
            Q[5] = fmaf(-mf * ez, ez, QC[5]);
        }
        store_node<QUAD>(nt, v, m, com, Q, C, comf, mh + ml);
        nt.dsum[2 * v] = make_float4(mh, Sh[0], Sh[1], Sh[2]);
        nt.dsum[2 * v + 1] = make_float4(ml, Sl[0], Sl[1], Sl[2]);
    }
}

// one internal cell v from its children (a leaf returns at once): mass and
// the sum of m x as float pairs, the children's pairs added by two_sum_acc
// (each addition errs by at most about 2^-47 of the magnitudes added, so a
// body's term collects at most depth x 2^-47 of relative error on its way
// to the root: 1.5e-13 at depth 21), the centre of mass as their float-pair
// quotient, both stored in FP64 too; second moments in FP32 by the parallel-axis rule
// from the children's, Q_v = sum_c Q_c + m_c d_c d_c^T, d_c = com_c - com_v
// formed in FP32 from the stored offsets of the centres of mass from their
// cube centres, d_c = (a_c - a_v) + (k_c - k_v) u (k the integer cube
// centres in units u = h/2, their difference exact)
template <bool QUAD>
__device__ __forceinline__ void level_node(int64_t v, const SysParams* __restrict__ sysp, NodeTables& nt)
{
    const int4 pb = nt.b[v];
    const int nch = pb.w >> 8;
    if (nch == 0) return;  // leaf: done by k_leaf_moments
    float mh = 0.f, ml = 0.f, Sh[3] = {0.f, 0.f, 0.f}, Sl[3] = {0.f, 0.f, 0.f};
    for (int k = 0; k < nch; k++) {
        const int64_t c = pb.z + k;
        const float4 h = nt.dsum[2 * c], l = nt.dsum[2 * c + 1];
        two_sum_acc(mh, ml, h.x, l.x);
        two_sum_acc(Sh[0], Sl[0], h.y, l.y);
        two_sum_acc(Sh[1], Sl[1], h.z, l.z);
        two_sum_acc(Sh[2], Sl[2], h.w, l.w);
    }
    const double m = widen(mh) + widen(ml);
    double com[3];
    float comf[3];
    pair_quotient(Sh, Sl, mh, ml, com, comf);
    nt.dsum[2 * v] = make_float4(mh, Sh[0], Sh[1], Sh[2]);
    nt.dsum[2 * v + 1] = make_float4(ml, Sl[0], Sl[1], Sl[2]);
    const int4 cc = nt.c[v];
    double C[3];
    cube_centre(sysp[cc.w], cc, C);
    float Q[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const float av[3] = {(float)(com[0] - C[0]), (float)(com[1] - C[1]), (float)(com[2] - C[2])};
    const float uf = sysp[cc.w].uf;
    for (int k = 0; QUAD && k < nch; k++) {
        const int64_t c = pb.z + k;
        const float4 ac = nt.a[c];
        const int4 kc = nt.c[c];
        const float mc = ac.w;
        const float d[3] = {fmaf((float)(kc.x - cc.x), uf, ac.x - av[0]), fmaf((float)(kc.y - cc.y), uf, ac.y - av[1]),
                            fmaf((float)(kc.z - cc.z), uf, ac.z - av[2])};
        const float* qc = nt.quad + 6 * c;
        Q[0] += fmaf(mc * d[0], d[0], qc[0]);
        Q[1] += fmaf(mc * d[0], d[1], qc[1]);
        Q[2] += fmaf(mc * d[0], d[2], qc[2]);
        Q[3] += fmaf(mc * d[1], d[1], qc[3]);
        Q[4] += fmaf(mc * d[1], d[2], qc[4]);
        Q[5] += fmaf(mc * d[2], d[2], qc[5]);
    }
    store_node<QUAD>(nt, v, m, com, Q, C, comf, mh + ml);
}

// internal cells of level `lev`: [level_start[lev], level_start[lev + 1])
template <bool QUAD>
__global__ void k_level_moments(int lev, const uint32_t* __restrict__ level_start,
                                const SysParams* __restrict__ sysp, const Info* info, NodeTables nt)
{
    if (capacity_failed(info)) return;
    const int64_t start = level_start[lev];
    const int64_t end = level_start[lev + 1];
    for (int64_t v = start + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < end;
         v += (int64_t)gridDim.x * blockDim.x)
        level_node<QUAD>(v, sysp, nt);
}

// every level from the deepest possible down to lev_lo, in one block: the
// cells past the depth a captured step expects (normally none)
template <bool QUAD>
__global__ void __launch_bounds__(256) k_level_moments_deep(int lev_lo, const uint32_t* __restrict__ level_start,
                                                             const SysParams* __restrict__ sysp, const Info* info,
                                                             NodeTables nt)
{
    if (capacity_failed(info)) return;
    for (int lev = kMaxLevel - 1; lev >= lev_lo; lev--) {
        const int64_t start = level_start[lev];
        const int64_t end = level_start[lev + 1];
        for (int64_t v = start + threadIdx.x; v < end; v += blockDim.x) level_node<QUAD>(v, sysp, nt);
        __syncthreads();
    }
}

// total mass of each system: its root's mass
__global__ void k_sys_mass(SysParams* __restrict__ sysp, int nsys, const NodeTables nt, const Info* info)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys || capacity_failed(info)) return;
    sysp[s].msys = (float)nt.mass64[s];
}

// ------------------------------------------------------------------ groups
// Bodies are walked in groups of at most gmax consecutive Morton-ordered
// bodies of one system.  A cube holding more than gmax bodies is split into
// groups: a leaf into consecutive chunks of gmax; an internal cube by packing
// runs of its consecutive children that hold at most gmax each, greedily left
// to right (children holding more than gmax are split in turn by their own
// thread).  A root holding at most gmax is one group.  Each group records a
// reference cube (itself, the leaf it was cut from, or the common parent of
// the packed children); the walk measures positions from that cube's centre.
__global__ void k_group_marks(const Info* info, const NodeTables nt, int gmax, uint32_t* __restrict__ gflag,
                              int32_t* __restrict__ gref_at)
{
    if (capacity_failed(info)) return;
    const int64_t M = info->M;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < M; v += (int64_t)gridDim.x * blockDim.x) {
        const int4 b = nt.b[v];
        const int nch = b.w >> 8;
        if (b.y <= gmax) {
            if ((b.w & 255) == 0) {  // a root
                gflag[b.x] = 1;
                gref_at[b.x] = (int32_t)v;
            }
            continue;
        }
        if (nch == 0) {
            for (int s = 0; s < b.y; s += gmax) {
                gflag[b.x + s] = 1;
                gref_at[b.x + s] = (int32_t)v;
            }
            continue;
        }
        int run_first = -1, run_count = 0, run_len = 0, run_only = -1;
        for (int k = 0; k < nch; k++) {
            const int c = b.z + k;
            const int4 cb = nt.b[c];
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
}

__global__ void k_group_table(const uint32_t* __restrict__ gflag, const uint32_t* __restrict__ gscan,
                              const int32_t* __restrict__ gref_at, int64_t n, const uint32_t* __restrict__ total,
                              int32_t* __restrict__ gfirst, int32_t* __restrict__ gref, Info* info)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s == 0) {
        gfirst[*total] = (int32_t)n;
        info->G = *total;
    }
    if (s >= n || !gflag[s]) return;
    const uint32_t g = gscan[s];
    gfirst[g] = (int32_t)s;
    gref[g] = gref_at[s];
}

// Groups split by size for the walk, so that a group of at most 32 bodies is
// summed one body per lane and one of at most 64 two per lane: class 0
// holds at most 32 bodies, class 1 at most 64, class 2 more.  Block b of
// kSplitBlocks takes the b-th contiguous range of the group table; a first
// pass counts each range's groups per class, a second gives every group its
// place (the counts of the ranges before it, then warp ballots within the
// range), keeping the group order within each class.
constexpr int kSplitBlocks = 256;
constexpr int kSplitThreads = 256;

__device__ __forceinline__ int size_class(const int32_t* __restrict__ gfirst, int64_t g)
{
    const int cnt = gfirst[g + 1] - gfirst[g];
    return cnt <= 32 ? 0 : (cnt <= 64 ? 1 : 2);
}

__device__ __forceinline__ void split_range(const Info* info, int64_t& lo, int64_t& hi)
{
    const int64_t G = capacity_failed(info) ? 0 : info->G;
    const int64_t per = (G + gridDim.x - 1) / gridDim.x;
    lo = min(G, (int64_t)blockIdx.x * per);
    hi = min(G, lo + per);
}

__device__ __forceinline__ int warp_sum_i(int v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(kSplitThreads) k_split_count(const int32_t* __restrict__ gfirst, const Info* info,
                                                               int32_t* __restrict__ bcount)
{
    __shared__ int red[kSplitThreads / 32][3];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    int64_t lo, hi;
    split_range(info, lo, hi);
    int c[3] = {0, 0, 0};
    for (int64_t g = lo + tid; g < hi; g += blockDim.x) {
        const int k = size_class(gfirst, g);
        c[0] += k == 0;
        c[1] += k == 1;
        c[2] += k == 2;
    }
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const int v = warp_sum_i(c[k]);
        if (lane == 0) red[w][k] = v;
    }
    __syncthreads();
    if (tid < 3) {
        int t = 0;
        for (int ww = 0; ww < kSplitThreads / 32; ww++) t += red[ww][tid];
        bcount[3 * blockIdx.x + tid] = t;
    }
}

__global__ void __launch_bounds__(kSplitThreads) k_split_scatter(const int32_t* __restrict__ gfirst, const Info* info,
                                                                 const int32_t* __restrict__ bcount, int64_t cap_g,
                                                                 int32_t* __restrict__ lists,
                                                                 int32_t* __restrict__ counts)
{
    constexpr int W = kSplitThreads / 32;
    __shared__ int red[W][6];
    __shared__ int wcnt[W][3];
    __shared__ int base[3];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    // this range's offsets (the ranges before it) and the class totals
    int v[6] = {0, 0, 0, 0, 0, 0};
    for (int j = tid; j < (int)gridDim.x; j += blockDim.x) {
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const int x = bcount[3 * j + k];
            if (j < (int)blockIdx.x) v[k] += x;
            v[3 + k] += x;
        }
    }
#pragma unroll
    for (int k = 0; k < 6; k++) {
        const int s = warp_sum_i(v[k]);
        if (lane == 0) red[w][k] = s;
    }
    __syncthreads();
    if (tid < 6) {
        int t = 0;
        for (int ww = 0; ww < W; ww++) t += red[ww][tid];
        if (tid < 3) base[tid] = t;
        else if (blockIdx.x == 0) counts[tid - 3] = t;
    }
    int64_t lo, hi;
    split_range(info, lo, hi);
    const unsigned lt = (1u << lane) - 1u;
    for (int64_t c0 = lo; c0 < hi; c0 += kSplitThreads) {
        const int64_t g = c0 + tid;
        const int cls = g < hi ? size_class(gfirst, g) : -1;
        unsigned m[3];
#pragma unroll
        for (int k = 0; k < 3; k++) m[k] = __ballot_sync(0xffffffffu, cls == k);
        __syncthreads();  // base is set; the previous chunk's readers of wcnt and base are done
        if (lane == 0)
            for (int k = 0; k < 3; k++) wcnt[w][k] = __popc(m[k]);
        __syncthreads();
        if (cls >= 0) {
            int off = base[cls] + __popc(m[cls] & lt);
            for (int ww = 0; ww < w; ww++) off += wcnt[ww][cls];
            lists[cls * cap_g + off] = (int32_t)g;
        }
        __syncthreads();
        if (tid < 3) {
            int t = 0;
            for (int ww = 0; ww < W; ww++) t += wcnt[ww][tid];
            base[tid] += t;
        }
    }
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }
// grid of a grid-stride kernel over a device-side count bounded by cap
inline unsigned gsgrid(int64_t cap, int t)
{
    int64_t g = (cap + t - 1) / t;
    const int64_t gmax = 16 * (int64_t)sm_count();
    if (g > gmax) g = gmax;
    return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

void launch_sys_ids(const int64_t* offsets, int nsys, int64_t n, uint32_t* sys_of, SysParams* sysp, cudaStream_t s)
{
    const int64_t m = n > nsys ? n : nsys;
    k_sys_ids<<<nblk(m, 256), 256, 0, s>>>(offsets, nsys, n, sys_of, sysp);
    count_launches(1);
}

void launch_bbox(const float* pos, const int4* chunks, int nchunks, SysParams* sysp, int nsys, int32_t* err,
                 cudaStream_t s)
{
    k_bbox_init<<<nblk(nsys, 128), 128, 0, s>>>(sysp, nsys);
    k_bbox<<<nchunks, kBboxThreads, 0, s>>>(pos, chunks, sysp, err);
    k_sys_cube<<<nblk(nsys, 128), 128, 0, s>>>(sysp, nsys);
    count_launches(3);
}

void launch_keys(const float* pos, const float* mass, int64_t n, const uint32_t* sys_of, const SysParams* sysp,
                 uint64_t* keys, uint32_t* idx, int32_t* err, cudaStream_t s)
{
    k_keys<<<nblk(n, 256), 256, 0, s>>>(pos, mass, n, sys_of, sysp, keys, idx, err);
    count_launches(1);
}

void launch_gather(const float* pos, const float* mass, const uint32_t* perm, int64_t n, float4* body,
                   cudaStream_t s)
{
    k_gather<<<nblk(n, 256), 256, 0, s>>>(pos, mass, perm, n, body);
    count_launches(1);
}

void launch_node_counts(const uint64_t* keys, const uint32_t* sys_of, int64_t n, int leaf_max, int8_t* w,
                        int8_t* delta, int8_t* top, uint32_t* nstart, int32_t* depth, cudaStream_t s)
{
    if (leaf_max <= kTileWindow) {
        k_node_counts_tiled<<<nblk(n, kCountThreads), kCountThreads, 0, s>>>(keys, sys_of, n, leaf_max, delta, top,
                                                                            nstart, depth);
        count_launches(1);
        return;
    }
    k_window<<<nblk(n, 256), 256, 0, s>>>(keys, sys_of, n, leaf_max, w);
    k_node_counts<<<nblk(n, 256), 256, 0, s>>>(keys, sys_of, w, n, leaf_max, delta, top, nstart, depth);
    count_launches(2);
}

void launch_check_capacity(const uint32_t* m_total, Info* info, cudaStream_t s)
{
    k_check_capacity<<<1, 1, 0, s>>>(m_total, info);
    count_launches(1);
}

void launch_emit_preorder(const int8_t* delta, const uint32_t* nstart, const uint32_t* prepos, int64_t n,
                          const Info* info, uint32_t* pre_level, uint32_t* pre_first, uint32_t* iota, cudaStream_t s)
{
    k_emit_preorder<<<nblk(n, 256), 256, 0, s>>>(delta, nstart, prepos, n, info, pre_level, pre_first, iota);
    count_launches(1);
}

void launch_inverse_perm(const uint32_t* perm, int64_t cap_m, const Info* info, uint32_t* inv, cudaStream_t s)
{
    k_inverse_perm<<<gsgrid(cap_m, 256), 256, 0, s>>>(perm, info, inv);
    count_launches(1);
}

void launch_node_finalize(const uint64_t* keys, const int8_t* top, const uint32_t* sys_of, const SysParams* sysp,
                          int64_t n, const uint32_t* bfs_level, const uint32_t* bfs_pre, const uint32_t* pre_first,
                          const uint32_t* bfs_of_pre, int64_t cap_m, const Info* info, NodeTables nt, cudaStream_t s)
{
    (void)n;
    k_node_finalize<<<gsgrid(cap_m, 128), 128, 0, s>>>(keys, top, sys_of, sysp, bfs_level, bfs_pre, pre_first,
                                                       bfs_of_pre, info, nt);
    count_launches(1);
}

void launch_moments(const float4* body, int64_t cap_m, int depth, int depth_hint, const uint32_t* level_start,
                    const uint32_t* sys_of, const SysParams* sysp, const Info* info, NodeTables nt, bool quad,
                    cudaStream_t s)
{
    (void)sys_of;
    const unsigned g = gsgrid(cap_m, 128);
    if (quad) k_leaf_moments<true><<<g, 128, 0, s>>>(body, sysp, info, nt);
    else k_leaf_moments<false><<<g, 128, 0, s>>>(body, sysp, info, nt);
    count_launches(1);
    // the level launches take a small grid (4 blocks per SM): most levels
    // hold few internal cells, the launches past the tree's depth none, and a
    // large grid costs more to start than they work
    const unsigned glim = 4u * (unsigned)sm_count();
    const unsigned gl = g < glim ? g : glim;
    int top = depth < 0 ? kMaxLevel : depth;
    if (depth < 0 && depth_hint >= 0 && depth_hint + 3 < kMaxLevel) {
        // depth unknown on the host (a captured step): the levels from the
        // expected depth + 3 down get a launch each, any deeper ones one block
        top = depth_hint + 3;
        if (quad) k_level_moments_deep<true><<<1, 256, 0, s>>>(top, level_start, sysp, info, nt);
        else k_level_moments_deep<false><<<1, 256, 0, s>>>(top, level_start, sysp, info, nt);
        count_launches(1);
    }
    for (int lev = top - 1; lev >= 0; lev--) {
        if (quad) k_level_moments<true><<<gl, 128, 0, s>>>(lev, level_start, sysp, info, nt);
        else k_level_moments<false><<<gl, 128, 0, s>>>(lev, level_start, sysp, info, nt);
        count_launches(1);
    }
}

size_t group_split_scratch() { return (size_t)3 * kSplitBlocks; }

void launch_group_split(const int32_t* gfirst, const Info* info, int64_t cap_g, int32_t* lists, int32_t* counts,
                        int32_t* scratch, cudaStream_t s)
{
    k_split_count<<<kSplitBlocks, kSplitThreads, 0, s>>>(gfirst, info, scratch);
    k_split_scatter<<<kSplitBlocks, kSplitThreads, 0, s>>>(gfirst, info, scratch, cap_g, lists, counts);
    count_launches(2);
}

void launch_sys_mass(SysParams* sysp, int nsys, const NodeTables nt, const Info* info, cudaStream_t s)
{
    k_sys_mass<<<nblk(nsys, 128), 128, 0, s>>>(sysp, nsys, nt, info);
    count_launches(1);
}

void launch_group_marks(int64_t cap_m, const Info* info, const NodeTables nt, int gmax, int64_t n, uint32_t* gflag,
                        int32_t* gref_at, cudaStream_t s)
{
    cudaMemsetAsync(gflag, 0, n * sizeof(uint32_t), s);
    k_group_marks<<<gsgrid(cap_m, 128), 128, 0, s>>>(info, nt, gmax, gflag, gref_at);
    count_launches(1);
}

void launch_group_table(const uint32_t* gflag, const uint32_t* gscan, const int32_t* gref_at, int64_t n,
                        const uint32_t* total, int32_t* gfirst, int32_t* gref, Info* info, cudaStream_t s)
{
    k_group_table<<<nblk(n, 256), 256, 0, s>>>(gflag, gscan, gref_at, n, total, gfirst, gref, info);
    count_launches(1);
}

}  // namespace tc
