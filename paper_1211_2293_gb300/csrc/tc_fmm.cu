// tc_fmm.cu -- the fast multipole method on the treecode's tree (Sec. 5
// names it as the treecode's O(N) successor and gives no formulation; the
// reading built here is stated in full in include/tc.h beside tc_ctx_fmm).
//
// Every cell carries a monopole at its centre of mass (the build's FP64
// reduction) and gets a third-order local expansion about it: the field L0,
// its Jacobian L1 (symmetric, 6 numbers), its second and third derivatives
// L2 and L3 (symmetric, 10 and 15 numbers).  The dual traversal decides which ordered pairs of
// cells interact through expansions (M2L) and which pairs of leaves
// directly (P2P): from (root, root), a pair of a cell with itself splits into
// all pairs of its children; a pair of distinct cells is accepted when
// r_A + r_B < theta |c_A - c_B| (r_X: the cell's radius about its centre of
// mass), else summed directly when both are leaves, else the target B is
// split when it is internal and (A is a leaf or r_B >= r_A), else the source
// A.  Per target cell B that is a walk: B's candidate sources are its
// parent's unresolved sources and its parent's children (B itself among
// them); B refines every candidate wider than itself, applies M2L to the
// accepted ones, and keeps the rest for its own children.  So the traversal runs level by level, top down, one warp per
// cell, and no pair list is ever written: a cell's unresolved candidates go
// to a pool its children read in the next launch, and its local expansion is
// its parent's moved to its own centre (L2L) plus its own M2L terms.  A leaf
// walks its candidates to the end: accepted cells feed its expansion, leaves
// it meets send their bodies to a shared-memory tile (P2P), and its
// expansion is evaluated at its bodies (L2P).  A leaf holds fewer bodies
// than a warp has lanes, so its P2P splits the tile: lane t + c k (c the
// leaf's bodies) sums the tile's pairs k, k + S, k + 2S, ... for body t
// (S = 32 / c slices), with the compensated summation of the treecode's
// force loop, and the slices are added at the end.
//
// Radii are FP64 (a bottom-up pass per level, leaves from their bodies,
// cells from their children's spheres), rounded to FP32 for the test; the
// same pass gathers each cell's walk record (centre of mass, cube centre,
// radius, body and child ranges) into one 48-byte run, one gather per
// candidate.  The
// acceptance test runs in FP32 on cell-relative values (integer cube centres
// in units of h/2 plus the float offset of each centre of mass from its cube
// centre), as the treecode walk does.
#include "tc_walk.cuh"

namespace tc {

namespace {

constexpr int kFmmWarps = 4;
constexpr int kFmmStack = 2048;  // refinement stack per warp (shared memory)
constexpr int kFmmTile = 128;
constexpr int kFmmBlocksPerSm = 4;
constexpr int kLocW = 36;        // floats per local expansion: L0 3, L1 6, L2 10, L3 15, two spare

// Symmetric storage of the expansion's coefficients: a sorted index tuple
// is stored once, in lexicographic order -- L1 (00 01 02 11 12 22), L2
// (000 001 ... 222, 10 entries), L3 (0000 ... 2222, 15 entries).  The
// positions are pure arithmetic on the indices, so in the unrolled loops
// below every one folds to a constant (the coefficients stay in registers).
__host__ __device__ constexpr int mn(int a, int b) { return a < b ? a : b; }
__host__ __device__ constexpr int mx(int a, int b) { return a < b ? b : a; }
// sorted pair x <= y over the alphabet 0..n-1
__host__ __device__ constexpr int si2n(int x, int y, int n) { return x * n - x * (x - 1) / 2 + (y - x); }
// sorted triples over 0..n-1 whose first element is below x
__host__ __device__ constexpr int off3n(int x, int n)
{
    return x == 0 ? 0 : (x == 1 ? n * (n + 1) / 2 : n * (n + 1) / 2 + (n - 1) * n / 2);
}
__host__ __device__ constexpr int si3s(int a, int b, int c, int n) { return off3n(a, n) + si2n(b - a, c - a, n - a); }
__host__ __device__ constexpr int si2(int i, int j) { return si2n(mn(i, j), mx(i, j), 3); }
__host__ __device__ constexpr int si3(int i, int j, int k)
{
    return si3s(mn(mn(i, j), k), i + j + k - mn(mn(i, j), k) - mx(mx(i, j), k), mx(mx(i, j), k), 3);
}
__host__ __device__ constexpr int si4(int i, int j, int k, int l)
{
    // a four-element sorting network: the extremes, then the middle pair
    return (mn(mn(i, j), mn(k, l)) == 0 ? 0 : (mn(mn(i, j), mn(k, l)) == 1 ? 10 : 14)) +
           si3s(mn(mx(mn(i, j), mn(k, l)), mn(mx(i, j), mx(k, l))) - mn(mn(i, j), mn(k, l)),
                mx(mx(mn(i, j), mn(k, l)), mn(mx(i, j), mx(k, l))) - mn(mn(i, j), mn(k, l)),
                mx(mx(i, j), mx(k, l)) - mn(mn(i, j), mn(k, l)), 3 - mn(mn(i, j), mn(k, l)));
}
static_assert(si2(2, 1) == 4 && si3(2, 0, 1) == 4 && si3(2, 1, 1) == 7 && si4(0, 1, 1, 2) == 7 &&
                  si4(2, 1, 2, 1) == 12 && si4(2, 2, 1, 2) == 13 && si4(2, 2, 2, 2) == 14 && si4(1, 0, 0, 0) == 1,
              "symmetric storage positions");

__device__ __forceinline__ float ipow(float x, int n)  // n in [0, 4], a constant after unrolling
{
    return n == 0 ? 1.f : (n == 1 ? x : (n == 2 ? x * x : (n == 3 ? x * x * x : (x * x) * (x * x))));
}

// the monomials of an offset t over the sorted pairs and triples
__device__ __forceinline__ void monomials(const float (&t)[3], float (&t2)[6], float (&t3)[10])
{
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = i; j < 3; j++) t2[si2(i, j)] = t[i] * t[j];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = i; j < 3; j++)
#pragma unroll
            for (int k = j; k < 3; k++) t3[si3(i, j, k)] = t2[si2(i, j)] * t[k];
}

// The Taylor series of the field about a cell's centre to third order:
// a(c + t) = L0 + L1 t + (1/2) L2 t t + (1/6) L3 t t t (L1 the Jacobian,
// L2, L3 the second and third derivatives).
struct Loc {
    float l0[3];
    float l1[6];
    float l2[10];
    float l3[15];
    __device__ void zero()
    {
#pragma unroll
        for (int k = 0; k < 3; k++) l0[k] = 0.f;
#pragma unroll
        for (int k = 0; k < 6; k++) l1[k] = 0.f;
#pragma unroll
        for (int k = 0; k < 10; k++) l2[k] = 0.f;
#pragma unroll
        for (int k = 0; k < 15; k++) l3[k] = 0.f;
    }
    // M2L: the softened field of mass gm (G M) seen from d = c_A - c_B and
    // its first three derivatives with respect to the evaluation point:
    //   L0_i    += gm d_i / rho^3
    //   L1_ij   += gm (3 d_i d_j / rho^5 - delta_ij / rho^3)
    //   L2_ijk  += gm (15 d_i d_j d_k / rho^7 - 3 (delta_ij d_k + delta_ik d_j + delta_jk d_i) / rho^5)
    //   L3_ijkl += gm (105 d_i d_j d_k d_l / rho^9 - 15 (6 terms delta d d) / rho^7
    //                  + 3 (3 terms delta delta) / rho^5)
    // For an L3 entry with axis counts (a, b, c) the six delta d d terms sum
    // to C(a,2) x^(a-2) y^b z^c + C(b,2) ... + C(c,2) ..., the three delta
    // delta terms to 3 for (4, 0, 0) and its permutations, 1 for (2, 2, 0)
    // and its permutations, 0 otherwise.
    __device__ void add_monopole(float gm, float dx, float dy, float dz, float eps2)
    {
        const float r2 = fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, eps2)));
        const float ri = rsqrtf(r2);
        const float ri2 = ri * ri;
        const float g3 = gm * ri * ri2;
        const float g5 = g3 * ri2;
        const float g7 = g5 * ri2;
        const float g9 = g7 * ri2;
        l0[0] = fmaf(g3, dx, l0[0]);
        l0[1] = fmaf(g3, dy, l0[1]);
        l0[2] = fmaf(g3, dz, l0[2]);
        const float t5 = 3.f * g5;
        l1[0] += fmaf(t5 * dx, dx, -g3);
        l1[1] += t5 * dx * dy;
        l1[2] += t5 * dx * dz;
        l1[3] += fmaf(t5 * dy, dy, -g3);
        l1[4] += t5 * dy * dz;
        l1[5] += fmaf(t5 * dz, dz, -g3);
        const float f7 = 15.f * g7;
        const float ax = f7 * dx, ay = f7 * dy, az = f7 * dz;
        l2[0] += fmaf(ax * dx, dx, -3.f * t5 * dx);
        l2[1] += fmaf(ax * dx, dy, -t5 * dy);
        l2[2] += fmaf(ax * dx, dz, -t5 * dz);
        l2[3] += fmaf(ax * dy, dy, -t5 * dx);
        l2[4] += ax * dy * dz;
        l2[5] += fmaf(ax * dz, dz, -t5 * dx);
        l2[6] += fmaf(ay * dy, dy, -3.f * t5 * dy);
        l2[7] += fmaf(ay * dy, dz, -t5 * dz);
        l2[8] += fmaf(ay * dz, dz, -t5 * dy);
        l2[9] += fmaf(az * dz, dz, -3.f * t5 * dz);
        const float h9 = 105.f * g9, m7 = -15.f * g7;
        // the L3 entries in storage order: axis counts (ca, cb, cc), ca
        // falling, then cb falling
        int k = 0;
#pragma unroll
        for (int ca = 4; ca >= 0; ca--)
#pragma unroll
            for (int cb = 4 - ca; cb >= 0; cb--) {
                const int cc = 4 - ca - cb;
                const float P = ipow(dx, ca) * ipow(dy, cb) * ipow(dz, cc);
                float S6 = 0.f;
                if (ca >= 2) S6 += (float)(ca * (ca - 1) / 2) * ipow(dx, ca - 2) * ipow(dy, cb) * ipow(dz, cc);
                if (cb >= 2) S6 += (float)(cb * (cb - 1) / 2) * ipow(dx, ca) * ipow(dy, cb - 2) * ipow(dz, cc);
                if (cc >= 2) S6 += (float)(cc * (cc - 1) / 2) * ipow(dx, ca) * ipow(dy, cb) * ipow(dz, cc - 2);
                const int S3 = (ca == 4 || cb == 4 || cc == 4) ? 3
                               : ((ca == 2 && cb == 2) || (ca == 2 && cc == 2) || (cb == 2 && cc == 2)) ? 1 : 0;
                l3[k] += fmaf(h9, P, fmaf(m7, S6, (float)(3 * S3) * g5));
                k++;
            }
    }
    // the field of the series at offset t from its centre (L2P, and the L0
    // part of L2L): L0 + L1 t + (1/2) L2 t t + (1/6) L3 t t t, each sum over
    // the sorted index tuples with their multiplicities
    __device__ void eval(const float (&t)[3], const float (&t2)[6], const float (&t3)[10], float (&o)[3]) const
    {
        eval_series(l0, l1, l2, l3, t, t2, t3, o);
    }
    // the same for any storage of the 34 coefficients (registers, or the
    // parent's record read in place)
    template <typename A0, typename A1, typename A2, typename A3>
    __device__ static void eval_series(const A0& l0, const A1& l1, const A2& l2, const A3& l3, const float (&t)[3],
                                       const float (&t2)[6], const float (&t3)[10], float (&o)[3])
    {
#pragma unroll
        for (int i = 0; i < 3; i++) {
            float s = l0[i];
#pragma unroll
            for (int j = 0; j < 3; j++) s = fmaf(l1[si2(i, j)], t[j], s);
            float s2 = 0.f;
#pragma unroll
            for (int j = 0; j < 3; j++)
#pragma unroll
                for (int k = j; k < 3; k++) s2 = fmaf((float)(j == k ? 1 : 2) * l2[si3(i, j, k)], t2[si2(j, k)], s2);
            float s3 = 0.f;
#pragma unroll
            for (int j = 0; j < 3; j++)
#pragma unroll
                for (int k = j; k < 3; k++)
#pragma unroll
                    for (int m = k; m < 3; m++) {
                        const int mult = (j == k && k == m) ? 1 : ((j == k || k == m) ? 3 : 6);
                        s3 = fmaf((float)mult * l3[si4(i, j, k, m)], t3[si3(j, k, m)], s3);
                    }
            o[i] = s + 0.5f * s2 + (1.f / 6.f) * s3;
        }
    }
    // this += parent's series moved to offset t (L2L):
    //   L0 += L0p + L1p t + (1/2) L2p t t + (1/6) L3p t t t
    //   L1 += L1p + L2p t + (1/2) L3p t t,  L2 += L2p + L3p t,  L3 += L3p
    // (the parent's record q: L0 at q[0..3), L1 at q[3..9), L2 at q[9..19),
    // L3 at q[19..34), read where it is)
    __device__ void add_shifted(const float* __restrict__ q, const float (&t)[3])
    {
        struct P {
            const float* b;
            __device__ float operator[](int k) const { return __ldg(b + k); }
        };
        const P p0{q}, p1{q + 3}, p2{q + 9}, p3{q + 19};
        struct {
            P l1, l2, l3;
        } p{p1, p2, p3};
        float t2[6], t3[10];
        monomials(t, t2, t3);
        float s[3];
        eval_series(p0, p.l1, p.l2, p.l3, t, t2, t3, s);
#pragma unroll
        for (int i = 0; i < 3; i++) l0[i] += s[i];
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = i; j < 3; j++) {
                float u = p.l1[si2(i, j)];
#pragma unroll
                for (int m = 0; m < 3; m++) u = fmaf(p.l2[si3(i, j, m)], t[m], u);
                float w = 0.f;
#pragma unroll
                for (int m = 0; m < 3; m++)
#pragma unroll
                    for (int n = m; n < 3; n++) w = fmaf((float)(m == n ? 1 : 2) * p.l3[si4(i, j, m, n)], t2[si2(m, n)], w);
                l1[si2(i, j)] += fmaf(0.5f, w, u);
            }
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = i; j < 3; j++)
#pragma unroll
                for (int m = j; m < 3; m++) {
                    float u = p.l2[si3(i, j, m)];
#pragma unroll
                    for (int n = 0; n < 3; n++) u = fmaf(p.l3[si4(i, j, m, n)], t[n], u);
                    l2[si3(i, j, m)] += u;
                }
#pragma unroll
        for (int k = 0; k < 15; k++) l3[k] += p.l3[k];
    }
};

struct FmmArgs {
    const float4* body;      // Morton order, absolute positions, mass
    const uint32_t* perm;    // Morton position -> original index
    const SysParams* sysp;
    NodeTables nt;
    const int32_t* parent;
    const Info* info;
    int32_t* err;
    float* loc;              // cap_m x kLocW
    const int32_t* near_in;  // the previous level's unresolved candidates
    int32_t* near_out;       // this level's
    unsigned long long* ctr; // [0, 1] pool fill per level parity, [2] pool need, [3] slab need, [4..7] statistics
    int par;                 // this level's parity
    int64_t pool_cap;
    int32_t* slab;           // one list of slab_cap entries per resident warp
    int64_t slab_cap;
    int64_t* near_off;       // per node: its list in the pool
    int32_t* near_cnt;
    float* acc;              // n x 3, original order
    unsigned long long* rec; // per node: M2L pairs, P2P pairs, their hashes (target = the node)
    const int4* fnode;       // per node, 3 entries: {com offset, mass}, {cube centre, r_X (FP32 bits)}, b
    int records;             // keep the pair-set hashes and the per-node records
    float theta2, eps2, G;
};

// P2P of one lane: body (X, Y, Z) against the pairs k, k + S, ... of a
// pair-interleaved tile, compensated across flushes
struct P2PSum {
    float sx, sy, sz, cx, cy, cz;
    __device__ void init() { sx = sy = sz = cx = cy = cz = 0.f; }
    __device__ void flush(float* tile, int n, f2 X, f2 Y, f2 Z, f2 E2, int k, int S)
    {
        if (n <= 0) return;
        if ((n & 1) && (threadIdx.x & 31) == 0) put_entry(tile, n, make_float4(0.f, 0.f, 0.f, 0.f));
        __syncwarp();
        const int np = (n + 1) >> 1;
        const ulonglong2* t2 = reinterpret_cast<const ulonglong2*>(tile);
        f2 ax = 0ull, ay = 0ull, az = 0ull;
#pragma unroll 4
        for (int p = k; p < np; p += S) {
            const ulonglong2 xy = t2[2 * p];
            const ulonglong2 zm = t2[2 * p + 1];
            const f2 dx = f2sub(xy.x, X);
            const f2 dy = f2sub(xy.y, Y);
            const f2 dz = f2sub(zm.x, Z);
            const f2 r2 = f2fma(dz, dz, f2fma(dy, dy, f2fma(dx, dx, E2)));
            float r2a, r2b;
            f2unpack(r2, r2a, r2b);
            const f2 ri = f2pack(rsqrt_sfu(r2a), rsqrt_sfu(r2b));
            const f2 mri3 = f2mul(f2mul(zm.y, ri), f2mul(ri, ri));
            ax = f2fma(dx, mri3, ax);
            ay = f2fma(dy, mri3, ay);
            az = f2fma(dz, mri3, az);
        }
        two_sum_acc(sx, cx, f2sum(ax));
        two_sum_acc(sy, cy, f2sum(ay));
        two_sum_acc(sz, cz, f2sum(az));
        __syncwarp();
    }
};

// r_X for the cells [start, end) of one level (FP64): a leaf's farthest
// body from its centre of mass, above, the farthest child sphere
__global__ void k_fmm_radius(const float4* __restrict__ body, NodeTables nt, double* __restrict__ rad,
                             int4* __restrict__ fnode, int64_t start, int64_t end)
{
    for (int64_t v = start + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < end;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int4 b = nt.b[v];
        const double c0 = nt.com64[3 * v], c1 = nt.com64[3 * v + 1], c2 = nt.com64[3 * v + 2];
        double r2max = 0.0, r = 0.0;
        const int nch = b.w >> 8;
        if (nch == 0) {
            for (int i = b.x; i < b.x + b.y; i++) {
                const float4 q = body[i];
                const double e0 = (double)q.x - c0, e1 = (double)q.y - c1, e2 = (double)q.z - c2;
                r2max = fmax(r2max, e0 * e0 + e1 * e1 + e2 * e2);
            }
            r = sqrt(r2max);
        } else {
            for (int k = b.z; k < b.z + nch; k++) {
                const double e0 = nt.com64[3 * k] - c0, e1 = nt.com64[3 * k + 1] - c1, e2 = nt.com64[3 * k + 2] - c2;
                r = fmax(r, sqrt(e0 * e0 + e1 * e1 + e2 * e2) + rad[k]);
            }
        }
        rad[v] = r;
        // the walk's record of the cell, gathered into one place
        const float4 na = nt.a[v];
        const int4 nc = nt.c[v];
        fnode[3 * v] = make_int4(__float_as_int(na.x), __float_as_int(na.y), __float_as_int(na.z), __float_as_int(na.w));
        fnode[3 * v + 1] = make_int4(nc.x, nc.y, nc.z, __float_as_int((float)r));
        fnode[3 * v + 2] = b;
    }
}

__global__ void k_fmm_level_starts(const Info* info, NodeTables nt, int64_t* __restrict__ lstart)
{
    const int64_t M = info->M;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < M; v += (int64_t)gridDim.x * blockDim.x) {
        const int lv = nt.b[v].w & 255;
        const int lp = v > 0 ? (nt.b[v - 1].w & 255) : -1;
        for (int l = lp + 1; l <= lv; l++) lstart[l] = v;
        if (v == M - 1)
            for (int l = lv + 1; l < kFmmLevelSlots; l++) lstart[l] = M;
    }
}

__global__ void k_fmm_parent(const Info* info, NodeTables nt, int32_t* __restrict__ parent)
{
    const int64_t M = info->M;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < M; v += (int64_t)gridDim.x * blockDim.x) {
        const int4 b = nt.b[v];
        if ((b.w & 255) == 0) parent[v] = -1;  // a system's root
        const int nch = b.w >> 8;
        for (int k = 0; k < nch; k++) parent[b.z + k] = (int32_t)v;
    }
}

// one warp per cell of [start, end): the target walk described above
__global__ void __launch_bounds__(kFmmWarps * 32, kFmmBlocksPerSm) k_fmm_level(FmmArgs a, int64_t start, int64_t end)
{
    __shared__ uint32_t stk_s[kFmmWarps][kFmmStack];
    __shared__ __align__(16) float tile_s[kFmmWarps][4 * tile_cap(kFmmTile)];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t* stk = stk_s[w];
    float* btile = tile_s[w];
    int32_t* slab = a.slab + ((int64_t)blockIdx.x * kFmmWarps + w) * a.slab_cap;
    const uint32_t lt = (1u << lane) - 1u;
    if ((*(volatile const int32_t*)&a.info->err & kErrCapacity) != 0) return;  // no tree
    const NodeTables nt = a.nt;
    const f2 E2 = f2pack(a.eps2, a.eps2);
    unsigned long long t_m2l = 0, t_p2p = 0, th_m2l = 0, th_p2p = 0;  // the warp's totals (lane 0)
    for (int64_t B = start + (int64_t)blockIdx.x * kFmmWarps + w; B < end; B += (int64_t)gridDim.x * kFmmWarps) {
        const int4 bb = nt.b[B];
        const float4 ba = nt.a[B];
        const int4 bc = nt.c[B];
        const SysParams& SP = a.sysp[bc.w];
        const float uf = SP.uf;
        const bool leafB = (bb.w >> 8) == 0;
        const float rB = __int_as_float(a.fnode[3 * B + 1].w);
        const int P = a.parent[B];
        // candidates: the parent's unresolved sources, then its children; a
        // root has none, or itself when it is a leaf
        int np = 0, nch = 0, pz = 0;
        int64_t poff = 0;
        if (P >= 0) {
            np = a.near_cnt[P];
            poff = a.near_off[P];
            const int4 pb = nt.b[P];
            nch = pb.w >> 8;
            pz = pb.z;
        } else if (leafB) {
            nch = 1;
            pz = (int)B;
        }
        const int ntot = np + nch;
        // a leaf's bodies, 32 per round (one per lane)
        const int rounds = leafB ? max(1, (bb.y + 31) >> 5) : 1;
        for (int r = 0; r < rounds; r++) {
            // lane = t + c k: body t of this round, tile slice k of S
            const int c = leafB ? min(32, bb.y - 32 * r) : 32;
            const int S = 32 / c;
            const int t = lane % c, ks = lane / c;
            const bool slice = leafB && ks < S;
            const int ib = 32 * r + t;
            float4 me = make_float4(0.f, 0.f, 0.f, 0.f);
            if (slice) me = a.body[bb.x + ib];
            const f2 XA = f2pack(me.x, me.x), YA = f2pack(me.y, me.y), ZA = f2pack(me.z, me.z);
            P2PSum fsum;
            fsum.init();
            const int k0 = slice ? ks : (1 << 30);  // lanes past the slices sum nothing
            Loc L;
            L.zero();
            int sp = 0, ip = 0, bn = 0;
            int64_t nn = 0;
            bool bad = false;
            unsigned long long n_m2l = 0, n_p2p = 0, h_m2l = 0, h_p2p = 0;  // this cell's pairs (per lane)
            while (true) {
                int A = -1;
                if (sp > 0) {
                    const int take = min(sp, 32);
                    if (lane < take) A = (int)stk[sp - take + lane];
                    sp -= take;
                } else if (ip < ntot) {
                    const int k = ip + lane;
                    if (k < ntot) A = k < np ? a.near_in[poff + k] : pz + (k - np);
                    ip += 32;
                } else {
                    break;
                }
                __syncwarp();
                bool m2l = false, p2p = false, keep = false, split = false;
                int4 ab = make_int4(0, 0, 0, 0);
                if (A >= 0) {
                    // the candidate's record: one 48-byte run
                    const int4* fr = a.fnode + 3 * (int64_t)A;
                    const int4 a0 = __ldg(fr), ac = __ldg(fr + 1);
                    ab = __ldg(fr + 2);
                    const bool leafA = (ab.w >> 8) == 0;
                    if (A == (int)B) {
                        p2p = leafB;  // an internal cell's self pair is its children's pairs
                    } else {
                        const float4 aa = make_float4(__int_as_float(a0.x), __int_as_float(a0.y), __int_as_float(a0.z),
                                                      __int_as_float(a0.w));
                        const float dx = fmaf((float)(ac.x - bc.x), uf, aa.x - ba.x);
                        const float dy = fmaf((float)(ac.y - bc.y), uf, aa.y - ba.y);
                        const float dz = fmaf((float)(ac.z - bc.z), uf, aa.z - ba.z);
                        const float rA = __int_as_float(ac.w);
                        const float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                        const float rr = rA + rB;
                        if (rr * rr < a.theta2 * d2) {
                            m2l = true;
                            L.add_monopole(a.G * aa.w, dx, dy, dz, a.eps2);
                        } else if (leafA && leafB) {
                            p2p = true;
                        } else if (!leafB && (leafA || rB >= rA)) {
                            keep = true;
                        } else {
                            split = true;
                        }
                    }
                    if (r == 0 && (m2l || p2p)) {
                        const unsigned long long hh =
                            a.records ? mix64(((unsigned long long)(unsigned)A << 32) ^ (unsigned long long)B) : 0ull;
                        if (m2l) {
                            n_m2l++;
                            h_m2l += hh;
                        } else {
                            n_p2p++;
                            h_p2p += hh;
                        }
                    }
                }
                // refined sources push their children
                const int npush = split ? (ab.w >> 8) : 0;
                int tot;
                const int excl = warp_excl_small(npush, lt, tot);
                if (sp + tot > kFmmStack) {
                    bad = true;
                    break;
                }
                for (int k = 0; k < npush; k++) stk[sp + excl + k] = (uint32_t)(ab.z + k);
                sp += tot;
                // unresolved sources go to the warp's slab (counted past its end)
                const unsigned km = __ballot_sync(0xffffffffu, keep);
                if (keep) {
                    const int64_t at = nn + __popc(km & lt);
                    if (at < a.slab_cap) slab[at] = A;
                }
                nn += __popc(km);
                // leaves met: their bodies to the tile, 32 at a time
                if (__any_sync(0xffffffffu, p2p)) {
                    const int cnt = p2p ? ab.y : 0;
                    const int incl_c = warp_incl_scan_i(cnt);
                    const int excl_c = incl_c - cnt;
                    const int T = __shfl_sync(0xffffffffu, incl_c, 31);
                    for (int o = 0; o < T; o += 32) {
                        const int t = min(o + lane, T - 1);
                        int pos = 0;
#pragma unroll
                        for (int step = 16; step; step >>= 1) {
                            const int e = __shfl_sync(0xffffffffu, excl_c, pos + step);
                            if (e <= t) pos += step;
                        }
                        const int f = __shfl_sync(0xffffffffu, ab.x, pos);
                        const int e0 = __shfl_sync(0xffffffffu, excl_c, pos);
                        if (o + lane < T) put_entry(btile, bn + lane, __ldg(&a.body[f + (t - e0)]));
                        bn += min(32, T - o);
                        if (bn >= kFmmTile) {
                            fsum.flush(btile, bn, XA, YA, ZA, E2, k0, S);
                            bn = 0;
                        }
                    }
                }
                __syncwarp();
            }
            if (bad) {
                if (lane == 0) {
                    atomicOr(a.err, kErrFmmStack);
                    if (!leafB) {
                        a.near_off[B] = 0;
                        a.near_cnt[B] = 0;
                    }
                }
                __syncwarp();
                break;
            }
            fsum.flush(btile, bn, XA, YA, ZA, E2, k0, S);
            // the slices' sums, added by the lanes of slice 0 (through the tile)
            float fx = 0.f, fy = 0.f, fz = 0.f;
            if (leafB) {
                btile[3 * lane + 0] = fsum.sx + fsum.cx;
                btile[3 * lane + 1] = fsum.sy + fsum.cy;
                btile[3 * lane + 2] = fsum.sz + fsum.cz;
                __syncwarp();
                if (ks == 0)
                    for (int k = 0; k < S; k++) {
                        fx += btile[3 * (t + c * k) + 0];
                        fy += btile[3 * (t + c * k) + 1];
                        fz += btile[3 * (t + c * k) + 2];
                    }
                __syncwarp();
            }
            if (r == 0) {
                // this cell's pair records
#pragma unroll
                for (int o = 16; o; o >>= 1) {
                    n_m2l += __shfl_xor_sync(0xffffffffu, n_m2l, o);
                    n_p2p += __shfl_xor_sync(0xffffffffu, n_p2p, o);
                    h_m2l += __shfl_xor_sync(0xffffffffu, h_m2l, o);
                    h_p2p += __shfl_xor_sync(0xffffffffu, h_p2p, o);
                }
                if (lane == 0) {
                    if (a.records) {
                        ulonglong4_32a* rec = reinterpret_cast<ulonglong4_32a*>(a.rec) + B;
                        *rec = make_ulonglong4_32a(n_m2l, n_p2p, h_m2l, h_p2p);
                    }
                    t_m2l += n_m2l;
                    t_p2p += n_p2p;
                    th_m2l += h_m2l;
                    th_p2p += h_p2p;
                }
            }
            // this cell's own M2L terms, summed over the lanes
#pragma unroll
            for (int k = 0; k < 3; k++)
#pragma unroll
                for (int o = 16; o; o >>= 1) L.l0[k] += __shfl_xor_sync(0xffffffffu, L.l0[k], o);
#pragma unroll
            for (int k = 0; k < 6; k++)
#pragma unroll
                for (int o = 16; o; o >>= 1) L.l1[k] += __shfl_xor_sync(0xffffffffu, L.l1[k], o);
#pragma unroll
            for (int k = 0; k < 10; k++)
#pragma unroll
                for (int o = 16; o; o >>= 1) L.l2[k] += __shfl_xor_sync(0xffffffffu, L.l2[k], o);
#pragma unroll
            for (int k = 0; k < 15; k++)
#pragma unroll
                for (int o = 16; o; o >>= 1) L.l3[k] += __shfl_xor_sync(0xffffffffu, L.l3[k], o);
            // plus the parent's expansion moved to this centre (L2L)
            if (P >= 0) {
                const float* q = a.loc + (int64_t)P * kLocW;
                const float4 pa = nt.a[P];
                const int4 pc = nt.c[P];
                const float t[3] = {fmaf((float)(bc.x - pc.x), uf, ba.x - pa.x), fmaf((float)(bc.y - pc.y), uf, ba.y - pa.y),
                                    fmaf((float)(bc.z - pc.z), uf, ba.z - pa.z)};
                L.add_shifted(q, t);
            }
            if (r == 0 && lane == 0) {
                float* o = a.loc + B * kLocW;
#pragma unroll
                for (int k = 0; k < 3; k++) o[k] = L.l0[k];
#pragma unroll
                for (int k = 0; k < 6; k++) o[3 + k] = L.l1[k];
#pragma unroll
                for (int k = 0; k < 10; k++) o[9 + k] = L.l2[k];
#pragma unroll
                for (int k = 0; k < 15; k++) o[19 + k] = L.l3[k];
            }
            if (!leafB) {
                // the unresolved candidates, from the slab to the pool
                long long off = -1;
                if (lane == 0) {
                    if (nn > a.slab_cap) {
                        atomicMax(&a.ctr[3], (unsigned long long)nn);
                        atomicOr(a.err, kErrFmmSlab);
                    } else {
                        const unsigned long long o = atomicAdd(&a.ctr[a.par], (unsigned long long)nn);
                        if ((int64_t)(o + nn) > a.pool_cap) {
                            atomicMax(&a.ctr[2], o + nn);
                            atomicOr(a.err, kErrFmmPool);
                        } else {
                            off = (long long)o;
                        }
                    }
                    a.near_off[B] = off < 0 ? 0 : off;
                    a.near_cnt[B] = off < 0 ? 0 : (int32_t)nn;
                }
                off = __shfl_sync(0xffffffffu, off, 0);
                __syncwarp();
                if (off >= 0)
                    for (int64_t k = lane; k < nn; k += 32) a.near_out[off + k] = slab[k];
            } else if (ks == 0) {
                // L2P at the lane's body, offset from the leaf's centre of mass
                const double cx = SP.c0[0] + (double)bc.x * 0.5 * SP.h, cy = SP.c0[1] + (double)bc.y * 0.5 * SP.h,
                             cz = SP.c0[2] + (double)bc.z * 0.5 * SP.h;
                const float ox = (float)((double)me.x - cx) - ba.x;
                const float oy = (float)((double)me.y - cy) - ba.y;
                const float oz = (float)((double)me.z - cz) - ba.z;
                const float ot[3] = {ox, oy, oz};
                float ot2[6], ot3[10], lo[3];
                monomials(ot, ot2, ot3);
                L.eval(ot, ot2, ot3, lo);
                const float lx = lo[0], ly = lo[1], lz = lo[2];
                const int64_t o = a.perm[bb.x + ib];
                a.acc[3 * o + 0] = fmaf(a.G, fx, lx);
                a.acc[3 * o + 1] = fmaf(a.G, fy, ly);
                a.acc[3 * o + 2] = fmaf(a.G, fz, lz);
            }
            __syncwarp();
        }
    }
    if (lane == 0 && (t_m2l | t_p2p)) {
        atomicAdd(&a.ctr[4], t_m2l);
        atomicAdd(&a.ctr[5], t_p2p);
        atomicAdd(&a.ctr[6], th_m2l);
        atomicAdd(&a.ctr[7], th_p2p);
    }
}

int fmm_grid_max() { return kFmmBlocksPerSm * sm_count(); }

}  // namespace

int64_t fmm_slab_warps() { return (int64_t)fmm_grid_max() * kFmmWarps; }
int fmm_loc_width() { return kLocW; }

void launch_fmm_level_starts(const Info* info, int64_t cap_m, NodeTables nt, int64_t* lstart, cudaStream_t s)
{
    int64_t g = (cap_m + 255) / 256;
    if (g > 8 * sm_count()) g = 8 * sm_count();
    k_fmm_level_starts<<<(unsigned)(g < 1 ? 1 : g), 256, 0, s>>>(info, nt, lstart);
    count_launches(1);
}

cudaError_t launch_fmm(const FmmLaunch& p, const int64_t* lstart_h, int depth, cudaStream_t s)
{
    int64_t g = (p.cap_m + 255) / 256;
    if (g > 8 * sm_count()) g = 8 * sm_count();
    k_fmm_parent<<<(unsigned)(g < 1 ? 1 : g), 256, 0, s>>>(p.info, p.nt, p.parent);
    count_launches(1);
    for (int l = depth; l >= 0; l--) {
        const int64_t start = lstart_h[l], end = lstart_h[l + 1];
        if (end <= start) continue;
        int64_t gb = (end - start + 127) / 128;
        if (gb > 8 * sm_count()) gb = 8 * sm_count();
        k_fmm_radius<<<(unsigned)gb, 128, 0, s>>>(p.body, p.nt, p.rad, p.fnode, start, end);
        count_launches(1);
    }
    FmmArgs a;
    a.body = p.body;
    a.perm = p.perm;
    a.sysp = p.sysp;
    a.nt = p.nt;
    a.parent = p.parent;
    a.info = p.info;
    a.err = p.err;
    a.loc = p.loc;
    a.ctr = p.ctr;
    a.pool_cap = p.pool_cap;
    a.slab = p.slab;
    a.slab_cap = p.slab_cap;
    a.near_off = p.near_off;
    a.near_cnt = p.near_cnt;
    a.acc = p.acc;
    a.rec = p.rec;
    a.fnode = p.fnode;
    a.records = p.records;
    a.theta2 = p.theta * p.theta;
    a.eps2 = p.eps * p.eps;
    a.G = p.G;
    const int gmax = fmm_grid_max();
    for (int l = 0; l <= depth; l++) {
        const int64_t start = lstart_h[l], end = lstart_h[l + 1];
        if (end <= start) continue;
        a.par = l & 1;
        a.near_in = p.pool[(l + 1) & 1];
        a.near_out = p.pool[l & 1];
        cudaError_t e = cudaMemsetAsync(&p.ctr[l & 1], 0, sizeof(unsigned long long), s);
        if (e != cudaSuccess) return e;
        int64_t blocks = (end - start + kFmmWarps - 1) / kFmmWarps;
        if (blocks > gmax) blocks = gmax;
        k_fmm_level<<<(unsigned)blocks, kFmmWarps * 32, 0, s>>>(a, start, end);
        count_launches(1);
    }
    return cudaGetLastError();
}

}  // namespace tc
