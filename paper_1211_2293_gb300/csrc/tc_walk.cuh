// tc_walk.cuh -- the force phase: tree walk with the cell-opening test,
// interaction lists staged in shared memory, softened monopole (optionally
// quadrupole) force loop.  The kernel templates live here; tc_walk_unit.cu
// instantiates them for one (bodies per lane, tile) pair per object (the
// build compiles it nine times, in parallel), tc_walk.cu holds the
// launchers.
//
// Paper, Sec. 3.1: the force on a body is evaluated by traversing the tree
// from the root; a cell distant enough joins the interaction list, otherwise
// the traversal continues with its children; the accumulated list of cells
// and bodies is then looped through with F = G m_a m_b / r^2.  Sec. 3.2: the
// summation for each body over its list is independent of every other body.
//
// GPU design.  One warp walks the tree once for a whole group of up to
// 32*B Morton-consecutive bodies (B bodies per lane) -- the list is built for
// the group, so every body of the group uses the same list.  The walk is a
// LIFO of node indices in shared memory; each step pops up to 32 nodes, one
// per lane, and applies the opening test in parallel:
//   * a node holding a body of the group is opened;
//   * otherwise, with s its cube side and d the distance from its centre of
//     mass to the group's bounding box, it is accepted iff s < theta * d
//     (compared as s^2 < theta^2 d^2);
//   * an opened internal node pushes its (contiguous) children, an opened
//     leaf sends its bodies to the body tile, an accepted node sends its
//     (centre of mass, mass) to the cell tile.
// Ballots and prefix sums compact the three outcomes.  When a tile reaches
// kTile entries every lane sums it for its B bodies (the force loop: one
// rsqrt and 12 FP32 FMA-pipe instructions per interaction) and the tile is
// reused, so lists never go to HBM.
//
// Precision.  The opening test and the cell sources are evaluated in a frame
// centred on the group's reference cube: cube centres are exact integers in
// units u = h/2, the group box is split into an integer part (units of u)
// and a float remainder, so every difference is formed without cancellation
// and the test's relative error stays ~1e-7.  Body-body terms use absolute
// float positions (their differences are exact or correctly rounded).  In
// the precise mode cell terms use the cell-relative frame and each tile's
// partial sum enters the per-body total through an error-free TwoSum
// (compensated accumulation); the plain mode uses absolute float centres of
// mass and plain accumulation.
#pragma once
#include "tc_internal.cuh"
#include "tc_mma.cuh"

namespace tc {

namespace {

// list tiles: a step adds at most 32 entries before the flush check, and a
// flush may pad one entry, so a tile of TILE entries needs TILE + 34 slots
__host__ __device__ constexpr int tile_cap(int tile) { return tile + 34; }

// ---------------------------------------------------------------- packed FP32
// Blackwell's paired FP32 instructions (add/sub/mul/fma .f32x2) work on a
// 64-bit register holding two floats.  A list tile is stored pair-interleaved
// -- {x_j, x_j+1}, {y_j, y_j+1}, {z_j, z_j+1}, {m_j, m_j+1} per pair of
// entries -- so one pair of 16-byte shared loads yields two sources already
// packed, and every FP32 operation of the force loop serves two sources.
typedef unsigned long long f2;

__device__ __forceinline__ f2 f2pack(float a, float b)
{
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void f2unpack(f2 r, float& a, float& b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ f2 f2sub(f2 a, f2 b)
{
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 f2mul(f2 a, f2 b)
{
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 f2fma(f2 a, f2 b, f2 c)
{
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ float f2sum(f2 a)
{
    float x, y;
    f2unpack(a, x, y);
    return x + y;
}

// entry k of a pair-interleaved tile
__device__ __forceinline__ void put_entry(float* tile, int k, float4 q)
{
    float* t = tile + 8 * (k >> 1) + (k & 1);
    t[0] = q.x;
    t[2] = q.y;
    t[4] = q.z;
    t[6] = q.w;
}

// entry k from global memory by cp.async: four 4-byte copies into the
// pair-interleaved tile, global -> shared without passing through
// registers; the copier waits for its copies (cp_async_wait_all, or an
// mbarrier that tracks them) before the tile is read
__device__ __forceinline__ void cp_async4(void* dst, const void* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}

__device__ __forceinline__ void put_entry_async(float* tile, int k, const float4* src)
{
    float* t = tile + 8 * (k >> 1) + (k & 1);
    const float* q = reinterpret_cast<const float*>(src);
    cp_async4(t, q);
    cp_async4(t + 2, q + 1);
    cp_async4(t + 4, q + 2);
    cp_async4(t + 6, q + 3);
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ unsigned long long mix64(unsigned long long z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ int warp_incl_scan_i(int x)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// exclusive warp prefix sum of x in [0, 15] (and the warp total) from four
// ballots: no shuffle chain
__device__ __forceinline__ int warp_excl_small(int x, unsigned lt, int& total)
{
    int e = 0, t = 0;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const unsigned bk = __ballot_sync(0xffffffffu, (x >> k) & 1);
        e += __popc(bk & lt) << k;
        t += __popc(bk) << k;
    }
    total = t;
    return e;
}

// Lf x 2^-level for a power-of-two Lf: exponent arithmetic when the result
// stays a normal float (fast, decided once per group), scalbnf otherwise
__device__ __forceinline__ float pow2_down(float Lf, int level, bool fast)
{
    return fast ? __int_as_float(__float_as_int(Lf) - (level << 23)) : scalbnf(Lf, -level);
}

// error-free sum: s + c absorbs x (Knuth's TwoSum)
__device__ __forceinline__ void two_sum_acc(float& s, float& c, float x)
{
    float t = __fadd_rn(s, x);
    float z = __fsub_rn(t, s);
    float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(x, z));
    s = t;
    c = __fadd_rn(c, e);
}

// 1/sqrt(x) on the SFU, flushing subnormals (x >= eps^2 > 0 is normal here),
// so no range fix-up surrounds the approximation
__device__ __forceinline__ float rsqrt_sfu(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// The force loop: npairs pairs of sources against the lane's B bodies.
// Body coordinates are held duplicated ({x, x}); the two halves of each
// accumulator collect the even and the odd sources of the tile.
//   r2 = |d|^2 + eps^2, ri = rsqrt(r2), a += d * m * ri^3, pot -= m * ri
template <int B, bool POT, int UNROLL>
__device__ __forceinline__ void sum_tile(const float* __restrict__ tile, int npairs, const f2 (&X)[B],
                                         const f2 (&Y)[B], const f2 (&Z)[B], f2 E2, f2 (&ax)[B],
                                         f2 (&ay)[B], f2 (&az)[B], f2 (&ph)[B])
{
    const ulonglong2* t2 = reinterpret_cast<const ulonglong2*>(tile);
#pragma unroll(UNROLL)
    for (int p = 0; p < npairs; p++) {
        const ulonglong2 xy = t2[2 * p];
        const ulonglong2 zm = t2[2 * p + 1];
#pragma unroll
        for (int b = 0; b < B; b++) {
            const f2 dx = f2sub(xy.x, X[b]);
            const f2 dy = f2sub(xy.y, Y[b]);
            const f2 dz = f2sub(zm.x, Z[b]);
            const f2 r2 = f2fma(dz, dz, f2fma(dy, dy, f2fma(dx, dx, E2)));
            float r2a, r2b;
            f2unpack(r2, r2a, r2b);
            const f2 ri = f2pack(rsqrt_sfu(r2a), rsqrt_sfu(r2b));
            const f2 mri = f2mul(zm.y, ri);
            const f2 mri3 = f2mul(mri, f2mul(ri, ri));
            ax[b] = f2fma(dx, mri3, ax[b]);
            ay[b] = f2fma(dy, mri3, ay[b]);
            az[b] = f2fma(dz, mri3, az[b]);
            if (POT) ph[b] = f2sub(ph[b], mri);
        }
    }
}

// quadrupole entry k of a pair-interleaved tile: {Qxx, Qxy, Qxz, Qyy, Qyz,
// Qzz, tr Q, 0} of entries 2p and 2p+1 as pairs
__device__ __forceinline__ void put_quad(float* qtile, int k, const float* q6)
{
    float* t = qtile + 16 * (k >> 1) + (k & 1);
    float qq[6];
#pragma unroll
    for (int i = 0; i < 6; i++) qq[i] = q6 ? __ldg(q6 + i) : 0.f;
#pragma unroll
    for (int i = 0; i < 6; i++) t[2 * i] = qq[i];
    t[12] = qq[0] + qq[3] + qq[5];
    t[14] = 0.f;
}

// The cell loop with quadrupole terms: per pair of cells and body, with
// d = com - x, rho^2 = |d|^2 + eps^2 and Q the cell's second moments about
// its centre of mass (second-order expansion of the softened potential):
//   a += (m rho^-3 + 7.5 d.Qd rho^-7 - 1.5 tr Q rho^-5) d - 3 rho^-5 Qd
//   pot -= m rho^-1 + 0.5 (3 d.Qd rho^-5 - tr Q rho^-3)
template <int B, bool POT, int UNROLL>
__device__ __forceinline__ void sum_tile_quad(const float* __restrict__ tile, const float* __restrict__ qtile,
                                              int npairs, const f2 (&X)[B], const f2 (&Y)[B], const f2 (&Z)[B],
                                              f2 E2, f2 (&ax)[B], f2 (&ay)[B], f2 (&az)[B], f2 (&ph)[B])
{
    const ulonglong2* t2 = reinterpret_cast<const ulonglong2*>(tile);
    const ulonglong2* q2 = reinterpret_cast<const ulonglong2*>(qtile);
    const f2 K75 = f2pack(7.5f, 7.5f), Km15 = f2pack(-1.5f, -1.5f), Km3 = f2pack(-3.f, -3.f);
    const f2 K15 = f2pack(1.5f, 1.5f), Kmh = f2pack(-0.5f, -0.5f);
#pragma unroll(UNROLL)
    for (int p = 0; p < npairs; p++) {
        const ulonglong2 xy = t2[2 * p];
        const ulonglong2 zm = t2[2 * p + 1];
        const ulonglong2 qa = q2[4 * p];      // Qxx, Qxy
        const ulonglong2 qb = q2[4 * p + 1];  // Qxz, Qyy
        const ulonglong2 qc = q2[4 * p + 2];  // Qyz, Qzz
        const ulonglong2 qd = q2[4 * p + 3];  // tr Q, 0
#pragma unroll
        for (int b = 0; b < B; b++) {
            const f2 dx = f2sub(xy.x, X[b]);
            const f2 dy = f2sub(xy.y, Y[b]);
            const f2 dz = f2sub(zm.x, Z[b]);
            const f2 r2 = f2fma(dz, dz, f2fma(dy, dy, f2fma(dx, dx, E2)));
            float r2a, r2b;
            f2unpack(r2, r2a, r2b);
            const f2 ri = f2pack(rsqrt_sfu(r2a), rsqrt_sfu(r2b));
            const f2 ri2 = f2mul(ri, ri);
            const f2 ri3 = f2mul(ri2, ri);
            const f2 ri5 = f2mul(ri3, ri2);
            const f2 ri7 = f2mul(ri5, ri2);
            const f2 qx = f2fma(qb.x, dz, f2fma(qa.y, dy, f2mul(qa.x, dx)));
            const f2 qy = f2fma(qc.x, dz, f2fma(qb.y, dy, f2mul(qa.y, dx)));
            const f2 qz = f2fma(qc.y, dz, f2fma(qc.x, dy, f2mul(qb.x, dx)));
            const f2 dqd = f2fma(dz, qz, f2fma(dy, qy, f2mul(dx, qx)));
            const f2 trr5 = f2mul(qd.x, ri5);
            // coefficient of d: m rho^-3 + 7.5 d.Qd rho^-7 - 1.5 tr rho^-5
            const f2 cd = f2fma(K75, f2mul(dqd, ri7), f2fma(Km15, trr5, f2mul(zm.y, ri3)));
            const f2 s3 = f2mul(Km3, ri5);
            ax[b] = f2fma(dx, cd, f2fma(qx, s3, ax[b]));
            ay[b] = f2fma(dy, cd, f2fma(qy, s3, ay[b]));
            az[b] = f2fma(dz, cd, f2fma(qz, s3, az[b]));
            if (POT) {
                // m rho^-1 + 1.5 d.Qd rho^-5 - 0.5 tr rho^-3
                ph[b] = f2sub(ph[b], f2fma(K15, f2mul(dqd, ri5), f2fma(Kmh, f2mul(qd.x, ri3), f2mul(zm.y, ri))));
            }
        }
    }
}

template <int B, bool PRECISE, bool POT, int UNROLL>
struct Accum {
    f2 ax[B], ay[B], az[B], ph[B];        // packed running sums (plain mode)
    float sx[B], sy[B], sz[B], sp[B];     // running sums (precise mode)
    float cx[B], cy[B], cz[B], cp[B];     // their compensations
    __device__ void init()
    {
#pragma unroll
        for (int b = 0; b < B; b++) {
            ax[b] = ay[b] = az[b] = ph[b] = 0ull;
            sx[b] = sy[b] = sz[b] = sp[b] = cx[b] = cy[b] = cz[b] = cp[b] = 0.f;
        }
    }
    // sums tile[0, n) (pads an odd count with a massless entry)
    __device__ void flush(float* tile, int n, const f2 (&X)[B], const f2 (&Y)[B], const f2 (&Z)[B], f2 E2)
    {
        if (n <= 0) return;
        if ((n & 1) && (threadIdx.x & 31) == 0) put_entry(tile, n, make_float4(0.f, 0.f, 0.f, 0.f));
        __syncwarp();
        const int np = (n + 1) >> 1;
        if (PRECISE) {
            f2 tx[B], ty[B], tz[B], tp[B];
#pragma unroll
            for (int b = 0; b < B; b++) tx[b] = ty[b] = tz[b] = tp[b] = 0ull;
            sum_tile<B, POT, UNROLL>(tile, np, X, Y, Z, E2, tx, ty, tz, tp);
#pragma unroll
            for (int b = 0; b < B; b++) {
                two_sum_acc(sx[b], cx[b], f2sum(tx[b]));
                two_sum_acc(sy[b], cy[b], f2sum(ty[b]));
                two_sum_acc(sz[b], cz[b], f2sum(tz[b]));
                if (POT) two_sum_acc(sp[b], cp[b], f2sum(tp[b]));
            }
        } else {
            sum_tile<B, POT, UNROLL>(tile, np, X, Y, Z, E2, ax, ay, az, ph);
        }
        __syncwarp();
    }
    // the same for a cell tile with quadrupole entries (precise mode)
    __device__ void flush_quad(float* tile, float* qtile, int n, const f2 (&X)[B], const f2 (&Y)[B],
                               const f2 (&Z)[B], f2 E2)
    {
        if (n <= 0) return;
        if ((n & 1) && (threadIdx.x & 31) == 0) {
            put_entry(tile, n, make_float4(0.f, 0.f, 0.f, 0.f));
            put_quad(qtile, n, nullptr);
        }
        __syncwarp();
        const int np = (n + 1) >> 1;
        f2 tx[B], ty[B], tz[B], tp[B];
#pragma unroll
        for (int b = 0; b < B; b++) tx[b] = ty[b] = tz[b] = tp[b] = 0ull;
        sum_tile_quad<B, POT, UNROLL>(tile, qtile, np, X, Y, Z, E2, tx, ty, tz, tp);
#pragma unroll
        for (int b = 0; b < B; b++) {
            two_sum_acc(sx[b], cx[b], f2sum(tx[b]));
            two_sum_acc(sy[b], cy[b], f2sum(ty[b]));
            two_sum_acc(sz[b], cz[b], f2sum(tz[b]));
            if (POT) two_sum_acc(sp[b], cp[b], f2sum(tp[b]));
        }
        __syncwarp();
    }
    __device__ void result(int b, float& fx, float& fy, float& fz, float& fp) const
    {
        if (PRECISE) {
            fx = sx[b];
            fy = sy[b];
            fz = sz[b];
            fp = sp[b];
        } else {
            fx = f2sum(ax[b]);
            fy = f2sum(ay[b]);
            fz = f2sum(az[b]);
            fp = f2sum(ph[b]);
        }
    }
    __device__ void comp(int b, float& fx, float& fy, float& fz, float& fp) const
    {
        fx = PRECISE ? cx[b] : 0.f;
        fy = PRECISE ? cy[b] : 0.f;
        fz = PRECISE ? cz[b] : 0.f;
        fp = PRECISE ? cp[b] : 0.f;
    }
};

// Learned correction.  Band cells found by a walk step are appended to a
// per-warp list of pending node indices; whenever 32 are pending, lane j
// builds the row of cell j -- 13 normalised features as BF16 pairs (8 words)
// and the factor G M s^2 / r^4 that turns a label into an acceleration --
// and the warp evaluates the rows 16 at a time on the tensor cores.
  // register cap of the learned walk: 65536 / (128 x this)
constexpr int kLearnedMinBlocks = 4;  // register cap of the learned walk: 65536 / (128 x this)
constexpr int kPend = 64;   // < 32 left over + 32 added by a step
constexpr int kRowW = 9;    // words per row
__host__ __device__ constexpr size_t mlp_frag_bytes() { return (sizeof(MlpFrag) + 15) & ~(size_t)15; }

// The network row of cell v seen from the group's box centre xgc (in the
// frame of the group's reference cube rc): d/s and s/r formed here, the
// other nine features from the node's record (k_node_features), and the
// factor G M s^2 / r^4 that turns a label into an acceleration
// what a row needs of its node: the walk record (b, a, c) and the packed
// cell-only features
struct BandNode {
    int4 nb;
    float4 na;
    int4 cc;
    uint4 c0;
    uint2 c1;
};

__device__ __forceinline__ BandNode band_node_load(const NodeTables& nt, int v)
{
    BandNode q;
    q.nb = __ldg(&nt.b[v]);
    q.na = __ldg(&nt.a[v]);
    q.cc = __ldg(&nt.c[v]);
    q.c0 = __ldg(&nt.feat[2 * v]);
    q.c1 = __ldg(reinterpret_cast<const uint2*>(&nt.feat[2 * v + 1]));
    return q;
}

__device__ __forceinline__ void band_row_from(const float* __restrict__ xscale, const float* __restrict__ xoff,
                                              const BandNode& q, int4 rc, float uf, float Lf, float inv_L,
                                              const float (&xgc)[3], float G, uint32_t (&w)[8], float& fac)
{
    // centre of mass in the group's reference frame, as in the walk
    const float dx = fmaf((float)(q.cc.x - rc.x), uf, q.na.x) - xgc[0];
    const float dy = fmaf((float)(q.cc.y - rc.y), uf, q.na.y) - xgc[1];
    const float dz = fmaf((float)(q.cc.z - rc.z), uf, q.na.z) - xgc[2];
    const float sz = scalbnf(Lf, -(q.nb.w & 255));
    const float inv_s = scalbnf(inv_L, q.nb.w & 255);  // exact: sides are powers of two
    const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    const float ri = rsqrtf(r2);
    const float Mc = q.na.w;
    const float f0 = fmaf(dx * inv_s, xscale[0], xoff[0]);
    const float f1 = fmaf(dy * inv_s, xscale[1], xoff[1]);
    const float f2 = fmaf(dz * inv_s, xscale[2], xoff[2]);
    const float f3 = fmaf(ri * sz, xscale[3], xoff[3]);
    w[0] = pack_bf16(f0, f1);
    w[1] = pack_bf16(f2, f3);
    w[2] = q.c0.x;
    w[3] = q.c0.y;
    w[4] = q.c0.z;
    w[5] = q.c0.w;
    w[6] = q.c1.x;
    w[7] = q.c1.y;
    const float ri2 = ri * ri;
    fac = G * Mc * (sz * sz) * (ri2 * ri2);  // G M s^2 / r^4
}

__device__ __forceinline__ void band_row(const MlpFrag& m, int v, const NodeTables& nt, int4 rc, float uf, float Lf,
                                         float inv_L, const float (&xgc)[3], float G, uint32_t (&w)[8], float& fac)
{
    band_row_from(m.xscale, m.xoff, band_node_load(nt, v), rc, uf, Lf, inv_L, xgc, G, w, fac);
}

// rows of the n <= 32 cells pend[0, n) evaluated, label x yscale x factor
// added to corr (lanes of q = 0 hold x, y; of q = 1 hold z).  Lane j builds
// the row of cell j.
__device__ __noinline__ void learned_rows(const MlpFrag& m, const uint32_t* pend, int n, uint32_t* rows,
                                          const NodeTables& nt, int4 rc, float uf, float Lf, float inv_L,
                                          const float (&xgc)[3], float eps, float inv_msys, float G,
                                          float (&corr)[3], int lane)
{
    (void)eps;
    (void)inv_msys;
    uint32_t w[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
    float fac = 0.f;
    if (lane < n) band_row(m, (int)pend[lane], nt, rc, uf, Lf, inv_L, xgc, G, w, fac);
    uint32_t* r = rows + lane * kRowW;
#pragma unroll
    for (int k = 0; k < 8; k++) r[k] = w[k];
    r[8] = __float_as_uint(fac);
    __syncwarp();
    const int g = lane >> 2, q = lane & 3;
    for (int t = 0; t < n; t += 16) {
        const uint32_t* r0 = rows + (t + g) * kRowW;
        const uint32_t* r1 = rows + (t + g + 8) * kRowW;
        const uint32_t x[4] = {r0[q], r1[q], r0[q + 4], r1[q + 4]};
        float y[4];
        mlp16_infer(m, x, y, lane);
        const float f0 = __uint_as_float(r0[8]), f1 = __uint_as_float(r1[8]);
        if (q == 0) {
            corr[0] += (y[0] * f0 + y[2] * f1) * m.yscale[0];
            corr[1] += (y[1] * f0 + y[3] * f1) * m.yscale[1];
        } else if (q == 1) {
            corr[2] += (y[0] * f0 + y[2] * f1) * m.yscale[2];
        }
    }
    __syncwarp();
}

// shared memory of one warp: cell and body tiles (the quadrupole walk adds
// the cells' second moments), the stack, and in learned mode the pending
// list and the rows (the block holds one copy of the network in front of the
// warps' regions)
__host__ __device__ constexpr size_t walk_warp_bytes(int tile, int stack, bool learned, bool quadw)
{
    return (size_t)2 * tile_cap(tile) * 16 + (quadw ? (size_t)tile_cap(tile) * 32 : 0) + (size_t)stack * 4 +
           (learned ? (size_t)(kPend + 32 * kRowW) * 4 : 0);
}

template <int B, int TILE, bool PRECISE, bool POT, bool LEARNED, bool QUADW>
__global__ void __launch_bounds__(128, LEARNED ? kLearnedMinBlocks : (B >= 4 ? 3 : 4)) k_walk(WalkArgs a, int stack_cap)
{
    constexpr int kTile = TILE;
    constexpr int kTileCap = tile_cap(TILE);
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const size_t head = LEARNED ? mlp_frag_bytes() : 0;
    const size_t per_warp = walk_warp_bytes(TILE, stack_cap, LEARNED, QUADW);
    float* ctile = reinterpret_cast<float*>(smem + head + wib * per_warp);
    float* qtile = ctile + 4 * kTileCap;  // quadrupole walk: 8 floats per cell entry
    float* btile = qtile + (QUADW ? 8 * kTileCap : 0);
    uint32_t* stk = reinterpret_cast<uint32_t*>(btile + 4 * kTileCap);
    uint32_t* pend = stk + stack_cap;  // learned: pending band cells, then the rows
    uint32_t* rows = pend + kPend;
    const f2 E2 = f2pack(a.eps2, a.eps2);
    const uint32_t lt = (1u << lane) - 1u;

    const Info* info = a.info;
    if (info->err & kErrCapacity) return;  // the build stopped: no tree to walk
    const bool list_mode = a.list_cells != nullptr;
    // list export walks one group: queue position 0 maps to list_group
    const int64_t G = list_mode ? (int64_t)a.list_group + 1 : (a.glist ? (int64_t)*a.glist_n : info->G);
    const int g_shift = list_mode ? a.list_group : 0;
    const NodeTables nt = a.nt;
    MlpFrag* mlp = reinterpret_cast<MlpFrag*>(smem);
    if (LEARNED) {
        // the inference part at the front of the device model
        for (int i = threadIdx.x; i < (int)(sizeof(MlpFrag) / 4); i += blockDim.x)
            reinterpret_cast<uint32_t*>(mlp)[i] = reinterpret_cast<const uint32_t*>(a.mlp)[i];
        __syncthreads();
    }

    for (;;) {
        cp_async_wait_all();  // a group that stopped early (list export, stack overflow) may have copies in flight
        int g = 0;
        if (lane == 0) g = (int)atomicAdd(&a.info->work[a.work_slot], 1u) + g_shift;
        g = __shfl_sync(0xffffffffu, g, 0);
        if (g >= G) break;
        if (a.glist) g = __ldg(a.glist + g);  // this launch's size class
        const int gfirst = a.gfirst[g];
        const int gend = a.gfirst[g + 1];
        // the group's system: its root cube and its root node (roots are
        // nodes 0..S-1 in system order)
        const uint32_t sysid = a.sys_of[gfirst];
        const SysParams& SP = a.sysp[sysid];
        const double ud = 0.5 * SP.h;
        const float uf = SP.uf;
        const float Lf = SP.Lf;
        const int4 rc = nt.c[a.gref[g]];
        const double gx = SP.c0[0] + (double)rc.x * ud, gy = SP.c0[1] + (double)rc.y * ud,
                     gz = SP.c0[2] + (double)rc.z * ud;

        // the group's bodies: absolute and reference-relative positions,
        // each coordinate duplicated into a packed pair
        f2 XA[B], YA[B], ZA[B], XR[B], YR[B], ZR[B];
        bool act[B];
        float mi[B];
        float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
#pragma unroll
        for (int b = 0; b < B; b++) {
            int i = gfirst + lane + 32 * b;
            act[b] = i < gend;
            float4 q = a.body[act[b] ? i : gfirst];
            XA[b] = f2pack(q.x, q.x);
            YA[b] = f2pack(q.y, q.y);
            ZA[b] = f2pack(q.z, q.z);
            mi[b] = q.w;
            if (PRECISE) {
                const float rx = (float)((double)q.x - gx), ry = (float)((double)q.y - gy),
                            rz = (float)((double)q.z - gz);
                XR[b] = f2pack(rx, rx);
                YR[b] = f2pack(ry, ry);
                ZR[b] = f2pack(rz, rz);
            }
            lo[0] = fminf(lo[0], q.x); hi[0] = fmaxf(hi[0], q.x);
            lo[1] = fminf(lo[1], q.y); hi[1] = fmaxf(hi[1], q.y);
            lo[2] = fminf(lo[2], q.z); hi[2] = fmaxf(hi[2], q.z);
        }
#pragma unroll
        for (int k = 0; k < 3; k++) {
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
                hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
            }
        }
        // group box relative to the reference centre: integer part (units
        // of u) + float remainder in [0, u).  Lane k < 6 splits one bound.
        int kb = 0;
        float fb = 0.f;
        if (lane < 6) {
            const int ax = lane % 3;
            const double gref = ax == 0 ? gx : (ax == 1 ? gy : gz);
            const double t = (double)(lane < 3 ? lo[ax] : hi[ax]) - gref;
            const double kf = floor(t / ud);
            kb = (int)kf;
            fb = (float)(t - kf * ud);
        }
        // the same bounds and the reference cube's centre as floats: integers
        // below 2^24, so their differences with a node's centre are exact
        int klo[3], khi[3];
        float klof[3], khif[3];
        const float rcf[3] = {(float)rc.x, (float)rc.y, (float)rc.z};
        float flo[3], fhi[3];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            klo[k] = __shfl_sync(0xffffffffu, kb, k);
            khi[k] = __shfl_sync(0xffffffffu, kb, k + 3);
            flo[k] = __shfl_sync(0xffffffffu, fb, k);
            fhi[k] = __shfl_sync(0xffffffffu, fb, k + 3);
            klof[k] = (float)klo[k];
            khif[k] = (float)khi[k];
        }

        // learned correction: evaluated at the centre of the group's box
        // (reference-relative), summed over the group's band cells
        float xgc[3] = {0.f, 0.f, 0.f};
        float corr[3] = {0.f, 0.f, 0.f};
        int qn = 0;
        unsigned long long nevals = 0;
        float inv_L = 0.f, inv_msys = 0.f;
        if (LEARNED) {
            inv_L = 1.0f / Lf;
            inv_msys = 1.0f / SP.msys;
#pragma unroll
            for (int k = 0; k < 3; k++)
                xgc[k] = 0.5f * (fmaf((float)klo[k], uf, flo[k]) + fmaf((float)khi[k], uf, fhi[k]));
        }

        // force-loop unroll: deep for one or two bodies per lane; shallower
        // with four (registers), in the quadrupole walk (registers) and in
        // the learned walk (measured: 4 deep is the fastest there)
        constexpr int kUnroll = QUADW ? 2 : (LEARNED || B >= 4 ? 4 : 8);
        // one running (compensated) sum per body collects the cell tiles and
        // the body tiles alike
        Accum<B, PRECISE, POT, kUnroll> fsum;
        fsum.init();
        int cn = 0, bn = 0, Lc = 0, Lb = 0, nleaf = 0;
        unsigned long long hsh = 0;
        const bool want_hash = a.hash != nullptr;  // list hashes only for verification
        const bool fast_side = ((__float_as_int(Lf) >> 23) & 255) > kMaxLevel + 1;
        bool overflow = false;
        int sp = 1;
        if (lane == 0) stk[0] = sysid;  // the system's root: holds every body, always opened
        __syncwarp();

        while (sp > 0) {
            const int np = min(sp, 32);
            int v = -1;
            if (lane < np) v = (int)stk[sp - np + lane];
            sp -= np;
            __syncwarp();
            int4 nb = make_int4(0, 0, 0, 0);
            bool acc = false, oleaf = false, oint = false;
            float4 src = make_float4(0.f, 0.f, 0.f, 0.f);
            float band_e2 = 0.f;
            if (v >= 0) {
                // the three node records are independent loads: issue together
                nb = __ldg(&nt.b[v]);
                const float4 na = __ldg(&nt.a[v]);
                const int4 cc = __ldg(&nt.c[v]);
                const int nch = nb.w >> 8;
                const bool overlap = (nb.x < gend) && (gfirst < nb.x + nb.y);
                if (!overlap) {
                    const float D[3] = {(float)cc.x - rcf[0], (float)cc.y - rcf[1], (float)cc.z - rcf[2]};
                    const float off[3] = {na.x, na.y, na.z};
                    float e2 = 0.f;
#pragma unroll
                    for (int k = 0; k < 3; k++) {
                        const float lo_c = fmaf(klof[k] - D[k], uf, flo[k]);  // box lo - cube centre
                        const float hi_c = fmaf(khif[k] - D[k], uf, fhi[k]);
                        const float e = fmaxf(fmaxf(lo_c - off[k], off[k] - hi_c), 0.f);
                        e2 = fmaf(e, e, e2);
                    }
                    const float s = pow2_down(Lf, nb.w & 255, fast_side);
                    acc = (s * s) < a.theta2 * e2;
                    band_e2 = e2;
                    if (acc) {
                        if (PRECISE || LEARNED) {
                            src = make_float4(fmaf(D[0], uf, off[0]), fmaf(D[1], uf, off[1]),
                                              fmaf(D[2], uf, off[2]), na.w);
                        } else {
                            src = nt.d[v];
                        }
                    }
                }
                if (!acc) {
                    oleaf = (nch == 0);
                    oint = (nch != 0);
                }
            }
            // opened internal nodes push their children
            const int npush = oint ? (nb.w >> 8) : 0;  // at most 8
            int tot;
            const int excl = warp_excl_small(npush, lt, tot);
            if (sp + tot > stack_cap) {
                overflow = true;
                break;
            }
            for (int k = 0; k < npush; k++) stk[sp + excl + k] = (uint32_t)(nb.z + k);
            sp += tot;
            // accepted cells -> cell tile
            const unsigned am = __ballot_sync(0xffffffffu, acc);
            if (list_mode && acc) {
                const int k = Lc + __popc(am & lt);
                if (k < a.list_cap) a.list_cells[k] = v;
            }
            if (acc) {
                put_entry(ctile, cn + __popc(am & lt), src);
                if (QUADW) put_quad(qtile, cn + __popc(am & lt), nt.quad + 6 * (int64_t)v);
                if (want_hash) hsh += mix64(2ull * (unsigned)v + 1ull);
            }
            cn += __popc(am);
            Lc += __popc(am);
            // band cells (s / d at or above the band, two bodies or more):
            // training pairs and learned corrections
            bool band = false;
            const bool pairs_on = !LEARNED && a.pair_body != nullptr;  // pair emission runs a plain walk
            if ((LEARNED || pairs_on) && acc && nb.y >= 2) {
                const float sz = pow2_down(Lf, nb.w & 255, fast_side);
                band = sz * sz >= a.band2 * band_e2;
            }
            if (pairs_on && band) {
                const unsigned long long hh = mix64(a.pair_seed ^ (((unsigned long long)g << 32) | (unsigned)v));
                if ((float)(hh >> 40) * (1.0f / 16777216.0f) < a.pair_prob) {
                    const unsigned long long k = atomicAdd(a.pair_count, 1ull);
                    if ((int64_t)k < a.pair_cap) {
                        a.pair_body[k] = gfirst + (int)((hh & 0xffffffffull) % (unsigned)(gend - gfirst));
                        a.pair_node[k] = v;
                    }
                }
            }
            if (LEARNED) {
                const unsigned bm = __ballot_sync(0xffffffffu, band);
                if (bm) {
                    if (band) pend[qn + __popc(bm & lt)] = (uint32_t)v;
                    qn += __popc(bm);
                    if (qn >= 32) {
                        __syncwarp();
                        learned_rows(*mlp, pend, 32, rows, nt, rc, uf, Lf, inv_L, xgc, a.eps, inv_msys, a.G, corr,
                                     lane);
                        nevals += 32;
                        // move the cells past the first 32 to the front (read all, then write)
                        const int rest = qn - 32;
                        const uint32_t t = lane < rest ? pend[32 + lane] : 0u;
                        __syncwarp();
                        if (lane < rest) pend[lane] = t;
                        qn = rest;
                    }
                    __syncwarp();
                }
            }
            // opened leaves -> body tile.  The bodies of all leaves opened in
            // this step are gathered 32 at a time: lane j takes body t of the
            // concatenated ranges, finding its leaf by a binary search over
            // the lanes' exclusive offsets.
            const unsigned lm = __ballot_sync(0xffffffffu, oleaf);
            if (list_mode && oleaf) {
                const int k = nleaf + __popc(lm & lt);
                if (k < a.list_cap) a.list_leaves[k] = v;
            }
            nleaf += __popc(lm);
            if (lm) {
                if (want_hash && oleaf) hsh += mix64(2ull * (unsigned)v + 2ull);
                const int cnt = oleaf ? nb.y : 0;
                const int incl_c = warp_incl_scan_i(cnt);
                const int excl_c = incl_c - cnt;
                const int T = __shfl_sync(0xffffffffu, incl_c, 31);
                Lb += T;
                for (int o = 0; o < T; o += 32) {
                    const int t = min(o + lane, T - 1);
                    int pos = 0;
#pragma unroll
                    for (int step = 16; step; step >>= 1) {
                        const int e = __shfl_sync(0xffffffffu, excl_c, pos + step);
                        if (e <= t) pos += step;
                    }
                    const int f = __shfl_sync(0xffffffffu, nb.x, pos);
                    const int e0 = __shfl_sync(0xffffffffu, excl_c, pos);
                    if (o + lane < T) put_entry_async(btile, bn + lane, &a.body[f + (t - e0)]);
                    bn += min(32, T - o);
                    if (bn >= kTile) {
                        cp_async_wait_all();
                        fsum.flush(btile, bn, XA, YA, ZA, E2);
                        bn = 0;
                    }
                }
            }
            __syncwarp();
            if (cn >= kTile) {
                if (QUADW) fsum.flush_quad(ctile, qtile, cn, XR, YR, ZR, E2);
                else if (PRECISE) fsum.flush(ctile, cn, XR, YR, ZR, E2);
                else fsum.flush(ctile, cn, XA, YA, ZA, E2);
                cn = 0;
            }
        }
        if (overflow) {
            if (lane == 0) atomicOr(&a.info->err, kErrStack);
            __syncwarp();
            continue;
        }
        if (QUADW) fsum.flush_quad(ctile, qtile, cn, XR, YR, ZR, E2);
        else if (PRECISE) fsum.flush(ctile, cn, XR, YR, ZR, E2);
        else fsum.flush(ctile, cn, XA, YA, ZA, E2);
        cp_async_wait_all();
        fsum.flush(btile, bn, XA, YA, ZA, E2);
        if (LEARNED) {
            if (qn > 0) {
                learned_rows(*mlp, pend, qn, rows, nt, rc, uf, Lf, inv_L, xgc, a.eps, inv_msys, a.G, corr, lane);
                nevals += qn;
            }
#pragma unroll
            for (int k = 0; k < 3; k++)
#pragma unroll
                for (int o = 16; o; o >>= 1) corr[k] += __shfl_xor_sync(0xffffffffu, corr[k], o);
        }

        if (list_mode) {
            if (lane == 0) {
                a.list_n[0] = Lc;
                a.list_n[1] = nleaf;
            }
            __syncwarp();
            continue;
        }
        // results, scattered back to the original body order
#pragma unroll
        for (int b = 0; b < B; b++) {
            if (!act[b]) continue;
            const int i = gfirst + lane + 32 * b;
            const int64_t o = a.perm[i];
            float sx_, sy_, sz_, sp_, kx, ky, kz, kp;
            fsum.result(b, sx_, sy_, sz_, sp_);
            fsum.comp(b, kx, ky, kz, kp);
            // the running sum with its compensation
            const float fx = sx_ + kx;
            const float fy = sy_ + ky;
            const float fz = sz_ + kz;
            const float fp = sp_ + kp;
            a.acc[3 * o + 0] = a.G * fx + corr[0];
            a.acc[3 * o + 1] = a.G * fy + corr[1];
            a.acc[3 * o + 2] = a.G * fz + corr[2];
            if (POT) {
                // remove the body's own term, -m_i / eps, summed with the list
                const float self = mi[b] * rsqrtf(a.eps2);
                a.pot[o] = a.G * (fp + self);
            }
        }
        // per-group list statistics
        if (want_hash) {
#pragma unroll
            for (int o = 16; o; o >>= 1) hsh += __shfl_xor_sync(0xffffffffu, hsh, o);
        }
        if (lane == 0) {
            const int gc = gend - gfirst;
            atomicAdd(&a.info->interactions, (unsigned long long)gc * (unsigned long long)(Lc + Lb));
            atomicAdd(&a.info->cells, (unsigned long long)gc * (unsigned long long)Lc);
            atomicAdd(&a.info->bodies, (unsigned long long)gc * (unsigned long long)Lb);
            if (LEARNED && a.mlp_evals) atomicAdd(a.mlp_evals, nevals);
            if (a.ncell) a.ncell[g] = Lc;
            if (a.nbody) a.nbody[g] = Lb;
            if (a.hash) a.hash[g] = hsh;
        }
        __syncwarp();
    }
}

}  // namespace
}  // namespace tc

#include "tc_walk_ws.cuh"

namespace tc {
namespace {

template <int B, int TILE, bool PRECISE, bool POT, bool LEARNED, bool QUADW>
cudaError_t prepare_t(const WalkConfig& c, int num_sms, int* grid, size_t* smem_out)
{
    const int warps = c.warps;
    const size_t head = LEARNED ? mlp_frag_bytes() : 0;
    const size_t smem = head + walk_warp_bytes(TILE, c.stack, LEARNED, QUADW) * warps;
    auto kern = k_walk<B, TILE, PRECISE, POT, LEARNED, QUADW>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, warps * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if (c.blocks_per_sm > 0 && c.blocks_per_sm < per_sm) per_sm = c.blocks_per_sm;
    *grid = num_sms * per_sm;
    *smem_out = smem;
    return cudaSuccess;
}

template <int B, int TILE, bool PRECISE, bool POT, bool LEARNED, bool QUADW>
cudaError_t launch_t(const WalkArgs& a, const WalkConfig& c, int grid, size_t smem, cudaStream_t s)
{
    k_walk<B, TILE, PRECISE, POT, LEARNED, QUADW><<<grid, c.warps * 32, smem, s>>>(a, c.stack);
    count_launches(1);
    return cudaGetLastError();
}

// dispatch over the mode for B bodies per lane and tiles of TT entries to
// the template instance F; the learned correction exists in the precise
// mode without potential, the quadrupole walk in the precise mode
template <int B, int TT, template <int, int, bool, bool, bool, bool> class F, typename... Args>
cudaError_t dispatch_modes(const WalkConfig& c, Args... args)
{
    const bool p = c.precise != 0, pot = c.want_pot != 0;
    if ((c.learned || c.quadw) && !p) return cudaErrorInvalidValue;
    if (c.learned && (pot || c.quadw)) return cudaErrorInvalidValue;
    if (c.learned) return F<B, TT, true, false, true, false>::run(args...);
    if (c.quadw && pot) return F<B, TT, true, true, false, true>::run(args...);
    if (c.quadw) return F<B, TT, true, false, false, true>::run(args...);
    if (p && pot) return F<B, TT, true, true, false, false>::run(args...);
    if (p && !pot) return F<B, TT, true, false, false, false>::run(args...);
    if (!p && pot) return F<B, TT, false, true, false, false>::run(args...);
    return F<B, TT, false, false, false, false>::run(args...);
}

// split = 1 runs the monopole walks (precise or plain, with or without the
// potential) on k_walk_ws, producer and consumer warps apart; the learned
// walk there records its band cells for k_band_eval instead of evaluating
// the network inside the walk
template <int B, int TILE, bool PRECISE, bool POT, bool LEARNED, bool QUADW>
struct PrepareF {
    static cudaError_t run(const WalkConfig* c, int num_sms, int* grid, size_t* smem)
    {
        if constexpr (!QUADW) {
            if (c->split) return prepare_ws_t<B, TILE, PRECISE, POT, LEARNED>(*c, num_sms, grid, smem);
        }
        return prepare_t<B, TILE, PRECISE, POT, LEARNED, QUADW>(*c, num_sms, grid, smem);
    }
};
template <int B, int TILE, bool PRECISE, bool POT, bool LEARNED, bool QUADW>
struct LaunchF {
    static cudaError_t run(const WalkArgs* a, const WalkConfig* c, int grid, size_t smem, cudaStream_t s)
    {
        if constexpr (!QUADW) {
            if (c->split) return launch_ws_t<B, TILE, PRECISE, POT, LEARNED>(*a, *c, grid, smem, s);
        }
        return launch_t<B, TILE, PRECISE, POT, LEARNED, QUADW>(*a, *c, grid, smem, s);
    }
};

}  // namespace

}  // namespace tc
