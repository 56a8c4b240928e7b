// tc_walk.cu -- the force phase: tree walk with the cell-opening test,
// interaction lists staged in shared memory, softened monopole force loop.
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
#include "tc_internal.cuh"

namespace tc {

namespace {

constexpr int kTile = 128;              // list entries per tile flush
constexpr int kTileCap = kTile + 32;    // a step adds at most 32 before a flush check

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

// error-free sum: s + c absorbs x (Knuth's TwoSum)
__device__ __forceinline__ void two_sum_acc(float& s, float& c, float x)
{
    float t = __fadd_rn(s, x);
    float z = __fsub_rn(t, s);
    float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(x, z));
    s = t;
    c = __fadd_rn(c, e);
}

template <int B, bool POT>
__device__ __forceinline__ void sum_tile(const float4* __restrict__ tile, int n, const float3 (&x)[B],
                                         float eps2, float (&ax)[B], float (&ay)[B], float (&az)[B],
                                         float (&ph)[B])
{
#pragma unroll 4
    for (int j = 0; j < n; j++) {
        const float4 s = tile[j];
#pragma unroll
        for (int b = 0; b < B; b++) {
            float dx = s.x - x[b].x;
            float dy = s.y - x[b].y;
            float dz = s.z - x[b].z;
            float r2 = fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, eps2)));
            float ri = rsqrtf(r2);
            float mri = s.w * ri;
            float mri3 = mri * (ri * ri);
            ax[b] = fmaf(dx, mri3, ax[b]);
            ay[b] = fmaf(dy, mri3, ay[b]);
            az[b] = fmaf(dz, mri3, az[b]);
            if (POT) ph[b] -= mri;
        }
    }
}

template <int B, bool PRECISE, bool POT>
struct Accum {
    float ax[B], ay[B], az[B], ph[B];     // running sums
    float cx[B], cy[B], cz[B], cp[B];     // compensations (precise)
    __device__ void init()
    {
#pragma unroll
        for (int b = 0; b < B; b++) ax[b] = ay[b] = az[b] = ph[b] = cx[b] = cy[b] = cz[b] = cp[b] = 0.f;
    }
    __device__ void flush(const float4* tile, int n, const float3 (&x)[B], float eps2)
    {
        if (n <= 0) return;
        __syncwarp();
        if (PRECISE) {
            float tx[B], ty[B], tz[B], tp[B];
#pragma unroll
            for (int b = 0; b < B; b++) tx[b] = ty[b] = tz[b] = tp[b] = 0.f;
            sum_tile<B, POT>(tile, n, x, eps2, tx, ty, tz, tp);
#pragma unroll
            for (int b = 0; b < B; b++) {
                two_sum_acc(ax[b], cx[b], tx[b]);
                two_sum_acc(ay[b], cy[b], ty[b]);
                two_sum_acc(az[b], cz[b], tz[b]);
                if (POT) two_sum_acc(ph[b], cp[b], tp[b]);
            }
        } else {
            sum_tile<B, POT>(tile, n, x, eps2, ax, ay, az, ph);
        }
        __syncwarp();
    }
};

template <int B, bool PRECISE, bool POT>
__global__ void __launch_bounds__(128) k_walk(WalkArgs a, int stack_cap)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const size_t per_warp = (size_t)2 * kTileCap * sizeof(float4) + (size_t)stack_cap * sizeof(uint32_t);
    float4* ctile = reinterpret_cast<float4*>(smem + wib * per_warp);
    float4* btile = ctile + kTileCap;
    uint32_t* stk = reinterpret_cast<uint32_t*>(btile + kTileCap);
    const uint32_t lt = (1u << lane) - 1u;

    const Info* info = a.info;
    const int64_t G = info->G;
    const double c0x = info->c0[0], c0y = info->c0[1], c0z = info->c0[2];
    const double ud = 0.5 * info->h;
    const float uf = info->uf;
    const float Lf = info->Lf;
    const NodeTables nt = a.nt;

    for (;;) {
        int g = 0;
        if (lane == 0) g = (int)atomicAdd(&a.info->work, 1u);
        g = __shfl_sync(0xffffffffu, g, 0);
        if (g >= G) break;
        const int gfirst = a.gfirst[g];
        const int gend = a.gfirst[g + 1];
        const int4 rc = nt.c[a.gref[g]];
        const double gx = c0x + (double)rc.x * ud, gy = c0y + (double)rc.y * ud, gz = c0z + (double)rc.z * ud;

        // the group's bodies: absolute and reference-relative positions
        float3 xa[B], xr[B];
        bool act[B];
        float mi[B];
        float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
#pragma unroll
        for (int b = 0; b < B; b++) {
            int i = gfirst + lane + 32 * b;
            act[b] = i < gend;
            float4 q = a.body[act[b] ? i : gfirst];
            xa[b] = make_float3(q.x, q.y, q.z);
            mi[b] = q.w;
            if (PRECISE)
                xr[b] = make_float3((float)((double)q.x - gx), (float)((double)q.y - gy), (float)((double)q.z - gz));
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
        int klo[3], khi[3];
        float flo[3], fhi[3];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            klo[k] = __shfl_sync(0xffffffffu, kb, k);
            khi[k] = __shfl_sync(0xffffffffu, kb, k + 3);
            flo[k] = __shfl_sync(0xffffffffu, fb, k);
            fhi[k] = __shfl_sync(0xffffffffu, fb, k + 3);
        }

        Accum<B, PRECISE, POT> cacc, bacc;
        cacc.init();
        bacc.init();
        int cn = 0, bn = 0, Lc = 0, Lb = 0;
        unsigned long long hsh = 0;
        bool overflow = false;
        int sp = 1;
        if (lane == 0) stk[0] = 0;  // the root: holds every body, always opened
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
            if (v >= 0) {
                nb = nt.b[v];
                const int nch = nb.w >> 8;
                const bool overlap = (nb.x < gend) && (gfirst < nb.x + nb.y);
                if (!overlap) {
                    const float4 na = nt.a[v];
                    const int4 cc = nt.c[v];
                    const int D[3] = {cc.x - rc.x, cc.y - rc.y, cc.z - rc.z};
                    const float off[3] = {na.x, na.y, na.z};
                    float e2 = 0.f;
#pragma unroll
                    for (int k = 0; k < 3; k++) {
                        const float lo_c = fmaf((float)(klo[k] - D[k]), uf, flo[k]);  // box lo - cube centre
                        const float hi_c = fmaf((float)(khi[k] - D[k]), uf, fhi[k]);
                        const float e = fmaxf(fmaxf(lo_c - off[k], off[k] - hi_c), 0.f);
                        e2 = fmaf(e, e, e2);
                    }
                    const float s = scalbnf(Lf, -(nb.w & 255));
                    acc = (s * s) < a.theta2 * e2;
                    if (acc) {
                        if (PRECISE) {
                            src = make_float4(fmaf((float)D[0], uf, off[0]), fmaf((float)D[1], uf, off[1]),
                                              fmaf((float)D[2], uf, off[2]), na.w);
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
            const int npush = oint ? (nb.w >> 8) : 0;
            const int incl = warp_incl_scan_i(npush);
            const int tot = __shfl_sync(0xffffffffu, incl, 31);
            if (sp + tot > stack_cap) {
                overflow = true;
                break;
            }
            for (int k = 0; k < npush; k++) stk[sp + incl - npush + k] = (uint32_t)(nb.z + k);
            sp += tot;
            // accepted cells -> cell tile
            const unsigned am = __ballot_sync(0xffffffffu, acc);
            if (acc) {
                ctile[cn + __popc(am & lt)] = src;
                hsh += mix64(2ull * (unsigned)v + 1ull);
            }
            cn += __popc(am);
            Lc += __popc(am);
            // opened leaves -> body tile
            unsigned lm = __ballot_sync(0xffffffffu, oleaf);
            if (oleaf) hsh += mix64(2ull * (unsigned)v + 2ull);
            while (lm) {
                const int srcl = __ffs(lm) - 1;
                lm &= lm - 1;
                const int f = __shfl_sync(0xffffffffu, nb.x, srcl);
                const int c = __shfl_sync(0xffffffffu, nb.y, srcl);
                Lb += c;
                for (int o = 0; o < c; o += 32) {
                    if (o + lane < c) btile[bn + lane] = a.body[f + o + lane];
                    bn += min(32, c - o);
                    if (bn >= kTile) {
                        bacc.flush(btile, bn, xa, a.eps2);
                        bn = 0;
                    }
                }
            }
            __syncwarp();
            if (cn >= kTile) {
                if (PRECISE) cacc.flush(ctile, cn, xr, a.eps2);
                else cacc.flush(ctile, cn, xa, a.eps2);
                cn = 0;
            }
        }
        if (overflow) {
            if (lane == 0) atomicOr(&a.info->err, kErrStack);
            __syncwarp();
            continue;
        }
        if (PRECISE) cacc.flush(ctile, cn, xr, a.eps2);
        else cacc.flush(ctile, cn, xa, a.eps2);
        bacc.flush(btile, bn, xa, a.eps2);

        // results, scattered back to the original body order
#pragma unroll
        for (int b = 0; b < B; b++) {
            if (!act[b]) continue;
            const int i = gfirst + lane + 32 * b;
            const int64_t o = a.perm[i];
            float fx, fy, fz, fp;
            if (PRECISE) {
                // (cell sum) + (body sum), each carried with its compensation
                fx = (cacc.ax[b] + bacc.ax[b]) + (cacc.cx[b] + bacc.cx[b]);
                fy = (cacc.ay[b] + bacc.ay[b]) + (cacc.cy[b] + bacc.cy[b]);
                fz = (cacc.az[b] + bacc.az[b]) + (cacc.cz[b] + bacc.cz[b]);
                fp = (cacc.ph[b] + bacc.ph[b]) + (cacc.cp[b] + bacc.cp[b]);
            } else {
                fx = cacc.ax[b] + bacc.ax[b];
                fy = cacc.ay[b] + bacc.ay[b];
                fz = cacc.az[b] + bacc.az[b];
                fp = cacc.ph[b] + bacc.ph[b];
            }
            a.acc[3 * o + 0] = a.G * fx;
            a.acc[3 * o + 1] = a.G * fy;
            a.acc[3 * o + 2] = a.G * fz;
            if (POT) {
                // remove the body's own term, -m_i / eps, summed with the list
                const float self = mi[b] * rsqrtf(a.eps2);
                a.pot[o] = a.G * (fp + self);
            }
        }
        // per-group list statistics
#pragma unroll
        for (int o = 16; o; o >>= 1) hsh += __shfl_xor_sync(0xffffffffu, hsh, o);
        if (lane == 0) {
            const int gc = gend - gfirst;
            atomicAdd(&a.info->interactions, (unsigned long long)gc * (unsigned long long)(Lc + Lb));
            atomicAdd(&a.info->cells, (unsigned long long)Lc);
            atomicAdd(&a.info->bodies, (unsigned long long)Lb);
            if (a.ncell) a.ncell[g] = Lc;
            if (a.nbody) a.nbody[g] = Lb;
            if (a.hash) a.hash[g] = hsh;
        }
        __syncwarp();
    }
}

template <int B, bool PRECISE, bool POT>
cudaError_t launch_t(const WalkArgs& a, const WalkConfig& c, int num_sms, cudaStream_t s)
{
    const int warps = c.warps;
    const size_t per_warp = (size_t)2 * kTileCap * sizeof(float4) + (size_t)c.stack * sizeof(uint32_t);
    const size_t smem = per_warp * warps;
    auto kern = k_walk<B, PRECISE, POT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, warps * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if (c.blocks_per_sm > 0 && c.blocks_per_sm < per_sm) per_sm = c.blocks_per_sm;
    kern<<<num_sms * per_sm, warps * 32, smem, s>>>(a, c.stack);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_walk(const WalkArgs& a, const WalkConfig& c, int num_sms, cudaStream_t s)
{
    cudaMemsetAsync(&a.info->work, 0, sizeof(uint32_t), s);
    cudaMemsetAsync(&a.info->interactions, 0, 3 * sizeof(unsigned long long), s);
    const bool p = c.precise != 0, pot = c.want_pot != 0;
#define TC_WALK_CASE(BB)                                                              \
    if (c.gmax == 32 * BB) {                                                          \
        if (p && pot) return launch_t<BB, true, true>(a, c, num_sms, s);              \
        if (p && !pot) return launch_t<BB, true, false>(a, c, num_sms, s);            \
        if (!p && pot) return launch_t<BB, false, true>(a, c, num_sms, s);            \
        return launch_t<BB, false, false>(a, c, num_sms, s);                          \
    }
    TC_WALK_CASE(1)
    TC_WALK_CASE(2)
    TC_WALK_CASE(4)
#undef TC_WALK_CASE
    return cudaErrorInvalidValue;
}

}  // namespace tc
