// tc_walk_ws.cuh -- the force phase with the tree walk and the force loop on
// different warps (included by tc_walk.cuh after k_walk).
//
// k_walk gives each warp a whole group: it walks a step, sums a full list
// tile, walks on.  Measured on a uniform cube of 2^20 bodies, its warps spend
// 44 % of their time walking and the walk and the sums of the other warps of
// an SM hardly overlap: the walk alone takes 0.45 ms, the whole kernel
// 1.52 ms, while the force loop alone would need about 1.1 ms.
//
// Here a block holds P producer/consumer pairs.  The producer warp walks a
// group exactly as k_walk does (opening test, ballots, list compaction into
// pair-interleaved tiles) but never sums: it fills the slots of a ring in
// shared memory, each slot carrying a cell part and a body part of up to
// one tile each, and hands a slot over when either part is full or the group
// ends.  The consumer warp holds the group's bodies in registers and sums
// every slot it is handed (the same compensated paired-FP32 loop), then
// writes the group's accelerations.  The ring has kWsSlots slots; one
// mbarrier per slot tells the consumer a slot is full, one tells the
// producer it is empty again.  Slots are filled and emptied in one order,
// one slot open at a time, so the two never wait on each other in a cycle.
//
// Every wait is bounded (about a second of SM clock): a wait that runs out
// raises kErrWorkLoop in the error word and its warp returns, so a fault in
// the protocol ends the kernel with an error instead of a hang.
#pragma once

namespace tc {

namespace {

constexpr int kWsSlots = 3;                      // ring depth per pair
constexpr int kWsMaxPairs = 4;                   // pairs per block (block = 2 x pairs warps)
constexpr long long kWsWaitCycles = 1ll << 31;   // about 1 s of SM clock

// slot header (64 bytes at the front of a slot)
struct WsHdr {
    int32_t flags;  // kWsFirst | kWsLast | kWsDone | kWsAbort
    int32_t cn;     // entries in the cell part
    int32_t bn;     // entries in the body part
    int32_t g;      // group
    int32_t gfirst, gend;
    int32_t pad[2];
    double ref[3];  // centre of the group's reference cube (absolute, FP64)
    double pad2;
};
static_assert(sizeof(WsHdr) == 64, "slot header");
enum : int32_t { kWsFirst = 1, kWsLast = 2, kWsDone = 4, kWsAbort = 8 };

__host__ __device__ constexpr size_t ws_slot_bytes(int tile) { return sizeof(WsHdr) + (size_t)2 * tile_cap(tile) * 16; }
// one pair: 2 x kWsSlots mbarriers (padded to 64 bytes), the slots, the
// producer's stack
__host__ __device__ constexpr size_t ws_pair_bytes(int tile, int stack)
{
    return 64 + kWsSlots * ws_slot_bytes(tile) + (size_t)stack * 4;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count) : "memory");
}

// every lane of the warp arrives (the barriers count 32 arrivals), each
// releasing its own writes to the slot
__device__ __forceinline__ void mbar_arrive(uint64_t* b)
{
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(smem_addr(b)) : "memory");
}

// the opened leaves' bodies reach a slot by cp.async (put_entry_async);
// before its arrival on the slot's full barrier every producer lane makes the
// barrier track its copies (cp.async.mbarrier.arrive without .noinc: the
// pending count rises now and falls when the lane's copies have landed), so
// the phase completes only once the bodies are in the tile
__device__ __forceinline__ void mbar_track_copies(uint64_t* b)
{
    asm volatile("cp.async.mbarrier.arrive.shared::cta.b64 [%0];" ::"r"(smem_addr(b)) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_addr(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

// wait for the phase of the given parity to complete, at most
// kWsWaitCycles; warp-uniform result (false if any lane ran out)
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity)
{
    bool ok = mbar_try(b, parity);
    if (!ok) {
        const long long t0 = clock64();
        while (!(ok = mbar_try(b, parity)))
            if (clock64() - t0 > kWsWaitCycles) break;
    }
    return __all_sync(0xffffffffu, ok);
}

// LEARNED: the producer also records the group's band cells (accepted, two
// bodies or more, s >= band d) for the network, which runs after the walk
// (k_band_eval) as (node, group) pairs, and each group's record (box centre
// and frame)
template <int B, int TILE, bool PRECISE, bool POT, bool LEARNED>
__global__ void __launch_bounds__(2 * 32 * kWsMaxPairs, B >= 4 ? 1 : 2) k_walk_ws(WalkArgs a, int stack_cap)
{
    constexpr int kTile = TILE;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int pairs = blockDim.x >> 6;
    const bool producer = warp < pairs;
    const int q = producer ? warp : warp - pairs;  // the pair
    unsigned char* base = smem + (size_t)q * ws_pair_bytes(TILE, stack_cap);
    uint64_t* full = reinterpret_cast<uint64_t*>(base);
    uint64_t* empty = full + kWsSlots;
    unsigned char* slots = base + 64;
    uint32_t* stk = reinterpret_cast<uint32_t*>(slots + kWsSlots * ws_slot_bytes(TILE));
    const uint32_t lt = (1u << lane) - 1u;

    const Info* info = a.info;
    if (info->err & kErrCapacity) return;  // the build stopped: no tree to walk (uniform: no barrier used yet)
    if (threadIdx.x < pairs) {
        for (int s = 0; s < kWsSlots; s++) {
            mbar_init(reinterpret_cast<uint64_t*>(smem + (size_t)threadIdx.x * ws_pair_bytes(TILE, stack_cap)) + s,
                      32);
            mbar_init(reinterpret_cast<uint64_t*>(smem + (size_t)threadIdx.x * ws_pair_bytes(TILE, stack_cap)) +
                          kWsSlots + s,
                      32);
        }
    }
    __syncthreads();
    auto slot_hdr = [&](int k) { return reinterpret_cast<WsHdr*>(slots + (size_t)(k % kWsSlots) * ws_slot_bytes(TILE)); };
    auto slot_cells = [&](int k) {
        return reinterpret_cast<float*>(slots + (size_t)(k % kWsSlots) * ws_slot_bytes(TILE) + sizeof(WsHdr));
    };
    auto slot_bodies = [&](int k) { return slot_cells(k) + 4 * tile_cap(TILE); };

    if (producer) {
        // ------------------------------------------------------------ producer
        const bool list_stats = a.hash != nullptr;
        const int64_t G = a.glist ? (int64_t)*a.glist_n : info->G;
        const NodeTables nt = a.nt;
        int k = 0;  // slots taken so far
        bool alive = true;
        // take slot k (wait until the consumer has emptied it)
        auto take = [&]() -> bool {
            if (!mbar_wait(&empty[k % kWsSlots], ((k / kWsSlots) & 1) ^ 1)) {
                if (lane == 0) atomicOr(&a.info->err, kErrWorkLoop);
                return false;
            }
            return true;
        };
        auto hand_over = [&](int flags, int cn, int bn) {
            WsHdr* h = slot_hdr(k);
            if (lane == 0) {
                h->flags |= flags;
                h->cn = cn;
                h->bn = bn;
            }
            __syncwarp();
            mbar_track_copies(&full[k % kWsSlots]);
            mbar_arrive(&full[k % kWsSlots]);
            k++;
        };
        // band cells: this warp's chunk of the record (cbase < 0: none yet)
        int64_t cbase = -1;
        int cused = kBandChunk;
        const int64_t band_lim = (a.band_cap / kBandChunk) * kBandChunk;
        auto band_append = [&](bool band, int v, int g) {
            const unsigned bm = __ballot_sync(0xffffffffu, band);
            const int c = __popc(bm);
            if (c == 0) return;
            const int rank = __popc(bm & lt);
            const int room = kBandChunk - cused;
            int64_t nbase = -1;
            if (c > room) {  // a new chunk for the cells that do not fit
                long long x = -1;
                if (lane == 0) {
                    x = (long long)atomicAdd(a.band_n, (unsigned long long)kBandChunk);
                    if (x + kBandChunk > band_lim) {
                        atomicOr(&a.info->err, kErrBand);
                        x = -1;
                    }
                }
                nbase = __shfl_sync(0xffffffffu, x, 0);
            }
            if (band) {
                int64_t pos = -1;
                if (rank < room) pos = cbase + cused + rank;
                else if (nbase >= 0) pos = nbase + (rank - room);
                if (pos >= 0) a.band[pos] = make_int2(v, g);
            }
            if (c > room) {
                cbase = nbase;
                cused = nbase >= 0 ? c - room : kBandChunk;
            } else {
                cused += c;
            }
        };
        auto open_slot = [&](int flags, int g) {
            WsHdr* h = slot_hdr(k);
            if (lane == 0) {
                h->flags = flags;
                h->g = g;
            }
        };
        for (;;) {
            int g = 0;
            if (lane == 0) g = (int)atomicAdd(&a.info->work[a.work_slot], 1u);
            g = __shfl_sync(0xffffffffu, g, 0);
            if (g >= G) {
                if (take()) {
                    open_slot(kWsDone, 0);
                    hand_over(0, 0, 0);
                }
                // the unused tail of the chunk: no cell
                if (LEARNED && cbase >= 0)
                    for (int j = cused + lane; j < kBandChunk; j += 32) a.band[cbase + j] = make_int2(-1, 0);
                break;
            }
            if (a.glist) g = __ldg(a.glist + g);
            const int gfirst = a.gfirst[g];
            const int gend = a.gfirst[g + 1];
            const uint32_t sysid = a.sys_of[gfirst];
            const SysParams& SP = a.sysp[sysid];
            const double ud = 0.5 * SP.h;
            const float uf = SP.uf;
            const float Lf = SP.Lf;
            const int4 rc = nt.c[a.gref[g]];
            const double gx = SP.c0[0] + (double)rc.x * ud, gy = SP.c0[1] + (double)rc.y * ud,
                         gz = SP.c0[2] + (double)rc.z * ud;
            // the group's bounding box
            float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
#pragma unroll
            for (int b = 0; b < B; b++) {
                const int i = gfirst + lane + 32 * b;
                if (i < gend) {
                    const float4 qb = a.body[i];
                    lo[0] = fminf(lo[0], qb.x); hi[0] = fmaxf(hi[0], qb.x);
                    lo[1] = fminf(lo[1], qb.y); hi[1] = fmaxf(hi[1], qb.y);
                    lo[2] = fminf(lo[2], qb.z); hi[2] = fmaxf(hi[2], qb.z);
                }
            }
#pragma unroll
            for (int kk = 0; kk < 3; kk++) {
#pragma unroll
                for (int o = 16; o; o >>= 1) {
                    lo[kk] = fminf(lo[kk], __shfl_xor_sync(0xffffffffu, lo[kk], o));
                    hi[kk] = fmaxf(hi[kk], __shfl_xor_sync(0xffffffffu, hi[kk], o));
                }
            }
            // box relative to the reference centre: integer part (units of
            // u) + float remainder; lane k < 6 splits one bound
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
            float klof[3], khif[3], flo[3], fhi[3];
            const float rcf[3] = {(float)rc.x, (float)rc.y, (float)rc.z};
#pragma unroll
            for (int kk = 0; kk < 3; kk++) {
                klof[kk] = (float)__shfl_sync(0xffffffffu, kb, kk);
                khif[kk] = (float)__shfl_sync(0xffffffffu, kb, kk + 3);
                flo[kk] = __shfl_sync(0xffffffffu, fb, kk);
                fhi[kk] = __shfl_sync(0xffffffffu, fb, kk + 3);
            }
            if (LEARNED && lane == 0) {
                // the group's record: box centre, reference-relative (as
                // k_walk forms it), and the frame the network's rows need
                float xc[3];
#pragma unroll
                for (int kk = 0; kk < 3; kk++) xc[kk] = 0.5f * (fmaf(klof[kk], uf, flo[kk]) + fmaf(khif[kk], uf, fhi[kk]));
                a.grec[2 * (int64_t)g] = make_float4(xc[0], xc[1], xc[2], uf);
                a.grec[2 * (int64_t)g + 1] =
                    make_float4(__int_as_float(rc.x), __int_as_float(rc.y), __int_as_float(rc.z), Lf);
            }
            if (!take()) {
                alive = false;
                break;
            }
            open_slot(kWsFirst, g);
            if (lane == 0) {
                WsHdr* h = slot_hdr(k);
                h->gfirst = gfirst;
                h->gend = gend;
                h->ref[0] = gx;
                h->ref[1] = gy;
                h->ref[2] = gz;
            }
            float* ctile = slot_cells(k);
            float* btile = slot_bodies(k);
            int cn = 0, bn = 0, Lc = 0, Lb = 0;
            unsigned long long hsh = 0;
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
                        for (int kk = 0; kk < 3; kk++) {
                            const float lo_c = fmaf(klof[kk] - D[kk], uf, flo[kk]);
                            const float hi_c = fmaf(khif[kk] - D[kk], uf, fhi[kk]);
                            const float e = fmaxf(fmaxf(lo_c - off[kk], off[kk] - hi_c), 0.f);
                            e2 = fmaf(e, e, e2);
                        }
                        const float sz = pow2_down(Lf, nb.w & 255, fast_side);
                        acc = (sz * sz) < a.theta2 * e2;
                        band_e2 = e2;
                        if (acc) {
                            if (PRECISE) {
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
                const int npush = oint ? (nb.w >> 8) : 0;
                int tot;
                const int excl = warp_excl_small(npush, lt, tot);
                if (sp + tot > stack_cap) {
                    overflow = true;
                    break;
                }
                for (int c = 0; c < npush; c++) stk[sp + excl + c] = (uint32_t)(nb.z + c);
                sp += tot;
                // accepted cells -> the slot's cell part
                const unsigned am = __ballot_sync(0xffffffffu, acc);
                if (acc) {
                    put_entry(ctile, cn + __popc(am & lt), src);
                    if (list_stats) hsh += mix64(2ull * (unsigned)v + 1ull);
                }
                cn += __popc(am);
                Lc += __popc(am);
                if (LEARNED) {
                    bool band = false;
                    if (acc && nb.y >= 2) {
                        const float sz = pow2_down(Lf, nb.w & 255, fast_side);
                        band = sz * sz >= a.band2 * band_e2;
                    }
                    band_append(band, v, g);
                }
                // opened leaves -> the slot's body part, 32 bodies at a time
                const unsigned lm = __ballot_sync(0xffffffffu, oleaf);
                if (lm) {
                    if (list_stats && oleaf) hsh += mix64(2ull * (unsigned)v + 2ull);
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
                            hand_over(0, cn, bn);
                            if (!take()) {
                                alive = false;
                                break;
                            }
                            open_slot(0, g);
                            ctile = slot_cells(k);
                            btile = slot_bodies(k);
                            cn = bn = 0;
                        }
                    }
                    if (!alive) break;
                }
                __syncwarp();
                if (cn >= kTile) {
                    hand_over(0, cn, bn);
                    if (!take()) {
                        alive = false;
                        break;
                    }
                    open_slot(0, g);
                    ctile = slot_cells(k);
                    btile = slot_bodies(k);
                    cn = bn = 0;
                }
            }
            if (!alive) break;
            if (overflow) {
                if (lane == 0) atomicOr(&a.info->err, kErrStack);
                hand_over(kWsLast | kWsAbort, 0, 0);
                continue;
            }
            hand_over(kWsLast, cn, bn);
            if (list_stats) {
#pragma unroll
                for (int o = 16; o; o >>= 1) hsh += __shfl_xor_sync(0xffffffffu, hsh, o);
            }
            if (lane == 0) {
                const int gc = gend - gfirst;
                atomicAdd(&a.info->interactions, (unsigned long long)gc * (unsigned long long)(Lc + Lb));
                atomicAdd(&a.info->cells, (unsigned long long)gc * (unsigned long long)Lc);
                atomicAdd(&a.info->bodies, (unsigned long long)gc * (unsigned long long)Lb);
                if (a.ncell) a.ncell[g] = Lc;
                if (a.nbody) a.nbody[g] = Lb;
                if (a.hash) a.hash[g] = hsh;
            }
            __syncwarp();
        }
        (void)alive;
        cp_async_wait_all();  // (a warp that gave up may still have copies in flight)
        return;
    }

    // ---------------------------------------------------------------- consumer
    constexpr int kUnroll = B >= 4 ? 4 : 8;
    const f2 E2 = f2pack(a.eps2, a.eps2);
    f2 XA[B], YA[B], ZA[B], XR[B], YR[B], ZR[B];
    float mi[B];
    bool act[B];
#pragma unroll
    for (int b = 0; b < B; b++) {
        XA[b] = YA[b] = ZA[b] = XR[b] = YR[b] = ZR[b] = 0ull;
        mi[b] = 0.f;
        act[b] = false;
    }
    int gfirst = 0;
    Accum<B, PRECISE, POT, kUnroll> fsum;
    fsum.init();
    for (int k = 0;; k++) {
        if (!mbar_wait(&full[k % kWsSlots], (k / kWsSlots) & 1)) {
            if (lane == 0) atomicOr(&a.info->err, kErrWorkLoop);
            return;
        }
        const WsHdr* h = slot_hdr(k);
        const int flags = h->flags;
        if (flags & kWsDone) return;
        const int cn = h->cn, bn = h->bn;
        if (flags & kWsFirst) {
            gfirst = h->gfirst;
            const int gend = h->gend;
            const double gx = h->ref[0], gy = h->ref[1], gz = h->ref[2];
#pragma unroll
            for (int b = 0; b < B; b++) {
                const int i = gfirst + lane + 32 * b;
                act[b] = i < gend;
                const float4 qb = a.body[act[b] ? i : gfirst];
                XA[b] = f2pack(qb.x, qb.x);
                YA[b] = f2pack(qb.y, qb.y);
                ZA[b] = f2pack(qb.z, qb.z);
                mi[b] = qb.w;
                if (PRECISE) {
                    const float rx = (float)((double)qb.x - gx), ry = (float)((double)qb.y - gy),
                                rz = (float)((double)qb.z - gz);
                    XR[b] = f2pack(rx, rx);
                    YR[b] = f2pack(ry, ry);
                    ZR[b] = f2pack(rz, rz);
                }
            }
            fsum.init();
        }
        float* ct = slot_cells(k);
        float* bt = slot_bodies(k);
        if (PRECISE) fsum.flush(ct, cn, XR, YR, ZR, E2);
        else fsum.flush(ct, cn, XA, YA, ZA, E2);
        fsum.flush(bt, bn, XA, YA, ZA, E2);
        __syncwarp();
        mbar_arrive(&empty[k % kWsSlots]);
        if ((flags & kWsLast) && !(flags & kWsAbort)) {
#pragma unroll
            for (int b = 0; b < B; b++) {
                if (!act[b]) continue;
                const int i = gfirst + lane + 32 * b;
                const int64_t o = a.perm[i];
                float sx_, sy_, sz_, sp_, kx, ky, kz, kp;
                fsum.result(b, sx_, sy_, sz_, sp_);
                fsum.comp(b, kx, ky, kz, kp);
                a.acc[3 * o + 0] = a.G * (sx_ + kx);
                a.acc[3 * o + 1] = a.G * (sy_ + ky);
                a.acc[3 * o + 2] = a.G * (sz_ + kz);
                if (POT) {
                    const float self = mi[b] * rsqrtf(a.eps2);
                    a.pot[o] = a.G * ((sp_ + kp) + self);
                }
            }
        }
    }
}

template <int B, int TILE, bool PRECISE, bool POT, bool LEARNED>
cudaError_t prepare_ws_t(const WalkConfig& c, int num_sms, int* grid, size_t* smem_out)
{
    const int pairs = c.warps < 1 ? 1 : (c.warps > kWsMaxPairs ? kWsMaxPairs : c.warps);
    const size_t smem = ws_pair_bytes(TILE, c.stack) * pairs;
    auto kern = k_walk_ws<B, TILE, PRECISE, POT, LEARNED>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, pairs * 64, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if (c.blocks_per_sm > 0 && c.blocks_per_sm < per_sm) per_sm = c.blocks_per_sm;
    *grid = num_sms * per_sm;
    *smem_out = smem;
    return cudaSuccess;
}

template <int B, int TILE, bool PRECISE, bool POT, bool LEARNED>
cudaError_t launch_ws_t(const WalkArgs& a, const WalkConfig& c, int grid, size_t smem, cudaStream_t s)
{
    // the split walk has no list export, training pairs or quadrupole
    // terms (those run on k_walk); its learned walk records band cells
    if (a.list_cells || a.pair_body) return cudaErrorInvalidValue;
    if (LEARNED && (!a.band || !a.band_n || !a.grec)) return cudaErrorInvalidValue;
    const int pairs = c.warps < 1 ? 1 : (c.warps > kWsMaxPairs ? kWsMaxPairs : c.warps);
    k_walk_ws<B, TILE, PRECISE, POT, LEARNED><<<grid, pairs * 64, smem, s>>>(a, c.stack);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace

}  // namespace tc
