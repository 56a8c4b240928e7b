// tc_mlp.cu -- the learned far-field correction's network on the GPU:
// batch inference, training (forward, backward, Adam) and the exact labels
// of training pairs.
//
// Network: 13 -> 64 -> 64 -> 3, ReLU after the hidden layers, BF16 operands
// on the tensor cores (warp-level mma.sync m16n8k16), FP32 accumulation,
// FP32 master weights.  Every kernel works on 16-row tiles, one warp each.
//
// Training loss: L = (1/B) sum_i w_i |y_i - t_i|^2 over a mini-batch of B
// pairs (targets pre-divided by the output scale; w_i = 1 without weights).
// Backward, per 16-row tile:
//   dY = 2 w (Y - T) / B,  dW3 = H2^T dY,  dH2 = (dY W3^T) * [H2 > 0],
//   dW2 = H1^T dH2,      dH1 = (dH2 W2^T) * [H1 > 0],   dW1 = X^T dH1,
// biases by column sums; the transposed operands are staged in shared
// memory.  Gradients are summed per block in shared memory, then added to
// the global gradient; a separate kernel applies Adam.
#include <cuda_bf16.h>

#include "tc_internal.cuh"
#include "tc_mma.cuh"

namespace tc {

namespace {

constexpr int kTrainWarps = 4;

// padded gradient layout in shared memory
constexpr int kGW1 = 0;                                   // [16][64]
constexpr int kGB1 = kGW1 + kMlpInPad * kMlpHid;          // [64]
constexpr int kGW2 = kGB1 + kMlpHid;                      // [64][64]
constexpr int kGB2 = kGW2 + kMlpHid * kMlpHid;            // [64]
constexpr int kGW3 = kGB2 + kMlpHid;                      // [64][8]
constexpr int kGB3 = kGW3 + kMlpHid * kMlpOutPad;         // [8]
constexpr int kGPad = kGB3 + kMlpOutPad;

// per-warp staging (BF16): X[16][16], H1[16][64], H2[16][64], dY[16][8],
// dH2[16][64], dH1[16][64]
constexpr int kStX = 0;
constexpr int kStH1 = kStX + 16 * kMlpInPad;
constexpr int kStH2 = kStH1 + 16 * kMlpHid;
constexpr int kStDY = kStH2 + 16 * kMlpHid;
constexpr int kStDH2 = kStDY + 16 * kMlpOutPad;
constexpr int kStDH1 = kStDH2 + 16 * kMlpHid;
constexpr int kStSize = kStDH1 + 16 * kMlpHid;

// store a C tile (16 x 8, column block nb) into a row-major BF16 matrix
__device__ __forceinline__ void store_c(__nv_bfloat16* M, int ld, int nb, const float (&c)[4], int lane)
{
    const int g = lane >> 2, q = lane & 3;
    M[g * ld + nb * 8 + 2 * q] = __float2bfloat16_rn(c[0]);
    M[g * ld + nb * 8 + 2 * q + 1] = __float2bfloat16_rn(c[1]);
    M[(g + 8) * ld + nb * 8 + 2 * q] = __float2bfloat16_rn(c[2]);
    M[(g + 8) * ld + nb * 8 + 2 * q + 1] = __float2bfloat16_rn(c[3]);
}

// A fragment of the transpose of a row-major BF16 matrix S (S is k x m:
// A[m][k] = S[k][m]), m-tile mt, one 16-deep k-step at k = 0
__device__ __forceinline__ void load_at(uint32_t (&a)[4], const __nv_bfloat16* S, int ld, int mt, int lane)
{
    const int g = lane >> 2, q = lane & 3;
    const int m0 = mt * 16 + g, k0 = 2 * q;
    a[0] = pack_raw(S[k0 * ld + m0], S[(k0 + 1) * ld + m0]);
    a[1] = pack_raw(S[k0 * ld + m0 + 8], S[(k0 + 1) * ld + m0 + 8]);
    a[2] = pack_raw(S[(k0 + 8) * ld + m0], S[(k0 + 9) * ld + m0]);
    a[3] = pack_raw(S[(k0 + 8) * ld + m0 + 8], S[(k0 + 9) * ld + m0 + 8]);
}

// B fragment of a row-major BF16 matrix S (B[k][n] = S[k][n]), k-step 0,
// column block nb
__device__ __forceinline__ void load_bs(uint32_t (&b)[2], const __nv_bfloat16* S, int ld, int nb, int lane)
{
    const int g = lane >> 2, q = lane & 3;
    const int n = nb * 8 + g, k = 2 * q;
    b[0] = pack_raw(S[k * ld + n], S[(k + 1) * ld + n]);
    b[1] = pack_raw(S[(k + 8) * ld + n], S[(k + 9) * ld + n]);
}

// B fragment of the transpose of a k-major weight W[n][k] (B[k][n] = W[n][k]
// with W stored [n][ldk]), k-step ks, column block nb
__device__ __forceinline__ void load_bt(uint32_t (&b)[2], const __nv_bfloat16* W, int ldk, int ks, int nb, int lane)
{
    const int g = lane >> 2, q = lane & 3;
    const int n = nb * 8 + g, k = ks * 16 + 2 * q;
    b[0] = pack_raw(W[n * ldk + k], W[n * ldk + k + 1]);
    b[1] = pack_raw(W[n * ldk + k + 8], W[n * ldk + k + 9]);
}

// G is the warp's own partial gradient: each element always belongs to the
// same lane, so the sums are plain additions in the warp's order of tiles
__device__ __forceinline__ void add_c(float* G, int ld, int mt, int nb, const float (&c)[4], int lane)
{
    const int g = lane >> 2, q = lane & 3;
    const int r = mt * 16 + g, col = nb * 8 + 2 * q;
    G[r * ld + col] += c[0];
    G[r * ld + col + 1] += c[1];
    G[(r + 8) * ld + col] += c[2];
    G[(r + 8) * ld + col + 1] += c[3];
}

// column sums of a C tile over its 16 rows into G[col]
__device__ __forceinline__ void colsum_c(float* G, int nb, const float (&c)[4], int lane)
{
    float s0 = c[0] + c[2], s1 = c[1] + c[3];
#pragma unroll
    for (int o = 4; o < 32; o <<= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    }
    if (lane < 4) {
        G[nb * 8 + 2 * lane] += s0;
        G[nb * 8 + 2 * lane + 1] += s1;
    }
}

// X: n x 16 normalised features (FP32, padding zero); T: n x 3 scaled
// targets; W: n weights (nullable); idx: the batch's row indices (B of
// them).  Every warp sums its tiles' gradient into its own partial (part,
// kGPad floats per warp of the grid) and its loss into lpart; k_grad_reduce
// adds the partials in warp order, so a training run repeats bit for bit.
__global__ void __launch_bounds__(kTrainWarps * 32) k_mlp_train(const float* __restrict__ X,
                                                                 const float* __restrict__ T,
                                                                 const float* __restrict__ W,
                                                                 const int32_t* __restrict__ idx, int B,
                                                                 const MlpDev* __restrict__ model,
                                                                 float* __restrict__ part, float* __restrict__ lpart)
{
    extern __shared__ __align__(16) unsigned char smem[];
    MlpDev& m = *reinterpret_cast<MlpDev*>(smem);
    __nv_bfloat16* stage = reinterpret_cast<__nv_bfloat16*>(smem + sizeof(MlpDev));
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __nv_bfloat16* st = stage + w * kStSize;
    float* gs = part + ((int64_t)blockIdx.x * kTrainWarps + w) * kGPad;  // this warp's partial
    for (int i = threadIdx.x; i < (int)(sizeof(MlpDev) / 4); i += blockDim.x)
        reinterpret_cast<uint32_t*>(&m)[i] = reinterpret_cast<const uint32_t*>(model)[i];
    for (int i = lane; i < kGPad; i += 32) gs[i] = 0.f;
    __syncthreads();
    const int g = lane >> 2, q = lane & 3;
    const float inv_b = 1.0f / (float)B;
    float lsum = 0.f;
    const int ntiles = (B + 15) / 16;
    for (int tile = blockIdx.x * kTrainWarps + w; tile < ntiles; tile += gridDim.x * kTrainWarps) {
        // rows of this tile (a row past B is all zero and has zero gradient)
        const int r0 = tile * 16 + g, r1 = r0 + 8;
        const bool v0 = r0 < B, v1 = r1 < B;
        const int64_t i0 = v0 ? idx[r0] : 0, i1 = v1 ? idx[r1] : 0;
        uint32_t x[4];
        {
            float a0 = v0 ? X[i0 * kMlpInPad + 2 * q] : 0.f, a1 = v0 ? X[i0 * kMlpInPad + 2 * q + 1] : 0.f;
            float a2 = v1 ? X[i1 * kMlpInPad + 2 * q] : 0.f, a3 = v1 ? X[i1 * kMlpInPad + 2 * q + 1] : 0.f;
            float a4 = v0 ? X[i0 * kMlpInPad + 2 * q + 8] : 0.f, a5 = v0 ? X[i0 * kMlpInPad + 2 * q + 9] : 0.f;
            float a6 = v1 ? X[i1 * kMlpInPad + 2 * q + 8] : 0.f, a7 = v1 ? X[i1 * kMlpInPad + 2 * q + 9] : 0.f;
            x[0] = pack_bf16(a0, a1);
            x[1] = pack_bf16(a2, a3);
            x[2] = pack_bf16(a4, a5);
            x[3] = pack_bf16(a6, a7);
            // X tile, row-major, for dW1 = X^T dH1
            st[kStX + g * 16 + 2 * q] = __float2bfloat16_rn(a0);
            st[kStX + g * 16 + 2 * q + 1] = __float2bfloat16_rn(a1);
            st[kStX + (g + 8) * 16 + 2 * q] = __float2bfloat16_rn(a2);
            st[kStX + (g + 8) * 16 + 2 * q + 1] = __float2bfloat16_rn(a3);
            st[kStX + g * 16 + 2 * q + 8] = __float2bfloat16_rn(a4);
            st[kStX + g * 16 + 2 * q + 9] = __float2bfloat16_rn(a5);
            st[kStX + (g + 8) * 16 + 2 * q + 8] = __float2bfloat16_rn(a6);
            st[kStX + (g + 8) * 16 + 2 * q + 9] = __float2bfloat16_rn(a7);
        }
        float h1[8][4], h2[8][4], y[4];
        mlp16(m, x, h1, h2, y, lane);
        // dY = 2 w (Y - T) / B on the 3 used columns of valid rows
        float dy[4] = {0.f, 0.f, 0.f, 0.f};
        {
            const int c0 = 2 * q, c1 = 2 * q + 1;
            const float w0 = (W && v0) ? W[i0] : 1.f, w1 = (W && v1) ? W[i1] : 1.f;
            if (v0 && c0 < 3) { const float e = y[0] - T[i0 * 3 + c0]; lsum += w0 * e * e; dy[0] = 2.f * w0 * e * inv_b; }
            if (v0 && c1 < 3) { const float e = y[1] - T[i0 * 3 + c1]; lsum += w0 * e * e; dy[1] = 2.f * w0 * e * inv_b; }
            if (v1 && c0 < 3) { const float e = y[2] - T[i1 * 3 + c0]; lsum += w1 * e * e; dy[2] = 2.f * w1 * e * inv_b; }
            if (v1 && c1 < 3) { const float e = y[3] - T[i1 * 3 + c1]; lsum += w1 * e * e; dy[3] = 2.f * w1 * e * inv_b; }
        }
        for (int nb = 0; nb < 8; nb++) {
            store_c(st + kStH1, kMlpHid, nb, h1[nb], lane);
            store_c(st + kStH2, kMlpHid, nb, h2[nb], lane);
        }
        store_c(st + kStDY, kMlpOutPad, 0, dy, lane);
        __syncwarp();
        colsum_c(gs + kGB3, 0, dy, lane);
        // dW3 = H2^T dY
        for (int mt = 0; mt < 4; mt++) {
            uint32_t a[4], b[2];
            load_at(a, st + kStH2, kMlpHid, mt, lane);
            load_bs(b, st + kStDY, kMlpOutPad, 0, lane);
            float c[4] = {0.f, 0.f, 0.f, 0.f};
            mma_bf16(c, a, b);
            add_c(gs + kGW3, kMlpOutPad, mt, 0, c, lane);
        }
        // dH2 = dY W3^T * [H2 > 0]; dY padded to a 16-deep k-step with zeros
        float dh2[8][4];
        {
            uint32_t a[4];
            a[0] = pack_bf16(dy[0], dy[1]);
            a[1] = pack_bf16(dy[2], dy[3]);
            a[2] = 0u;
            a[3] = 0u;
            for (int nb = 0; nb < 8; nb++) {
                const int n = nb * 8 + g, k = 2 * q;
                uint32_t b[2];
                b[0] = pack_raw(m.w3[n * kMlpOutPad + k], m.w3[n * kMlpOutPad + k + 1]);
                b[1] = 0u;
                dh2[nb][0] = dh2[nb][1] = dh2[nb][2] = dh2[nb][3] = 0.f;
                mma_bf16(dh2[nb], a, b);
#pragma unroll
                for (int e = 0; e < 4; e++) dh2[nb][e] = h2[nb][e] > 0.f ? dh2[nb][e] : 0.f;
                store_c(st + kStDH2, kMlpHid, nb, dh2[nb], lane);
                colsum_c(gs + kGB2, nb, dh2[nb], lane);
            }
        }
        __syncwarp();
        // dW2 = H1^T dH2
        for (int mt = 0; mt < 4; mt++) {
            uint32_t a[4];
            load_at(a, st + kStH1, kMlpHid, mt, lane);
            for (int nb = 0; nb < 8; nb++) {
                uint32_t b[2];
                load_bs(b, st + kStDH2, kMlpHid, nb, lane);
                float c[4] = {0.f, 0.f, 0.f, 0.f};
                mma_bf16(c, a, b);
                add_c(gs + kGW2, kMlpHid, mt, nb, c, lane);
            }
        }
        // dH1 = dH2 W2^T * [H1 > 0]
        float dh1[8][4];
        for (int nb = 0; nb < 8; nb++) dh1[nb][0] = dh1[nb][1] = dh1[nb][2] = dh1[nb][3] = 0.f;
        for (int ks = 0; ks < 4; ks++) {
            uint32_t a[4];
            c_to_a(a, dh2[2 * ks], dh2[2 * ks + 1]);
            for (int nb = 0; nb < 8; nb++) {
                uint32_t b[2];
                load_bt(b, m.w2, kMlpHid, ks, nb, lane);
                mma_bf16(dh1[nb], a, b);
            }
        }
        for (int nb = 0; nb < 8; nb++) {
#pragma unroll
            for (int e = 0; e < 4; e++) dh1[nb][e] = h1[nb][e] > 0.f ? dh1[nb][e] : 0.f;
            store_c(st + kStDH1, kMlpHid, nb, dh1[nb], lane);
            colsum_c(gs + kGB1, nb, dh1[nb], lane);
        }
        __syncwarp();
        // dW1 = X^T dH1
        {
            uint32_t a[4];
            load_at(a, st + kStX, kMlpInPad, 0, lane);
            for (int nb = 0; nb < 8; nb++) {
                uint32_t b[2];
                load_bs(b, st + kStDH1, kMlpHid, nb, lane);
                float c[4] = {0.f, 0.f, 0.f, 0.f};
                mma_bf16(c, a, b);
                add_c(gs + kGW1, kMlpHid, 0, nb, c, lane);
            }
        }
        __syncwarp();
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if (lane == 0) lpart[(int64_t)blockIdx.x * kTrainWarps + w] = lsum * inv_b;
}

// the partials of nw warps, added in one fixed order, into the packed
// gradient (W1[13][64], b1, W2, b2, W3[64][3], b3) and the loss (element
// kMlpNParam, added to *loss).  A block takes 32 elements; its 8 warps sum
// the warps k = y, y + 8, ... in turn, and warp 0 adds the 8 sums in order.
constexpr int kReduceSlices = 8;
__global__ void __launch_bounds__(32 * kReduceSlices) k_grad_reduce(const float* __restrict__ part,
                                                                    const float* __restrict__ lpart, int nw,
                                                                    float* __restrict__ grad, float* __restrict__ loss)
{
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int e = blockIdx.x * 32 + tx;
    // packed index -> the padded index of a warp's partial (stride kGPad),
    // or the loss partials (stride 1)
    const float* src = nullptr;
    int64_t stride = kGPad;
    constexpr int kB1 = kMlpIn * kMlpHid, kW2 = kB1 + kMlpHid, kB2 = kW2 + kMlpHid * kMlpHid;
    constexpr int kW3 = kB2 + kMlpHid, kB3 = kW3 + kMlpHid * kMlpOut;
    static_assert(kB3 + kMlpOut == kMlpNParam, "packed gradient layout");
    if (e < kB1) src = part + kGW1 + e;
    else if (e < kW2) src = part + kGB1 + (e - kB1);
    else if (e < kB2) src = part + kGW2 + (e - kW2);
    else if (e < kW3) src = part + kGB2 + (e - kB2);
    else if (e < kB3) src = part + kGW3 + ((e - kW3) / kMlpOut) * kMlpOutPad + ((e - kW3) % kMlpOut);
    else if (e < kMlpNParam) src = part + kGB3 + (e - kB3);
    else if (e == kMlpNParam) { src = lpart; stride = 1; }
    float s = 0.f;
    if (src)
        for (int k = ty; k < nw; k += kReduceSlices) s += src[(int64_t)k * stride];
    __shared__ float red[kReduceSlices][33];
    red[ty][tx] = s;
    __syncthreads();
    if (ty == 0 && src) {
        float t = red[0][tx];
#pragma unroll
        for (int j = 1; j < kReduceSlices; j++) t += red[j][tx];
        if (e < kMlpNParam) grad[e] = t;
        else *loss += t;
    }
}

// packed FP32 parameters + feature/output maps -> device BF16 model: the
// k-major weights for training and the fragment-arranged inference copy
__global__ void k_mlp_pack(const float* __restrict__ p, const float* __restrict__ maps, MlpDev* __restrict__ m)
{
    const float* W1 = p;
    const float* b1 = W1 + kMlpIn * kMlpHid;
    const float* W2 = b1 + kMlpHid;
    const float* b2 = W2 + kMlpHid * kMlpHid;
    const float* W3 = b2 + kMlpHid;
    const float* b3 = W3 + kMlpHid * kMlpOut;
    // padded weights: input rows past 13 and output columns past 3 are zero
    auto w1 = [&](int k, int n) { return k < kMlpIn ? W1[k * kMlpHid + n] : 0.f; };
    auto w3 = [&](int k, int n) { return n < kMlpOut ? W3[k * kMlpOut + n] : 0.f; };
    auto bf = [](float lo, float hi) {
        __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
        return *reinterpret_cast<uint32_t*>(&v);
    };
    for (int i = threadIdx.x; i < kMlpInPad * kMlpHid; i += blockDim.x)
        m->w1[i] = __float2bfloat16_rn(w1(i / kMlpHid, i % kMlpHid));
    for (int i = threadIdx.x; i < kMlpHid * kMlpHid; i += blockDim.x) m->w2[i] = __float2bfloat16_rn(W2[i]);
    for (int i = threadIdx.x; i < kMlpHid * kMlpOutPad; i += blockDim.x)
        m->w3[i] = __float2bfloat16_rn(w3(i / kMlpOutPad, i % kMlpOutPad));
    // B fragments: lane (g, q) of column block nb, k-step ks holds
    // {W[16 ks + 2q][n], W[16 ks + 2q + 1][n]}, {W[16 ks + 2q + 8][n], W[16 ks + 2q + 9][n]}, n = 8 nb + g
    MlpFrag& f = m->frag;
    for (int i = threadIdx.x; i < 8 * 32; i += blockDim.x) {
        const int nb = i / 32, lane = i % 32, g = lane >> 2, q = lane & 3, n = nb * 8 + g, k = 2 * q;
        f.f1[nb][lane] = make_uint2(bf(w1(k, n), w1(k + 1, n)), bf(w1(k + 8, n), w1(k + 9, n)));
    }
    for (int i = threadIdx.x; i < 4 * 8 * 32; i += blockDim.x) {
        const int ks = i / 256, nb = (i / 32) % 8, lane = i % 32, g = lane >> 2, q = lane & 3;
        const int n = nb * 8 + g, k = ks * 16 + 2 * q;
        f.f2[ks][nb][lane] = make_uint2(bf(W2[k * kMlpHid + n], W2[(k + 1) * kMlpHid + n]),
                                        bf(W2[(k + 8) * kMlpHid + n], W2[(k + 9) * kMlpHid + n]));
    }
    for (int i = threadIdx.x; i < 4 * 32; i += blockDim.x) {
        const int ks = i / 32, lane = i % 32, g = lane >> 2, q = lane & 3, k = ks * 16 + 2 * q;
        f.f3[ks][lane] = make_uint2(bf(w3(k, g), w3(k + 1, g)), bf(w3(k + 8, g), w3(k + 9, g)));
    }
    for (int i = threadIdx.x; i < kMlpHid; i += blockDim.x) {
        m->b1[i] = b1[i];
        m->b2[i] = b2[i];
    }
    for (int i = threadIdx.x; i < 32; i += blockDim.x) {
        const int nb = i / 4, q = i % 4;
        f.b1[nb][q] = make_float2(b1[nb * 8 + 2 * q], b1[nb * 8 + 2 * q + 1]);
        f.b2[nb][q] = make_float2(b2[nb * 8 + 2 * q], b2[nb * 8 + 2 * q + 1]);
    }
    for (int i = threadIdx.x; i < kMlpOutPad; i += blockDim.x) {
        m->b3[i] = i < kMlpOut ? b3[i] : 0.f;
        f.yscale[i] = i < kMlpOut ? maps[2 * kMlpIn + i] : 0.f;
    }
    for (int i = threadIdx.x; i < 4; i += blockDim.x)
        f.b3[i] = make_float2(2 * i < kMlpOut ? b3[2 * i] : 0.f, 2 * i + 1 < kMlpOut ? b3[2 * i + 1] : 0.f);
    for (int i = threadIdx.x; i < kMlpInPad; i += blockDim.x) {
        f.xscale[i] = i < kMlpIn ? maps[kMlpIn + i] : 0.f;
        f.xoff[i] = i < kMlpIn ? -maps[i] * maps[kMlpIn + i] : 0.f;
    }
}

// Adam on the FP32 master parameters
__global__ void k_adam(float* __restrict__ p, float* __restrict__ mom, float* __restrict__ vel,
                       const float* __restrict__ g, int n, float lr, float b1, float b2, float eps, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * mom[i] + (1.f - b1) * gi;
    const float vi = b2 * vel[i] + (1.f - b2) * gi * gi;
    mom[i] = mi;
    vel[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// batch inference: Y (n x 3) = network(X) * yscale, X normalised n x 16 --
// the same fragment path the walk evaluates its corrections with
__global__ void __launch_bounds__(128) k_mlp_infer(const float* __restrict__ X, int64_t n,
                                                   const MlpDev* __restrict__ model, float* __restrict__ Y)
{
    __shared__ MlpFrag m;
    for (int i = threadIdx.x; i < (int)(sizeof(MlpFrag) / 4); i += blockDim.x)
        reinterpret_cast<uint32_t*>(&m)[i] = reinterpret_cast<const uint32_t*>(&model->frag)[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int g = lane >> 2, q = lane & 3;
    const int64_t ntiles = (n + 15) / 16;
    for (int64_t tile = (int64_t)blockIdx.x * 4 + w; tile < ntiles; tile += (int64_t)gridDim.x * 4) {
        const int64_t r0 = tile * 16 + g, r1 = r0 + 8;
        const bool v0 = r0 < n, v1 = r1 < n;
        auto xv = [&](int64_t r, bool v, int c) { return v ? X[r * kMlpInPad + c] : 0.f; };
        uint32_t x[4];
        x[0] = pack_bf16(xv(r0, v0, 2 * q), xv(r0, v0, 2 * q + 1));
        x[1] = pack_bf16(xv(r1, v1, 2 * q), xv(r1, v1, 2 * q + 1));
        x[2] = pack_bf16(xv(r0, v0, 2 * q + 8), xv(r0, v0, 2 * q + 9));
        x[3] = pack_bf16(xv(r1, v1, 2 * q + 8), xv(r1, v1, 2 * q + 9));
        float y[4];
        mlp16_infer(m, x, y, lane);
        const int c0 = 2 * q, c1 = 2 * q + 1;
        if (v0 && c0 < 3) Y[r0 * 3 + c0] = y[0] * m.yscale[c0];
        if (v0 && c1 < 3) Y[r0 * 3 + c1] = y[1] * m.yscale[c1];
        if (v1 && c0 < 3) Y[r1 * 3 + c0] = y[2] * m.yscale[c0];
        if (v1 && c1 < 3) Y[r1 * 3 + c1] = y[3] * m.yscale[c1];
    }
}

// Features, exact label and label factor of (body, cell) pairs, one thread
// per pair: features at the body's position; factor F = G M s^2 / r^4 (the
// scale of the quadrupole term); label = (a_exact - a_mono) / F with a_exact
// the softened sum over the cell's bodies (FP64 accumulation).
__global__ void k_pair_labels(const int32_t* __restrict__ pb, const int32_t* __restrict__ pv, int64_t np,
                              const float4* __restrict__ body, const uint32_t* __restrict__ sys_of,
                              const SysParams* __restrict__ sysp, NodeTables nt, float eps, float G,
                              float* __restrict__ feat, float* __restrict__ lab, float* __restrict__ fac)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= np) return;
    const int64_t ib = pb[k], v = pv[k];
    const float4 xb = body[ib];
    const double x[3] = {xb.x, xb.y, xb.z};
    const int4 b = nt.b[v];
    const int4 cc = nt.c[v];
    const SysParams& P = sysp[cc.w];
    const double s = ldexp(P.L, -(b.w & 255));
    const double M = nt.mass64[v];
    const double* com = &nt.com64[3 * v];
    double d[3], r2 = 0.0;
    for (int a = 0; a < 3; a++) {
        d[a] = com[a] - x[a];
        r2 += d[a] * d[a];
    }
    const double r = sqrt(r2);
    float* f = feat + k * kMlpIn;
    for (int a = 0; a < 3; a++) f[a] = (float)(d[a] / s);
    f[3] = (float)(s / r);
    f[4] = (float)(eps / s);
    f[5] = (float)log2((double)b.y);
    f[6] = (float)(M / nt.mass64[cc.w]);  // the system's root is node cc.w
    for (int q = 0; q < 6; q++) f[7 + q] = (float)((double)nt.quad[6 * v + q] / (M * s * s));
    const double e2 = (double)eps * (double)eps;
    double ae[3] = {0, 0, 0};
    for (int j = b.x; j < b.x + b.y; j++) {
        const float4 y = body[j];
        const double dx = (double)y.x - x[0], dy = (double)y.y - x[1], dz = (double)y.z - x[2];
        const double q2 = dx * dx + dy * dy + dz * dz + e2;
        const double ri = 1.0 / sqrt(q2);
        const double fm = (double)y.w * ri * ri * ri;
        ae[0] += fm * dx;
        ae[1] += fm * dy;
        ae[2] += fm * dz;
    }
    const double rm = 1.0 / sqrt(r2 + e2);
    const double fmo = M * rm * rm * rm;
    const double F = (double)G * M * s * s / (r2 * r2);
    for (int a = 0; a < 3; a++) lab[k * 3 + a] = (float)((double)G * (ae[a] - fmo * d[a]) / F);
    if (fac) fac[k] = (float)F;
}

// ---------------------------------------------------------------- node features
// The nine features of a cell that do not depend on the point it is
// evaluated at -- eps/s, log2(count), M / M_sys and the six moment ratios
// Q_ab / (M s^2) -- normalised with the model's maps and packed as BF16
// pairs in the order of a network row (words 2..7: features 4..12, then the
// zero padding), once per node and force phase, so a walk that evaluates a
// cell forms only d/s and s/r itself.
__global__ void k_node_features(const Info* info, const SysParams* __restrict__ sysp, NodeTables nt, float eps,
                                const MlpDev* __restrict__ model)
{
    if ((*(volatile const int32_t*)&info->err & kErrCapacity) != 0) return;
    const int64_t M = info->M;
    const MlpFrag& m = model->frag;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < M; v += (int64_t)gridDim.x * blockDim.x) {
        const int4 nb = nt.b[v];
        const float4 na = nt.a[v];
        const int4 cc = nt.c[v];
        const SysParams& P = sysp[cc.w];
        const int level = nb.w & 255;
        const float inv_s = scalbnf(1.0f / P.Lf, level);  // exact: sides are powers of two
        const float Mc = na.w;
        const float iq = __fdividef(inv_s * inv_s, Mc);
        const float* qd = nt.quad + 6 * v;
        float f[kMlpInPad];
#pragma unroll
        for (int k = 0; k < kMlpInPad; k++) f[k] = 0.f;
        f[4] = eps * inv_s;
        f[5] = __log2f((float)nb.y);
        f[6] = Mc * (1.0f / P.msys);
#pragma unroll
        for (int k = 0; k < 6; k++) f[7 + k] = qd[k] * iq;
#pragma unroll
        for (int k = 4; k < kMlpIn; k++) f[k] = fmaf(f[k], m.xscale[k], m.xoff[k]);
        nt.feat[2 * v] = make_uint4(pack_bf16(f[4], f[5]), pack_bf16(f[6], f[7]), pack_bf16(f[8], f[9]),
                                    pack_bf16(f[10], f[11]));
        nt.feat[2 * v + 1] = make_uint4(pack_bf16(f[12], 0.f), 0u, 0u, 0u);
    }
}

// ---------------------------------------------------------------- training data
// Sums over the n training pairs, in FP64: column c of blockIdx.y takes
//   c < 13: x_c,  13 <= c < 26: x_(c-13)^2,  26 <= c < 29: t_(c-26)^2,
//   c = 29: F^2 (the pairs' label factors; F null: skipped)
__global__ void k_mlp_sums(const float* __restrict__ X, const float* __restrict__ T, const float* __restrict__ F,
                           int64_t n, double* __restrict__ sums)
{
    const int c = blockIdx.y;
    if (c == kMlpSums - 1 && !F) return;
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double v;
        if (c < kMlpIn) v = X[i * kMlpIn + c];
        else if (c < 2 * kMlpIn) { v = X[i * kMlpIn + c - kMlpIn]; v *= v; }
        else if (c < 2 * kMlpIn + kMlpOut) { v = T[i * kMlpOut + c - 2 * kMlpIn]; v *= v; }
        else { v = F[i]; v *= v; }
        s += v;
    }
    __shared__ double red[32];
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) atomicAdd(&sums[c], s);
    }
}

// the model's maps from the sums: feature means and inverse standard
// deviations (0 for a constant feature), output RMS (1 for an all-zero
// output); and the factor-weight scale n / sum F^2
__global__ void k_mlp_maps(const double* __restrict__ sums, int64_t n, float* __restrict__ maps,
                           float* __restrict__ wscale)
{
    const int k = threadIdx.x;
    const double inv_n = 1.0 / (double)n;
    if (k < kMlpIn) {
        const double mean = sums[k] * inv_n;
        const double var = fmax(0.0, sums[kMlpIn + k] * inv_n - mean * mean);
        maps[k] = (float)mean;
        maps[kMlpIn + k] = var > 1e-30 ? (float)(1.0 / sqrt(var)) : 0.f;
    } else if (k < kMlpIn + kMlpOut) {
        const double rms = sqrt(sums[2 * kMlpIn + k - kMlpIn] * inv_n);
        maps[2 * kMlpIn + k - kMlpIn] = rms > 1e-30 ? (float)rms : 1.f;
    } else if (k == kMlpIn + kMlpOut) {
        const double s2 = sums[kMlpSums - 1];
        *wscale = s2 > 0.0 ? (float)((double)n / s2) : 0.f;
    }
}

// normalised padded rows (x - mean) * scale, each operation rounded on its
// own (no contraction), zero padding; targets t / yscale
__global__ void k_mlp_rows(const float* __restrict__ X, const float* __restrict__ T, int64_t n,
                           const float* __restrict__ maps, float* __restrict__ rows, float* __restrict__ tout)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * kMlpInPad;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / kMlpInPad;
        const int k = (int)(e % kMlpInPad);
        rows[e] = k < kMlpIn ? __fmul_rn(__fsub_rn(X[i * kMlpIn + k], maps[k]), maps[kMlpIn + k]) : 0.f;
        if (T && k < kMlpOut) tout[i * kMlpOut + k] = __fdiv_rn(T[i * kMlpOut + k], maps[2 * kMlpIn + k]);
    }
}

// loss weights in place: mode 0 checks the given weights (finite, >= 0;
// *bad = 1 otherwise), mode 1 turns label factors F into F^2 n / sum F^2
__global__ void k_mlp_weights(float* __restrict__ w, int64_t n, int mode, const float* __restrict__ wscale,
                              int32_t* __restrict__ bad)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float v = w[i];
        if (!isfinite(v) || (mode == 0 && v < 0.f)) {
            *bad = 1;
            continue;
        }
        if (mode == 1) w[i] = __fmul_rn(__fmul_rn(v, v), *wscale);
    }
}

// Fresh parameters: weights and biases of layer l uniform in +-1/sqrt(fan-in)
// from a counter-based generator (SplitMix64 of seed and index)
__device__ __forceinline__ uint64_t splitmix(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void k_mlp_init(float* __restrict__ p, uint64_t seed)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kMlpNParam) return;
    const int l1 = kMlpIn * kMlpHid + kMlpHid;
    const double fan = i < l1 ? (double)kMlpIn : (double)kMlpHid;
    const double u = (double)(splitmix(seed * 0x100000001B3ull + (uint64_t)i) >> 11) * (1.0 / 9007199254740992.0);
    p[i] = (float)((2.0 * u - 1.0) / sqrt(fan));
}

// A random permutation of [0, n) without sorting: a 4-round Feistel network
// is a bijection on [0, 4^h) (4^h >= n, h the half width in bits); walking
// its cycle from i until the value falls below n gives a bijection on
// [0, n) (the walk ends: the cycle through i < n returns to i).  Key 0
// gives the identity.
__device__ __forceinline__ uint32_t feistel(uint32_t x, int h, uint64_t key)
{
    const uint32_t mask = (1u << h) - 1u;
    uint32_t L = x >> h, R = x & mask;
#pragma unroll
    for (int r = 0; r < 4; r++) {
        const uint32_t f = (uint32_t)splitmix(key + 0x632BE59BD9B4E019ull * (uint64_t)r + R) & mask;
        const uint32_t t = L ^ f;
        L = R;
        R = t;
    }
    return (L << h) | R;
}

__global__ void k_mlp_shuffle(int64_t n, int h, uint64_t key, int32_t* __restrict__ idx)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t x = (uint32_t)i;
        if (key != 0) {
            do {
                x = feistel(x, h, key);
            } while ((int64_t)x >= n);
        }
        idx[i] = (int32_t)x;
    }
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

size_t mlp_train_smem() { return sizeof(MlpDev) + (size_t)kTrainWarps * kStSize * 2; }
int64_t mlp_train_part_floats(int blocks) { return (int64_t)blocks * kTrainWarps * (kGPad + 1); }

cudaError_t launch_mlp_train(const float* X, const float* T, const float* W, const int32_t* idx, int B,
                             const void* model, float* grad, float* loss, float* part, int blocks, cudaStream_t s)
{
    const size_t smem = mlp_train_smem();
    cudaError_t e = cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int nw = blocks * kTrainWarps;
    float* lpart = part + (int64_t)nw * kGPad;
    k_mlp_train<<<blocks, kTrainWarps * 32, smem, s>>>(X, T, W, idx, B, (const MlpDev*)model, part, lpart);
    k_grad_reduce<<<(kMlpNParam + 1 + 31) / 32, 32 * kReduceSlices, 0, s>>>(part, lpart, nw, grad, loss);
    count_launches(2);
    return cudaGetLastError();
}

void launch_mlp_pack(const float* params, const float* maps, void* model, cudaStream_t s)
{
    k_mlp_pack<<<1, 256, 0, s>>>(params, maps, (MlpDev*)model);
    count_launches(1);
}

void launch_adam(float* p, float* m, float* v, const float* g, int n, float lr, int t, cudaStream_t s)
{
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    k_adam<<<nblk(n, 256), 256, 0, s>>>(p, m, v, g, n, lr, b1, b2, 1e-8f, c1, c2);
    count_launches(1);
}

void launch_mlp_infer(const float* X, int64_t n, const void* model, float* Y, cudaStream_t s)
{
    int64_t g = (n + 63) / 64;
    if (g > 4096) g = 4096;
    k_mlp_infer<<<(unsigned)(g < 1 ? 1 : g), 128, 0, s>>>(X, n, (const MlpDev*)model, Y);
    count_launches(1);
}

namespace {
// (body, node) pairs as sort keys (body position in the high half) and back
__global__ void k_pair_keys(const int32_t* __restrict__ pb, const int32_t* __restrict__ pv, int64_t np,
                            uint64_t* __restrict__ keys, uint32_t* __restrict__ vals)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < np; k += (int64_t)gridDim.x * blockDim.x) {
        keys[k] = ((uint64_t)(uint32_t)pb[k] << 32) | (uint32_t)pv[k];
        vals[k] = (uint32_t)k;
    }
}

__global__ void k_pair_unkey(const uint64_t* __restrict__ keys, int64_t np, int32_t* __restrict__ pb,
                             int32_t* __restrict__ pv)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < np; k += (int64_t)gridDim.x * blockDim.x) {
        pb[k] = (int32_t)(keys[k] >> 32);
        pv[k] = (int32_t)(keys[k] & 0xffffffffu);
    }
}
}  // namespace

void launch_pair_order(int32_t* pb, int32_t* pv, int64_t np, uint64_t* keys, uint32_t* vals, SortBufs& b,
                       cudaStream_t s)
{
    int64_t g = nblk(np, 256);
    if (g > 8 * sm_count()) g = 8 * sm_count();
    k_pair_keys<<<(unsigned)(g < 1 ? 1 : g), 256, 0, s>>>(pb, pv, np, keys, vals);
    count_launches(1);
    radix_sort_u64(keys, vals, np, 63, nullptr, 0, b, s);
    k_pair_unkey<<<(unsigned)(g < 1 ? 1 : g), 256, 0, s>>>(keys, np, pb, pv);
    count_launches(1);
}

void launch_pair_labels(const int32_t* pb, const int32_t* pv, int64_t np, const float4* body, const uint32_t* sys_of,
                        const SysParams* sysp, NodeTables nt, float eps, float G, float* feat, float* lab,
                        float* fac, cudaStream_t s)
{
    k_pair_labels<<<nblk(np, 128), 128, 0, s>>>(pb, pv, np, body, sys_of, sysp, nt, eps, G, feat, lab, fac);
    count_launches(1);
}

void launch_mlp_sums(const float* X, const float* T, const float* F, int64_t n, double* sums, cudaStream_t s)
{
    // one block per column: each sum is taken in one fixed order, so the
    // maps (and the training that follows) repeat bit for bit
    cudaMemsetAsync(sums, 0, kMlpSums * sizeof(double), s);
    k_mlp_sums<<<dim3(1, kMlpSums), 1024, 0, s>>>(X, T, F, n, sums);
    count_launches(1);
}

void launch_mlp_maps(const double* sums, int64_t n, float* maps, float* wscale, cudaStream_t s)
{
    k_mlp_maps<<<1, 32, 0, s>>>(sums, n, maps, wscale);
    count_launches(1);
}

void launch_mlp_rows(const float* X, const float* T, int64_t n, const float* maps, float* rows, float* tout,
                     cudaStream_t s)
{
    int64_t g = (n * kMlpInPad + 255) / 256;
    if (g > 16 * sm_count()) g = 16 * sm_count();
    k_mlp_rows<<<(unsigned)(g < 1 ? 1 : g), 256, 0, s>>>(X, T, n, maps, rows, tout);
    count_launches(1);
}

void launch_mlp_weights(float* w, int64_t n, int mode, const float* wscale, int32_t* bad, cudaStream_t s)
{
    int64_t g = (n + 255) / 256;
    if (g > 16 * sm_count()) g = 16 * sm_count();
    k_mlp_weights<<<(unsigned)(g < 1 ? 1 : g), 256, 0, s>>>(w, n, mode, wscale, bad);
    count_launches(1);
}

void launch_mlp_init(float* params, uint64_t seed, cudaStream_t s)
{
    k_mlp_init<<<nblk(kMlpNParam, 256), 256, 0, s>>>(params, seed);
    count_launches(1);
}

void launch_mlp_shuffle(int64_t n, uint64_t key, int32_t* idx, cudaStream_t s)
{
    int h = 1;
    while (((int64_t)1 << (2 * h)) < n) h++;
    int64_t g = (n + 255) / 256;
    if (g > 16 * sm_count()) g = 16 * sm_count();
    k_mlp_shuffle<<<(unsigned)(g < 1 ? 1 : g), 256, 0, s>>>(n, h, key, idx);
    count_launches(1);
}

void launch_node_features(const Info* info, int64_t cap_m, const SysParams* sysp, NodeTables nt, float eps,
                          const void* model, cudaStream_t s)
{
    int64_t g = (cap_m + 255) / 256;
    if (g > 16 * sm_count()) g = 16 * sm_count();
    k_node_features<<<(unsigned)(g < 1 ? 1 : g), 256, 0, s>>>(info, sysp, nt, eps, (const MlpDev*)model);
    count_launches(1);
}

size_t mlp_dev_size() { return sizeof(MlpDev); }
size_t mlp_frag_size() { return sizeof(MlpFrag); }

}  // namespace tc
