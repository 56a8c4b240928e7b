// tc_mma.cuh -- warp-level BF16 tensor-core tile product (FP32 accumulate)
// and the 13 -> 64 -> 64 -> 3 MLP of the learned far-field correction.
//
// One mma.sync.m16n8k16 multiplies a 16x16 BF16 tile A (row-major) by a
// 16x8 BF16 tile B and adds into a 16x8 FP32 tile C.  Fragment ownership
// (PTX ISA, m16n8k16 with 16-bit operands), g = lane / 4, q = lane % 4:
//   A: {A[g][2q..2q+1], A[g+8][2q..2q+1], A[g][2q+8..2q+9], A[g+8][2q+8..2q+9]}
//   B: {B[2q..2q+1][g], B[2q+8..2q+9][g]}
//   C: {C[g][2q], C[g][2q+1], C[g+8][2q], C[g+8][2q+1]}
// so the C tiles of two neighbouring column blocks are exactly the A
// fragment of the next layer's 16-column k-step.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

namespace tc {

constexpr int kMlpIn = 13;
constexpr int kMlpInPad = 16;
constexpr int kMlpHid = 64;
constexpr int kMlpOut = 3;
constexpr int kMlpOutPad = 8;
constexpr int kMlpNParam = kMlpIn * kMlpHid + kMlpHid + kMlpHid * kMlpHid + kMlpHid + kMlpHid * kMlpOut + kMlpOut;

// Device copy of a model: BF16 weights laid out k-major ([in][out], padded),
// FP32 biases, and the affine maps of the features and of the output.
struct MlpDev {
    __nv_bfloat16 w1[kMlpInPad * kMlpHid];
    __nv_bfloat16 w2[kMlpHid * kMlpHid];
    __nv_bfloat16 w3[kMlpHid * kMlpOutPad];
    float b1[kMlpHid];
    float b2[kMlpHid];
    float b3[kMlpOutPad];
    float xmean[kMlpInPad];
    float xscale[kMlpInPad];   // 1 / std of each feature (0 for the padding)
    float yscale[kMlpOutPad];  // network output x yscale = label
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ uint32_t pack_raw(__nv_bfloat16 lo, __nv_bfloat16 hi)
{
    __nv_bfloat162 v;
    v.x = lo;
    v.y = hi;
    return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// B fragment of a k-major BF16 matrix W[k][n] (row stride ld), k-step ks,
// column block nb
__device__ __forceinline__ void load_b(uint32_t (&b)[2], const __nv_bfloat16* W, int ld, int ks, int nb, int lane)
{
    const int g = lane >> 2, q = lane & 3;
    const int n = nb * 8 + g, k = ks * 16 + 2 * q;
    b[0] = pack_raw(W[(k) * ld + n], W[(k + 1) * ld + n]);
    b[1] = pack_raw(W[(k + 8) * ld + n], W[(k + 9) * ld + n]);
}

// A fragment from C tiles (FP32) of column blocks 2ks and 2ks+1
__device__ __forceinline__ void c_to_a(uint32_t (&a)[4], const float (&c0)[4], const float (&c1)[4])
{
    a[0] = pack_bf16(c0[0], c0[1]);
    a[1] = pack_bf16(c0[2], c0[3]);
    a[2] = pack_bf16(c1[0], c1[1]);
    a[3] = pack_bf16(c1[2], c1[3]);
}

// The MLP on 16 rows: x holds the A fragment of the (normalised, padded)
// features; y returns the C tile of the output (columns 0..2 used).  The
// hidden activations are returned too (for training): h1, h2 as C tiles
// after ReLU.
__device__ __forceinline__ void mlp16(const MlpDev& m, const uint32_t (&x)[4], float (&h1)[8][4], float (&h2)[8][4],
                                      float (&y)[4], int lane)
{
    const int q = lane & 3;
#pragma unroll
    for (int nb = 0; nb < 8; nb++) {
        const float bb0 = m.b1[nb * 8 + 2 * q], bb1 = m.b1[nb * 8 + 2 * q + 1];
        h1[nb][0] = bb0;
        h1[nb][1] = bb1;
        h1[nb][2] = bb0;
        h1[nb][3] = bb1;
        uint32_t b[2];
        load_b(b, m.w1, kMlpHid, 0, nb, lane);
        mma_bf16(h1[nb], x, b);
#pragma unroll
        for (int e = 0; e < 4; e++) h1[nb][e] = fmaxf(h1[nb][e], 0.f);
    }
#pragma unroll
    for (int nb = 0; nb < 8; nb++) {
        const float bb0 = m.b2[nb * 8 + 2 * q], bb1 = m.b2[nb * 8 + 2 * q + 1];
        h2[nb][0] = bb0;
        h2[nb][1] = bb1;
        h2[nb][2] = bb0;
        h2[nb][3] = bb1;
    }
#pragma unroll
    for (int ks = 0; ks < 4; ks++) {
        uint32_t a[4];
        c_to_a(a, h1[2 * ks], h1[2 * ks + 1]);
#pragma unroll
        for (int nb = 0; nb < 8; nb++) {
            uint32_t b[2];
            load_b(b, m.w2, kMlpHid, ks, nb, lane);
            mma_bf16(h2[nb], a, b);
        }
    }
#pragma unroll
    for (int nb = 0; nb < 8; nb++)
#pragma unroll
        for (int e = 0; e < 4; e++) h2[nb][e] = fmaxf(h2[nb][e], 0.f);
    y[0] = m.b3[2 * q];
    y[1] = m.b3[2 * q + 1];
    y[2] = y[0];
    y[3] = y[1];
#pragma unroll
    for (int ks = 0; ks < 4; ks++) {
        uint32_t a[4];
        c_to_a(a, h2[2 * ks], h2[2 * ks + 1]);
        uint32_t b[2];
        load_b(b, m.w3, kMlpOutPad, ks, 0, lane);
        mma_bf16(y, a, b);
    }
}

// A fragment of 16 feature rows stored as FP32 rows of kMlpInPad (already
// normalised, padding zero)
__device__ __forceinline__ void load_x(uint32_t (&a)[4], const float* X, int ld, int lane)
{
    const int g = lane >> 2, q = lane & 3;
    a[0] = pack_bf16(X[g * ld + 2 * q], X[g * ld + 2 * q + 1]);
    a[1] = pack_bf16(X[(g + 8) * ld + 2 * q], X[(g + 8) * ld + 2 * q + 1]);
    a[2] = pack_bf16(X[g * ld + 2 * q + 8], X[g * ld + 2 * q + 9]);
    a[3] = pack_bf16(X[(g + 8) * ld + 2 * q + 8], X[(g + 8) * ld + 2 * q + 9]);
}

}  // namespace tc
