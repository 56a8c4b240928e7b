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

// Inference copy of a model: the BF16 weights pre-arranged as the B
// fragments of mma.m16n8k16 (one 64-bit word per lane and fragment, so a
// fragment is one shared-memory load), the FP32 bias pairs each lane adds,
// and the affine maps of the features and of the output.
struct MlpFrag {
    uint2 f1[8][32];       // layer 1: [column block][lane] (inputs padded to 16)
    uint2 f2[4][8][32];    // layer 2: [k-step][column block][lane]
    uint2 f3[4][32];       // layer 3: [k-step][lane] (outputs padded to 8)
    float2 b1[8][4];       // [column block][q]: biases of columns 8 nb + 2q, + 1
    float2 b2[8][4];
    float2 b3[4];
    float xscale[kMlpInPad];  // 1 / std of each feature (0 for the padding)
    float xoff[kMlpInPad];    // -mean x scale: a feature enters as f x scale + off
    float yscale[kMlpOutPad]; // network output x yscale = label
};

// Device copy of a model: the inference part, then the k-major weights
// ([in][out], padded) the training kernel reads its transposes from.
struct MlpDev {
    MlpFrag frag;
    __nv_bfloat16 w1[kMlpInPad * kMlpHid];
    __nv_bfloat16 w2[kMlpHid * kMlpHid];
    __nv_bfloat16 w3[kMlpHid * kMlpOutPad];
    float b1[kMlpHid];
    float b2[kMlpHid];
    float b3[kMlpOutPad];
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

// round-to-nearest BF16 pair of max(lo, 0), max(hi, 0): ReLU fused into the
// conversion (the first operand of the instruction fills the upper half)
__device__ __forceinline__ uint32_t pack_relu(float lo, float hi)
{
    uint32_t d;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
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

__device__ __forceinline__ void mma_frag(float (&c)[4], const uint32_t (&a)[4], uint2 w)
{
    const uint32_t b[2] = {w.x, w.y};
    mma_bf16(c, a, b);
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

// the same with the ReLU applied first
__device__ __forceinline__ void c_to_a_relu(uint32_t (&a)[4], const float (&c0)[4], const float (&c1)[4])
{
    a[0] = pack_relu(c0[0], c0[1]);
    a[1] = pack_relu(c0[2], c0[3]);
    a[2] = pack_relu(c1[0], c1[1]);
    a[3] = pack_relu(c1[2], c1[3]);
}

__device__ __forceinline__ void bias_init(float (&c)[4], float2 b)
{
    c[0] = b.x;
    c[1] = b.y;
    c[2] = b.x;
    c[3] = b.y;
}

// Inference on 16 rows: x holds the A fragment of the (normalised, padded)
// features; y returns the C tile of the output (columns 0..2 used).  Same
// products in the same order as mlp16 below, so the two agree bit for bit.
__device__ __forceinline__ void mlp16_infer(const MlpFrag& m, const uint32_t (&x)[4], float (&y)[4], int lane)
{
    const int q = lane & 3;
    uint32_t a1[4][4];
#pragma unroll
    for (int ks = 0; ks < 4; ks++) {
        float c0[4], c1[4];
        bias_init(c0, m.b1[2 * ks][q]);
        bias_init(c1, m.b1[2 * ks + 1][q]);
        mma_frag(c0, x, m.f1[2 * ks][lane]);
        mma_frag(c1, x, m.f1[2 * ks + 1][lane]);
        c_to_a_relu(a1[ks], c0, c1);
    }
    // layer 2 in two halves of four column blocks: the first half feeds
    // k-steps 0, 1 of layer 3, the second k-steps 2, 3 (fewer live registers)
    bias_init(y, m.b3[q]);
#pragma unroll
    for (int half = 0; half < 2; half++) {
        float h2[4][4];
#pragma unroll
        for (int j = 0; j < 4; j++) bias_init(h2[j], m.b2[4 * half + j][q]);
#pragma unroll
        for (int ks = 0; ks < 4; ks++)
#pragma unroll
            for (int j = 0; j < 4; j++) mma_frag(h2[j], a1[ks], m.f2[ks][4 * half + j][lane]);
#pragma unroll
        for (int k = 0; k < 2; k++) {
            uint32_t a[4];
            c_to_a_relu(a, h2[2 * k], h2[2 * k + 1]);
            mma_frag(y, a, m.f3[2 * half + k][lane]);
        }
    }
}

// The MLP on 16 rows for training, from the k-major weights: returns the
// hidden activations too (h1, h2 as C tiles after ReLU).
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

}  // namespace tc
