// tc_step.cu -- moving the bodies (kick-drift-kick leapfrog), FP64
// diagnostics and the direct-summation reference.
//
// Paper, Sec. 3.1: after the force summation each body updates its position
// and velocity.  The integrator is not named; the kick-drift-kick leapfrog
// (velocity Verlet) is used: v += a dt/2; x += v dt; forces; v += a dt/2.
#include "tc_internal.cuh"

namespace tc {

namespace {

// v' = v + a*hk, x' = x + v'*dt, each a separately rounded float32 op.  A
// step whose build or walk raised the error word leaves the state as it is
// (the error is reported at the next synchronisation).
__device__ __forceinline__ bool failed(const Info* info) { return *(volatile const int32_t*)&info->err != 0; }

// The update is elementwise over the 3 n floats of the state: x += (v +=
// a hk) dt.  Each thread takes float4 runs (grid-stride) when the arrays are
// 16-byte aligned, else single floats; the error word is read once per warp.
__device__ __forceinline__ bool warp_failed(const Info* info)
{
    bool f = false;
    if ((threadIdx.x & 31) == 0) f = failed(info);
    return __shfl_sync(0xffffffffu, f, 0);
}

__device__ __forceinline__ float kick1(float v, float a, float hk) { return __fadd_rn(v, __fmul_rn(a, hk)); }
__device__ __forceinline__ float drift1(float x, float v, float dt) { return __fadd_rn(x, __fmul_rn(v, dt)); }

template <bool DRIFT, bool VEC>
__global__ void k_kick_drift(float* __restrict__ pos, float* __restrict__ vel, const float* __restrict__ acc,
                             int64_t n3, float hk, float dt, const Info* info)
{
    if (warp_failed(info)) return;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t done = 0;
    if (VEC) {
        const int64_t n4 = n3 >> 2;
        float4* v4 = reinterpret_cast<float4*>(vel);
        float4* p4 = reinterpret_cast<float4*>(pos);
        const float4* a4 = reinterpret_cast<const float4*>(acc);
        for (int64_t i = i0; i < n4; i += stride) {
            const float4 a = a4[i];
            float4 v = v4[i];
            v.x = kick1(v.x, a.x, hk);
            v.y = kick1(v.y, a.y, hk);
            v.z = kick1(v.z, a.z, hk);
            v.w = kick1(v.w, a.w, hk);
            v4[i] = v;
            if (DRIFT) {
                float4 x = p4[i];
                x.x = drift1(x.x, v.x, dt);
                x.y = drift1(x.y, v.y, dt);
                x.z = drift1(x.z, v.z, dt);
                x.w = drift1(x.w, v.w, dt);
                p4[i] = x;
            }
        }
        done = n4 << 2;
    }
    for (int64_t i = done + i0; i < n3; i += stride) {
        const float v = kick1(vel[i], acc[i], hk);
        vel[i] = v;
        if (DRIFT) pos[i] = drift1(pos[i], v, dt);
    }
}

// KE, PE = 1/2 sum m pot, P, L in FP64; block sums, then FP64 atomics
__global__ void k_diag(const float* __restrict__ pos, const float* __restrict__ vel, const float* __restrict__ mass,
                       const float* __restrict__ pot, int64_t n, double* __restrict__ out)
{
    __shared__ double sm[8][8];
    double q[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double m = mass[i];
        double x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
        double vx = vel[3 * i], vy = vel[3 * i + 1], vz = vel[3 * i + 2];
        q[0] += 0.5 * m * (vx * vx + vy * vy + vz * vz);
        if (pot) q[1] += 0.5 * m * (double)pot[i];
        q[2] += m * vx;
        q[3] += m * vy;
        q[4] += m * vz;
        q[5] += m * (y * vz - z * vy);
        q[6] += m * (z * vx - x * vz);
        q[7] += m * (x * vy - y * vx);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 8; k++) {
#pragma unroll
        for (int o = 16; o; o >>= 1) q[k] += __shfl_xor_sync(0xffffffffu, q[k], o);
        if (lane == 0) sm[k][w] = q[k];
    }
    __syncthreads();
    if (threadIdx.x < 8) {
        double s = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) s += sm[threadIdx.x][k];
        atomicAdd(&out[threadIdx.x], s);
    }
}

// Direct summation for ns targets over the bodies of each target's system
// (original order).  FP32 terms; each 256-source tile is summed in FP32 and
// added in FP64.  One block serves targets of a single system at a time:
// blocks are laid out per target and loop over [first, end) of the
// target's system, so threads of a block may walk different ranges; the
// tile holds the union for the block's smallest system range.
constexpr int kDirTile = 256;
__global__ void __launch_bounds__(kDirTile) k_direct(const float* __restrict__ pos, const float* __restrict__ mass,
                                                     const uint32_t* __restrict__ sys_of,
                                                     const SysParams* __restrict__ sysp,
                                                     const int64_t* __restrict__ idx, int64_t ns,
                                                     float eps2, float G, double* __restrict__ acc,
                                                     double* __restrict__ pot)
{
    __shared__ float4 tile[kDirTile];
    __shared__ int64_t lo_sh, hi_sh;
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool act = t < ns;
    int64_t i = act ? idx[t] : idx[(int64_t)blockIdx.x * blockDim.x];
    const uint32_t sy = sys_of[i];
    const int64_t j0 = sysp[sy].first, j1 = sysp[sy].end;
    // the block sweeps the union of its targets' system ranges
    if (threadIdx.x == 0) {
        lo_sh = j0;
        hi_sh = j1;
    }
    __syncthreads();
    atomicMin((unsigned long long*)&lo_sh, (unsigned long long)j0);
    atomicMax((unsigned long long*)&hi_sh, (unsigned long long)j1);
    __syncthreads();
    const int64_t blo = lo_sh, bhi = hi_sh;
    float xi = pos[3 * i], yi = pos[3 * i + 1], zi = pos[3 * i + 2];
    double ax = 0, ay = 0, az = 0, ph = 0;
    for (int64_t base = blo; base < bhi; base += kDirTile) {
        int64_t j = base + threadIdx.x;
        __syncthreads();
        // sources outside this thread's system are masked by zero mass below
        tile[threadIdx.x] = j < bhi ? make_float4(pos[3 * j], pos[3 * j + 1], pos[3 * j + 2], mass[j])
                                    : make_float4(0.f, 0.f, 0.f, 0.f);
        __syncthreads();
        const int cnt = (int)min((int64_t)kDirTile, bhi - base);
        const int k0 = (int)max((int64_t)0, min((int64_t)cnt, j0 - base));
        const int k1 = (int)max((int64_t)0, min((int64_t)cnt, j1 - base));
        float tx = 0.f, ty = 0.f, tz = 0.f, tp = 0.f;
        for (int k = k0; k < k1; k++) {
            float4 s = tile[k];
            float dx = s.x - xi, dy = s.y - yi, dz = s.z - zi;
            float r2 = fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, eps2)));
            float ri = rsqrtf(r2);
            float mri = s.w * ri;
            float mri3 = mri * ri * ri;
            tx = fmaf(dx, mri3, tx);
            ty = fmaf(dy, mri3, ty);
            tz = fmaf(dz, mri3, tz);
            tp -= mri;
        }
        ax += tx;
        ay += ty;
        az += tz;
        ph += tp;
    }
    if (!act) return;
    acc[3 * t] = (double)G * ax;
    acc[3 * t + 1] = (double)G * ay;
    acc[3 * t + 2] = (double)G * az;
    if (pot) pot[t] = (double)G * (ph + (double)(mass[i] * rsqrtf(eps2)));
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

namespace {
template <bool DRIFT>
void launch_update(float* pos, float* vel, const float* acc, int64_t n, float hkick, float dt, const Info* info,
                   cudaStream_t s)
{
    const bool vec = ((reinterpret_cast<uintptr_t>(vel) | reinterpret_cast<uintptr_t>(acc) |
                       (DRIFT ? reinterpret_cast<uintptr_t>(pos) : 0)) & 15u) == 0;
    int64_t g = nblk(vec ? (3 * n + 3) / 4 : 3 * n, 256);
    if (g > 8 * sm_count()) g = 8 * sm_count();
    if (g < 1) g = 1;
    if (vec) k_kick_drift<DRIFT, true><<<(unsigned)g, 256, 0, s>>>(pos, vel, acc, 3 * n, hkick, dt, info);
    else k_kick_drift<DRIFT, false><<<(unsigned)g, 256, 0, s>>>(pos, vel, acc, 3 * n, hkick, dt, info);
    count_launches(1);
}
}  // namespace

void launch_kick_drift(float* pos, float* vel, const float* acc, int64_t n, float hkick, float dt, const Info* info,
                       cudaStream_t s)
{
    launch_update<true>(pos, vel, acc, n, hkick, dt, info, s);
}

void launch_kick(float* vel, const float* acc, int64_t n, float hkick, const Info* info, cudaStream_t s)
{
    launch_update<false>(nullptr, vel, acc, n, hkick, 0.f, info, s);
}

// FP32 throughput probe: every thread runs 8 independent chains of `iters`
// fused multiply-adds (scalar, or paired f32x2 instructions), 2 flops each;
// the chains' ends are folded into one store so nothing is dead code.
template <bool PAIRED>
__global__ void __launch_bounds__(256) k_fp32_probe(int iters, float seed, float* out)
{
    if (PAIRED) {
        unsigned long long a[4], m, c;
        const float x = seed + threadIdx.x * 1e-7f;
        asm("mov.b64 %0, {%1, %1};" : "=l"(m) : "f"(0.999999f));
        asm("mov.b64 %0, {%1, %1};" : "=l"(c) : "f"(1e-7f));
#pragma unroll
        for (int k = 0; k < 4; k++) asm("mov.b64 %0, {%1, %2};" : "=l"(a[k]) : "f"(x + k), "f"(x - k));
        for (int i = 0; i < iters; i++) {
#pragma unroll
            for (int k = 0; k < 4; k++) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[k]) : "l"(m), "l"(c));
        }
        float sum = 0.f;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            float lo, hi;
            asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a[k]));
            sum += lo + hi;
        }
        if (sum == 12345.f) out[0] = sum;
    } else {
        float a[8];
        const float x = seed + threadIdx.x * 1e-7f;
#pragma unroll
        for (int k = 0; k < 8; k++) a[k] = x + k;
        for (int i = 0; i < iters; i++) {
#pragma unroll
            for (int k = 0; k < 8; k++) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(a[k]) : "f"(0.999999f), "f"(1e-7f));
        }
        float sum = 0.f;
#pragma unroll
        for (int k = 0; k < 8; k++) sum += a[k];
        if (sum == 12345.f) out[0] = sum;
    }
}

void launch_fp32_probe(bool paired, int blocks, int iters, float* out, cudaStream_t s)
{
    if (paired) k_fp32_probe<true><<<blocks, 256, 0, s>>>(iters, 1.0f, out);
    else k_fp32_probe<false><<<blocks, 256, 0, s>>>(iters, 1.0f, out);
    count_launches(1);
}

void launch_diag(const float* pos, const float* vel, const float* mass, const float* pot, int64_t n, Info* info,
                 cudaStream_t s)
{
    cudaMemsetAsync(info->diag, 0, 8 * sizeof(double), s);
    unsigned nb = nblk(n, 256);
    if (nb > 1024) nb = 1024;
    k_diag<<<nb, 256, 0, s>>>(pos, vel, mass, pot, n, info->diag);
    count_launches(1);
}

void launch_direct(const float* pos, const float* mass, const uint32_t* sys_of, const SysParams* sysp,
                   const int64_t* idx, int64_t ns, float eps2, float G, double* acc, double* pot, cudaStream_t s)
{
    k_direct<<<nblk(ns, kDirTile), kDirTile, 0, s>>>(pos, mass, sys_of, sysp, idx, ns, eps2, G, acc, pot);
    count_launches(1);
}

}  // namespace tc
