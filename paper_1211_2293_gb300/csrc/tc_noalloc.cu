// tc_noalloc.cu -- direct summation into caller buffers, with no device
// allocation at all (tc_direct_static in include/tc.h).
//
// tc_direct stages its index list and results in buffers the context
// allocates.  Some callers cannot let a library call cudaMalloc: a host
// framework whose caching allocator already owns the device's memory budget
// (a cudaMalloc behind its back can fail or fragment that budget), or a
// latency-critical loop that cannot afford the implicit device
// synchronisation of cudaMalloc/cudaFree.  For them this entry point keeps
// its only scratch -- the per-slice partial sums -- in a fixed file-scope
// device array, so a call only reads the caller's inputs and writes the
// caller's outputs.
//
// The array is a static __device__ object: every GPU that loads libtc holds
// its kDirectScratchBytes until the process exits.  Kernels reach it through
// the device address that cudaGetSymbolAddress returns; the host-side name
// of the array is only a stand-in and must never be passed to a kernel.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/tc.h"
#include "tc_internal.cuh"

namespace tc {

namespace {

constexpr int64_t kStaticNsMax = 8192;  // targets per call
constexpr int kSlicesMax = 16;          // source slices per target
constexpr int kThreads = 256;
constexpr size_t kDirectScratchBytes = (size_t)kStaticNsMax * kSlicesMax * 4 * sizeof(double);  // 4 MiB
constexpr int kMaxDevices = 64;

// partial sums (ax, ay, az, pot) of target t over source slice s at
// [(t * S + s) * 4]; every call overwrites the slots it reads
static __device__ __align__(256) double g_direct_scratch[kStaticNsMax * kSlicesMax * 4];
static_assert(sizeof(g_direct_scratch) == kDirectScratchBytes, "scratch size");

std::mutex g_setup_mu;
double* g_scratch_dev[kMaxDevices] = {};  // device address of the scratch, per device
int g_sms[kMaxDevices] = {};              // streaming multiprocessors, per device

// Block (bx, s) sums targets [bx * 256, +256) over source slice s: FP32 terms
// per 256-source tile, tiles added in FP64.
__global__ void __launch_bounds__(kThreads) k_direct_slices(const float* __restrict__ pos,
                                                            const float* __restrict__ mass, int64_t n,
                                                            const int64_t* __restrict__ idx, int64_t ns, int S,
                                                            float eps2, double* __restrict__ scratch)
{
    __shared__ float4 tile[kThreads];
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t it = t < ns ? idx[t] : 0;
    const bool act = t < ns && it >= 0 && it < n;  // an index outside [0, n) is never dereferenced
    const int64_t i = act ? it : 0;
    const float xi = pos[3 * i], yi = pos[3 * i + 1], zi = pos[3 * i + 2];
    const int64_t per = (n + S - 1) / S;
    const int64_t j0 = (int64_t)blockIdx.y * per;
    const int64_t j1 = j0 + per < n ? j0 + per : n;
    double ax = 0, ay = 0, az = 0, ph = 0;
    for (int64_t base = j0; base < j1; base += kThreads) {
        const int64_t j = base + threadIdx.x;
        __syncthreads();
        tile[threadIdx.x] = j < j1 ? make_float4(pos[3 * j], pos[3 * j + 1], pos[3 * j + 2], mass[j])
                                   : make_float4(0.f, 0.f, 0.f, 0.f);
        __syncthreads();
        const int cnt = (int)(j1 - base < kThreads ? j1 - base : kThreads);
        float tx = 0.f, ty = 0.f, tz = 0.f, tp = 0.f;
        for (int k = 0; k < cnt; k++) {
            const float4 s = tile[k];
            const float dx = s.x - xi, dy = s.y - yi, dz = s.z - zi;
            const float r2 = fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, eps2)));
            const float ri = rsqrtf(r2);
            const float mri = s.w * ri;
            const float mri3 = mri * ri * ri;
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
    double* o = scratch + ((size_t)t * S + blockIdx.y) * 4;
    o[0] = ax;
    o[1] = ay;
    o[2] = az;
    o[3] = ph;
}

// slices summed in order (deterministic); the potential drops the target's
// own -m_i / eps term
__global__ void k_direct_reduce(const double* __restrict__ scratch, const float* __restrict__ mass,
                                const int64_t* __restrict__ idx, int64_t n, int64_t ns, int S, float eps2, float G,
                                double* __restrict__ acc, double* __restrict__ pot)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ns) return;
    const int64_t i = idx[t];
    if (i < 0 || i >= n) {  // invalid index: NaN results, nothing else touched
        acc[3 * t] = acc[3 * t + 1] = acc[3 * t + 2] = NAN;
        if (pot) pot[t] = NAN;
        return;
    }
    double s[4] = {0, 0, 0, 0};
    for (int k = 0; k < S; k++)
        for (int c = 0; c < 4; c++) s[c] += scratch[((size_t)t * S + k) * 4 + c];
    acc[3 * t] = (double)G * s[0];
    acc[3 * t + 1] = (double)G * s[1];
    acc[3 * t + 2] = (double)G * s[2];
    if (pot) pot[t] = (double)G * (s[3] + (double)(mass[i] * rsqrtf(eps2)));
}

// memory a kernel on device `dev` can read and write in place: device memory
// of that device (another device's memory may not be peer-mapped), managed
// memory, or mapped pinned host memory
bool device_reachable(const void* p, int dev)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeDevice) return at.device == dev;
    return at.type == cudaMemoryTypeManaged || (at.type == cudaMemoryTypeHost && at.devicePointer != nullptr);
}

}  // namespace
}  // namespace tc

using namespace tc;

extern "C" int tc_direct_static(const float* pos, const float* mass, int64_t n, const int64_t* idx, int64_t ns,
                                float eps, float G, double* acc, double* pot, void* stream)
{
    char msg[256];
    auto bad = [&](int code, const char* what) {
        snprintf(msg, sizeof(msg), "tc_direct_static: %s", what);
        set_thread_error(msg);
        return code;
    };
    if (!pos || !mass || !idx || !acc) return bad(TC_EINVAL, "null pointer");
    if (n < 1 || n >= ((int64_t)1 << 31)) return bad(TC_EINVAL, "n must be in [1, 2^31)");
    if (ns < 1 || ns > kStaticNsMax) return bad(TC_EINVAL, "ns must be in [1, 8192] (the fixed scratch holds 8192 targets)");
    if (!(eps > 0.f) || !std::isfinite(eps) || !std::isfinite(G))
        return bad(TC_EINVAL, "eps must be > 0 and finite, G finite");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return bad(TC_ECUDA, "no usable current device");
    }
    if (!device_reachable(pos, dev) || !device_reachable(mass, dev) || !device_reachable(idx, dev) ||
        !device_reachable(acc, dev) || (pot && !device_reachable(pot, dev)))
        return bad(TC_EINVAL,
                   "every pointer must be memory the current device reaches in place (its own device memory, "
                   "managed or mapped host memory; nothing is staged)");
    double* scratch = nullptr;
    int sms = 0;
    {
        // once per device, with that device current: the device address of
        // the static scratch array and the device's SM count
        std::lock_guard<std::mutex> lk(g_setup_mu);
        if (!g_scratch_dev[dev]) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_direct_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                snprintf(msg, sizeof(msg), "tc_direct_static: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
                set_thread_error(msg);
                return TC_ECUDA;
            }
            int c = 0;
            e = cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess || c < 1) {
                cudaGetLastError();
                return bad(TC_ECUDA, "cudaDeviceGetAttribute(MultiProcessorCount) failed");
            }
            g_sms[dev] = c;
            g_scratch_dev[dev] = (double*)p;
        }
        scratch = g_scratch_dev[dev];
        sms = g_sms[dev];
    }
    // an error left pending by earlier, unrelated work is reported as such
    // (and not cleared) instead of being taken for this call's launch failure
    {
        const cudaError_t pe = cudaPeekAtLastError();
        if (pe != cudaSuccess) {
            snprintf(msg, sizeof(msg), "tc_direct_static: a CUDA error was already pending before the launch: %s",
                     cudaGetErrorString(pe));
            set_thread_error(msg);
            return TC_ECUDA;
        }
    }

    cudaStream_t s = (cudaStream_t)stream;
    const int64_t nbx = (ns + kThreads - 1) / kThreads;
    int S = (int)((4 * (int64_t)sms + nbx - 1) / nbx);
    if (S > kSlicesMax) S = kSlicesMax;
    if (S > n) S = (int)n;
    if (S < 1) S = 1;
    const float eps2 = eps * eps;
    k_direct_slices<<<dim3((unsigned)nbx, (unsigned)S), kThreads, 0, s>>>(pos, mass, n, idx, ns, S, eps2, scratch);
    k_direct_reduce<<<(unsigned)nbx, kThreads, 0, s>>>(scratch, mass, idx, n, ns, S, eps2, G, acc, pot);
    count_launches(2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        snprintf(msg, sizeof(msg), "tc_direct_static: launch failed: %s", cudaGetErrorString(e));
        set_thread_error(msg);
        return TC_ECUDA;
    }
    return TC_OK;
}
