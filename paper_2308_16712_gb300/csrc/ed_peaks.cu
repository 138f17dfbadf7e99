// ed_peaks.cu -- measured throughput ceilings of this GPU for the rooflines of
// the product kernels (diagnostics; not part of the computation):
//
//  - integer: chains of the representative search's own operation mix (a
//    funnel-shift rotation, a three-input logic operation, an unsigned min and
//    an add) over every SM;
//  - fp64 and fp32 fused multiply-adds (the Lanczos vector arithmetic, the
//    products' accumulation);
//  - random 32-byte reads from a caller's buffer (the pattern of the index
//    lookups and x gathers of a product over a sector far larger than L2).
//
// Each kernel runs many independent dependency chains per thread so that the
// issue rate, not the latency, bounds it.  Times are CUDA events on the
// caller's stream.
#include <cuda_runtime.h>

#include <algorithm>

#include "ed_kernels.cuh"

namespace edk {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kChains = 8;

// integer mix: per chain and iteration 4 operations (shf, lop3, min, add)
__global__ void __launch_bounds__(kPeakThreads) k_peak_int(int iters, uint32_t seed, uint32_t *out)
{
    uint32_t x[kChains], m[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        x[c] = seed ^ (threadIdx.x * 0x9E3779B9u + c * 0x85EBCA6Bu + blockIdx.x);
        m[c] = ~x[c];
    }
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            const uint32_t r = __funnelshift_l(x[c], x[c], 7);
            uint32_t t;
            asm("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(t) : "r"(r), "r"(m[c]), "r"(0x5bd1e995u));
            m[c] = min(m[c], t);
            x[c] = t + m[c];
        }
    }
    uint32_t acc = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        acc ^= x[c] ^ m[c];
    if (acc == 0x12345678u)  // practically never: keeps the chains live
        out[blockIdx.x] = acc;
}

template <typename T>
__global__ void __launch_bounds__(kPeakThreads) k_peak_fma(int iters, T seed, T *out)
{
    T a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        a[c] = seed + (T)(threadIdx.x + c);
    const T b = (T)0.999999, d = (T)1e-7;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c)
            a[c] = fma(a[c], b, d);
    }
    T acc = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        acc += a[c];
    if (acc == (T)-1.2345)
        out[blockIdx.x] = acc;
}

__device__ __forceinline__ uint64_t peak_mix(uint64_t x)
{
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdULL;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ULL;
    x ^= x >> 33;
    return x;
}

// random 32-byte chunks of buf (n32 chunks), 4 independent reads in flight
__global__ void __launch_bounds__(kPeakThreads) k_peak_gather(const uint4 *buf, uint64_t n32, int iters,
                                                              uint32_t *out)
{
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t acc = 0;
    for (int it = 0; it < iters; it += 4) {
        uint4 v[4][2];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint64_t c = peak_mix(tid * 0x9E3779B97F4A7C15ULL + (uint64_t)(it + u)) % n32;
            v[u][0] = __ldg(buf + 2 * c);
            v[u][1] = __ldg(buf + 2 * c + 1);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            acc ^= v[u][0].x ^ v[u][0].w ^ v[u][1].y ^ v[u][1].z;
    }
    if (acc == 0x9abcdef0u)
        out[blockIdx.x] = acc;
}

float elapsed(cudaEvent_t a, cudaEvent_t b)
{
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    return ms;
}

}  // namespace
}  // namespace edk

// Diagnostics hook: kind 0 = integer op mix (ops/s), 1 = fp64 FMA (FMA/s),
// 2 = fp32 FMA (FMA/s), 3 = random 32-byte reads of buf (reads/s; buf holds
// bytes >= 32 bytes, 16-byte aligned).  *ms_out = device time of the timed
// launches; returns the rate, or a negative value on error.
extern "C" double edx_peak(int kind, const void *buf, uint64_t bytes, double *ms_out, void *stream)
{
    using namespace edk;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = sms * 8;
    uint32_t *out = nullptr;
    if (cudaMalloc(&out, (size_t)blocks * sizeof(double)) != cudaSuccess)
        return -1.0;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int reps = 3;
    double work = 0.0;
    auto launch = [&](int iters) {
        switch (kind) {
        case 0: k_peak_int<<<blocks, kPeakThreads, 0, st>>>(iters, 12345u, out); break;
        case 1: k_peak_fma<double><<<blocks, kPeakThreads, 0, st>>>(iters, 0.5, (double *)out); break;
        case 2: k_peak_fma<float><<<blocks, kPeakThreads, 0, st>>>(iters, 0.5f, (float *)out); break;
        case 3:
            k_peak_gather<<<blocks, kPeakThreads, 0, st>>>((const uint4 *)buf, bytes / 32, iters, out);
            break;
        }
        count_launch();
    };
    int iters = 0;
    double per_iter = 0.0;  // work units per thread per iteration
    switch (kind) {
    case 0: iters = 1 << 14; per_iter = 4.0 * kChains; break;
    case 1: iters = 1 << 10; per_iter = kChains; break;
    case 2: iters = 1 << 14; per_iter = kChains; break;
    case 3: iters = 256; per_iter = 1.0; break;
    default: cudaFree(out); return -1.0;
    }
    if (kind == 3 && (!buf || bytes < 32 || ((uintptr_t)buf & 15))) {
        cudaFree(out);
        return -1.0;
    }
    launch(iters);  // warm-up
    cudaEventRecord(e0, st);
    for (int r = 0; r < reps; ++r)
        launch(iters);
    cudaEventRecord(e1, st);
    const cudaError_t err = cudaEventSynchronize(e1);
    const double ms = elapsed(e0, e1);
    work = (double)reps * blocks * kPeakThreads * iters * per_iter;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (err != cudaSuccess || ms <= 0.0)
        return -1.0;
    if (ms_out)
        *ms_out = ms;
    return work / (ms * 1e-3);
}
