// Measured throughput of the FP32 and FP64 fused multiply-add pipes: the
// denominators of the force kernel's roofline, taken on the device the
// library runs on rather than derived from unit counts and a nominal clock
// (the clock under a dense arithmetic load sits below its maximum).
//
// Every thread runs kChains independent multiply-add chains, so that each
// scheduler always has an independent FMA ready (FP32 latency ~4 cycles,
// FP64 longer); the multiplier and addend keep the values bounded and normal,
// and the sum is stored (to a device variable) only under a condition the
// values never meet, which
// keeps every chain live without a memory store in the loop.  The FMAs are
// inline PTX so that the compiler can neither fold nor reassociate them.
#include <string>

#include "md.h"
#include "md_internal.cuh"

namespace mdg {

constexpr int kPeakThreads = 256;
constexpr int kChains = 8;
constexpr int kUnroll = 16;

__device__ __forceinline__ float fma_pipe(float a, float b, float c)
{
    float d;
    asm volatile("fma.rn.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
__device__ __forceinline__ double fma_pipe(double a, double b, double c)
{
    double d;
    asm volatile("fma.rn.f64 %0, %1, %2, %3;" : "=d"(d) : "d"(a), "d"(b), "d"(c));
    return d;
}

__device__ float g_peak_sink_f;
__device__ double g_peak_sink_d;
__device__ __forceinline__ void sink(float v) { g_peak_sink_f = v; }
__device__ __forceinline__ void sink(double v) { g_peak_sink_d = v; }

template <typename T>
__global__ void __launch_bounds__(kPeakThreads) k_fma_peak(long long iters)
{
    T a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = T(1) + T(threadIdx.x + k) * T(1e-3);
    const T m = T(0.9999), c = T(1e-4);   // fixed point 1: the chains stay near 1
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = fma_pipe(a[k], m, c);
    }
    T s = T(0);
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == T(-1)) sink(s);   // never taken: the chains converge to 1
}

}  // namespace mdg

using namespace mdg;

extern "C" md_status md_fma_peak(int precision, int64_t iters, int blocks_per_sm, double* flops_per_s,
                                 double* seconds, void* cuda_stream)
{
    if (!flops_per_s || iters < 1 || blocks_per_sm < 1 || blocks_per_sm > 64 ||
        (precision != MD_PREC_MIXED && precision != MD_PREC_FP64)) {
        set_global_error("md_fma_peak: bad argument");
        return MD_ERR_INVALID_ARG;
    }
    const cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0, n_sm = 0;
    cudaEvent_t a = nullptr, b = nullptr;
    auto err = [&](cudaError_t e, const char* what) {
        set_global_error(std::string("md_fma_peak: ") + what + ": " + cudaGetErrorString(e));
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
        return MD_ERR_CUDA;
    };
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return err(e, "cudaGetDevice");
    if ((e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return err(e, "cudaDeviceGetAttribute");
    if ((e = cudaEventCreate(&a)) != cudaSuccess) return err(e, "cudaEventCreate");
    if ((e = cudaEventCreate(&b)) != cudaSuccess) return err(e, "cudaEventCreate");
    const int blocks = n_sm * blocks_per_sm;
    cudaEventRecord(a, s);
    if (precision == MD_PREC_MIXED) k_fma_peak<float><<<blocks, kPeakThreads, 0, s>>>(iters);
    else k_fma_peak<double><<<blocks, kPeakThreads, 0, s>>>(iters);
    cudaEventRecord(b, s);
    if ((e = cudaGetLastError()) != cudaSuccess) return err(e, "launch");
    if ((e = cudaEventSynchronize(b)) != cudaSuccess) return err(e, "cudaEventSynchronize");
    float ms = 0.0f;
    if ((e = cudaEventElapsedTime(&ms, a, b)) != cudaSuccess) return err(e, "cudaEventElapsedTime");
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    const double flops = 2.0 * (double)blocks * kPeakThreads * (double)iters * kUnroll * kChains;
    *flops_per_s = flops / (1e-3 * (double)ms);
    if (seconds) *seconds = 1e-3 * (double)ms;
    return MD_OK;
}
