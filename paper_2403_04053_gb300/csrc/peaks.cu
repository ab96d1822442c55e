// Measured arithmetic peaks of this GPU: the FP32 and FP64 fused multiply-add rates that the
// ALU-bound kernels of the library (the surface transform, the auxiliary-wave evaluation and
// the FP64 stepping passes) are judged against.  Not part of the paper's method.
//
// Each thread runs ILP independent FMA chains a = a * m + c for ITERS rounds; the grid fills
// every SM several times over.  FLOPs = 2 * chains * ITERS * threads per launch.
#include <cuda_runtime.h>

#include "pstd_internal.h"

namespace {

constexpr int kPeakIlp = 8;
constexpr int kPeakIters = 4096;
constexpr int kPeakThreads = 256;

template <typename T> __global__ void __launch_bounds__(kPeakThreads) fma_peak_kernel(T m, T c, T* sink)
{
    T a[kPeakIlp];
#pragma unroll
    for (int i = 0; i < kPeakIlp; ++i) a[i] = T(threadIdx.x + i) * T(1e-3);
    for (int it = 0; it < kPeakIters; ++it) {
#pragma unroll
        for (int i = 0; i < kPeakIlp; ++i) a[i] = fma(a[i], m, c);
    }
    T s = T(0);
#pragma unroll
    for (int i = 0; i < kPeakIlp; ++i) s += a[i];
    if (s == T(-12345.678)) *sink = s;   // never true for these inputs; keeps the chains live
}

template <typename T> pstd_status measure(double* tflops)
{
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return PSTD_ECUDA;
    T* sink = nullptr;
    if (cudaMalloc(&sink, sizeof(T)) != cudaSuccess) return PSTD_ENOMEM;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    pstd_status st = PSTD_OK;
    const int blocks = nsm * 8;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = PSTD_ECUDA;
    float best = 0.0f;
    for (int rep = 0; rep < 6 && st == PSTD_OK; ++rep) {
        cudaEventRecord(e0, 0);
        fma_peak_kernel<T><<<blocks, kPeakThreads>>>(T(0.999999), T(1e-7), sink);
        cudaEventRecord(e1, 0);
        if (cudaEventSynchronize(e1) != cudaSuccess) { st = PSTD_ECUDA; break; }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && (best == 0.0f || ms < best)) best = ms;   // the first launch warms up
    }
    if (st == PSTD_OK) {
        const double flops = 2.0 * kPeakIlp * kPeakIters * (double)kPeakThreads * blocks;
        *tflops = flops / (best * 1e-3) / 1e12;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    return st;
}

}  // namespace

extern "C" pstd_status pstd_measure_fma_peak(int precision, double* tflops)
{
    if (!tflops || (precision != PSTD_F32 && precision != PSTD_F64)) return PSTD_EINVAL;
    return precision == PSTD_F32 ? measure<float>(tflops) : measure<double>(tflops);
}

// ---------------------------------------------------------------------------------------
// Self-test of the bounded mbarrier wait that the TMA-fed passes use: a barrier on which
// nothing ever arrives, waited on with a caller-given limit.  The wait must give up after
// the limit and the kernel return normally, leaving the context usable.
// ---------------------------------------------------------------------------------------
#include "step_kernels.cuh"

namespace {

__global__ void wait_probe_kernel(unsigned long long limit_ns, unsigned long long* out)
{
    __shared__ __align__(8) unsigned long long bar;
    if (threadIdx.x == 0) {
        pstd::mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const unsigned long long t0 = pstd::global_ns();
    const bool completed = pstd::mbar_wait_bounded(&bar, 0, limit_ns);   // nothing arrives
    const unsigned long long waited = pstd::global_ns() - t0;
    if (threadIdx.x == 0) {
        out[0] = completed ? 1ull : 0ull;
        out[1] = waited;
    }
}

}  // namespace

extern "C" pstd_status pstd_selftest_bounded_wait(double limit_s, double* waited_s)
{
    if (!(limit_s > 0.0) || limit_s > 1.0 || !waited_s) return PSTD_EINVAL;
    unsigned long long* d = nullptr;
    if (cudaMalloc(&d, 2 * sizeof(unsigned long long)) != cudaSuccess) return PSTD_ENOMEM;
    unsigned long long h[2] = {2, 0};
    pstd_status st = PSTD_ECUDA;
    wait_probe_kernel<<<1, 32>>>((unsigned long long)(limit_s * 1e9), d);
    if (cudaGetLastError() == cudaSuccess && cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost) == cudaSuccess) {
        *waited_s = (double)h[1] * 1e-9;
        st = h[0] == 0 ? PSTD_ETIMEOUT : PSTD_OK;
    }
    cudaFree(d);
    return st;
}
