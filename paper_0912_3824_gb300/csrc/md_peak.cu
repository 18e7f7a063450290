// md_peak.cu -- FMA-chain microbenchmark of the CUDA-core arithmetic peaks.
//
// The step kernel is bound by the FP32 / INT32 lanes, not by tensor cores, so
// its roofline needs the FP32 FMA peak of the GPU it runs on; the FP64 leg
// needs the FP64 peak.  Neither is a published, fixed number for a part whose
// clock moves with power, so they are measured: every thread runs kChains
// independent chains of fused multiply-adds (enough in flight to cover the
// FMA latency on every scheduler), the grid fills every SM several times over,
// and the launch is timed with CUDA events.  One FMA counts as 2 flops.
#include <cuda_runtime.h>

#include "md_bench.h"

namespace {

constexpr int kChains = 8;
constexpr int kBlock = 256;

// Written only if the chains produce an impossible value, so the compiler
// keeps every FMA; never read.
__device__ double g_peak_sink;

template <typename T>
__global__ void __launch_bounds__(kBlock) k_fma_chains(long long iters, T b, T c)
{
    T x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k)
        x[k] = (T)(threadIdx.x + k) * (T)1e-3;
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int k = 0; k < kChains; ++k)
                x[k] = fma(x[k], b, c);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k)
        s += x[k];
    if (s == (T)-12345.0)
        g_peak_sink = (double)s;
}

}  // namespace

extern "C" int md_fma_peak(int32_t precision, int64_t iters, double *tflops, double *ms)
{
    if (!tflops || iters < 1 || (precision != 0 && precision != 2))
        return 1;
    int dev = 0, nsm = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 3;
    const void *f = precision == 0 ? (const void *)k_fma_chains<double> : (const void *)k_fma_chains<float>;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, kBlock, 0) != cudaSuccess || per_sm < 1)
        return 3;
    const int grid = nsm * per_sm * 4;              // four full waves
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess)
        return 3;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return 3;
    }
    float best = 0.f;
    int rc = 0;
    for (int rep = 0; rep < 4 && rc == 0; ++rep) {  // the first launch warms the clocks up
        cudaEventRecord(e0, 0);
        if (precision == 0)
            k_fma_chains<double><<<grid, kBlock>>>(iters, 1.0000000001, 1e-12);
        else
            k_fma_chains<float><<<grid, kBlock>>>(iters, 1.000001f, 1e-7f);
        cudaEventRecord(e1, 0);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
            rc = 3;
            break;
        }
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        if (rep == 0 || t < best)
            best = t;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc)
        return rc;
    const double fmas = (double)grid * kBlock * (double)iters * 16.0 * kChains;
    *tflops = 2.0 * fmas / ((double)best * 1e-3) / 1e12;
    if (ms)
        *ms = best;
    return 0;
}
