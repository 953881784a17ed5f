// Arithmetic peak probes: many independent FMA chains per thread, timed
// with CUDA events.  They give the FP64 (DFMA) and FP32 (FFMA) rates this
// GPU sustains, the denominators of the ALU rooflines of the kernels.
#include <cuda_runtime.h>

#include "../../include/aderdg.h"

namespace {

template <typename T, int CHAINS>
__global__ void __launch_bounds__(256) k_fma_chains(int iters, T a, T b, T *sink)
{
    T x[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = T(threadIdx.x + c) * T(1e-3);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) x[c] = x[c] * a + b;
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += x[c];
    if (s == T(12345.678)) sink[threadIdx.x] = s;  // never true; keeps the chains alive
}

template <typename T, int CHAINS>
int run(int iters, double *tflops)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return ADERDG_E_CUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    T *sink = nullptr;
    if (cudaMalloc(&sink, 256 * sizeof(T)) != cudaSuccess) return ADERDG_E_NOMEM;
    const int blocks = sms * 8, threads = 256;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_fma_chains<T, CHAINS><<<blocks, threads>>>(iters / 10, T(0.999999), T(1e-7), sink);  // warm-up
    cudaEventRecord(e0);
    k_fma_chains<T, CHAINS><<<blocks, threads>>>(iters, T(0.999999), T(1e-7), sink);
    cudaEventRecord(e1);
    cudaError_t err = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (err != cudaSuccess) return ADERDG_E_CUDA;
    const double flops = 2.0 * CHAINS * (double)iters * blocks * threads;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return ADERDG_OK;
}

}  // namespace

extern "C" int aderdg_peak_tflops(int kind, double *tflops)
{
    if (!tflops) return ADERDG_E_INVAL;
    if (kind == 0) return run<double, 8>(20000, tflops);
    if (kind == 1) return run<float, 16>(200000, tflops);
    return ADERDG_E_INVAL;
}
