// Arithmetic peak probes: many independent FMA chains per thread, timed
// with CUDA events.  They give the FP64 (DFMA) and FP32 (FFMA) rates this
// GPU sustains, the denominators of the ALU rooflines of the kernels.
// Also the check of the device reciprocal the flux kernels use.
#include <cuda_runtime.h>

#include "../../include/aderdg.h"
#include "common.cuh"

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

__global__ void k_recip(const double *x, double *y, long long n, int single)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = single ? (double)aderdg::recip((float)x[i]) : aderdg::recip(x[i]);
}

}  // namespace

extern "C" int aderdg_device_recip(const double *x, double *y, long long n, int precision)
{
    if (n < 0 || (n > 0 && (!x || !y)) || (precision != ADERDG_FP64 && precision != ADERDG_MIXED_FP32))
        return ADERDG_E_INVAL;
    if (n == 0) return ADERDG_OK;
    if (n > (1ll << 26)) return ADERDG_E_INVAL;
    double *d = nullptr;
    if (cudaMalloc(&d, 2 * n * sizeof(double)) != cudaSuccess) return ADERDG_E_NOMEM;
    cudaError_t e = cudaMemcpy(d, x, n * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_recip<<<(int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096), 256>>>(d, d + n, n,
                                                                             precision == ADERDG_MIXED_FP32);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(y, d + n, n * sizeof(double), cudaMemcpyDeviceToHost);
    cudaFree(d);
    return e == cudaSuccess ? ADERDG_OK : ADERDG_E_CUDA;
}

extern "C" int aderdg_peak_tflops(int kind, double *tflops)
{
    if (!tflops) return ADERDG_E_INVAL;
    if (kind == 0) return run<double, 8>(20000, tflops);
    if (kind == 1) return run<float, 16>(200000, tflops);
    return ADERDG_E_INVAL;
}
