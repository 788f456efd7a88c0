// Measured FP32 and FP64 FMA throughput of the current GPU: the roofline denominators of the
// ALU-bound kernels (the near field and MtL in FP32, the singular integrals in FP64 or
// float-float). Each thread runs eight independent FMA chains for a fixed count, on enough
// blocks to fill every SM; the rate is 2 x FMAs / elapsed time between two CUDA events.
#include <cuda_runtime.h>

#include "pb_internal.cuh"

template <class T>
__global__ void __launch_bounds__(256) k_fma_chain(T* __restrict__ out, int iters, T a, T b)
{
    T x[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = T(threadIdx.x + c) * T(1e-3);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int c = 0; c < 8; ++c) x[c] = fma(x[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <class T>
static int time_chain(cudaStream_t st, int nsm, int iters, double* tflops)
{
    const int blocks = nsm * 8, threads = 256;
    T* out = nullptr;
    if (cudaMallocAsync(&out, sizeof(T) * blocks * threads, st) != cudaSuccess) return PB_ERR_NOMEM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_fma_chain<T><<<blocks, threads, 0, st>>>(out, iters / 8, T(0.9999), T(1e-4));  // warm-up
    cudaEventRecord(e0, st);
    k_fma_chain<T><<<blocks, threads, 0, st>>>(out, iters, T(0.9999), T(1e-4));
    cudaEventRecord(e1, st);
    int rc = cudaEventSynchronize(e1) == cudaSuccess ? PB_OK : PB_ERR_CUDA;
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(out, st);
    cudaStreamSynchronize(st);
    const double fmas = (double)blocks * threads * iters * 32.0;
    *tflops = ms > 0 ? 2.0 * fmas / (ms * 1e-3) / 1e12 : 0.0;
    return rc;
}

extern "C" int pb_measure_alu_peaks(void* stream, double* fp32_tflops, double* fp64_tflops)
{
    if (!fp32_tflops || !fp64_tflops) return PB_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return PB_ERR_CUDA;
    int rc = time_chain<float>(st, nsm, 20000, fp32_tflops);
    if (!rc) rc = time_chain<double>(st, nsm, 400, fp64_tflops);
    return rc;
}
