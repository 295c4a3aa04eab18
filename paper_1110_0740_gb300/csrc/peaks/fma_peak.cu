// fma_peak.cu -- FMA-throughput microbenchmark of the non-tensor pipes
// (float32 FFMA, float64 DFMA): the measured ALU peaks beside which the
// step's arithmetic roofline is read.  Every thread runs CHAINS independent
// dependency chains of fused multiply-adds; the grid fills every SM several
// times over.  The result depends on the operands, so nothing is folded
// away, and is stored only in a branch no input takes.
#include <cuda_runtime.h>

#include "ctu_peaks.h"

namespace {

constexpr int CHAINS = 8;
constexpr int FMA_BLOCK = 256;

template <class T>
__global__ void __launch_bounds__(FMA_BLOCK) k_fma(T a, T b, int iters, T *sink)
{
    T x[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
#pragma unroll 16
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) x[c] = fma(x[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += x[c];
    if (s == (T)-1.25e-7) sink[blockIdx.x] = s;
}

template <class T>
ctu_status run(int iters, double *flops_per_s, void *stream)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return CTU_ECUDA;
    T *sink = nullptr;
    const int blocks = sms * 16;
    if (cudaMalloc(&sink, sizeof(T) * blocks) != cudaSuccess) return CTU_ENOMEM;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // a = 1 - 2^-20 keeps the chains bounded without denormals
    const T a = (T)0.99999904632568359375, b = (T)1e-6;
    k_fma<T><<<blocks, FMA_BLOCK, 0, s>>>(a, b, iters / 8 + 1, sink);  // warm-up
    cudaEventRecord(e0, s);
    k_fma<T><<<blocks, FMA_BLOCK, 0, s>>>(a, b, iters, sink);
    cudaEventRecord(e1, s);
    ctu_status st = CTU_OK;
    float ms = 0.0f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.0f)
        st = CTU_ECUDA;
    else
        *flops_per_s = 2.0 * CHAINS * (double)iters * blocks * FMA_BLOCK / (ms * 1e-3);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    return st;
}

} // namespace

extern "C" ctu_status ctu_fma_peak(int fp64, int iters, double *flops_per_s, void *stream)
{
    if (!flops_per_s || iters < 1) return CTU_EINVAL;
    return fp64 ? run<double>(iters, flops_per_s, stream) : run<float>(iters, flops_per_s, stream);
}
