// peak_kernels.cu -- FMA-chain measurement of the CUDA-core FP32 / FP64 pipes.
//
// Each thread runs kChains independent FMA chains of kIters steps, so the
// pipe, not the latency of one chain, is the limit.  Grid: 8 CTAs of 256
// threads per SM.  Used as the denominator of the roofline of the build
// kernels, whose work is CUDA-core FMA arithmetic (small ragged QRs).
#include "kernels.h"

namespace rsai {

constexpr int kChains = 8;
constexpr int kIters = 4096;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chain(T *out, T a, T b) {
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == (T)123.456) out[0] = s;  // keeps the chains alive, never true in practice
}

cudaError_t run_peak_fma(bool fp64, cudaStream_t st, double *flops_per_s) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = sms * 8, threads = 256;
    void *out = nullptr;
    cudaError_t e = cudaMallocAsync(&out, 16, st);
    if (e != cudaSuccess) return e;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best_ms = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(e0, st);
        if (fp64) k_fma_chain<double><<<grid, threads, 0, st>>>((double *)out, 0.999999, 1e-7);
        else k_fma_chain<float><<<grid, threads, 0, st>>>((float *)out, 0.999999f, 1e-7f);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best_ms) best_ms = ms;  // first launch is warm-up
    }
    e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(out, st);
    cudaStreamSynchronize(st);
    double flops = 2.0 * (double)grid * threads * kChains * (double)kIters;
    *flops_per_s = flops / (best_ms * 1e-3);
    return e;
}

}  // namespace rsai
