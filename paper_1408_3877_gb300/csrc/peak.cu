// Throughput of dependent-free multiply-add streams on this device (FP32 or FP64): the
// ALU ceiling the operator kernels are compared with.  Each thread runs 8 independent
// chains; the chains' results are summed into one store so that nothing is optimised away.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"

namespace {

template <typename T, int ITERS>
__global__ void __launch_bounds__(256) k_fma_peak(T *out, T a, T b) {
    T x[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = (T)(threadIdx.x + c);
#pragma unroll 16
    for (int i = 0; i < ITERS; ++i) {
#pragma unroll
        for (int c = 0; c < 8; ++c) x[c] = x[c] * a + b;
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += x[c];
    if (s == (T)-1.2345) out[0] = s;  // practically never: keeps the chains alive
}

template <typename T>
int run(double *tflops) {
    constexpr int ITERS = 4096;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return FESTUNG_ECUDA;
    T *out = nullptr;
    if (cudaMalloc(&out, sizeof(T)) != cudaSuccess) return FESTUNG_ENOMEM;
    const int blocks = sms * 8, threads = 256;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const T a = (T)0.999999, b = (T)1e-7;
    k_fma_peak<T, ITERS><<<blocks, threads>>>(out, a, b);  // warm-up
    float best = 1e30f;
    for (int rep = 0; rep < 5; ++rep) {
        cudaEventRecord(e0);
        k_fma_peak<T, ITERS><<<blocks, threads>>>(out, a, b);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        best = std::min(best, ms);
    }
    const cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (err != cudaSuccess) return FESTUNG_ECUDA;
    const double flops = 2.0 * 8.0 * ITERS * (double)blocks * threads;
    *tflops = flops / (best * 1e-3) / 1e12;
    return FESTUNG_OK;
}

}  // namespace

extern "C" int festung_fma_peak(int prec, double *tflops) {
    if (!tflops || (prec != FESTUNG_FP32 && prec != FESTUNG_FP64)) return FESTUNG_EINVAL;
    return prec == FESTUNG_FP32 ? run<float>(tflops) : run<double>(tflops);
}
