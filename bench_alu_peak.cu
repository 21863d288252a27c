// Measured FP64 and FP32 fused multiply-add throughput of the device: the
// denominators of the FP64 and FP32 stage kernels' ALU rooflines, beside the
// nominal figures (152 SMs x lanes x 2 flops x clock).
//
// Every thread runs eight independent multiply-add chains x <- x a + b for
// `iters` iterations (a, b runtime values, so nothing folds); the grid holds
// eight 256-thread blocks per SM. The sum of the chains is stored only if it
// is negative, which it never is, so the work cannot be removed. Built as its
// own library (libgbr_probe.so) from beside the benchmark: it is
// measurement, not part of the solver.
#include <cuda_runtime.h>

namespace {

template <typename T>
__global__ void __launch_bounds__(256) fma_chains(T* out, T a, T b, int iters)
{
    T x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = T(threadIdx.x) * T(1e-3) + T(k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
    }
    T s = T(0);
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    if (s < T(0)) out[blockIdx.x] = s;
}

template <typename T>
int run(int iters, double* gflops)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -2;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -2;
    const int blocks = 8 * sms;
    T* out = nullptr;
    if (cudaMalloc(&out, sizeof(T) * blocks) != cudaSuccess) return -2;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const T a = T(0.999999), b = T(1e-6);
    fma_chains<T><<<blocks, 256>>>(out, a, b, iters);  // warm-up
    float best = 0.f;
    for (int r = 0; r < 5; ++r) {
        cudaEventRecord(e0);
        fma_chains<T><<<blocks, 256>>>(out, a, b, iters);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r == 0 || ms < best) best = ms;
    }
    const cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (err != cudaSuccess || best <= 0.f) return -2;
    const double flops = 2.0 * 8.0 * (double)iters * (double)blocks * 256.0;
    *gflops = flops / (best * 1e-3) / 1e9;
    return 0;
}

}  // namespace

// GFLOP/s of FP64 (precision 64) or FP32 (precision 32) fused multiply-adds
// on the current device, best of five timed launches. Returns 0, -1 for bad
// arguments, -2 for a CUDA error.
extern "C" int gbr_probe_fma_gflops(int precision, int iters, double* gflops)
{
    if (!gflops || iters <= 0) return -1;
    if (precision == 64) return run<double>(iters, gflops);
    if (precision == 32) return run<float>(iters, gflops);
    return -1;
}
