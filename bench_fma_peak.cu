// bench_fma_peak.cu -- measured FP32 and FP64 FMA throughput of the current GPU (libbench_fma_peak.so, built by bench.py).
//
// A measurement probe for the benchmark, not part of the lattice Boltzmann library: it shows
// where the FP32 and FP64 arithmetic ceilings lie relative to the step kernels, which are bound
// by HBM bandwidth (FP32, 16-bit storage) or by FP64 arithmetic (FP64 storage).
//
//   int fma_peak(int fp64, double* tflops)
// runs eight independent FMA chains per thread on 8 blocks of 256 threads per SM, times one
// launch with CUDA events after a warm-up launch, and writes 2 x FMAs / time in TFLOP/s.
// Returns 0, or the CUDA error code.
#include <cuda_runtime.h>

namespace {

template <class T>
__global__ void __launch_bounds__(256) k_fma(T* __restrict__ out, int iters, T a, T b) {
    T x0 = T(threadIdx.x) * T(1e-3), x1 = x0 + T(1), x2 = x0 + T(2), x3 = x0 + T(3);
    T x4 = x0 + T(4), x5 = x0 + T(5), x6 = x0 + T(6), x7 = x0 + T(7);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            x0 = fma(x0, a, b);
            x1 = fma(x1, a, b);
            x2 = fma(x2, a, b);
            x3 = fma(x3, a, b);
            x4 = fma(x4, a, b);
            x5 = fma(x5, a, b);
            x6 = fma(x6, a, b);
            x7 = fma(x7, a, b);
        }
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
}

template <class T>
int run(int iters, double* tflops) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return (int)e;
    const int blocks = 8 * sms, threads = 256;
    T* out = nullptr;
    e = cudaMalloc(&out, sizeof(T) * (size_t)blocks * threads);
    if (e != cudaSuccess) return (int)e;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // a just below 1 and a small b keep every chain in the normal range
    k_fma<T><<<blocks, threads>>>(out, iters, T(0.999999), T(1e-6));
    cudaEventRecord(e0);
    k_fma<T><<<blocks, threads>>>(out, iters, T(0.999999), T(1e-6));
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess) return (int)e;
    const double fmas = (double)blocks * threads * iters * 16.0 * 8.0;
    *tflops = 2.0 * fmas / (ms * 1e-3) / 1e12;
    return 0;
}

}  // namespace

extern "C" int fma_peak(int fp64, double* tflops) {
    if (!tflops) return -1;
    return fp64 ? run<double>(256, tflops) : run<float>(16384, tflops);
}
