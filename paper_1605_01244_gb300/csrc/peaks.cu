// CUDA-core FMA throughput microbenchmark (FP64 and FP32), used to state the
// ALU roofline of the window sums: many independent FMA chains per thread,
// every SM busy, timed with CUDA events.
#include "internal.cuh"

namespace {

template <typename R>
__global__ void __launch_bounds__(256) fma_chains_kernel(R *out, int iters, R b, R c) {
    R a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = (R)(threadIdx.x + k) * (R)1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int k = 0; k < 8; ++k) a[k] = fma(a[k], b, c);
        }
    }
    R s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    if (s == (R)-12345.0) out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains live
}

template <typename R> double run(int iters, cudaStream_t st) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = sms * 8, threads = 256;
    R *out = nullptr;
    if (cudaMalloc(&out, sizeof(R) * blocks * threads) != cudaSuccess) return -1.0;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    fma_chains_kernel<R><<<blocks, threads, 0, st>>>(out, 2, (R)0.999999, (R)1e-7);  // warm-up
    cudaEventRecord(e0, st);
    fma_chains_kernel<R><<<blocks, threads, 0, st>>>(out, iters, (R)0.999999, (R)1e-7);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (cudaGetLastError() != cudaSuccess || ms <= 0.f) return -1.0;
    const double flops = 2.0 * 8 * 16 * (double)iters * blocks * threads;
    return flops / (ms * 1e-3) / 1e12;
}

}  // namespace

extern "C" int nfft3_fma_peak(int prec, int iters, void *stream, double *tflops) {
    if (!tflops || (prec != 64 && prec != 32) || iters <= 0) return NFFT3_ERR_ARG;
    const double v = prec == 64 ? run<double>(iters, (cudaStream_t)stream)
                                : run<float>(iters, (cudaStream_t)stream);
    if (v < 0) return NFFT3_ERR_CUDA;
    *tflops = v;
    return NFFT3_OK;
}
