// Largest input magnitude of a call, as the exponent rank the FP64 family's
// range scaling needs (value_rank in internal.cuh): one grid-stride pass over
// the input doubles, a warp max, one atomicMax per warp.
#include "internal.cuh"

namespace gbnfft {
namespace {

__global__ void __launch_bounds__(256) value_rank_kernel(const unsigned long long *__restrict__ v, int64_t count,
                                                         int *__restrict__ rank) {
    int best = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int r = value_rank(__ldg(v + i));
        best = r > best ? r : best;
    }
    best = __reduce_max_sync(0xffffffffu, (unsigned)best);
    if ((threadIdx.x & 31) == 0 && best > 0) atomicMax(rank, best);
}

}  // namespace

cudaError_t launch_value_rank(const double *v, int64_t count, int *rank, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (count + 255) / 256;
    const int64_t cap = (int64_t)(sms > 0 ? sms : 1) * 8;
    value_rank_kernel<<<(unsigned)(want < cap ? want : cap), 256, 0, st>>>(
        reinterpret_cast<const unsigned long long *>(v), count, rank);
    return cudaGetLastError();
}

}  // namespace gbnfft
