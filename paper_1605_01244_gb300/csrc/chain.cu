// Chain rule for the point coordinates (the backward pass of f = A(x) c):
// with G_j = dL/d(Re f_j) + i dL/d(Im f_j) and the gradient d_d f_j of
// nfft3*_eval_grad (Sec. 2, the series differentiated term by term),
//     dL/dx_{j,d} = Re(conj(G_j) d_d f_j) = Re G_j Re d_d f_j + Im G_j Im d_d f_j.
// One thread per point: one complex G load, three complex gradient loads, three
// doubles stored -- HBM-bound, coalesced along j.
#include "internal.cuh"

namespace gbnfft {
namespace {

template <typename R>
__global__ void __launch_bounds__(256) chain_x_kernel(const R *__restrict__ G, const R *__restrict__ grad,
                                                      double *__restrict__ gx, int64_t M) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < M;
         j += (int64_t)gridDim.x * blockDim.x) {
        const double gr = (double)G[2 * j], gi = (double)G[2 * j + 1];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const int64_t e = 2 * (3 * j + d);
            gx[3 * j + d] = fma(gr, (double)grad[e], gi * (double)grad[e + 1]);
        }
    }
}

}  // namespace

template <typename R>
cudaError_t launch_chain_x(const R *G, const R *grad, double *gx, int64_t M, cudaStream_t st) {
    if (M <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (M + 255) / 256;
    const int64_t cap = (int64_t)(sms > 0 ? sms : 1) * 8;
    chain_x_kernel<R><<<(unsigned)(want < cap ? want : cap), 256, 0, st>>>(G, grad, gx, M);
    return cudaGetLastError();
}

template cudaError_t launch_chain_x<double>(const double *, const double *, double *, int64_t, cudaStream_t);
template cudaError_t launch_chain_x<float>(const float *, const float *, double *, int64_t, cudaStream_t);

}  // namespace gbnfft
