// Double-float gathers, one thread per point: the grid split and the value
// gather (the kernels are in gather_df.cuh).
#include "gather_df.cuh"

namespace gbnfft {
namespace {

// Split every FP64 complex grid value into float4 (re_hi, re_lo, im_hi, im_lo),
// in place (same 16 bytes per element).
__global__ void grid_to_df_kernel(double2 *__restrict__ G, int64_t total) {
    float4 *out = reinterpret_cast<float4 *>(G);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = G[e];
        const float rh = __double2float_rn(v.x);
        const float ih = __double2float_rn(v.y);
        float4 o;
        o.x = rh;
        o.y = __double2float_rn(v.x - (double)rh);
        o.z = ih;
        o.w = __double2float_rn(v.y - (double)ih);
        out[e] = o;
    }
}


int grid_blocks_df(int64_t total, int threads) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t want = (total + threads - 1) / threads;
    int64_t cap = (int64_t)sms * 16;
    return (int)(want < cap ? (want < 1 ? 1 : want) : cap);
}

}  // namespace

cudaError_t launch_grid_to_df(double2 *G, int64_t total, cudaStream_t st) {
    const int threads = 256;
    grid_to_df_kernel<<<grid_blocks_df(total, threads), threads, 0, st>>>(G, total);
    return cudaGetLastError();
}

cudaError_t launch_gather_df(const float4 *G, Grid3 g, int m, PointsView<double> pts,
                             const WinTableDF &w, double2 *f, cudaStream_t st) {
    return df_select<1>(G, g, m, pts, w, f, nullptr, st);
}

}  // namespace gbnfft
