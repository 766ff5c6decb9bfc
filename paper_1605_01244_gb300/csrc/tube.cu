// Tube refinement step of the paper's vortex-tube evaluation (Sec. 4.3,
// sftubeeval3): of M points x_j with values psi_j, keep those with density
// rho_j = |psi_j|^2 <= rhobar and replace each kept point xi by the 27 points
// of the regular grid of step h_d / 3 centred on it,
//     xi + (a h1/3, b h2/3, c h3/3),  a, b, c in {-1, 0, 1}  (c fastest).
// Deterministic: a flag per point, an exclusive scan of the flags, then kept
// point number r writes its children at 27 r (the order of the input points).
#include "internal.cuh"

namespace gbnfft {
namespace {

template <typename C>
__global__ void tube_flag_kernel(const C *__restrict__ psi, int64_t M, double rhobar, int *__restrict__ flag) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j <= M; j += (int64_t)gridDim.x * blockDim.x) {
        if (j == M) {
            flag[j] = 0;   // makes pos[M] the number of kept points
            continue;
        }
        const double re = (double)psi[j].x, im = (double)psi[j].y;
        const double rho = __dadd_rn(__dmul_rn(re, re), __dmul_rn(im, im));
        flag[j] = rho <= rhobar ? 1 : 0;
    }
}

__global__ void tube_children_kernel(const double *__restrict__ x, const int *__restrict__ flag,
                                     const int *__restrict__ pos, int64_t M, double3 h3, double *__restrict__ out,
                                     int64_t cap) {
    // one thread per (point, child)
    const int64_t total = M * 27;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = t / 27;
        if (!flag[j]) continue;
        const int k = (int)(t - j * 27);
        const int64_t o = (int64_t)pos[j] * 27 + k;
        if (o >= cap) continue;
        const int a = k / 9 - 1, b = (k / 3) % 3 - 1, c = k % 3 - 1;
        out[3 * o + 0] = __dadd_rn(x[3 * j + 0], (double)a * h3.x);
        out[3 * o + 1] = __dadd_rn(x[3 * j + 1], (double)b * h3.y);
        out[3 * o + 2] = __dadd_rn(x[3 * j + 2], (double)c * h3.z);
    }
}

int grid_for(int64_t n) {
    const int64_t b = (n + 255) / 256;
    return (int)(b < 1 ? 1 : (b > 65535 * 8 ? 65535 * 8 : b));
}

}  // namespace
}  // namespace gbnfft

using namespace gbnfft;

extern "C" {

size_t nfft3_tube_workspace_bytes(int64_t M) {
    if (M < 0) return 0;
    return sizeof(int) * (2 * (size_t)(M + 1) + scan_tmp_ints(M + 1));
}

int nfft3_tube_refine(int prec, const double *x, const void *psi, int64_t M, double rhobar, const double *h,
                      double *out, int64_t cap, int64_t *kept, void *workspace, size_t ws_bytes, void *stream) {
    if ((prec != 64 && prec != 32) || M < 0 || !h || !kept || cap < 0) return NFFT3_ERR_ARG;
    if (M > (int64_t)1 << 30) return NFFT3_ERR_TOO_LARGE;   // pos[] is int and 27 * kept must fit
    if (M > 0 && (!x || !psi || !workspace || (cap > 0 && !out))) return NFFT3_ERR_ARG;
    if (ws_bytes < nfft3_tube_workspace_bytes(M)) return NFFT3_ERR_ARG;
    *kept = 0;
    if (M == 0) return NFFT3_OK;
    cudaStream_t st = (cudaStream_t)stream;
    int *flag = (int *)workspace;
    int *pos = flag + (M + 1);
    int *tmp = pos + (M + 1);
    if (prec == 64)
        tube_flag_kernel<double2><<<grid_for(M + 1), 256, 0, st>>>((const double2 *)psi, M, rhobar, flag);
    else
        tube_flag_kernel<float2><<<grid_for(M + 1), 256, 0, st>>>((const float2 *)psi, M, rhobar, flag);
    if (cudaGetLastError() != cudaSuccess) return NFFT3_ERR_CUDA;
    if (exclusive_scan(flag, pos, M + 1, tmp, st) != cudaSuccess) return NFFT3_ERR_CUDA;
    const double3 h3 = make_double3(h[0] / 3.0, h[1] / 3.0, h[2] / 3.0);
    if (cap > 0) {
        tube_children_kernel<<<grid_for(27 * M), 256, 0, st>>>(x, flag, pos, M, h3, out, cap);
        if (cudaGetLastError() != cudaSuccess) return NFFT3_ERR_CUDA;
    }
    int total = 0;
    if (cudaMemcpyAsync(&total, pos + M, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return NFFT3_ERR_CUDA;
    *kept = total;
    return 27 * (int64_t)total > cap ? NFFT3_ERR_TOO_LARGE : NFFT3_OK;
}

}  // extern "C"
