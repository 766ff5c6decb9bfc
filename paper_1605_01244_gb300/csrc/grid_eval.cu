// Evaluation of the truncated series on a rectilinear grid (the paper's
// igridftn / ndcovlt, Sec. 2.1):
//   f[i1, i2, i3] = sum_k c_k E1[i1, k1] E2[i2, k2] E3[i3, k3],
//   E_d[i, k] = exp(+2 pi i (k - N_d/2) y_d[i])        (torus coordinates y_d),
// as three dense complex contractions, one dimension at a time:
//   T1[k1, k2, i3] = sum_k3 c[k1, k2, k3] E3[i3, k3]
//   T2[k1, i2, i3] = sum_k2 E2[i2, k2] T1[k1, k2, i3]      (batched over k1)
//   f [i1, i2, i3] = sum_k1 E1[i1, k1] T2[k1, i2, i3]
// The exponential matrices come from this file's kernel (phase reduced
// exactly before the sine/cosine); the contractions are this library's
// complex matrix products (cgemm.cu: FP32 for the mixed family, FP64 or,
// with GBNFFT_GRID_DF=1, double-float for the FP64 family).  The paper's own
// regular-grid check compares this evaluation with the inverse FFT.
#include <cstdlib>
#include <cstring>

#include "internal.cuh"

namespace gbnfft {
namespace {

// E[i, k] = exp(2 pi i kk y_i), kk = k - N/2, with kk y_i reduced to [-1/2, 1/2]
// exactly: p + e = kk y_i (error-free product), r = (p - rint(p)) + e.
template <typename C>
__global__ void exp_matrix_kernel(const double *__restrict__ y, int M, int N, C *__restrict__ E) {
    const int64_t total = (int64_t)M * N;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(t / N), k = (int)(t - (int64_t)i * N);
        const double kk = (double)(k - N / 2);
        const double p = __dmul_rn(kk, y[i]);
        const double e = fma(kk, y[i], -p);
        const double r = __dadd_rn(__dsub_rn(p, rint(p)), e);
        double s, c;
        sincospi(2.0 * r, &s, &c);
        E[t].x = c;
        E[t].y = s;
    }
}

int grid_blocks(int64_t n) {
    const int64_t b = (n + 255) / 256;
    return (int)(b < 1 ? 1 : (b > 152 * 64 ? 152 * 64 : b));
}

size_t ws_elems(int N1, int N2, int N3, int M1, int M2, int M3) {
    // + 1 element: the range word of the double-float variant
    return (size_t)M1 * N1 + (size_t)M2 * N2 + (size_t)M3 * N3 + (size_t)N1 * N2 * M3 + (size_t)N1 * M2 * M3 + 1;
}

template <typename C>
int grid_eval(const C *c, int N1, int N2, int N3, const double *y1, int M1, const double *y2, int M2,
              const double *y3, int M3, C *f, void *workspace, size_t ws_bytes, cudaStream_t st) {
    if (N1 < 1 || N2 < 1 || N3 < 1 || M1 < 0 || M2 < 0 || M3 < 0) return NFFT3_ERR_ARG;
    if ((int64_t)N1 * N2 > INT32_MAX || (int64_t)M2 * M3 > INT32_MAX) return NFFT3_ERR_TOO_LARGE;
    if ((int64_t)N1 * N2 > 65535 * 64 || M1 > 65535 * 64 || M2 > 65535 * 64 || N1 > 65535)
        return NFFT3_ERR_TOO_LARGE;   // grid limits of the product kernels
    if ((int64_t)M1 * M2 * M3 == 0) return NFFT3_OK;
    if (!c || !y1 || !y2 || !y3 || !f || !workspace) return NFFT3_ERR_ARG;
    if (ws_bytes < sizeof(C) * ws_elems(N1, N2, N3, M1, M2, M3)) return NFFT3_ERR_ARG;
    C *E1 = (C *)workspace, *E2 = E1 + (size_t)M1 * N1, *E3 = E2 + (size_t)M2 * N2;
    C *T1 = E3 + (size_t)M3 * N3, *T2 = T1 + (size_t)N1 * N2 * M3;
    int *rank = (int *)(T2 + (size_t)N1 * M2 * M3);
    exp_matrix_kernel<C><<<grid_blocks((int64_t)M1 * N1), 256, 0, st>>>(y1, M1, N1, E1);
    exp_matrix_kernel<C><<<grid_blocks((int64_t)M2 * N2), 256, 0, st>>>(y2, M2, N2, E2);
    exp_matrix_kernel<C><<<grid_blocks((int64_t)M3 * N3), 256, 0, st>>>(y3, M3, N3, E3);
    if (cudaGetLastError() != cudaSuccess) return NFFT3_ERR_CUDA;
    int arith = kGemmF32;
    const int *vexp = nullptr;
    if constexpr (sizeof(C) == 16) {
        // FP64 family: FP64 products by default; GBNFFT_GRID_DF=1 selects the
        // double-float products (scaled into range by c's largest magnitude)
        const char *v = std::getenv("GBNFFT_GRID_DF");
        arith = v && !std::strcmp(v, "1") ? kGemmDF : kGemmF64;
        if (arith == kGemmDF) {
            if (cudaMemsetAsync(rank, 0, sizeof(int), st) != cudaSuccess ||
                launch_value_rank((const double *)c, 2 * (int64_t)N1 * N2 * N3, rank, st) != cudaSuccess)
                return NFFT3_ERR_CUDA;
            vexp = rank;
        }
    }
    // T1 (N1 N2 x M3) = c (N1 N2 x N3) E3^T            (E3 read transposed)
    // T2[k1] (M2 x M3) = E2 (M2 x N2) T1[k1] (N2 x M3)  (batched over k1)
    // f (M1 x M2 M3) = E1 (M1 x N1) T2 (N1 x M2 M3)
    cudaError_t e = launch_cgemm(arith, c, N3, 0, E3, N3, 0, true, T1, M3, 0, N1 * N2, M3, N3, 1, vexp, 1, 0, st);
    if (e == cudaSuccess)
        e = launch_cgemm(arith, E2, N2, 0, T1, M3, (int64_t)N2 * M3, false, T2, M3, (int64_t)M2 * M3, M2, M3, N2, N1,
                         nullptr, 0, 0, st);
    if (e == cudaSuccess)
        e = launch_cgemm(arith, E1, N1, 0, T2, (int64_t)M2 * M3, 0, false, f, (int64_t)M2 * M3, 0, M1, M2 * M3, N1,
                         1, vexp, 0, 1, st);
    return e == cudaSuccess ? NFFT3_OK : NFFT3_ERR_CUDA;
}

}  // namespace
}  // namespace gbnfft

using namespace gbnfft;

extern "C" {

size_t nfft3_grid_eval_workspace_bytes(int prec, int N1, int N2, int N3, int M1, int M2, int M3) {
    if (N1 < 1 || N2 < 1 || N3 < 1 || M1 < 0 || M2 < 0 || M3 < 0) return 0;
    return (prec == 64 ? 16 : 8) * ws_elems(N1, N2, N3, M1, M2, M3);
}

int nfft3d_grid_eval(const double *c, int N1, int N2, int N3, const double *y1, int M1, const double *y2, int M2,
                     const double *y3, int M3, double *f, void *workspace, size_t ws_bytes, void *stream) {
    return grid_eval<double2>((const double2 *)c, N1, N2, N3, y1, M1, y2, M2, y3, M3, (double2 *)f, workspace,
                              ws_bytes, (cudaStream_t)stream);
}

int nfft3f_grid_eval(const float *c, int N1, int N2, int N3, const double *y1, int M1, const double *y2, int M2,
                     const double *y3, int M3, float *f, void *workspace, size_t ws_bytes, void *stream) {
    return grid_eval<float2>((const float2 *)c, N1, N2, N3, y1, M1, y2, M2, y3, M3, (float2 *)f, workspace,
                             ws_bytes, (cudaStream_t)stream);
}

}  // extern "C"
