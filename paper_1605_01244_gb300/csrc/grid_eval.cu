// Evaluation of the truncated series on a rectilinear grid (the paper's
// igridftn / ndcovlt, Sec. 2.1):
//   f[i1, i2, i3] = sum_k c_k E1[i1, k1] E2[i2, k2] E3[i3, k3],
//   E_d[i, k] = exp(+2 pi i (k - N_d/2) y_d[i])        (torus coordinates y_d),
// as three dense complex contractions, one dimension at a time:
//   T1[k1, k2, i3] = sum_k3 c[k1, k2, k3] E3[i3, k3]
//   T2[k1, i2, i3] = sum_k2 E2[i2, k2] T1[k1, k2, i3]      (batched over k1)
//   f [i1, i2, i3] = sum_k1 E1[i1, k1] T2[k1, i2, i3]
// The exponential matrices come from this file's kernel (phase reduced
// exactly before the sine/cosine); the contractions are plain cuBLAS
// Z/CGEMMs.  The paper's own regular-grid check compares this evaluation with
// the inverse FFT.
#include <cublas_v2.h>

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

// one cuBLAS handle per host thread, bound to the call's stream
cublasHandle_t handle_for(cudaStream_t st, int *err) {
    static thread_local cublasHandle_t h = nullptr;
    static thread_local int dev = -1;
    int d = 0;
    cudaGetDevice(&d);
    if (h && d != dev) {
        cublasDestroy(h);
        h = nullptr;
    }
    if (!h) {
        if (cublasCreate(&h) != CUBLAS_STATUS_SUCCESS) {
            h = nullptr;
            *err = 1;
            return nullptr;
        }
        dev = d;
    }
    *err = cublasSetStream(h, st) != CUBLAS_STATUS_SUCCESS;
    return h;
}

size_t ws_elems(int N1, int N2, int N3, int M1, int M2, int M3) {
    return (size_t)M1 * N1 + (size_t)M2 * N2 + (size_t)M3 * N3 + (size_t)N1 * N2 * M3 + (size_t)N1 * M2 * M3;
}

template <typename C>
int grid_eval(const C *c, int N1, int N2, int N3, const double *y1, int M1, const double *y2, int M2,
              const double *y3, int M3, C *f, void *workspace, size_t ws_bytes, cudaStream_t st) {
    if (N1 < 1 || N2 < 1 || N3 < 1 || M1 < 0 || M2 < 0 || M3 < 0) return NFFT3_ERR_ARG;
    if ((int64_t)N1 * N2 > INT32_MAX || (int64_t)M2 * M3 > INT32_MAX) return NFFT3_ERR_TOO_LARGE;
    if ((int64_t)M1 * M2 * M3 == 0) return NFFT3_OK;
    if (!c || !y1 || !y2 || !y3 || !f || !workspace) return NFFT3_ERR_ARG;
    if (ws_bytes < sizeof(C) * ws_elems(N1, N2, N3, M1, M2, M3)) return NFFT3_ERR_ARG;
    C *E1 = (C *)workspace, *E2 = E1 + (size_t)M1 * N1, *E3 = E2 + (size_t)M2 * N2;
    C *T1 = E3 + (size_t)M3 * N3, *T2 = T1 + (size_t)N1 * N2 * M3;
    exp_matrix_kernel<C><<<grid_blocks((int64_t)M1 * N1), 256, 0, st>>>(y1, M1, N1, E1);
    exp_matrix_kernel<C><<<grid_blocks((int64_t)M2 * N2), 256, 0, st>>>(y2, M2, N2, E2);
    exp_matrix_kernel<C><<<grid_blocks((int64_t)M3 * N3), 256, 0, st>>>(y3, M3, N3, E3);
    if (cudaGetLastError() != cudaSuccess) return NFFT3_ERR_CUDA;
    int herr = 0;
    cublasHandle_t h = handle_for(st, &herr);
    if (herr) return NFFT3_ERR_CUDA;
    // Row-major X (r x s) is column-major X^T (s x r, leading dimension s).
    // T1 (N1N2 x M3) = c (N1N2 x N3) E3^T:  col-major T1^T = E3 c^T.
    // T2[k1] (M2 x M3) = E2 (M2 x N2) T1[k1]:  col-major T2[k1]^T = T1[k1]^T E2^T.
    // f (M1 x M2M3) = E1 (M1 x N1) T2:  col-major f^T = T2^T E1^T.
    cublasStatus_t s;
    if constexpr (sizeof(C) == 16) {
        const cuDoubleComplex one = make_cuDoubleComplex(1.0, 0.0), zero = make_cuDoubleComplex(0.0, 0.0);
        using Z = cuDoubleComplex;
        s = cublasZgemm(h, CUBLAS_OP_T, CUBLAS_OP_N, M3, N1 * N2, N3, &one, (const Z *)E3, N3, (const Z *)c, N3,
                        &zero, (Z *)T1, M3);
        if (s == CUBLAS_STATUS_SUCCESS)
            s = cublasZgemmStridedBatched(h, CUBLAS_OP_N, CUBLAS_OP_N, M3, M2, N2, &one, (const Z *)T1, M3,
                                          (long long)N2 * M3, (const Z *)E2, N2, 0, &zero, (Z *)T2, M3,
                                          (long long)M2 * M3, N1);
        if (s == CUBLAS_STATUS_SUCCESS)
            s = cublasZgemm(h, CUBLAS_OP_N, CUBLAS_OP_N, M2 * M3, M1, N1, &one, (const Z *)T2, M2 * M3,
                            (const Z *)E1, N1, &zero, (Z *)f, M2 * M3);
    } else {
        const cuComplex one = make_cuComplex(1.f, 0.f), zero = make_cuComplex(0.f, 0.f);
        using Q = cuComplex;
        s = cublasCgemm(h, CUBLAS_OP_T, CUBLAS_OP_N, M3, N1 * N2, N3, &one, (const Q *)E3, N3, (const Q *)c, N3,
                        &zero, (Q *)T1, M3);
        if (s == CUBLAS_STATUS_SUCCESS)
            s = cublasCgemmStridedBatched(h, CUBLAS_OP_N, CUBLAS_OP_N, M3, M2, N2, &one, (const Q *)T1, M3,
                                          (long long)N2 * M3, (const Q *)E2, N2, 0, &zero, (Q *)T2, M3,
                                          (long long)M2 * M3, N1);
        if (s == CUBLAS_STATUS_SUCCESS)
            s = cublasCgemm(h, CUBLAS_OP_N, CUBLAS_OP_N, M2 * M3, M1, N1, &one, (const Q *)T2, M2 * M3,
                            (const Q *)E1, N1, &zero, (Q *)f, M2 * M3);
    }
    if (s != CUBLAS_STATUS_SUCCESS) return NFFT3_ERR_CUDA;
    return cudaGetLastError() == cudaSuccess ? NFFT3_OK : NFFT3_ERR_CUDA;
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
