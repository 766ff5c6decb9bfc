// Vortex-core location: Newton iteration on the zeros of psi (a curve in R^3)
// and de-duplication of converged points.
//
// psi: R^3 -> C gives two real equations F = (Re psi, Im psi) in three
// unknowns; with J = [Re grad psi; Im grad psi] (2 x 3) the minimum-norm
// Gauss-Newton step is  dx = -J^T (J J^T)^{-1} F.  The paper locates cores by
// thresholding rho = |psi|^2 on refined point sets (Sec. 4.3, sftubeeval3);
// this iteration refines such candidates to the zero set of the series.
#include <cmath>

#include "internal.cuh"

namespace gbnfft {
namespace {

template <typename C> __device__ __forceinline__ void load_c(const C *p, int64_t i, double &re, double &im) {
    const C v = p[i];
    re = (double)v.x;
    im = (double)v.y;
}

// status: 0 active, 1 converged (|psi| < tol), 2 singular J J^T, 3 step larger
// than max_step (the seed is not in the basin of a core)
template <typename C>
__global__ void newton_step_kernel(int64_t M, double *__restrict__ x, const C *__restrict__ f,
                                   const C *__restrict__ grad, int *__restrict__ status,
                                   double *__restrict__ resid, double tol, double max_step) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < M;
         j += (int64_t)gridDim.x * blockDim.x) {
        if (status[j] != 0) continue;
        double fr, fi;
        load_c(f, j, fr, fi);
        const double r = sqrt(fr * fr + fi * fi);
        resid[j] = r;
        if (r < tol) {
            status[j] = 1;
            continue;
        }
        double a[3], b[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) load_c(grad, 3 * j + d, a[d], b[d]);
        const double aa = a[0] * a[0] + a[1] * a[1] + a[2] * a[2];
        const double bb = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
        const double ab = a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
        const double det = aa * bb - ab * ab;
        const double scale = (aa + bb) * (aa + bb);
        if (!(det > 1e-30 * scale) || !(scale > 0)) {
            status[j] = 2;
            continue;
        }
        // y = (J J^T)^{-1} F
        const double y0 = (bb * fr - ab * fi) / det;
        const double y1 = (aa * fi - ab * fr) / det;
        double dx[3], n2 = 0;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            dx[d] = -(y0 * a[d] + y1 * b[d]);
            n2 += dx[d] * dx[d];
        }
        if (!(sqrt(n2) <= max_step)) {
            status[j] = 3;
            continue;
        }
#pragma unroll
        for (int d = 0; d < 3; ++d) x[3 * j + d] += dx[d];
    }
}

// keep[i] = 1 if point i converged and no converged point with a lower index
// lies within `radius` (periodic distance on the unit torus); 0 otherwise.
__global__ void dedupe_kernel(int64_t M, const double *__restrict__ x, const int *__restrict__ status,
                              double radius, int *__restrict__ keep) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M;
         i += (int64_t)gridDim.x * blockDim.x) {
        int k = status[i] == 1;
        if (k) {
            const double r2 = radius * radius;
            for (int64_t j = 0; j < i && k; ++j) {
                if (status[j] != 1) continue;
                double d2 = 0;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    double t = x[3 * i + d] - x[3 * j + d];
                    t -= rint(t);
                    d2 += t * t;
                }
                if (d2 <= r2) k = 0;
            }
        }
        keep[i] = k;
    }
}

int blocks_for(int64_t n, int threads) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (n + threads - 1) / threads, cap = (int64_t)sms * 8;
    return (int)(want < cap ? (want < 1 ? 1 : want) : cap);
}

}  // namespace
}  // namespace gbnfft

using namespace gbnfft;

extern "C" int nfft3_newton_step(int prec, int64_t M, double *x, const void *f, const void *grad,
                                 int *status, double *resid, double tol, double max_step,
                                 void *stream) {
    if ((prec != 64 && prec != 32) || M < 0) return NFFT3_ERR_ARG;
    if (M == 0) return NFFT3_OK;
    if (!x || !f || !grad || !status || !resid) return NFFT3_ERR_ARG;
    const cudaStream_t st = (cudaStream_t)stream;
    if (prec == 64)
        newton_step_kernel<double2><<<blocks_for(M, 256), 256, 0, st>>>(
            M, x, (const double2 *)f, (const double2 *)grad, status, resid, tol, max_step);
    else
        newton_step_kernel<float2><<<blocks_for(M, 256), 256, 0, st>>>(
            M, x, (const float2 *)f, (const float2 *)grad, status, resid, tol, max_step);
    return cudaGetLastError() == cudaSuccess ? NFFT3_OK : NFFT3_ERR_CUDA;
}

extern "C" int nfft3_dedupe(int64_t M, const double *x, const int *status, double radius, int *keep,
                            void *stream) {
    if (M < 0 || !(radius >= 0)) return NFFT3_ERR_ARG;
    if (M == 0) return NFFT3_OK;
    if (!x || !status || !keep) return NFFT3_ERR_ARG;
    dedupe_kernel<<<blocks_for(M, 128), 128, 0, (cudaStream_t)stream>>>(M, x, status, radius, keep);
    return cudaGetLastError() == cudaSuccess ? NFFT3_OK : NFFT3_ERR_CUDA;
}
