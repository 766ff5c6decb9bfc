// One- and two-dimensional NFFT (the paper's infft and infft2, Appendix B):
//   f_j = sum_{k in I_N} c_k exp(+2 pi i k.x_j),   k_d in [-N_d/2, N_d/2),  d < dim,
// FP64, the same approximation as the 3D path: Kaiser-Bessel window of
// half-width alpha = m + 1/2 in grid units, deconvolution by
// (-1)^k phi(0) / Phi(k / n), unnormalised inverse FFT of the zero-padded
// n_1 (x n_2) grid, window sum over the 2m+1 (squared) taps.
// Three steps on the stream: deconvolve + zero-pad (this file), cuFFT Z2Z
// (inverse), gather (this file, one thread per point, window weights from
// their closed form, coordinates reduced exactly as in set_points).
#include <cufft.h>

#include <map>
#include <tuple>

#include "reduce.cuh"

namespace gbnfft {
namespace {

constexpr double kPi = 3.141592653589793238462643383279502884;

// I0 by its positive power series (accurate to rounding for x < 60)
__device__ double bessel_i0_dev(double x) {
    const double t = 0.25 * x * x;
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 400; ++k) {
        term *= t / ((double)k * (double)k);
        sum += term;
        if (term < 1e-17 * sum) break;
    }
    return sum;
}

struct LowArgs {
    int dim, N1, N2, n1, n2, m;
    double b1, b2;
};

// D_d[i] = (-1)^k phi(0) / Phi(k / n_d), k = i - N_d / 2, phi(0) = sinh(b alpha) / (pi alpha)
__global__ void low_deconv_table_kernel(LowArgs a, double *D1, double *D2) {
    const double al = a.m + 0.5;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < a.N1 + a.N2; t += gridDim.x * blockDim.x) {
        const bool first = t < a.N1;
        const int Nd = first ? a.N1 : a.N2, nd = first ? a.n1 : a.n2, i = first ? t : t - a.N1;
        const double b = first ? a.b1 : a.b2;
        const int k = i - Nd / 2;
        const double nu = 2.0 * kPi * (double)k / (double)nd;
        const double phi0 = sinh(b * al) / (kPi * al);
        const double v = ((k & 1) ? -1.0 : 1.0) * phi0 / bessel_i0_dev(al * sqrt(b * b - nu * nu));
        (first ? D1 : D2)[i] = v;
    }
}

// G[k mod n] = c_k D1[k1] (D2[k2]), zero elsewhere
__global__ void low_deconv_scatter_kernel(const double2 *__restrict__ c, LowArgs a, const double *__restrict__ D1,
                                          const double *__restrict__ D2, double2 *__restrict__ G) {
    const int64_t total = (int64_t)a.n1 * a.n2;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int l1 = (int)(t / a.n2), l2 = (int)(t - (int64_t)l1 * a.n2);
        const int k1 = l1 < a.N1 / 2 ? l1 : (l1 >= a.n1 - a.N1 / 2 ? l1 - a.n1 : INT32_MIN);
        const int k2 = a.dim == 1 ? 0 : (l2 < a.N2 / 2 ? l2 : (l2 >= a.n2 - a.N2 / 2 ? l2 - a.n2 : INT32_MIN));
        double2 v = make_double2(0.0, 0.0);
        if (k1 != INT32_MIN && k2 != INT32_MIN) {
            const int i1 = k1 + a.N1 / 2, i2 = a.dim == 1 ? 0 : k2 + a.N2 / 2;
            const double d = D1[i1] * (a.dim == 1 ? 1.0 : D2[i2]);
            const double2 cv = c[(int64_t)i1 * (a.dim == 1 ? 1 : a.N2) + i2];
            v = make_double2(cv.x * d, cv.y * d);
        }
        G[t] = v;
    }
}

// normalised window weight of tap a at offset s: (alpha / q) sinh(b q) / sinh(b alpha),
// q = sqrt((s + a)(2m + 1 - s - a)) (value alpha b / sinh(b alpha) at q = 0)
__device__ __forceinline__ double low_weight(double s, int tap, int m, double b) {
    const double al = m + 0.5;
    const double q2 = (s + tap) * (2 * m + 1 - s - tap);
    if (q2 <= 0.0) return al * b / sinh(b * al);
    const double q = sqrt(q2);
    return (al / q) * sinh(b * q) / sinh(b * al);
}

__global__ void low_gather_kernel(const double2 *__restrict__ G, LowArgs a, const double *__restrict__ x,
                                  int64_t M, double2 *__restrict__ f, int *__restrict__ status) {
    const int W = 2 * a.m + 1;
    const CoordParams cp1 = coord_params(a.n1, a.m), cp2 = coord_params(a.n2, a.m);
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < M; j += (int64_t)gridDim.x * blockDim.x) {
        const Reduced r1 = reduce_coord(x[(int64_t)a.dim * j], cp1, status);
        Reduced r2{0, 0.0};
        if (a.dim == 2) r2 = reduce_coord(x[2 * j + 1], cp2, status);
        double w2[kMaxTaps];
        if (a.dim == 2)
            for (int q = 0; q < W; ++q) w2[q] = low_weight(r2.s, q, a.m, a.b2);
        double re = 0.0, im = 0.0;
        for (int p = 0; p < W; ++p) {
            int i1 = r1.l0 + p;
            while (i1 >= a.n1) i1 -= a.n1;
            const double w1 = low_weight(r1.s, p, a.m, a.b1);
            if (a.dim == 1) {
                const double2 g = G[i1];
                re = fma(w1, g.x, re);
                im = fma(w1, g.y, im);
                continue;
            }
            double sr = 0.0, si = 0.0;
            for (int q = 0; q < W; ++q) {
                int i2 = r2.l0 + q;
                while (i2 >= a.n2) i2 -= a.n2;
                const double2 g = G[(int64_t)i1 * a.n2 + i2];
                sr = fma(w2[q], g.x, sr);
                si = fma(w2[q], g.y, si);
            }
            re = fma(w1, sr, re);
            im = fma(w1, si, im);
        }
        f[j] = make_double2(re, im);
    }
}

int oversampled(int N, double sigma) {
    int n = (int)std::ceil(sigma * (double)N - 1e-9);
    if (n < N) n = N;
    if (n % 2) ++n;
    auto smooth = [](int v) {
        for (int p : {2, 3, 5, 7})
            while (v % p == 0) v /= p;
        return v == 1;
    };
    while (!smooth(n)) n += 2;
    return n;
}

bool low_args(int dim, const int *N, int m, double sigma, LowArgs &a) {
    if (dim != 1 && dim != 2) return false;
    if (sigma <= 0) sigma = 2.0;
    if (!(sigma >= 1.25 && sigma <= 8.0) || m < 1 || m > kMaxM) return false;
    a.dim = dim;
    a.N1 = N[0];
    a.N2 = dim == 2 ? N[1] : 1;
    if (a.N1 < 2 || a.N1 % 2 || (dim == 2 && (a.N2 < 2 || a.N2 % 2))) return false;
    if (a.N1 > (1 << 22) || a.N2 > (1 << 14)) return false;
    a.n1 = oversampled(a.N1, sigma);
    a.n2 = dim == 2 ? oversampled(a.N2, sigma) : 1;
    a.m = m;
    a.b1 = kPi * (2.0 - (double)a.N1 / a.n1);
    a.b2 = dim == 2 ? kPi * (2.0 - (double)a.N2 / a.n2) : 0.0;
    return true;
}

size_t low_ws(const LowArgs &a) {
    return sizeof(double2) * (size_t)a.n1 * a.n2 + sizeof(double) * (size_t)(a.N1 + a.N2) + 256;
}

// cuFFT plans kept per host thread and size (created on first use)
cufftHandle low_plan(const LowArgs &a, int *err) {
    static thread_local std::map<std::tuple<int, int, int, int>, cufftHandle> plans;
    int dev = 0;
    cudaGetDevice(&dev);
    const auto key = std::make_tuple(dev, a.dim, a.n1, a.n2);
    auto it = plans.find(key);
    if (it != plans.end()) return it->second;
    cufftHandle h;
    const cufftResult r = a.dim == 1 ? cufftPlan1d(&h, a.n1, CUFFT_Z2Z, 1) : cufftPlan2d(&h, a.n1, a.n2, CUFFT_Z2Z);
    if (r != CUFFT_SUCCESS) {
        *err = 1;
        return 0;
    }
    plans[key] = h;
    return h;
}

int grid_of(int64_t n) {
    const int64_t b = (n + 255) / 256;
    return (int)(b < 1 ? 1 : (b > 152 * 32 ? 152 * 32 : b));
}

}  // namespace
}  // namespace gbnfft

using namespace gbnfft;

extern "C" {

size_t nfft_lowdim_workspace_bytes(int dim, const int *N, int m, double sigma) {
    LowArgs a;
    if (!N || !low_args(dim, N, m, sigma, a)) return 0;
    return low_ws(a);
}

int nfft_lowdim_eval(int dim, const int *N, int64_t M, int m, double sigma, const double *x, const double *c,
                     double *f, void *workspace, size_t ws_bytes, void *stream) {
    LowArgs a;
    if (!N || !low_args(dim, N, m, sigma, a) || M < 0) return NFFT3_ERR_ARG;
    if (M == 0) return NFFT3_OK;
    if (!x || !c || !f || !workspace || ws_bytes < low_ws(a)) return NFFT3_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    double2 *G = (double2 *)workspace;
    double *D1 = (double *)(G + (size_t)a.n1 * a.n2);
    double *D2 = D1 + a.N1;
    int *status = (int *)(D2 + a.N2);
    if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return NFFT3_ERR_CUDA;
    low_deconv_table_kernel<<<grid_of(a.N1 + a.N2), 256, 0, st>>>(a, D1, D2);
    low_deconv_scatter_kernel<<<grid_of((int64_t)a.n1 * a.n2), 256, 0, st>>>((const double2 *)c, a, D1, D2, G);
    if (cudaGetLastError() != cudaSuccess) return NFFT3_ERR_CUDA;
    int err = 0;
    cufftHandle h = low_plan(a, &err);
    if (err) return NFFT3_ERR_CUFFT;
    if (cufftSetStream(h, st) != CUFFT_SUCCESS ||
        cufftExecZ2Z(h, (cufftDoubleComplex *)G, (cufftDoubleComplex *)G, CUFFT_INVERSE) != CUFFT_SUCCESS)
        return NFFT3_ERR_CUFFT;
    low_gather_kernel<<<grid_of(M), 256, 0, st>>>(G, a, x, M, (double2 *)f, status);
    if (cudaGetLastError() != cudaSuccess) return NFFT3_ERR_CUDA;
    int hs = 0;
    if (cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return NFFT3_ERR_CUDA;
    return (hs & 1) ? NFFT3_ERR_POINTS : NFFT3_OK;
}

}  // extern "C"
