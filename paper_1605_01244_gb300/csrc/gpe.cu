// Time-splitting pseudospectral (TSSP) integration of the Gross-Pitaevskii
// equation of the paper's Sec. 3, eq. (GPE),
//     psi_t = (i/2) Lap psi + (i/2) (1 - |psi|^2) psi,
// on a periodic box of sides L1 x L2 x L3 sampled at n1 x n2 x n3 points
// (FP64, complex interleaved, row-major with i3 fastest), by the Strang
// splitting of Sec. 3.1: a half step of the potential part (solved exactly,
// |psi| being constant under it: psi <- exp(i t (1 - |psi|^2) / 2) psi), a
// full step of the kinetic part (solved exactly in Fourier space: psi_hat_k
// <- exp(-i t |kappa_k|^2 / 2) psi_hat_k, kappa_d = 2 pi k_d / L_d), and
// another potential half step.  Consecutive potential half steps of a run
// are merged into one full step (exact for the continuous flow, since the
// step only rotates the phase by an amount fixed by |psi|).
//
// The kinetic factor is separable: exp(-i t (kx^2 + ky^2 + kz^2) / 2) =
// e1[k1] e2[k2] e3[k3], three 1D tables built on the host per step size,
// with the 1/(n1 n2 n3) of the inverse FFT folded into e1.  The FFTs are
// cuFFT Z2Z (the paper's solver uses the same transforms).
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include "internal.cuh"

struct gpe_plan_s {
    int n[3];
    double L[3];
    cudaStream_t stream;
    cufftHandle fft;
    double2 *tab;          // e1 | e2 | e3 (n1 + n2 + n3 complex), for the step size tab_tau
    double tab_tau;
    double2 *work;         // n1 n2 n3 complex: the transform of psi for the energy
    double *partial;       // per-block partial sums of the diagnostics
    int nblocks;
    int64_t launches;
};

namespace {

constexpr int kThreads = 256;

// signed frequency of FFT index i on an axis of n points
__host__ __device__ __forceinline__ int freq(int i, int n) { return i < (n + 1) / 2 ? i : i - n; }

// psi <- exp(i c (1 - |psi|^2)) psi  (c = t / 2 for a potential step of length t)
__global__ void __launch_bounds__(kThreads) gpe_potential_kernel(double2 *__restrict__ psi, int64_t total,
                                                                 double c) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = psi[e];
        const double ph = c * (1.0 - (v.x * v.x + v.y * v.y));
        double s, co;
        sincos(ph, &s, &co);
        psi[e] = make_double2(v.x * co - v.y * s, v.x * s + v.y * co);
    }
}

// psi_hat[k] <- e1[k1] e2[k2] e3[k3] psi_hat[k]
__global__ void __launch_bounds__(kThreads) gpe_kinetic_kernel(double2 *__restrict__ h, int n1, int n2, int n3,
                                                               const double2 *__restrict__ tab) {
    const int64_t total = (int64_t)n1 * n2 * n3;
    const double2 *e1 = tab, *e2 = tab + n1, *e3 = tab + n1 + n2;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i3 = (int)(e % n3);
        const int64_t r = e / n3;
        const int i2 = (int)(r % n2), i1 = (int)(r / n2);
        const double2 a = e1[i1], b = e2[i2], c = e3[i3];
        const double2 ab = make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
        const double2 f = make_double2(ab.x * c.x - ab.y * c.y, ab.x * c.y + ab.y * c.x);
        const double2 v = h[e];
        h[e] = make_double2(v.x * f.x - v.y * f.y, v.x * f.y + v.y * f.x);
    }
}

// Per-block partial sums, in a fixed order (the result does not depend on
// scheduling): part[3 b + 0] = sum |psi|^2, part[3 b + 1] = sum (1 - |psi|^2)^2,
// part[3 b + 2] = sum |kappa|^2 |psi_hat|^2.
__global__ void __launch_bounds__(kThreads) gpe_sums_kernel(const double2 *__restrict__ psi,
                                                            const double2 *__restrict__ h, int n1, int n2,
                                                            int n3, double k1s, double k2s, double k3s,
                                                            double *__restrict__ part) {
    const int64_t total = (int64_t)n1 * n2 * n3;
    double m = 0, u = 0, kin = 0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = psi[e];
        const double rho = v.x * v.x + v.y * v.y;
        m += rho;
        u += (1.0 - rho) * (1.0 - rho);
        const int i3 = (int)(e % n3);
        const int64_t r = e / n3;
        const int i2 = (int)(r % n2), i1 = (int)(r / n2);
        const double q1 = k1s * freq(i1, n1), q2 = k2s * freq(i2, n2), q3 = k3s * freq(i3, n3);
        const double2 w = h[e];
        kin += (q1 * q1 + q2 * q2 + q3 * q3) * (w.x * w.x + w.y * w.y);
    }
    __shared__ double sm[3][kThreads];
    sm[0][threadIdx.x] = m;
    sm[1][threadIdx.x] = u;
    sm[2][threadIdx.x] = kin;
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int q = 0; q < 3; ++q) sm[q][threadIdx.x] += sm[q][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < 3; ++q) part[3 * blockIdx.x + q] = sm[q][0];
}

int blocks_for(int64_t total) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (total + kThreads - 1) / kThreads, cap = (int64_t)sms * 8;
    return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

// kinetic tables for step size tau: e_d[i] = exp(-i tau kappa^2 / 2), kappa =
// 2 pi freq(i) / L_d, with 1 / (n1 n2 n3) folded into e1
int build_tables(gpe_plan p, double tau) {
    const int tot = p->n[0] + p->n[1] + p->n[2];
    double2 *h = (double2 *)std::malloc(sizeof(double2) * tot);
    if (!h) return NFFT3_ERR_ALLOC;
    const long double two_pi = 6.283185307179586476925286766559005768L;
    const long double scale = 1.0L / ((long double)p->n[0] * p->n[1] * p->n[2]);
    int o = 0;
    for (int d = 0; d < 3; ++d)
        for (int i = 0; i < p->n[d]; ++i, ++o) {
            const long double kap = two_pi * (long double)freq(i, p->n[d]) / (long double)p->L[d];
            const long double ph = -0.5L * (long double)tau * kap * kap;
            const long double sc = d == 0 ? scale : 1.0L;
            h[o] = make_double2((double)(sc * cosl(ph)), (double)(sc * sinl(ph)));
        }
    const cudaError_t e = cudaMemcpyAsync(p->tab, h, sizeof(double2) * tot, cudaMemcpyHostToDevice, p->stream);
    const cudaError_t e2 = cudaStreamSynchronize(p->stream);
    std::free(h);
    if (e != cudaSuccess || e2 != cudaSuccess) return NFFT3_ERR_CUDA;
    p->tab_tau = tau;
    return NFFT3_OK;
}

void release(gpe_plan p) {
    if (!p) return;
    if (p->fft) cufftDestroy(p->fft);
    if (p->tab) cudaFree(p->tab);
    if (p->work) cudaFree(p->work);
    if (p->partial) cudaFree(p->partial);
    delete p;
}

}  // namespace

extern "C" {

int gpe_plan_create(gpe_plan *out, int n1, int n2, int n3, double L1, double L2, double L3, void *stream) {
    if (!out) return NFFT3_ERR_ARG;
    *out = nullptr;
    if (n1 < 1 || n2 < 1 || n3 < 1 || !(L1 > 0) || !(L2 > 0) || !(L3 > 0)) return NFFT3_ERR_ARG;
    if ((int64_t)n1 * n2 * n3 > ((int64_t)1 << 31)) return NFFT3_ERR_TOO_LARGE;
    gpe_plan p = new (std::nothrow) gpe_plan_s;
    if (!p) return NFFT3_ERR_ALLOC;
    std::memset(p, 0, sizeof(*p));
    p->n[0] = n1, p->n[1] = n2, p->n[2] = n3;
    p->L[0] = L1, p->L[1] = L2, p->L[2] = L3;
    p->stream = (cudaStream_t)stream;
    p->tab_tau = std::nan("");
    const int64_t total = (int64_t)n1 * n2 * n3;
    p->nblocks = blocks_for(total);
    if (cudaMalloc(&p->tab, sizeof(double2) * (n1 + n2 + n3)) != cudaSuccess ||
        cudaMalloc(&p->work, sizeof(double2) * total) != cudaSuccess ||
        cudaMalloc(&p->partial, sizeof(double) * 3 * p->nblocks) != cudaSuccess) {
        cudaGetLastError();
        release(p);
        return NFFT3_ERR_ALLOC;
    }
    if (cufftPlan3d(&p->fft, n1, n2, n3, CUFFT_Z2Z) != CUFFT_SUCCESS) {
        p->fft = 0;
        release(p);
        return NFFT3_ERR_CUFFT;
    }
    if (cufftSetStream(p->fft, p->stream) != CUFFT_SUCCESS) {
        release(p);
        return NFFT3_ERR_CUFFT;
    }
    *out = p;
    return NFFT3_OK;
}

int gpe_steps(gpe_plan p, double *psi, double tau, int nsteps) {
    if (!p || !psi || nsteps < 0 || !std::isfinite(tau)) return NFFT3_ERR_ARG;
    if (nsteps == 0) return NFFT3_OK;
    if (!(p->tab_tau == tau)) {
        const int st = build_tables(p, tau);
        if (st != NFFT3_OK) return st;
    }
    double2 *v = (double2 *)psi;
    const int64_t total = (int64_t)p->n[0] * p->n[1] * p->n[2];
    const int nb = p->nblocks;
    // potential half step, then (kinetic step, potential step) with the
    // middle potential half steps merged, and a final potential half step
    gpe_potential_kernel<<<nb, kThreads, 0, p->stream>>>(v, total, 0.25 * tau);
    if (cudaGetLastError() != cudaSuccess) return NFFT3_ERR_CUDA;
    for (int s = 0; s < nsteps; ++s) {
        if (cufftExecZ2Z(p->fft, (cufftDoubleComplex *)v, (cufftDoubleComplex *)v, CUFFT_FORWARD) != CUFFT_SUCCESS)
            return NFFT3_ERR_CUFFT;
        gpe_kinetic_kernel<<<nb, kThreads, 0, p->stream>>>(v, p->n[0], p->n[1], p->n[2], p->tab);
        if (cudaGetLastError() != cudaSuccess) return NFFT3_ERR_CUDA;
        if (cufftExecZ2Z(p->fft, (cufftDoubleComplex *)v, (cufftDoubleComplex *)v, CUFFT_INVERSE) != CUFFT_SUCCESS)
            return NFFT3_ERR_CUFFT;
        gpe_potential_kernel<<<nb, kThreads, 0, p->stream>>>(v, total, (s + 1 < nsteps ? 0.5 : 0.25) * tau);
        if (cudaGetLastError() != cudaSuccess) return NFFT3_ERR_CUDA;
    }
    p->launches += 1 + 2 * (int64_t)nsteps;
    return NFFT3_OK;
}

int gpe_mass_energy(gpe_plan p, const double *psi, double *mass, double *energy) {
    if (!p || !psi) return NFFT3_ERR_ARG;
    const int64_t total = (int64_t)p->n[0] * p->n[1] * p->n[2];
    if (cudaMemcpyAsync(p->work, psi, sizeof(double2) * total, cudaMemcpyDeviceToDevice, p->stream) != cudaSuccess)
        return NFFT3_ERR_CUDA;
    if (cufftExecZ2Z(p->fft, (cufftDoubleComplex *)p->work, (cufftDoubleComplex *)p->work, CUFFT_FORWARD) !=
        CUFFT_SUCCESS)
        return NFFT3_ERR_CUFFT;
    const double two_pi = 6.283185307179586476925286766559;
    gpe_sums_kernel<<<p->nblocks, kThreads, 0, p->stream>>>((const double2 *)psi, p->work, p->n[0], p->n[1],
                                                            p->n[2], two_pi / p->L[0], two_pi / p->L[1],
                                                            two_pi / p->L[2], p->partial);
    if (cudaGetLastError() != cudaSuccess) return NFFT3_ERR_CUDA;
    p->launches += 1;
    double *h = (double *)std::malloc(sizeof(double) * 3 * p->nblocks);
    if (!h) return NFFT3_ERR_ALLOC;
    if (cudaMemcpyAsync(h, p->partial, sizeof(double) * 3 * p->nblocks, cudaMemcpyDeviceToHost, p->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(p->stream) != cudaSuccess) {
        std::free(h);
        return NFFT3_ERR_CUDA;
    }
    double m = 0, u = 0, kin = 0;
    for (int b = 0; b < p->nblocks; ++b) m += h[3 * b], u += h[3 * b + 1], kin += h[3 * b + 2];
    std::free(h);
    // cell volume dV = L1 L2 L3 / (n1 n2 n3); Parseval: sum_x |grad psi|^2 =
    // (1 / (n1 n2 n3)) sum_k |kappa|^2 |psi_hat_k|^2 (unnormalised forward FFT)
    const double dV = p->L[0] * p->L[1] * p->L[2] / (double)total;
    if (mass) *mass = dV * m;
    if (energy) *energy = dV * (0.5 * kin / (double)total + 0.25 * u);
    return NFFT3_OK;
}

int gpe_destroy(gpe_plan p) {
    release(p);
    return NFFT3_OK;
}

}  // extern "C"
