// Dense local-grid core detection: lattice point generation and the
// plaquette (phase-winding) test.
//
// A vortex core of psi is a curve where psi = 0 and the phase of psi winds by
// +-2 pi around it.  On a fine lattice, a core crosses the face (plaquette)
// of four neighbouring nodes when the phase differences around the face,
// each wrapped into (-pi, pi], sum to +-2 pi.  The paper instead marks
// lattice nodes with rho = |psi|^2 below a level (Sec. 5: isosurfaces at
// rho = 0.0012 on 321^3 and 281^3 grids); the winding test gives a
// point per crossing that Newton refinement can start from.
#include <cmath>

#include "internal.cuh"

namespace {

// x[(i1 R2 + i2) R3 + i3] = lo + i h  (torus coordinates, M = R1 R2 R3 points)
__global__ void lattice_kernel(double *__restrict__ x, int R1, int R2, int R3, double lo1, double lo2,
                               double lo3, double h1, double h2, double h3) {
    const int64_t total = (int64_t)R1 * R2 * R3;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i3 = (int)(e % R3);
        const int64_t r = e / R3;
        const int i2 = (int)(r % R2);
        const int i1 = (int)(r / R2);
        x[3 * e + 0] = lo1 + i1 * h1;
        x[3 * e + 1] = lo2 + i2 * h2;
        x[3 * e + 2] = lo3 + i3 * h3;
    }
}

template <typename C> __device__ __forceinline__ double phase(const C *p, int64_t i) {
    const C v = p[i];
    return atan2((double)v.y, (double)v.x);
}

// phase difference b - a wrapped into (-pi, pi]
__device__ __forceinline__ double wrapd(double d) {
    const double pi = 3.141592653589793238462643383279502884;
    while (d > pi) d -= 2 * pi;
    while (d <= -pi) d += 2 * pi;
    return d;
}

// winding of the phase around the quad p0 -> p1 -> p2 -> p3 -> p0, in turns
__device__ __forceinline__ int winding(double t0, double t1, double t2, double t3) {
    const double s = wrapd(t1 - t0) + wrapd(t2 - t1) + wrapd(t3 - t2) + wrapd(t0 - t3);
    return (int)rint(s / (2 * 3.141592653589793238462643383279502884));
}

// One thread per lattice cell corner (i1, i2, i3) with i_d < R_d - 1 in the two
// in-face directions: tests the three faces whose lowest corner it is
// (normal 1: (i2, i3) plane at i1; normal 2: (i1, i3) at i2; normal 3: (i1, i2) at i3).
template <typename C>
__global__ void plaquette_kernel(const C *__restrict__ psi, int R1, int R2, int R3, double lo1,
                                 double lo2, double lo3, double h1, double h2, double h3,
                                 double *__restrict__ out, int *__restrict__ out_dir, int64_t cap,
                                 unsigned long long *__restrict__ count) {
    const int64_t total = (int64_t)R1 * R2 * R3;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i3 = (int)(e % R3);
        const int64_t r = e / R3;
        const int i2 = (int)(r % R2);
        const int i1 = (int)(r / R2);
        const int64_t s1 = (int64_t)R2 * R3, s2 = R3;
        const double t000 = phase(psi, e);
        for (int dir = 0; dir < 3; ++dir) {
            // the two in-face directions (u, v) for the face with normal `dir`
            int64_t su, sv;
            bool ok;
            double cu[3] = {0.5, 0.5, 0.5};
            if (dir == 0) {
                ok = i2 + 1 < R2 && i3 + 1 < R3;
                su = s2, sv = 1;
                cu[0] = 0.0;
            } else if (dir == 1) {
                ok = i1 + 1 < R1 && i3 + 1 < R3;
                su = s1, sv = 1;
                cu[1] = 0.0;
            } else {
                ok = i1 + 1 < R1 && i2 + 1 < R2;
                su = s1, sv = s2;
                cu[2] = 0.0;
            }
            if (!ok) continue;
            const double tu = phase(psi, e + su), tuv = phase(psi, e + su + sv), tv = phase(psi, e + sv);
            const int w = winding(t000, tu, tuv, tv);
            if (w != 0) {
                const unsigned long long slot = atomicAdd(count, 1ull);
                if ((int64_t)slot < cap) {
                    out[3 * slot + 0] = lo1 + (i1 + cu[0]) * h1;
                    out[3 * slot + 1] = lo2 + (i2 + cu[1]) * h2;
                    out[3 * slot + 2] = lo3 + (i3 + cu[2]) * h3;
                    out_dir[slot] = (dir + 1) * (w > 0 ? 1 : -1);
                }
            }
        }
    }
}

int blocks_for(int64_t n, int threads) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (n + threads - 1) / threads, cap = (int64_t)sms * 16;
    return (int)(want < cap ? (want < 1 ? 1 : want) : cap);
}

}  // namespace

extern "C" int nfft3_lattice_points(double *x, int R1, int R2, int R3, const double *lo,
                                    const double *h, void *stream) {
    if (!x || !lo || !h || R1 < 1 || R2 < 1 || R3 < 1) return NFFT3_ERR_ARG;
    const int64_t total = (int64_t)R1 * R2 * R3;
    lattice_kernel<<<blocks_for(total, 256), 256, 0, (cudaStream_t)stream>>>(
        x, R1, R2, R3, lo[0], lo[1], lo[2], h[0], h[1], h[2]);
    return cudaGetLastError() == cudaSuccess ? NFFT3_OK : NFFT3_ERR_CUDA;
}

extern "C" int nfft3_plaquette_crossings(int prec, const void *psi, int R1, int R2, int R3,
                                         const double *lo, const double *h, double *out,
                                         int *out_dir, int64_t cap, unsigned long long *count,
                                         void *stream) {
    if ((prec != 64 && prec != 32) || !psi || !lo || !h || !out || !out_dir || !count || cap < 0 ||
        R1 < 1 || R2 < 1 || R3 < 1)
        return NFFT3_ERR_ARG;
    const cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(count, 0, sizeof(unsigned long long), st) != cudaSuccess) return NFFT3_ERR_CUDA;
    const int64_t total = (int64_t)R1 * R2 * R3;
    if (prec == 64)
        plaquette_kernel<double2><<<blocks_for(total, 256), 256, 0, st>>>(
            (const double2 *)psi, R1, R2, R3, lo[0], lo[1], lo[2], h[0], h[1], h[2], out, out_dir, cap,
            count);
    else
        plaquette_kernel<float2><<<blocks_for(total, 256), 256, 0, st>>>(
            (const float2 *)psi, R1, R2, R3, lo[0], lo[1], lo[2], h[0], h[1], h[2], out, out_dir, cap,
            count);
    return cudaGetLastError() == cudaSuccess ? NFFT3_OK : NFFT3_ERR_CUDA;
}
