// Grid kernels of the NFFT: deconvolve+scatter, window gather (value and
// gradient), adjoint spread and the adjoint's deconvolve+gather.
//
// Templates only: kernels.cu instantiates them for the mixed family (float)
// and kernels_f64.cu for the FP64 family, so that the two compile in parallel.
#pragma once
#include "internal.cuh"

namespace gbnfft {
namespace {

// Weights of the 2m+1 taps of one dimension for offset s in [0, 1):
// Horner in t = 2s - 1 with the plan's coefficients (kernel parameters,
// read from the constant bank by every thread at the same index).
template <typename R, int MM>
__device__ __forceinline__ void window_row(R s, const R (&c)[2 * MM + 1][PolyDeg<R>::value + 1],
                                           R out[2 * MM + 1]) {
    constexpr int D = PolyDeg<R>::value;
    const R t = (R)2 * s - (R)1;
#pragma unroll
    for (int a = 0; a <= 2 * MM; ++a) {
        R v = c[a][D];
#pragma unroll
        for (int k = D - 1; k >= 0; --k) v = fma(v, t, c[a][k]);
        out[a] = v;
    }
}

__device__ __forceinline__ int wrap_add(int base, int off, int n) {
    int v = base + off;
    while (v >= n) v -= n;
    return v;
}

template <typename C> __device__ __forceinline__ C cmul_real(C z, decltype(z.x) r) {
    C o;
    o.x = z.x * r;
    o.y = z.y * r;
    return o;
}

// ----------------------------------------------------------------------------
// (a) deconvolve and zero-pad: G[l] = c_k D1[k1] D2[k2] D3[k3] at l = k mod n,
// zero elsewhere.  One block per grid row (l1, l2), threads along the
// contiguous dimension l3; whether the row lies in the band |k1|, |k2| < N/2
// is decided once per row.  With with_grad, four grids are written back to
// back: G, then 2 pi i k_d G for d = 1..3.  With vexp (FP64 family) every
// coefficient is first scaled by 2^value_shift(vexp).
// ----------------------------------------------------------------------------
template <typename R>
__global__ void deconv_scatter_kernel(const typename Cplx<R>::T *__restrict__ c, int N1, int N2,
                                      int N3, const R *__restrict__ D1, const R *__restrict__ D2,
                                      const R *__restrict__ D3, typename Cplx<R>::T *__restrict__ G,
                                      Grid3 g, int with_grad, const int *__restrict__ vexp) {
    using C = typename Cplx<R>::T;
    const int vs = value_shift(vexp);
    const int64_t total = (int64_t)g.n1 * g.n2 * g.n3;
    const R two_pi = (R)6.283185307179586476925286766559;
    const int64_t rows = (int64_t)g.n1 * g.n2;
    for (int64_t row = blockIdx.x; row < rows; row += gridDim.x) {
        const int l2 = (int)(row % g.n2);
        const int l1 = (int)(row / g.n2);
        // frequency of grid index l: k = l (l < N/2) or l - n (l >= n - N/2)
        const int k1 = l1 < N1 / 2 ? l1 : (l1 >= g.n1 - N1 / 2 ? l1 - g.n1 : INT32_MIN);
        const int k2 = l2 < N2 / 2 ? l2 : (l2 >= g.n2 - N2 / 2 ? l2 - g.n2 : INT32_MIN);
        const bool row_in = k1 != INT32_MIN && k2 != INT32_MIN;
        C *out = G + row * g.n3;
        if (!row_in) {
            C z;
            z.x = 0;
            z.y = 0;
            for (int l3 = threadIdx.x; l3 < g.n3; l3 += blockDim.x) {
                out[l3] = z;
                if (with_grad)
                    for (int d = 1; d < 4; ++d) out[d * total + l3] = z;
            }
            continue;
        }
        const int i1 = k1 + N1 / 2, i2 = k2 + N2 / 2;
        const R d12 = D1[i1] * D2[i2];
        const C *crow = c + ((int64_t)i1 * N2 + i2) * N3;
        for (int l3 = threadIdx.x; l3 < g.n3; l3 += blockDim.x) {
            const int k3 = l3 < N3 / 2 ? l3 : (l3 >= g.n3 - N3 / 2 ? l3 - g.n3 : INT32_MIN);
            C v;
            v.x = 0;
            v.y = 0;
            if (k3 != INT32_MIN) {
                const int i3 = k3 + N3 / 2;
                v = cmul_real(scale_value(crow[i3], vs), d12 * D3[i3]);
            }
            out[l3] = v;
            if (with_grad) {
                const R kk[3] = {(R)k1, (R)k2, (R)(k3 != INT32_MIN ? k3 : 0)};
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    // 2 pi i k_d v
                    C t;
                    t.x = -two_pi * kk[d] * v.y;
                    t.y = two_pi * kk[d] * v.x;
                    out[(d + 1) * total + l3] = t;
                }
            }
        }
    }
}

// ----------------------------------------------------------------------------
// (c) window gather, one thread per sorted point:
//   f_j = sum_a w1[a] sum_b w2[b] sum_c w3[c] g[l0 + (a,b,c) mod n]
// ----------------------------------------------------------------------------
template <typename R, int MM, int NG>
__global__ void __launch_bounds__(128) gather_kernel(const typename Cplx<R>::T *__restrict__ G,
                                                     Grid3 g, PointsView<R> pts,
                                                     const __grid_constant__ Poly<R, MM> P,
                                                     typename Cplx<R>::T *__restrict__ f,
                                                     typename Cplx<R>::T *__restrict__ grad) {
    using C = typename Cplx<R>::T;
    constexpr int W = 2 * MM + 1;
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= pts.M) return;
    const int4 key = pts.key[j];
    R w1[W], w2[W], w3[W];
    window_row<R, MM>(pts.s1[j], P.c[0], w1);
    window_row<R, MM>(pts.s2[j], P.c[1], w2);
    window_row<R, MM>(pts.s3[j], P.c[2], w3);
    int i3[W];
#pragma unroll
    for (int c = 0; c < W; ++c) i3[c] = wrap_add(key.z, c, g.n3);
    const int64_t gsz = (int64_t)g.n1 * g.n2 * g.n3;
    R acc[NG][2];
#pragma unroll
    for (int q = 0; q < NG; ++q) acc[q][0] = acc[q][1] = 0;
    // a loop rolled; w1 rotates through registers so that every index is static
    int ia = key.x;
#pragma unroll 1
    for (int a = 0; a < W; ++a) {
        R mid[NG][2];
#pragma unroll
        for (int q = 0; q < NG; ++q) mid[q][0] = mid[q][1] = 0;
        int ib = key.y;
#pragma unroll
        for (int b = 0; b < W; ++b) {
            const int64_t row = ((int64_t)ia * g.n2 + ib) * g.n3;
#pragma unroll
            for (int q = 0; q < NG; ++q) {
                R in0 = 0, in1 = 0;
#pragma unroll
                for (int c = 0; c < W; ++c) {
                    const C v = __ldg(&G[q * gsz + row + i3[c]]);
                    in0 += w3[c] * v.x;
                    in1 += w3[c] * v.y;
                }
                mid[q][0] += w2[b] * in0;
                mid[q][1] += w2[b] * in1;
            }
            if (++ib == g.n2) ib = 0;
        }
#pragma unroll
        for (int q = 0; q < NG; ++q) {
            acc[q][0] += w1[0] * mid[q][0];
            acc[q][1] += w1[0] * mid[q][1];
        }
#pragma unroll
        for (int k = 0; k < W - 1; ++k) w1[k] = w1[k + 1];
        if (++ia == g.n1) ia = 0;
    }
    const int64_t o = key.w;
    const int vs = -value_shift(pts.vexp);
    if (NG == 1) {
        C r;
        r.x = acc[0][0];
        r.y = acc[0][1];
        f[o] = scale_value(r, vs);
    } else {
        if (f) {
            C r;
            r.x = acc[0][0];
            r.y = acc[0][1];
            f[o] = scale_value(r, vs);
        }
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            C r;
            r.x = acc[d + 1][0];
            r.y = acc[d + 1][1];
            grad[3 * o + d] = scale_value(r, vs);
        }
    }
}

// ----------------------------------------------------------------------------
// adjoint spread, one thread per sorted point: H[l0 + (a,b,c) mod n] +=
// f_j w1[a] w2[b] w3[c]  (global atomics).
// ----------------------------------------------------------------------------
template <typename R, int MM>
__global__ void __launch_bounds__(128) spread_kernel(const typename Cplx<R>::T *__restrict__ f,
                                                     Grid3 g, PointsView<R> pts,
                                                     const __grid_constant__ Poly<R, MM> P,
                                                     typename Cplx<R>::T *__restrict__ H) {
    using C = typename Cplx<R>::T;
    constexpr int W = 2 * MM + 1;
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= pts.M) return;
    const int4 key = pts.key[j];
    const C fv = scale_value(f[key.w], value_shift(pts.vexp));
    R w1[W], w2[W], w3[W];
    window_row<R, MM>(pts.s1[j], P.c[0], w1);
    window_row<R, MM>(pts.s2[j], P.c[1], w2);
    window_row<R, MM>(pts.s3[j], P.c[2], w3);
    int i3[W];
#pragma unroll
    for (int c = 0; c < W; ++c) i3[c] = wrap_add(key.z, c, g.n3);
    int ia = key.x;
#pragma unroll 1
    for (int a = 0; a < W; ++a) {
        int ib = key.y;
#pragma unroll
        for (int b = 0; b < W; ++b) {
            const R wab = w1[0] * w2[b];
            const R fr = fv.x * wab, fi = fv.y * wab;
            R *row = reinterpret_cast<R *>(H + ((int64_t)ia * g.n2 + ib) * g.n3);
#pragma unroll
            for (int c = 0; c < W; ++c) {
                atomicAdd(row + 2 * i3[c], fr * w3[c]);
                atomicAdd(row + 2 * i3[c] + 1, fi * w3[c]);
            }
            if (++ib == g.n2) ib = 0;
        }
#pragma unroll
        for (int k = 0; k < W - 1; ++k) w1[k] = w1[k + 1];
        if (++ia == g.n1) ia = 0;
    }
}

// adjoint deconvolution: c[i] = H[k mod n] D1[i1] D2[i2] D3[i3], one thread per
// coefficient; with vexp the result is scaled back by 2^-value_shift(vexp).
template <typename R>
__global__ void deconv_gather_kernel(const typename Cplx<R>::T *__restrict__ H, Grid3 g,
                                     const R *__restrict__ D1, const R *__restrict__ D2,
                                     const R *__restrict__ D3, int N1, int N2, int N3,
                                     typename Cplx<R>::T *__restrict__ c, const int *__restrict__ vexp) {
    const int64_t total = (int64_t)N1 * N2 * N3;
    const int vs = -value_shift(vexp);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i3 = (int)(e % N3);
        const int64_t r = e / N3;
        const int i2 = (int)(r % N2);
        const int i1 = (int)(r / N2);
        const int l1 = i1 - N1 / 2 < 0 ? i1 - N1 / 2 + g.n1 : i1 - N1 / 2;
        const int l2 = i2 - N2 / 2 < 0 ? i2 - N2 / 2 + g.n2 : i2 - N2 / 2;
        const int l3 = i3 - N3 / 2 < 0 ? i3 - N3 / 2 + g.n3 : i3 - N3 / 2;
        const R d = D1[i1] * D2[i2] * D3[i3];
        c[e] = scale_value(cmul_real(H[((int64_t)l1 * g.n2 + l2) * g.n3 + l3], d), vs);
    }
}

int grid_blocks(int64_t total, int threads) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t want = (total + threads - 1) / threads;
    int64_t cap = (int64_t)sms * 16;
    return (int)(want < cap ? (want < 1 ? 1 : want) : cap);
}

template <typename R, int MM, int NG>
cudaError_t gather_dispatch(const typename Cplx<R>::T *G, Grid3 g, PointsView<R> pts,
                            const WinTable<R> &w, typename Cplx<R>::T *f,
                            typename Cplx<R>::T *grad, cudaStream_t st) {
    const int threads = 128;
    const int64_t blocks = (pts.M + threads - 1) / threads;
    gather_kernel<R, MM, NG><<<(unsigned)blocks, threads, 0, st>>>(G, g, pts, make_poly<R, MM>(w),
                                                                   f, grad);
    return cudaGetLastError();
}

template <typename R, int NG>
cudaError_t gather_select(const typename Cplx<R>::T *G, Grid3 g, int m, PointsView<R> pts,
                          const WinTable<R> &w, typename Cplx<R>::T *f, typename Cplx<R>::T *grad,
                          cudaStream_t st) {
    if (pts.M == 0) return cudaSuccess;
    switch (m) {
        case 1: return gather_dispatch<R, 1, NG>(G, g, pts, w, f, grad, st);
        case 2: return gather_dispatch<R, 2, NG>(G, g, pts, w, f, grad, st);
        case 3: return gather_dispatch<R, 3, NG>(G, g, pts, w, f, grad, st);
        case 4: return gather_dispatch<R, 4, NG>(G, g, pts, w, f, grad, st);
        case 5: return gather_dispatch<R, 5, NG>(G, g, pts, w, f, grad, st);
        case 6: return gather_dispatch<R, 6, NG>(G, g, pts, w, f, grad, st);
        case 7: return gather_dispatch<R, 7, NG>(G, g, pts, w, f, grad, st);
        case 8: return gather_dispatch<R, 8, NG>(G, g, pts, w, f, grad, st);
        default: return cudaErrorInvalidValue;
    }
}

template <typename R, int MM>
cudaError_t spread_dispatch(const typename Cplx<R>::T *f, Grid3 g, PointsView<R> pts,
                            const WinTable<R> &w, typename Cplx<R>::T *H, cudaStream_t st) {
    const int threads = 128;
    const int64_t blocks = (pts.M + threads - 1) / threads;
    spread_kernel<R, MM><<<(unsigned)blocks, threads, 0, st>>>(f, g, pts, make_poly<R, MM>(w), H);
    return cudaGetLastError();
}

}  // namespace

template <typename R>
cudaError_t launch_deconv_scatter(const typename Cplx<R>::T *c, int N1, int N2, int N3,
                                  const R *D1, const R *D2, const R *D3, typename Cplx<R>::T *G,
                                  Grid3 g, int with_grad, const int *vexp, cudaStream_t st) {
    const int threads = 128;
    const int64_t rows = (int64_t)g.n1 * g.n2;
    deconv_scatter_kernel<R><<<(unsigned)(rows < (1ll << 30) ? rows : (1ll << 30)), threads, 0, st>>>(
        c, N1, N2, N3, D1, D2, D3, G, g, with_grad, vexp);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_gather(const typename Cplx<R>::T *G, Grid3 g, int m, PointsView<R> pts,
                          const WinTable<R> &w, typename Cplx<R>::T *f, cudaStream_t st) {
    return gather_select<R, 1>(G, g, m, pts, w, f, nullptr, st);
}

template <typename R>
cudaError_t launch_gather_grad(const typename Cplx<R>::T *G4, Grid3 g, int m, PointsView<R> pts,
                               const WinTable<R> &w, typename Cplx<R>::T *f,
                               typename Cplx<R>::T *grad, cudaStream_t st) {
    return gather_select<R, 4>(G4, g, m, pts, w, f, grad, st);
}

template <typename R>
cudaError_t launch_spread(const typename Cplx<R>::T *f, Grid3 g, int m, PointsView<R> pts,
                          const WinTable<R> &w, typename Cplx<R>::T *H, cudaStream_t st) {
    if (pts.M == 0) return cudaSuccess;
    switch (m) {
        case 1: return spread_dispatch<R, 1>(f, g, pts, w, H, st);
        case 2: return spread_dispatch<R, 2>(f, g, pts, w, H, st);
        case 3: return spread_dispatch<R, 3>(f, g, pts, w, H, st);
        case 4: return spread_dispatch<R, 4>(f, g, pts, w, H, st);
        case 5: return spread_dispatch<R, 5>(f, g, pts, w, H, st);
        case 6: return spread_dispatch<R, 6>(f, g, pts, w, H, st);
        case 7: return spread_dispatch<R, 7>(f, g, pts, w, H, st);
        case 8: return spread_dispatch<R, 8>(f, g, pts, w, H, st);
        default: return cudaErrorInvalidValue;
    }
}

template <typename R>
cudaError_t launch_deconv_gather(const typename Cplx<R>::T *H, Grid3 g, const R *D1, const R *D2,
                                 const R *D3, int N1, int N2, int N3, typename Cplx<R>::T *c,
                                 const int *vexp, cudaStream_t st) {
    const int threads = 256;
    const int64_t total = (int64_t)N1 * N2 * N3;
    deconv_gather_kernel<R><<<grid_blocks(total, threads), threads, 0, st>>>(H, g, D1, D2, D3, N1,
                                                                             N2, N3, c, vexp);
    return cudaGetLastError();
}

// Load the kernels of deconvolve + scatter and the 4-grid gather for cutoff m
// onto the current device now (CUDA loads modules lazily, on first use, and
// a load may allocate device memory).
template <typename R> cudaError_t preload_grad_kernels(int m) {
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, deconv_scatter_kernel<R>);
    switch (m) {
        case 1: if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, gather_kernel<R, 1, 4>); break;
        case 2: if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, gather_kernel<R, 2, 4>); break;
        case 3: if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, gather_kernel<R, 3, 4>); break;
        case 4: if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, gather_kernel<R, 4, 4>); break;
        case 5: if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, gather_kernel<R, 5, 4>); break;
        case 6: if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, gather_kernel<R, 6, 4>); break;
        case 7: if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, gather_kernel<R, 7, 4>); break;
        case 8: if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, gather_kernel<R, 8, 4>); break;
        default: return cudaErrorInvalidValue;
    }
    return e;
}

#define GBNFFT_INSTANTIATE(R)                                                                     \
    template cudaError_t preload_grad_kernels<R>(int);                                            \
    template cudaError_t launch_deconv_scatter<R>(const Cplx<R>::T *, int, int, int, const R *,    \
                                                  const R *, const R *, Cplx<R>::T *, Grid3, int,  \
                                                  const int *, cudaStream_t);                      \
    template cudaError_t launch_gather<R>(const Cplx<R>::T *, Grid3, int, PointsView<R>,          \
                                          const WinTable<R> &, Cplx<R>::T *, cudaStream_t);        \
    template cudaError_t launch_gather_grad<R>(const Cplx<R>::T *, Grid3, int, PointsView<R>,     \
                                               const WinTable<R> &, Cplx<R>::T *, Cplx<R>::T *,    \
                                               cudaStream_t);                                      \
    template cudaError_t launch_spread<R>(const Cplx<R>::T *, Grid3, int, PointsView<R>,          \
                                          const WinTable<R> &, Cplx<R>::T *, cudaStream_t);        \
    template cudaError_t launch_deconv_gather<R>(const Cplx<R>::T *, Grid3, const R *, const R *, \
                                                 const R *, int, int, int, Cplx<R>::T *,           \
                                                 const int *, cudaStream_t);

}  // namespace gbnfft
