// Shared part of the one-thread-per-point double-float gathers, instantiated
// in three translation units that compile in parallel: gather_df.cu (value),
// gather_df_grad.cu (value + gradient grids, m <= 6) and gather_df_grad_hi.cu
// (the same for m = 7, 8).
//
// FP64-accurate window gather on the FP32 pipe ("double-float" arithmetic).
//
// GB300 runs FP32 FMAs ~62x faster than FP64 FMAs, so the FP64 family's
// window sums are carried out on pairs of floats (hi, lo) with error-free
// transformations (Dekker/Knuth products and sums via FMA): a grid value is
// split once into hi + lo (24 + 24 significant bits), a window weight is a
// double-float polynomial in t = 2s - 1, and every accumulation is a
// two-sum whose rounding error is carried in a second float.  The result
// keeps about 2^-48 relative accuracy per operation (the dropped lo*lo
// cross terms and the FP32 sum of the error terms), far below the 1e-12
// target.
#pragma once
#include "internal.cuh"

namespace gbnfft {
namespace {

// (ah, al) += (xh, xl) * (yh, yl); all operations rounded explicitly so the
// compiler cannot contract them into FMAs that would break the error terms.
__device__ __forceinline__ void df_mac(float &ah, float &al, float xh, float xl, float yh,
                                       float yl) {
    const float p = __fmul_rn(xh, yh);
    float e = __fmaf_rn(xh, yh, -p);        // exact error of the high product
    e = __fmaf_rn(xh, yl, e);
    e = __fmaf_rn(xl, yh, e);
    const float s = __fadd_rn(ah, p);       // two-sum of the accumulator and p
    const float bb = __fsub_rn(s, ah);
    const float err = __fadd_rn(__fsub_rn(ah, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    al = __fadd_rn(al, __fadd_rn(err, e));
    ah = s;
}

// renormalise so that |al| <= ulp(ah)/2
__device__ __forceinline__ void df_norm(float &ah, float &al) {
    const float s = __fadd_rn(ah, al);
    al = __fsub_rn(al, __fsub_rn(s, ah));
    ah = s;
}

// v = v * t + c in double-float (Horner step)
__device__ __forceinline__ void df_horner_step(float &vh, float &vl, float th, float tl, float ch,
                                               float cl) {
    const float p = __fmul_rn(vh, th);
    float e = __fmaf_rn(vh, th, -p);
    e = __fmaf_rn(vh, tl, e);
    e = __fmaf_rn(vl, th, e);
    const float s = __fadd_rn(p, ch);
    const float bb = __fsub_rn(s, p);
    float err = __fadd_rn(__fsub_rn(p, __fsub_rn(s, bb)), __fsub_rn(ch, bb));
    err = __fadd_rn(err, __fadd_rn(e, cl));
    vh = __fadd_rn(s, err);
    vl = __fsub_rn(err, __fsub_rn(vh, s));
}

template <int MM>
__device__ __forceinline__ void df_window_row(double s, const float (&ch)[2 * MM + 1][kPolyDegDF + 1],
                                              const float (&cl)[2 * MM + 1][kPolyDegDF + 1],
                                              float wh[2 * MM + 1], float wl[2 * MM + 1]) {
    const double t = 2.0 * s - 1.0;               // exact
    const float th = __double2float_rn(t);
    const float tl = __double2float_rn(t - (double)th);
#pragma unroll
    for (int a = 0; a <= 2 * MM; ++a) {
        float vh = ch[a][kPolyDegDF], vl = cl[a][kPolyDegDF];
#pragma unroll
        for (int k = kPolyDegDF - 1; k >= 0; --k) df_horner_step(vh, vl, th, tl, ch[a][k], cl[a][k]);
        wh[a] = vh;
        wl[a] = vl;
    }
}

__device__ __forceinline__ int wrap_add(int base, int off, int n) {
    int v = base + off;
    while (v >= n) v -= n;
    return v;
}

// One thread per sorted point; NG = 1 (value) or 4 (value + gradient grids,
// written back to back).  f / grad are FP64 complex.
template <int MM, int NG>
__global__ void __launch_bounds__(128) gather_df_kernel(const float4 *__restrict__ G, Grid3 g,
                                                        PointsView<double> pts,
                                                        const __grid_constant__ PolyDF<MM> P,
                                                        double2 *__restrict__ f,
                                                        double2 *__restrict__ grad) {
    constexpr int W = 2 * MM + 1;
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= pts.M) return;
    const int4 key = pts.key[j];
    float w1h[W], w1l[W], w2h[W], w2l[W], w3h[W], w3l[W];
    df_window_row<MM>(pts.s1[j], P.ch[0], P.cl[0], w1h, w1l);
    df_window_row<MM>(pts.s2[j], P.ch[1], P.cl[1], w2h, w2l);
    df_window_row<MM>(pts.s3[j], P.ch[2], P.cl[2], w3h, w3l);
    int i3[W];
#pragma unroll
    for (int c = 0; c < W; ++c) i3[c] = wrap_add(key.z, c, g.n3);
    const int64_t gsz = (int64_t)g.n1 * g.n2 * g.n3;
    float acc[NG][4];
#pragma unroll
    for (int q = 0; q < NG; ++q) acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = 0.f;
    int ia = key.x;
#pragma unroll 1
    for (int a = 0; a < W; ++a) {
        float mid[NG][4];
#pragma unroll
        for (int q = 0; q < NG; ++q) mid[q][0] = mid[q][1] = mid[q][2] = mid[q][3] = 0.f;
        int ib = key.y;
#pragma unroll
        for (int b = 0; b < W; ++b) {
            const int64_t row = ((int64_t)ia * g.n2 + ib) * g.n3;
#pragma unroll
            for (int q = 0; q < NG; ++q) {
                // inner sum over the contiguous dimension: (re_h, re_l, im_h, im_l)
                float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
#pragma unroll
                for (int c = 0; c < W; ++c) {
                    const float4 v = __ldg(&G[q * gsz + row + i3[c]]);
                    df_mac(rh, rl, v.x, v.y, w3h[c], w3l[c]);
                    df_mac(ih, il, v.z, v.w, w3h[c], w3l[c]);
                }
                df_norm(rh, rl);
                df_norm(ih, il);
                df_mac(mid[q][0], mid[q][1], rh, rl, w2h[b], w2l[b]);
                df_mac(mid[q][2], mid[q][3], ih, il, w2h[b], w2l[b]);
            }
            if (++ib == g.n2) ib = 0;
        }
#pragma unroll
        for (int q = 0; q < NG; ++q) {
            df_norm(mid[q][0], mid[q][1]);
            df_norm(mid[q][2], mid[q][3]);
            df_mac(acc[q][0], acc[q][1], mid[q][0], mid[q][1], w1h[0], w1l[0]);
            df_mac(acc[q][2], acc[q][3], mid[q][2], mid[q][3], w1h[0], w1l[0]);
        }
#pragma unroll
        for (int k = 0; k < W - 1; ++k) {
            w1h[k] = w1h[k + 1];
            w1l[k] = w1l[k + 1];
        }
        if (++ia == g.n1) ia = 0;
    }
    const int64_t o = key.w;
    double2 r[NG];
#pragma unroll
    for (int q = 0; q < NG; ++q)
        r[q] = scale_value(make_double2((double)acc[q][0] + (double)acc[q][1], (double)acc[q][2] + (double)acc[q][3]),
                           -value_shift(pts.vexp));
    if (NG == 1) {
        f[o] = r[0];
    } else {
        if (f) f[o] = r[0];
#pragma unroll
        for (int d = 0; d < 3; ++d) grad[3 * o + d] = r[(d + 1) % NG];
    }
}

template <int MM, int NG>
cudaError_t df_dispatch(const float4 *G, Grid3 g, PointsView<double> pts, const WinTableDF &w,
                        double2 *f, double2 *grad, cudaStream_t st) {
    const int threads = 128;
    const int64_t blocks = (pts.M + threads - 1) / threads;
    gather_df_kernel<MM, NG><<<(unsigned)blocks, threads, 0, st>>>(G, g, pts, make_poly_df<MM>(w),
                                                                  f, grad);
    return cudaGetLastError();
}

template <int NG>
cudaError_t df_select(const float4 *G, Grid3 g, int m, PointsView<double> pts,
                      const WinTableDF &w, double2 *f, double2 *grad, cudaStream_t st) {
    if (pts.M == 0) return cudaSuccess;
    switch (m) {
        case 1: return df_dispatch<1, NG>(G, g, pts, w, f, grad, st);
        case 2: return df_dispatch<2, NG>(G, g, pts, w, f, grad, st);
        case 3: return df_dispatch<3, NG>(G, g, pts, w, f, grad, st);
        case 4: return df_dispatch<4, NG>(G, g, pts, w, f, grad, st);
        case 5: return df_dispatch<5, NG>(G, g, pts, w, f, grad, st);
        case 6: return df_dispatch<6, NG>(G, g, pts, w, f, grad, st);
        case 7: return df_dispatch<7, NG>(G, g, pts, w, f, grad, st);
        case 8: return df_dispatch<8, NG>(G, g, pts, w, f, grad, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

// gradient gathers by cutoff (gather_df_grad.cu, gather_df_grad_hi.cu)
cudaError_t gather_grad_df_m_le6(const float4 *G4, Grid3 g, int m, PointsView<double> pts, const WinTableDF &w,
                                 double2 *f, double2 *grad, cudaStream_t st);
cudaError_t gather_grad_df_m_gt6(const float4 *G4, Grid3 g, int m, PointsView<double> pts, const WinTableDF &w,
                                 double2 *f, double2 *grad, cudaStream_t st);

}  // namespace gbnfft
