// Column-parallel window gather: one point per group of GS = 2^ceil(log2(2m+1))
// lanes, lane c of the group owning column c of the stencil's contiguous
// dimension.  For every stencil row (a, b) the group reads 2m+1 consecutive
// grid values, so a warp's load touches a few contiguous segments instead of
// 32 scattered sectors.  Each lane accumulates
//     T_c = sum_a w1[a] sum_b w2[b] g[l1+a, l2+b, l3+c]
// and the group finishes f = sum_c w3[c] T_c with a shuffle reduction.
// Window weights: lane c evaluates the polynomials of tap c for the three
// dimensions (coefficients staged in shared memory), then w1 and w2 are
// broadcast to the group's registers by shuffles, once per point.
//
// The kernels read a ghost-padded copy of the grid, P[p] = g[(p - shift) mod n]
// for p in [0, n + 2m) per dimension (written by pad_grid_*), so a stencil
// never wraps and a row's address is a pointer increment.  shift = 0 (the
// column kernels): a stencil with first node l0 starts at padded index l0.
// shift = m (the tile-staged kernel): it starts at its centre (l0 + m) mod n,
// so all points of an 8^3 tile of centres read one contiguous box.
//
// Two arithmetic variants: FP32 (mixed family) and double-float on the FP32
// pipe (FP64 family; see gather_df.cu for the arithmetic).
#include <cstdlib>

#include "col_common.cuh"

namespace gbnfft {
namespace {

// ---- FP32 (mixed family) -----------------------------------------------------
template <int MM, int NG>
__global__ void __launch_bounds__(256) gather_col_f32_kernel(const float2 *__restrict__ G, Grid3 pg,
                                                             PointsView<float> pts,
                                                             const __grid_constant__ Poly<float, MM> P,
                                                             float2 *__restrict__ f,
                                                             float2 *__restrict__ grad,
                                                             const int *__restrict__ sel, int64_t nwork) {
    constexpr int W = 2 * MM + 1;
    constexpr int GS = GroupSize<W>::value;
    constexpr int D = PolyDeg<float>::value;
    __shared__ float coef[3][W][D + 1];
    for (int i = threadIdx.x; i < 3 * W * (D + 1); i += blockDim.x)
        (&coef[0][0][0])[i] = (&P.c[0][0][0])[i];
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int sub = lane & (GS - 1);
    const int gbase = lane & ~(GS - 1);
    // work item w: sorted point sel[w] (sel given) or w
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / GS;
    const bool valid = w < nwork;
    const int64_t jj = valid ? (sel ? (int64_t)sel[w] : w) : (sel ? (int64_t)sel[0] : 0);
    const int4 key = pts.key[jj];
    const int tap = sub < W ? sub : 0;
    float myw[3];
    {
        const float s[3] = {pts.s1[jj], pts.s2[jj], pts.s3[jj]};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const float t = 2.f * s[d] - 1.f;
            float v = coef[d][tap][D];
#pragma unroll
            for (int k = D - 1; k >= 0; --k) v = fmaf(v, t, coef[d][tap][k]);
            myw[d] = sub < W ? v : 0.f;
        }
    }
    float w1[W], w2[W];
#pragma unroll
    for (int a = 0; a < W; ++a) {
        w1[a] = __shfl_sync(0xffffffffu, myw[0], gbase + a);
        w2[a] = __shfl_sync(0xffffffffu, myw[1], gbase + a);
    }
    // pg: padded dims (origin layout): the stencil starts at padded index l0
    const int64_t s1 = (int64_t)pg.n2 * pg.n3, gsz = (int64_t)pg.n1 * s1;
    const float2 *base = G + (int64_t)key.x * s1 + (int64_t)key.y * pg.n3 + key.z + tap;
    float T[NG][2];
#pragma unroll
    for (int q = 0; q < NG; ++q) T[q][0] = T[q][1] = 0.f;
#pragma unroll 1
    for (int a = 0; a < W; ++a) {
        float S[NG][2];
#pragma unroll
        for (int q = 0; q < NG; ++q) S[q][0] = S[q][1] = 0.f;
        const float2 *row = base;
#pragma unroll
        for (int b = 0; b < W; ++b) {
#pragma unroll
            for (int q = 0; q < NG; ++q) {
                const float2 v = __ldg(row + q * gsz);
                S[q][0] = fmaf(w2[b], v.x, S[q][0]);
                S[q][1] = fmaf(w2[b], v.y, S[q][1]);
            }
            row += pg.n3;
        }
#pragma unroll
        for (int q = 0; q < NG; ++q) {
            T[q][0] = fmaf(w1[0], S[q][0], T[q][0]);
            T[q][1] = fmaf(w1[0], S[q][1], T[q][1]);
        }
#pragma unroll
        for (int k = 0; k < W - 1; ++k) w1[k] = w1[k + 1];
        base += s1;
    }
    // f = sum_c w3[c] T_c over the group (lanes >= W contribute 0)
#pragma unroll
    for (int q = 0; q < NG; ++q) {
        float re = myw[2] * T[q][0], im = myw[2] * T[q][1];
#pragma unroll
        for (int off = GS / 2; off > 0; off >>= 1) {
            re += __shfl_xor_sync(0xffffffffu, re, off, GS);
            im += __shfl_xor_sync(0xffffffffu, im, off, GS);
        }
        T[q][0] = re;
        T[q][1] = im;
    }
    if (valid && sub == 0) {
        if (NG == 1) {
            f[key.w] = make_float2(T[0][0], T[0][1]);
        } else {
            if (f) f[key.w] = make_float2(T[0][0], T[0][1]);
#pragma unroll
            for (int d = 0; d < 3; ++d)
                grad[3 * (int64_t)key.w + d] = make_float2(T[(d + 1) % NG][0], T[(d + 1) % NG][1]);
        }
    }
}

// Same sum for grids whose three dimensions share one window table (equal
// N_d and n_d, e.g. cubes), value only: the lane's tap polynomial (D + 1
// floats) lives in registers for the whole kernel, and each warp walks
// 32/GS consecutive sorted points per iteration (grid-stride, warp-uniform),
// so no shared-memory table read is repeated per point.
template <int MM>
__global__ void __launch_bounds__(256) gather_col_f32_cube_kernel(const float2 *__restrict__ G, Grid3 pg,
                                                                  PointsView<float> pts,
                                                                  const __grid_constant__ Poly<float, MM> P,
                                                                  float2 *__restrict__ f,
                                                                  const int *__restrict__ sel, int64_t nwork) {
    constexpr int W = 2 * MM + 1;
    constexpr int GS = GroupSize<W>::value;
    constexpr int PPW = 32 / GS;
    constexpr int D = PolyDeg<float>::value;
    const int lane = threadIdx.x & 31;
    const int sub = lane & (GS - 1);
    const int gbase = lane & ~(GS - 1);
    const int tap = sub < W ? sub : 0;
    float cf[D + 1];
#pragma unroll
    for (int k = 0; k <= D; ++k) cf[k] = P.c[0][tap][k];
    const int64_t s1 = (int64_t)pg.n2 * pg.n3;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    // work item w: sorted point sel[w] (sel given) or w
    for (int64_t wb = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * PPW; wb < nwork;
         wb += nwarps * PPW) {
        const int64_t w = wb + lane / GS;
        const bool valid = w < nwork;
        const int64_t ww = valid ? w : wb;
        const int64_t jj = sel ? (int64_t)sel[ww] : ww;
        const int4 key = pts.key[jj];
        float myw[3];
        {
            const float s[3] = {pts.s1[jj], pts.s2[jj], pts.s3[jj]};
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const float t = 2.f * s[d] - 1.f;
                float v = cf[D];
#pragma unroll
                for (int k = D - 1; k >= 0; --k) v = fmaf(v, t, cf[k]);
                myw[d] = sub < W ? v : 0.f;
            }
        }
        float w2[W];
#pragma unroll
        for (int b = 0; b < W; ++b) w2[b] = __shfl_sync(0xffffffffu, myw[1], gbase + b);
        const float2 *base = G + (int64_t)key.x * s1 + (int64_t)key.y * pg.n3 + key.z + tap;
        float Tr = 0.f, Ti = 0.f;
#pragma unroll 1
        for (int a = 0; a < W; ++a) {
            float Sr = 0.f, Si = 0.f;
            const float2 *row = base;
#pragma unroll
            for (int b = 0; b < W; ++b) {
                const float2 v = __ldg(row);
                Sr = fmaf(w2[b], v.x, Sr);
                Si = fmaf(w2[b], v.y, Si);
                row += pg.n3;
            }
            const float w1 = __shfl_sync(0xffffffffu, myw[0], gbase + a);
            Tr = fmaf(w1, Sr, Tr);
            Ti = fmaf(w1, Si, Ti);
            base += s1;
        }
        float re = myw[2] * Tr, im = myw[2] * Ti;
#pragma unroll
        for (int off = GS / 2; off > 0; off >>= 1) {
            re += __shfl_xor_sync(0xffffffffu, re, off, GS);
            im += __shfl_xor_sync(0xffffffffu, im, off, GS);
        }
        if (valid && sub == 0) f[key.w] = make_float2(re, im);
    }
}

// ---- double-float (FP64 family) ----------------------------------------------
#ifndef GBNFFT_SLOT_MINB
#define GBNFFT_SLOT_MINB 3   // resident 256-thread blocks per SM the slot kernel is compiled for (2: 38.4 ms vs 31.6)
#endif
#ifndef GBNFFT_DF_MINB
#define GBNFFT_DF_MINB 3   // resident 256-thread blocks per SM the value kernel is compiled for
#endif

// Value gather with the W^2 taps of each stencil plane spread over all GS
// lanes of the group ("slots"): lane l owns taps s = l + GS t, (b, c) =
// (s / W, s mod W), t < NSLOT = ceil(W^2 / GS), instead of one column each.
// For W = 13 (m = 6) that fills 169 of 176 lane slots (96 %) instead of
// 13 of 16 columns (81 %); for W = 11 or 17 the gain is larger.  Each slot's
// weight w2[b] w3[c] is formed once per point; per plane a lane adds its
// slots' products and the plane weight w1[a] multiplies the lane sum; the
// group reduces the lane sums at the end.  Double-float throughout.
template <int MM, class Wt>
__global__ void __launch_bounds__(256, GBNFFT_SLOT_MINB) gather_slot_df_kernel(
    const float4 *__restrict__ G, Grid3 pg, PointsView<double> pts,
    const __grid_constant__ typename Wt::Table P, double2 *__restrict__ f) {
    constexpr int W = 2 * MM + 1;
    constexpr int GS = GroupSize<W>::value;
    constexpr int NSLOT = (W * W + GS - 1) / GS;
    __shared__ Wt wt;
    wt.load(P);
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int sub = lane & (GS - 1);
    const int gbase = lane & ~(GS - 1);
    const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / GS;
    const bool valid = j < pts.M;
    const int64_t jj = valid ? j : 0;
    const int4 key = pts.M > 0 ? pts.key[jj] : make_int4(0, 0, 0, 0);
    const int tap = sub < W ? sub : 0;
    float wh[3], wl[3];
    {
        const double s[3] = {pts.s1[jj], pts.s2[jj], pts.s3[jj]};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            wt.eval(d, tap, s[d], wh[d], wl[d]);
            if (sub >= W) wh[d] = wl[d] = 0.f;
        }
    }
    // slot offsets within a plane and slot weights w2[b] w3[c]
    int off[NSLOT];
    float w23h[NSLOT], w23l[NSLOT];
#pragma unroll
    for (int t = 0; t < NSLOT; ++t) {
        const int sidx = sub + GS * t;
        const bool in = sidx < W * W;
        const int b = in ? sidx / W : 0, c = in ? sidx - (sidx / W) * W : 0;
        const float bh = __shfl_sync(0xffffffffu, wh[1], gbase + b);
        const float bl = __shfl_sync(0xffffffffu, wl[1], gbase + b);
        const float ch = __shfl_sync(0xffffffffu, wh[2], gbase + c);
        const float cl = __shfl_sync(0xffffffffu, wl[2], gbase + c);
        float ph = 0.f, pl = 0.f;
        df_mac(ph, pl, bh, bl, ch, cl);
        df_norm(ph, pl);
        w23h[t] = in ? ph : 0.f;
        w23l[t] = in ? pl : 0.f;
        off[t] = b * pg.n3 + c;
    }
    const int64_t s1 = (int64_t)pg.n2 * pg.n3;
    const float4 *base = G + (int64_t)key.x * s1 + (int64_t)key.y * pg.n3 + key.z;
    float T[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 1
    for (int a = 0; a < W; ++a) {
        float S[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int t = 0; t < NSLOT; ++t) {
            const float4 v = __ldg(base + off[t]);
            df_mac(S[0], S[1], v.x, v.y, w23h[t], w23l[t]);
            df_mac(S[2], S[3], v.z, v.w, w23h[t], w23l[t]);
        }
        const float w1h = __shfl_sync(0xffffffffu, wh[0], gbase + a);
        const float w1l = __shfl_sync(0xffffffffu, wl[0], gbase + a);
        df_norm(S[0], S[1]);
        df_norm(S[2], S[3]);
        df_mac(T[0], T[1], S[0], S[1], w1h, w1l);
        df_mac(T[2], T[3], S[2], S[3], w1h, w1l);
        base += s1;
    }
    df_norm(T[0], T[1]);
    df_norm(T[2], T[3]);
#pragma unroll
    for (int o = GS / 2; o > 0; o >>= 1) {
        const float orh = __shfl_xor_sync(0xffffffffu, T[0], o, GS);
        const float orl = __shfl_xor_sync(0xffffffffu, T[1], o, GS);
        const float oih = __shfl_xor_sync(0xffffffffu, T[2], o, GS);
        const float oil = __shfl_xor_sync(0xffffffffu, T[3], o, GS);
        df_add(T[0], T[1], orh, orl);
        df_add(T[2], T[3], oih, oil);
    }
    if (valid && sub == 0)
        f[key.w] = scale_value(make_double2((double)T[0] + (double)T[1], (double)T[2] + (double)T[3]),
                               -value_shift(pts.vexp));
}

template <int MM, int NG, class Wt>
__global__ void __launch_bounds__(256, NG == 1 ? GBNFFT_DF_MINB : 2) gather_col_df_kernel(const float4 *__restrict__ G, Grid3 pg,
                                                            PointsView<double> pts,
                                                            const __grid_constant__ typename Wt::Table P,
                                                            double2 *__restrict__ f,
                                                            double2 *__restrict__ grad) {
    constexpr int W = 2 * MM + 1;
    constexpr int GS = GroupSize<W>::value;
    __shared__ Wt wt;
    wt.load(P);
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int sub = lane & (GS - 1);
    const int gbase = lane & ~(GS - 1);
    const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / GS;
    const bool valid = j < pts.M;
    const int64_t jj = valid ? j : 0;
    const int4 key = pts.M > 0 ? pts.key[jj] : make_int4(0, 0, 0, 0);
    const int tap = sub < W ? sub : 0;
    float mwh[3], mwl[3];
    {
        const double s[3] = {pts.s1[jj], pts.s2[jj], pts.s3[jj]};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            wt.eval(d, tap, s[d], mwh[d], mwl[d]);
            if (sub >= W) mwh[d] = mwl[d] = 0.f;
        }
    }
    float w2h[W], w2l[W];
#pragma unroll
    for (int b = 0; b < W; ++b) {
        w2h[b] = __shfl_sync(0xffffffffu, mwh[1], gbase + b);
        w2l[b] = __shfl_sync(0xffffffffu, mwl[1], gbase + b);
    }
    const int64_t s1 = (int64_t)pg.n2 * pg.n3, gsz = (int64_t)pg.n1 * s1;
    const float4 *base = G + (int64_t)key.x * s1 + (int64_t)key.y * pg.n3 + key.z + tap;
    float T[NG][4];
#pragma unroll
    for (int q = 0; q < NG; ++q) T[q][0] = T[q][1] = T[q][2] = T[q][3] = 0.f;
#pragma unroll 1
    for (int a = 0; a < W; ++a) {
        float S[NG][4];
#pragma unroll
        for (int q = 0; q < NG; ++q) S[q][0] = S[q][1] = S[q][2] = S[q][3] = 0.f;
        const float4 *row = base;
#pragma unroll
        for (int b = 0; b < W; ++b) {
#pragma unroll
            for (int q = 0; q < NG; ++q) {
                const float4 v = __ldg(row + q * gsz);
                df_mac(S[q][0], S[q][1], v.x, v.y, w2h[b], w2l[b]);
                df_mac(S[q][2], S[q][3], v.z, v.w, w2h[b], w2l[b]);
            }
            row += pg.n3;
        }
        const float w1h = __shfl_sync(0xffffffffu, mwh[0], gbase + a);
        const float w1l = __shfl_sync(0xffffffffu, mwl[0], gbase + a);
#pragma unroll
        for (int q = 0; q < NG; ++q) {
            df_norm(S[q][0], S[q][1]);
            df_norm(S[q][2], S[q][3]);
            df_mac(T[q][0], T[q][1], S[q][0], S[q][1], w1h, w1l);
            df_mac(T[q][2], T[q][3], S[q][2], S[q][3], w1h, w1l);
        }
        base += s1;
    }
    double2 out[NG];
#pragma unroll
    for (int q = 0; q < NG; ++q) {
        df_norm(T[q][0], T[q][1]);
        df_norm(T[q][2], T[q][3]);
        float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
        df_mac(rh, rl, T[q][0], T[q][1], mwh[2], mwl[2]);
        df_mac(ih, il, T[q][2], T[q][3], mwh[2], mwl[2]);
#pragma unroll
        for (int off = GS / 2; off > 0; off >>= 1) {
            const float orh = __shfl_xor_sync(0xffffffffu, rh, off, GS);
            const float orl = __shfl_xor_sync(0xffffffffu, rl, off, GS);
            const float oih = __shfl_xor_sync(0xffffffffu, ih, off, GS);
            const float oil = __shfl_xor_sync(0xffffffffu, il, off, GS);
            df_add(rh, rl, orh, orl);
            df_add(ih, il, oih, oil);
        }
        out[q] = scale_value(make_double2((double)rh + (double)rl, (double)ih + (double)il), -value_shift(pts.vexp));
    }
    if (valid && sub == 0) {
        if (NG == 1) {
            f[key.w] = out[0];
        } else {
            if (f) f[key.w] = out[0];
#pragma unroll
            for (int d = 0; d < 3; ++d) grad[3 * (int64_t)key.w + d] = out[(d + 1) % NG];
        }
    }
}

// Padded copies P[p1, p2, p3] = g[p1 mod n1, p2 mod n2, p3 mod n3] of ng grids:
// one block per padded row (q, p1, p2), threads along p3.

// source index of padded index p: (p - shift) mod n, for p in [0, n + 2m)
__device__ __forceinline__ int pad_src(int p, int m, int n) {
    int s = p - m;
    while (s < 0) s += n;
    while (s >= n) s -= n;
    return s;
}

__global__ void pad_grid_f32_kernel(const float2 *__restrict__ G, Grid3 g, float2 *__restrict__ P,
                                    Grid3 pg, int ng, int m) {
    // m here is the layout shift (0 or the window cutoff)
    const int64_t rows = (int64_t)ng * pg.n1 * pg.n2;
    for (int64_t row = blockIdx.x; row < rows; row += gridDim.x) {
        const int p2 = (int)(row % pg.n2);
        const int64_t r = row / pg.n2;
        const int p1 = (int)(r % pg.n1);
        const int q = (int)(r / pg.n1);
        const int s1 = pad_src(p1, m, g.n1), s2 = pad_src(p2, m, g.n2);
        const float2 *src = G + ((int64_t)q * g.n1 + s1) * g.n2 * g.n3 + (int64_t)s2 * g.n3;
        float2 *dst = P + row * pg.n3;
        for (int p3 = threadIdx.x; p3 < pg.n3; p3 += blockDim.x) dst[p3] = src[pad_src(p3, m, g.n3)];
    }
}

// FP64 grids to padded double-float (re_hi, re_lo, im_hi, im_lo).
__global__ void pad_grid_df_kernel(const double2 *__restrict__ G, Grid3 g, float4 *__restrict__ P,
                                   Grid3 pg, int ng, int m) {
    const int64_t rows = (int64_t)ng * pg.n1 * pg.n2;
    for (int64_t row = blockIdx.x; row < rows; row += gridDim.x) {
        const int p2 = (int)(row % pg.n2);
        const int64_t r = row / pg.n2;
        const int p1 = (int)(r % pg.n1);
        const int q = (int)(r / pg.n1);
        const int s1 = pad_src(p1, m, g.n1), s2 = pad_src(p2, m, g.n2);
        const double2 *src = G + ((int64_t)q * g.n1 + s1) * g.n2 * g.n3 + (int64_t)s2 * g.n3;
        float4 *dst = P + row * pg.n3;
        for (int p3 = threadIdx.x; p3 < pg.n3; p3 += blockDim.x) {
            const double2 v = src[pad_src(p3, m, g.n3)];
            float4 o;
            split_df(v.x, o.x, o.y);
            split_df(v.y, o.z, o.w);
            dst[p3] = o;
        }
    }
}

int pad_blocks(int64_t rows) {
    return (int)(rows < (int64_t)1 << 30 ? rows : (int64_t)1 << 30);
}

template <int MM, int NG>
cudaError_t col_f32_dispatch(const float2 *G, Grid3 g, PointsView<float> pts,
                             const WinTable<float> &w, float2 *f, float2 *grad, const int *sel, int64_t nwork,
                             cudaStream_t st) {
    constexpr int W = 2 * MM + 1;
    constexpr int GS = GroupSize<W>::value;
    const int threads = 256;
    const int64_t want = (nwork * GS + threads - 1) / threads;
    bool shared_table = NG == 1 && !std::getenv("GBNFFT_F32_NO_CUBE");
    for (int d = 1; d < 3 && shared_table; ++d)
        for (int a = 0; a < W && shared_table; ++a)
            for (int k = 0; k <= PolyDeg<float>::value; ++k)
                if (w.coef[d][a][k] != w.coef[0][a][k]) shared_table = false;
    if (shared_table) {
        static int resident = 0;   // blocks per SM x SMs for this instantiation
        if (resident == 0) {
            int dev = 0, sms = 0, per_sm = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gather_col_f32_cube_kernel<MM>, threads, 0);
            resident = (sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
        }
        const int64_t blocks = want < resident ? want : resident;
        gather_col_f32_cube_kernel<MM><<<(unsigned)blocks, threads, 0, st>>>(G, g, pts, make_poly<float, MM>(w), f,
                                                                              sel, nwork);
        return cudaGetLastError();
    }
    gather_col_f32_kernel<MM, NG><<<(unsigned)want, threads, 0, st>>>(G, g, pts, make_poly<float, MM>(w), f, grad,
                                                                       sel, nwork);
    return cudaGetLastError();
}

// ---- dense batches (mixed family) --------------------------------------------
// One warp per batch of <= 32 sorted points that share their first stencil
// nodes in dimensions 1 and 2 (they come from one sort key: one tile and one
// (x, y) cell of stencil centres), one point per lane.  Each lane evaluates
// its own 3 (2m+1) tap weights; for every stencil row (a, b) the row's start
// is the same for the whole warp and the lanes' third-dimension origins lie
// within 8 cells of each other (away from the grid's first and last tiles,
// where they wrap), so each load instruction of the warp touches one span of
// at most 2m + 8 grid values (one or two 128-byte lines) instead of one line
// per point as in the column kernel.
template <int MM>
__global__ void __launch_bounds__(256) gather_dense_f32_kernel(const float2 *__restrict__ G, Grid3 pg,
                                                               PointsView<float> pts,
                                                               const __grid_constant__ Poly<float, MM> P,
                                                               const int2 *__restrict__ batches, int nbatch,
                                                               float2 *__restrict__ f) {
    constexpr int W = 2 * MM + 1;
    constexpr int D = PolyDeg<float>::value;
    const int lane = threadIdx.x & 31;
    const int64_t s1 = (int64_t)pg.n2 * pg.n3;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < nbatch; b += nwarps) {
        const int2 bt = batches[b];
        const bool valid = lane < bt.y;
        const int64_t j = (int64_t)bt.x + (valid ? lane : 0);
        const int4 key = pts.key[j];
        float w1[W], w2[W], w3[W];
        {
            const float t1 = 2.f * pts.s1[j] - 1.f, t2 = 2.f * pts.s2[j] - 1.f, t3 = 2.f * pts.s3[j] - 1.f;
#pragma unroll
            for (int a = 0; a < W; ++a) {
                float v1 = P.c[0][a][D], v2 = P.c[1][a][D], v3 = P.c[2][a][D];
#pragma unroll
                for (int k = D - 1; k >= 0; --k) {
                    v1 = fmaf(v1, t1, P.c[0][a][k]);
                    v2 = fmaf(v2, t2, P.c[1][a][k]);
                    v3 = fmaf(v3, t3, P.c[2][a][k]);
                }
                w1[a] = v1;
                w2[a] = v2;
                w3[a] = v3;
            }
        }
        // rows are read as 16-byte pairs of values from the even node at or
        // below the stencil's first one (rows start at even nodes: the padded
        // row length is even); the third-dimension weights shift by one slot
        // for an odd first node and the slot past the stencil weighs zero
        constexpr int W2 = (W + 2) / 2;   // pairs covering W + 1 values
        const int odd = key.z & 1;
        float w3s[2 * W2];
#pragma unroll
        for (int c = 0; c < 2 * W2; ++c) {
            const float lo = c < W ? w3[c] : 0.f, hi = c >= 1 && c - 1 < W ? w3[c - 1] : 0.f;
            w3s[c] = odd ? hi : lo;
        }
        const float4 *base = reinterpret_cast<const float4 *>(G + (int64_t)key.x * s1 + (int64_t)key.y * pg.n3 +
                                                                (key.z - odd));
        const int64_t rstep = pg.n3 / 2;   // float4 per padded row
        float Tr = 0.f, Ti = 0.f;
#pragma unroll 1
        for (int a = 0; a < W; ++a) {
            float Sr = 0.f, Si = 0.f;
            const float4 *row = base;
#pragma unroll
            for (int bb = 0; bb < W; ++bb) {
                float Rr = 0.f, Ri = 0.f;
#pragma unroll
                for (int c = 0; c < W2; ++c) {
                    const float4 v = __ldg(row + c);
                    Rr = fmaf(w3s[2 * c], v.x, Rr);
                    Ri = fmaf(w3s[2 * c], v.y, Ri);
                    Rr = fmaf(w3s[2 * c + 1], v.z, Rr);
                    Ri = fmaf(w3s[2 * c + 1], v.w, Ri);
                }
                Sr = fmaf(w2[bb], Rr, Sr);
                Si = fmaf(w2[bb], Ri, Si);
                row += rstep;
            }
            Tr = fmaf(w1[0], Sr, Tr);
            Ti = fmaf(w1[0], Si, Ti);
#pragma unroll
            for (int k = 0; k < W - 1; ++k) w1[k] = w1[k + 1];
            base += s1 / 2;
        }
        if (valid) f[key.w] = make_float2(Tr, Ti);
    }
}

template <int MM>
cudaError_t split_f32_dispatch(const float2 *G, Grid3 g, PointsView<float> pts, const WinTable<float> &w,
                               const int2 *batches, int nbatch, const int *sparse_idx, int nsparse, float2 *f,
                               cudaStream_t st) {
    if (nbatch > 0) {
        static int resident = 0;   // blocks per SM x SMs for this instantiation
        if (resident == 0) {
            int dev = 0, sms = 0, per_sm = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gather_dense_f32_kernel<MM>, 256, 0);
            resident = (sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
        }
        const int64_t want = ((int64_t)nbatch * 32 + 255) / 256;
        gather_dense_f32_kernel<MM><<<(unsigned)(want < resident ? want : resident), 256, 0, st>>>(
            G, g, pts, make_poly<float, MM>(w), batches, nbatch, f);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (nsparse > 0) return col_f32_dispatch<MM, 1>(G, g, pts, w, f, nullptr, sparse_idx, nsparse, st);
    return cudaSuccess;
}

template <int MM, int NG>
cudaError_t col_df_dispatch(const float4 *G, Grid3 g, PointsView<double> pts, const WinTableDF &w,
                            const WinTable<double> &w64, bool fp64_weights, double2 *f, double2 *grad,
                            cudaStream_t st, const HalfTables *half) {
    constexpr int GS = GroupSize<2 * MM + 1>::value;
    const int threads = 256;
    const int64_t blocks = (pts.M * GS + threads - 1) / threads;
    const int hmode = half ? half->mode : 0;
    if (NG == 1 && fp64_weights && !std::getenv("GBNFFT_DF_COLUMNS")) {
        if (hmode == 1)
            gather_slot_df_kernel<MM, WeightsFP64H<MM>><<<(unsigned)blocks, threads, 0, st>>>(
                G, g, pts, make_poly_n<double, MM, kPolyDegHalf>(half->w64), f);
        else if (hmode == 2)
            gather_slot_df_kernel<MM, WeightsDFH<MM>><<<(unsigned)blocks, threads, 0, st>>>(
                G, g, pts, make_poly_dfn<MM, kPolyDegHalf>(half->wdf), f);
        else
            gather_slot_df_kernel<MM, WeightsFP64<MM>><<<(unsigned)blocks, threads, 0, st>>>(
                G, g, pts, make_poly<double, MM>(w64), f);
    } else if (fp64_weights)
        gather_col_df_kernel<MM, NG, WeightsFP64<MM>><<<(unsigned)blocks, threads, 0, st>>>(
            G, g, pts, make_poly<double, MM>(w64), f, grad);
    else
        gather_col_df_kernel<MM, NG, WeightsDF<MM>><<<(unsigned)blocks, threads, 0, st>>>(
            G, g, pts, make_poly_df<MM>(w), f, grad);
    return cudaGetLastError();
}

template <int NG>
cudaError_t col_f32_select(const float2 *G, Grid3 g, int m, PointsView<float> pts,
                           const WinTable<float> &w, float2 *f, float2 *grad, cudaStream_t st) {
    if (pts.M == 0) return cudaSuccess;
    switch (m) {
        case 1: return col_f32_dispatch<1, NG>(G, g, pts, w, f, grad, nullptr, pts.M, st);
        case 2: return col_f32_dispatch<2, NG>(G, g, pts, w, f, grad, nullptr, pts.M, st);
        case 3: return col_f32_dispatch<3, NG>(G, g, pts, w, f, grad, nullptr, pts.M, st);
        case 4: return col_f32_dispatch<4, NG>(G, g, pts, w, f, grad, nullptr, pts.M, st);
        case 5: return col_f32_dispatch<5, NG>(G, g, pts, w, f, grad, nullptr, pts.M, st);
        case 6: return col_f32_dispatch<6, NG>(G, g, pts, w, f, grad, nullptr, pts.M, st);
        case 7: return col_f32_dispatch<7, NG>(G, g, pts, w, f, grad, nullptr, pts.M, st);
        case 8: return col_f32_dispatch<8, NG>(G, g, pts, w, f, grad, nullptr, pts.M, st);
        default: return cudaErrorInvalidValue;
    }
}

template <int NG>
cudaError_t col_df_select(const float4 *G, Grid3 g, int m, PointsView<double> pts,
                          const WinTableDF &w, const WinTable<double> &w64, bool fp64_weights, double2 *f,
                          double2 *grad, cudaStream_t st, const HalfTables *half) {
    if (pts.M == 0) return cudaSuccess;
    switch (m) {
        case 1: return col_df_dispatch<1, NG>(G, g, pts, w, w64, fp64_weights, f, grad, st, half);
        case 2: return col_df_dispatch<2, NG>(G, g, pts, w, w64, fp64_weights, f, grad, st, half);
        case 3: return col_df_dispatch<3, NG>(G, g, pts, w, w64, fp64_weights, f, grad, st, half);
        case 4: return col_df_dispatch<4, NG>(G, g, pts, w, w64, fp64_weights, f, grad, st, half);
        case 5: return col_df_dispatch<5, NG>(G, g, pts, w, w64, fp64_weights, f, grad, st, half);
        case 6: return col_df_dispatch<6, NG>(G, g, pts, w, w64, fp64_weights, f, grad, st, half);
        case 7: return col_df_dispatch<7, NG>(G, g, pts, w, w64, fp64_weights, f, grad, st, half);
        case 8: return col_df_dispatch<8, NG>(G, g, pts, w, w64, fp64_weights, f, grad, st, half);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_pad_grid_f32(const float2 *G, Grid3 g, float2 *P, Grid3 pg, int ng, int shift,
                                cudaStream_t st) {
    const int64_t rows = (int64_t)ng * pg.n1 * pg.n2;
    pad_grid_f32_kernel<<<pad_blocks(rows), 128, 0, st>>>(G, g, P, pg, ng, shift);
    return cudaGetLastError();
}

cudaError_t launch_pad_grid_df(const double2 *G, Grid3 g, float4 *P, Grid3 pg, int ng, int shift,
                               cudaStream_t st) {
    const int64_t rows = (int64_t)ng * pg.n1 * pg.n2;
    pad_grid_df_kernel<<<pad_blocks(rows), 128, 0, st>>>(G, g, P, pg, ng, shift);
    return cudaGetLastError();
}

cudaError_t launch_gather_col_f32(const float2 *G, Grid3 g, int m, PointsView<float> pts,
                                  const WinTable<float> &w, float2 *f, float2 *grad, int ng,
                                  cudaStream_t st) {
    return ng == 4 ? col_f32_select<4>(G, g, m, pts, w, f, grad, st)
                   : col_f32_select<1>(G, g, m, pts, w, f, nullptr, st);
}

cudaError_t launch_gather_split_f32(const float2 *G, Grid3 g, int m, PointsView<float> pts,
                                    const WinTable<float> &w, const int2 *batches, int nbatch,
                                    const int *sparse_idx, int nsparse, float2 *f, cudaStream_t st) {
    if (pts.M == 0) return cudaSuccess;
    switch (m) {
        case 1: return split_f32_dispatch<1>(G, g, pts, w, batches, nbatch, sparse_idx, nsparse, f, st);
        case 2: return split_f32_dispatch<2>(G, g, pts, w, batches, nbatch, sparse_idx, nsparse, f, st);
        case 3: return split_f32_dispatch<3>(G, g, pts, w, batches, nbatch, sparse_idx, nsparse, f, st);
        case 4: return split_f32_dispatch<4>(G, g, pts, w, batches, nbatch, sparse_idx, nsparse, f, st);
        case 5: return split_f32_dispatch<5>(G, g, pts, w, batches, nbatch, sparse_idx, nsparse, f, st);
        case 6: return split_f32_dispatch<6>(G, g, pts, w, batches, nbatch, sparse_idx, nsparse, f, st);
        case 7: return split_f32_dispatch<7>(G, g, pts, w, batches, nbatch, sparse_idx, nsparse, f, st);
        case 8: return split_f32_dispatch<8>(G, g, pts, w, batches, nbatch, sparse_idx, nsparse, f, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_gather_col_df(const float4 *G, Grid3 g, int m, PointsView<double> pts,
                                 const WinTableDF &w, const WinTable<double> &w64, bool fp64_weights,
                                 double2 *f, double2 *grad, int ng, cudaStream_t st, const HalfTables *half) {
    return ng == 4 ? col_df_select<4>(G, g, m, pts, w, w64, fp64_weights, f, grad, st, nullptr)
                   : col_df_select<1>(G, g, m, pts, w, w64, fp64_weights, f, nullptr, st, half);
}

}  // namespace gbnfft
