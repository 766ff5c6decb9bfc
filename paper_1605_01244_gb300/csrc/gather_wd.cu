// Window-derivative gradient gather: value and gradient of the NFFT
// approximation from ONE padded grid (origin layout), by differentiating the
// window instead of the series:
//   f        = sum_a w1[a]  sum_b w2[b]  sum_c w3[c]  g[l0 + (a, b, c)]
//   d f/dx1  = sum_a w1'[a] sum_b w2[b]  sum_c w3[c]  g
//   d f/dx2  = sum_a w1[a]  sum_b w2'[b] sum_c w3[c]  g
//   d f/dx3  = sum_a w1[a]  sum_b w2[b]  sum_c w3'[c] g
// with w'[a] = d/dx_d phi(u_d - l_d) = n_d phi'(u_d - l_d) (torus units).
// Same column-parallel layout as gather_col.cu: lane c of a group owns stencil
// column c and accumulates, per plane a, S = sum_b w2 g and S' = sum_b w2' g,
// then T = sum_a w1 S, T1 = sum_a w1' S, T2 = sum_a w1 S'; the group reduces
// f = sum_c w3 T, g1 = sum_c w3 T1, g2 = sum_c w3 T2, g3 = sum_c w3' T.
// Per tap this is two multiply-adds per real part (one grid read) instead of
// four grids and four multiply-adds of the i k-weighted method, and the
// transform runs once instead of four times.
#include "col_common.cuh"

namespace gbnfft {
namespace {

// ---- FP64 family: double-float sums, FP64 weights ---------------------------
template <int MM>
__global__ void __launch_bounds__(256, 2) gather_wd_df_kernel(const float4 *__restrict__ G, Grid3 pg,
                                                              PointsView<double> pts, double3 dxs,
                                                              const __grid_constant__ Poly<double, MM> P,
                                                              double2 *__restrict__ f,
                                                              double2 *__restrict__ grad) {
    constexpr int W = 2 * MM + 1;
    constexpr int GS = GroupSize<W>::value;
    __shared__ WeightsFP64D<MM> wt;
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
    float wh[3], wl[3], dh[3], dl[3];
    {
        const double s[3] = {pts.s1[jj], pts.s2[jj], pts.s3[jj]};
        const double sc[3] = {dxs.x, dxs.y, dxs.z};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            wt.eval(d, tap, s[d], sc[d], wh[d], wl[d], dh[d], dl[d]);
            if (sub >= W) wh[d] = wl[d] = dh[d] = dl[d] = 0.f;
        }
    }
    float w2h[W], w2l[W], d2h[W], d2l[W];
#pragma unroll
    for (int b = 0; b < W; ++b) {
        w2h[b] = __shfl_sync(0xffffffffu, wh[1], gbase + b);
        w2l[b] = __shfl_sync(0xffffffffu, wl[1], gbase + b);
        d2h[b] = __shfl_sync(0xffffffffu, dh[1], gbase + b);
        d2l[b] = __shfl_sync(0xffffffffu, dl[1], gbase + b);
    }
    const int64_t s1 = (int64_t)pg.n2 * pg.n3;
    const float4 *base = G + (int64_t)key.x * s1 + (int64_t)key.y * pg.n3 + key.z + tap;
    // accumulators (re_hi, re_lo, im_hi, im_lo): T value, T1 d/dx1, T2 d/dx2
    float T[4] = {0.f, 0.f, 0.f, 0.f}, T1[4] = {0.f, 0.f, 0.f, 0.f}, T2[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 1
    for (int a = 0; a < W; ++a) {
        float S[4] = {0.f, 0.f, 0.f, 0.f}, Sd[4] = {0.f, 0.f, 0.f, 0.f};
        const float4 *row = base;
#pragma unroll
        for (int b = 0; b < W; ++b) {
            const float4 v = __ldg(row);
            df_mac(S[0], S[1], v.x, v.y, w2h[b], w2l[b]);
            df_mac(S[2], S[3], v.z, v.w, w2h[b], w2l[b]);
            df_mac(Sd[0], Sd[1], v.x, v.y, d2h[b], d2l[b]);
            df_mac(Sd[2], Sd[3], v.z, v.w, d2h[b], d2l[b]);
            row += pg.n3;
        }
        const float w1h = __shfl_sync(0xffffffffu, wh[0], gbase + a);
        const float w1l = __shfl_sync(0xffffffffu, wl[0], gbase + a);
        const float d1h = __shfl_sync(0xffffffffu, dh[0], gbase + a);
        const float d1l = __shfl_sync(0xffffffffu, dl[0], gbase + a);
        df_norm(S[0], S[1]);
        df_norm(S[2], S[3]);
        df_norm(Sd[0], Sd[1]);
        df_norm(Sd[2], Sd[3]);
        df_mac(T[0], T[1], S[0], S[1], w1h, w1l);
        df_mac(T[2], T[3], S[2], S[3], w1h, w1l);
        df_mac(T1[0], T1[1], S[0], S[1], d1h, d1l);
        df_mac(T1[2], T1[3], S[2], S[3], d1h, d1l);
        df_mac(T2[0], T2[1], Sd[0], Sd[1], w1h, w1l);
        df_mac(T2[2], T2[3], Sd[2], Sd[3], w1h, w1l);
        base += s1;
    }
    df_norm(T[0], T[1]);
    df_norm(T[2], T[3]);
    df_norm(T1[0], T1[1]);
    df_norm(T1[2], T1[3]);
    df_norm(T2[0], T2[1]);
    df_norm(T2[2], T2[3]);
    // per-lane column sums: f (w3 T), g1 (w3 T1), g2 (w3 T2), g3 (w3' T)
    float R[4][4] = {};
    df_mac(R[0][0], R[0][1], T[0], T[1], wh[2], wl[2]);
    df_mac(R[0][2], R[0][3], T[2], T[3], wh[2], wl[2]);
    df_mac(R[1][0], R[1][1], T1[0], T1[1], wh[2], wl[2]);
    df_mac(R[1][2], R[1][3], T1[2], T1[3], wh[2], wl[2]);
    df_mac(R[2][0], R[2][1], T2[0], T2[1], wh[2], wl[2]);
    df_mac(R[2][2], R[2][3], T2[2], T2[3], wh[2], wl[2]);
    df_mac(R[3][0], R[3][1], T[0], T[1], dh[2], dl[2]);
    df_mac(R[3][2], R[3][3], T[2], T[3], dh[2], dl[2]);
    double2 out[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
#pragma unroll
        for (int off = GS / 2; off > 0; off >>= 1) {
            float o[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) o[i] = __shfl_xor_sync(0xffffffffu, R[q][i], off, GS);
            df_add(R[q][0], R[q][1], o[0], o[1]);
            df_add(R[q][2], R[q][3], o[2], o[3]);
        }
        out[q] = scale_value(make_double2((double)R[q][0] + (double)R[q][1], (double)R[q][2] + (double)R[q][3]),
                             -value_shift(pts.vexp));
    }
    if (valid && sub == 0) {
        if (f) f[key.w] = out[0];
#pragma unroll
        for (int d = 0; d < 3; ++d) grad[3 * (int64_t)key.w + d] = out[d + 1];
    }
}

// ---- mixed family: FP32 -------------------------------------------------------
template <int MM>
__global__ void __launch_bounds__(256) gather_wd_f32_kernel(const float2 *__restrict__ G, Grid3 pg,
                                                            PointsView<float> pts, float3 dxs,
                                                            const __grid_constant__ Poly<float, MM> P,
                                                            float2 *__restrict__ f, float2 *__restrict__ grad) {
    constexpr int W = 2 * MM + 1;
    constexpr int GS = GroupSize<W>::value;
    __shared__ WeightsF32D<MM> wt;
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
    float w[3], dw[3];
    {
        const float s[3] = {pts.s1[jj], pts.s2[jj], pts.s3[jj]};
        const float sc[3] = {dxs.x, dxs.y, dxs.z};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            wt.eval(d, tap, s[d], sc[d], w[d], dw[d]);
            if (sub >= W) w[d] = dw[d] = 0.f;
        }
    }
    float w2[W], d2[W];
#pragma unroll
    for (int b = 0; b < W; ++b) {
        w2[b] = __shfl_sync(0xffffffffu, w[1], gbase + b);
        d2[b] = __shfl_sync(0xffffffffu, dw[1], gbase + b);
    }
    const int64_t s1 = (int64_t)pg.n2 * pg.n3;
    const float2 *base = G + (int64_t)key.x * s1 + (int64_t)key.y * pg.n3 + key.z + tap;
    float2 T = make_float2(0.f, 0.f), T1 = T, T2 = T;
#pragma unroll 1
    for (int a = 0; a < W; ++a) {
        float2 S = make_float2(0.f, 0.f), Sd = S;
        const float2 *row = base;
#pragma unroll
        for (int b = 0; b < W; ++b) {
            const float2 v = __ldg(row);
            S.x = fmaf(w2[b], v.x, S.x);
            S.y = fmaf(w2[b], v.y, S.y);
            Sd.x = fmaf(d2[b], v.x, Sd.x);
            Sd.y = fmaf(d2[b], v.y, Sd.y);
            row += pg.n3;
        }
        const float w1 = __shfl_sync(0xffffffffu, w[0], gbase + a);
        const float d1 = __shfl_sync(0xffffffffu, dw[0], gbase + a);
        T.x = fmaf(w1, S.x, T.x);
        T.y = fmaf(w1, S.y, T.y);
        T1.x = fmaf(d1, S.x, T1.x);
        T1.y = fmaf(d1, S.y, T1.y);
        T2.x = fmaf(w1, Sd.x, T2.x);
        T2.y = fmaf(w1, Sd.y, T2.y);
        base += s1;
    }
    float R[4][2] = {{w[2] * T.x, w[2] * T.y}, {w[2] * T1.x, w[2] * T1.y}, {w[2] * T2.x, w[2] * T2.y},
                     {dw[2] * T.x, dw[2] * T.y}};
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int off = GS / 2; off > 0; off >>= 1) {
            R[q][0] += __shfl_xor_sync(0xffffffffu, R[q][0], off, GS);
            R[q][1] += __shfl_xor_sync(0xffffffffu, R[q][1], off, GS);
        }
    if (valid && sub == 0) {
        if (f) f[key.w] = make_float2(R[0][0], R[0][1]);
#pragma unroll
        for (int d = 0; d < 3; ++d) grad[3 * (int64_t)key.w + d] = make_float2(R[d + 1][0], R[d + 1][1]);
    }
}

template <int MM>
cudaError_t wd_df_dispatch(const float4 *G, Grid3 pg, PointsView<double> pts, const WinTable<double> &w,
                           double3 dxs, double2 *f, double2 *grad, cudaStream_t st) {
    constexpr int GS = GroupSize<2 * MM + 1>::value;
    const int64_t blocks = (pts.M * GS + 255) / 256;
    gather_wd_df_kernel<MM><<<(unsigned)blocks, 256, 0, st>>>(G, pg, pts, dxs, make_poly<double, MM>(w), f, grad);
    return cudaGetLastError();
}

template <int MM>
cudaError_t wd_f32_dispatch(const float2 *G, Grid3 pg, PointsView<float> pts, const WinTable<float> &w,
                            float3 dxs, float2 *f, float2 *grad, cudaStream_t st) {
    constexpr int GS = GroupSize<2 * MM + 1>::value;
    const int64_t blocks = (pts.M * GS + 255) / 256;
    gather_wd_f32_kernel<MM><<<(unsigned)blocks, 256, 0, st>>>(G, pg, pts, dxs, make_poly<float, MM>(w), f, grad);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gather_wd_df(const float4 *G, Grid3 pg, int m, PointsView<double> pts,
                                const WinTable<double> &w, const int n[3], double2 *f, double2 *grad,
                                cudaStream_t st) {
    if (pts.M == 0) return cudaSuccess;
    const double3 dxs = make_double3(-2.0 * n[0], -2.0 * n[1], -2.0 * n[2]);
    switch (m) {
        case 1: return wd_df_dispatch<1>(G, pg, pts, w, dxs, f, grad, st);
        case 2: return wd_df_dispatch<2>(G, pg, pts, w, dxs, f, grad, st);
        case 3: return wd_df_dispatch<3>(G, pg, pts, w, dxs, f, grad, st);
        case 4: return wd_df_dispatch<4>(G, pg, pts, w, dxs, f, grad, st);
        case 5: return wd_df_dispatch<5>(G, pg, pts, w, dxs, f, grad, st);
        case 6: return wd_df_dispatch<6>(G, pg, pts, w, dxs, f, grad, st);
        case 7: return wd_df_dispatch<7>(G, pg, pts, w, dxs, f, grad, st);
        case 8: return wd_df_dispatch<8>(G, pg, pts, w, dxs, f, grad, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_gather_wd_f32(const float2 *G, Grid3 pg, int m, PointsView<float> pts,
                                 const WinTable<float> &w, const int n[3], float2 *f, float2 *grad,
                                 cudaStream_t st) {
    if (pts.M == 0) return cudaSuccess;
    const float3 dxs = make_float3(-2.f * n[0], -2.f * n[1], -2.f * n[2]);
    switch (m) {
        case 1: return wd_f32_dispatch<1>(G, pg, pts, w, dxs, f, grad, st);
        case 2: return wd_f32_dispatch<2>(G, pg, pts, w, dxs, f, grad, st);
        case 3: return wd_f32_dispatch<3>(G, pg, pts, w, dxs, f, grad, st);
        case 4: return wd_f32_dispatch<4>(G, pg, pts, w, dxs, f, grad, st);
        case 5: return wd_f32_dispatch<5>(G, pg, pts, w, dxs, f, grad, st);
        case 6: return wd_f32_dispatch<6>(G, pg, pts, w, dxs, f, grad, st);
        case 7: return wd_f32_dispatch<7>(G, pg, pts, w, dxs, f, grad, st);
        case 8: return wd_f32_dispatch<8>(G, pg, pts, w, dxs, f, grad, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace gbnfft
