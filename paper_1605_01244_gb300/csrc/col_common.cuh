// Shared pieces of the column-parallel gathers (gather_col.cu, gather_wd.cu):
// lane-group size, double-float arithmetic helpers and the per-lane tap
// weight evaluators (value, and value + derivative for the window-derivative
// gradient).
#pragma once
#include "internal.cuh"

namespace gbnfft {
namespace {

template <int W> struct GroupSize {
    static constexpr int value = W <= 2 ? 2 : W <= 4 ? 4 : W <= 8 ? 8 : W <= 16 ? 16 : 32;
};

// ---- packed pairs of floats (f32x2) -----------------------------------------
// Two FP32 values in one 64-bit register, operated on by a single add, sub,
// mul or fma instruction (PTX .f32x2, sm_100 and later; IEEE round to
// nearest, subnormals kept, like the scalar intrinsics).  The FP64 family's
// double-float arithmetic on complex values treats the real and imaginary
// parts as one pair, which halves its instruction count.
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 x2_pack(float a, float b) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void x2_unpack(f32x2 v, float &a, float &b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f32x2 x2_add(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 x2_sub(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 x2_mul(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 x2_fma(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
// v XOR z with z = 0 supplied at run time (a kernel argument): the same
// bits, but a value the code generator cannot trace back to the instruction
// that made it.  Measured on sm_103a: a packed product fed straight into a
// packed add was fused into one multiply-add (a single rounding), and
// fma(x, y, -(x y)) was folded to zero, although both break the explicitly
// rounded operations' semantics; passing the product through this exclusive
// or keeps each operation as written (checked bit for bit against the scalar
// df_mac and df_norm below).
__device__ __forceinline__ f32x2 x2_opaque(f32x2 v, f32x2 z) {
    f32x2 r;
    asm("xor.b64 %0, %1, %2;" : "=l"(r) : "l"(v), "l"(z));
    return r;
}
// (sh, sl) += (xh, xl) (yh, yl) on both halves of the pairs: the operations
// of df_mac below, in the same order (so the same results), packed; z: a
// run-time zero (x2_opaque)
__device__ __forceinline__ void x2_df_mac(f32x2 &sh, f32x2 &sl, f32x2 xh, f32x2 xl, f32x2 yh, f32x2 yl,
                                          f32x2 z) {
    const f32x2 p = x2_opaque(x2_mul(xh, yh), z);
    f32x2 e = x2_fma(xh, yh, x2_sub(0ull, p));
    e = x2_fma(xh, yl, e);
    e = x2_fma(xl, yh, e);
    const f32x2 s = x2_add(sh, p);
    const f32x2 bb = x2_sub(s, sh);
    const f32x2 err = x2_add(x2_sub(sh, x2_sub(s, bb)), x2_sub(p, bb));
    sl = x2_add(sl, x2_add(err, e));
    sh = s;
}
// (ph, pl) = (xh, xl) (yh, yl), normalised, on both halves of the pairs: the
// exact product of the high parts, its error and the cross terms, then one
// fast two-sum; z: a run-time zero (x2_opaque)
__device__ __forceinline__ void x2_df_mul(f32x2 &ph, f32x2 &pl, f32x2 xh, f32x2 xl, f32x2 yh, f32x2 yl,
                                          f32x2 z) {
    const f32x2 p = x2_opaque(x2_mul(xh, yh), z);
    f32x2 e = x2_fma(xh, yh, x2_sub(0ull, p));
    e = x2_fma(xh, yl, e);
    e = x2_fma(xl, yh, e);
    ph = x2_add(p, e);
    pl = x2_sub(e, x2_sub(ph, p));
}
// (sh, sl) += (xh, xl) (yh, yl) on both halves, for a multiplier x that is
// reused: nxh = -xh and nxl = -xl are passed in (made once, through
// x2_opaque), so the product's error is carried negated, ne = -e, by
// multiply-adds alone.  The product of the high parts is fma(xh, yh, z) with
// the run-time zero z: the same value as the product, but not a product the
// code generator could fuse into the two-sum's addition.  The same results as
// x2_df_mac, up to the sign of zero.
__device__ __forceinline__ void x2_df_mac_neg(f32x2 &sh, f32x2 &sl, f32x2 xh, f32x2 nxh, f32x2 nxl, f32x2 yh,
                                              f32x2 yl, f32x2 z) {
    const f32x2 p = x2_fma(xh, yh, z);
    f32x2 ne = x2_fma(nxh, yh, p);
    ne = x2_fma(nxh, yl, ne);
    ne = x2_fma(nxl, yh, ne);
    const f32x2 s = x2_add(sh, p);
    const f32x2 bb = x2_sub(s, sh);
    const f32x2 err = x2_add(x2_sub(sh, x2_sub(s, bb)), x2_sub(p, bb));
    sl = x2_add(sl, x2_sub(err, ne));
    sh = s;
}
// df_norm on both halves
__device__ __forceinline__ void x2_df_norm(f32x2 &sh, f32x2 &sl) {
    const f32x2 s = x2_add(sh, sl);
    sl = x2_sub(sl, x2_sub(s, sh));
    sh = s;
}

// ---- double-float helpers (same arithmetic as gather_df.cu) ------------------
__device__ __forceinline__ void df_mac(float &ah, float &al, float xh, float xl, float yh,
                                       float yl) {
    const float p = __fmul_rn(xh, yh);
    float e = __fmaf_rn(xh, yh, -p);
    e = __fmaf_rn(xh, yl, e);
    e = __fmaf_rn(xl, yh, e);
    const float s = __fadd_rn(ah, p);
    const float bb = __fsub_rn(s, ah);
    const float err = __fadd_rn(__fsub_rn(ah, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    al = __fadd_rn(al, __fadd_rn(err, e));
    ah = s;
}
__device__ __forceinline__ void df_norm(float &ah, float &al) {
    const float s = __fadd_rn(ah, al);
    al = __fsub_rn(al, __fsub_rn(s, ah));
    ah = s;
}
__device__ __forceinline__ void df_add(float &ah, float &al, float bh, float bl) {
    const float s = __fadd_rn(ah, bh);
    const float bb = __fsub_rn(s, ah);
    const float err = __fadd_rn(__fsub_rn(ah, __fsub_rn(s, bb)), __fsub_rn(bh, bb));
    al = __fadd_rn(al, __fadd_rn(err, bl));
    ah = s;
}
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

// Tap weights of the double-float gather, per lane (its tap) and dimension,
// as float pairs.  WeightsDF: Horner in double-float on the FP32 pipe with the
// hi/lo coefficient table.  WeightsFP64: Horner in FP64 on the FP64 pipe --
// which the window sums leave idle, so it runs alongside them -- then an exact
// integer split of each weight into hi + lo.
template <int MM> struct WeightsDF {
    using Table = PolyDF<MM>;
    static constexpr int W = 2 * MM + 1, D = kPolyDegDF;
    float ch[3][W][D + 1];
    float cl[3][W][D + 1];
    __device__ void load(const Table &P) {
        for (int i = threadIdx.x; i < 3 * W * (D + 1); i += blockDim.x) {
            (&ch[0][0][0])[i] = (&P.ch[0][0][0])[i];
            (&cl[0][0][0])[i] = (&P.cl[0][0][0])[i];
        }
    }
    __device__ __forceinline__ void eval(int d, int tap, double s, float &wh, float &wl) const {
        const double t = 2.0 * s - 1.0;
        const float th = __double2float_rn(t);
        const float tl = __double2float_rn(t - (double)th);
        float vh = ch[d][tap][D], vl = cl[d][tap][D];
#pragma unroll
        for (int k = D - 1; k >= 0; --k) df_horner_step(vh, vl, th, tl, ch[d][tap][k], cl[d][tap][k]);
        wh = vh;
        wl = vl;
    }
};
template <int MM> struct WeightsFP64 {
    using Table = Poly<double, MM>;
    static constexpr int W = 2 * MM + 1, D = PolyDeg<double>::value;
    double c[3][W][D + 1];
    __device__ void load(const Table &P) {
        for (int i = threadIdx.x; i < 3 * W * (D + 1); i += blockDim.x) (&c[0][0][0])[i] = (&P.c[0][0][0])[i];
    }
    __device__ __forceinline__ void eval(int d, int tap, double s, float &wh, float &wl) const {
        const double t = 2.0 * s - 1.0;
        double v = c[d][tap][D];
#pragma unroll
        for (int k = D - 1; k >= 0; --k) v = fma(v, t, c[d][tap][k]);
        split_df(v, wh, wl);
    }
};

// Half-interval tables (HalfTables in internal.cuh): the row and argument u
// in [-1, 1] of tap `tap` at offset s.  4s - 3 is exact for s in [1/2, 1);
// 1 - 4s is exact for s >= 1/8 and within 2^-53 below.
template <int MM> __device__ __forceinline__ void half_arg(int tap, double s, int &row, double &u) {
    const bool up = s >= 0.5;
    row = up ? tap : 2 * MM - tap;
    u = up ? fma(4.0, s, -3.0) : fma(-4.0, s, 1.0);
}
template <int MM> struct WeightsFP64H {
    using Table = PolyN<double, MM, kPolyDegHalf>;
    static constexpr int W = 2 * MM + 1, D = kPolyDegHalf;
    double c[3][W][D + 1];
    __device__ void load(const Table &P) {
        for (int i = threadIdx.x; i < 3 * W * (D + 1); i += blockDim.x) (&c[0][0][0])[i] = (&P.c[0][0][0])[i];
    }
    __device__ __forceinline__ void eval(int d, int tap, double s, float &wh, float &wl) const {
        int row;
        double u;
        half_arg<MM>(tap, s, row, u);
        double v = c[d][row][D];
#pragma unroll
        for (int k = D - 1; k >= 0; --k) v = fma(v, u, c[d][row][k]);
        split_df(v, wh, wl);
    }
};
template <int MM> struct WeightsDFH {
    using Table = PolyDFN<MM, kPolyDegHalf>;
    static constexpr int W = 2 * MM + 1, D = kPolyDegHalf;
    float ch[3][W][D + 1];
    float cl[3][W][D + 1];
    __device__ void load(const Table &P) {
        for (int i = threadIdx.x; i < 3 * W * (D + 1); i += blockDim.x) {
            (&ch[0][0][0])[i] = (&P.ch[0][0][0])[i];
            (&cl[0][0][0])[i] = (&P.cl[0][0][0])[i];
        }
    }
    __device__ __forceinline__ void eval(int d, int tap, double s, float &wh, float &wl) const {
        int row;
        double u;
        half_arg<MM>(tap, s, row, u);
        const float uh = __double2float_rn(u);
        const float ul = __double2float_rn(u - (double)uh);
        float vh = ch[d][row][D], vl = cl[d][row][D];
#pragma unroll
        for (int k = D - 1; k >= 0; --k) df_horner_step(vh, vl, uh, ul, ch[d][row][k], cl[d][row][k]);
        wh = vh;
        wl = vl;
    }
};

// Value and derivative weights: P(t) and dP/dx = -2 n_d P'(t) (t = 2s - 1,
// s decreases by n_d per unit of x), Horner for P and P' together.
template <int MM> struct WeightsFP64D {
    using Table = Poly<double, MM>;
    static constexpr int W = 2 * MM + 1, D = PolyDeg<double>::value;
    double c[3][W][D + 1];
    __device__ void load(const Table &P) {
        for (int i = threadIdx.x; i < 3 * W * (D + 1); i += blockDim.x) (&c[0][0][0])[i] = (&P.c[0][0][0])[i];
    }
    // value (hi, lo) and derivative (hi, lo) scaled by dxs = -2 n_d
    __device__ __forceinline__ void eval(int d, int tap, double s, double dxs, float &wh, float &wl, float &dh,
                                         float &dl) const {
        const double t = 2.0 * s - 1.0;
        double v = c[d][tap][D], dv = 0.0;
#pragma unroll
        for (int k = D - 1; k >= 0; --k) {
            dv = fma(dv, t, v);
            v = fma(v, t, c[d][tap][k]);
        }
        split_df(v, wh, wl);
        split_df(dv * dxs, dh, dl);
    }
};
template <int MM> struct WeightsF32D {
    using Table = Poly<float, MM>;
    static constexpr int W = 2 * MM + 1, D = PolyDeg<float>::value;
    float c[3][W][D + 1];
    __device__ void load(const Table &P) {
        for (int i = threadIdx.x; i < 3 * W * (D + 1); i += blockDim.x) (&c[0][0][0])[i] = (&P.c[0][0][0])[i];
    }
    __device__ __forceinline__ void eval(int d, int tap, float s, float dxs, float &w, float &dw) const {
        const float t = 2.f * s - 1.f;
        float v = c[d][tap][D], dv = 0.f;
#pragma unroll
        for (int k = D - 1; k >= 0; --k) {
            dv = fmaf(dv, t, v);
            v = fmaf(v, t, c[d][tap][k]);
        }
        w = v;
        dw = dv * dxs;
    }
};

}  // namespace
}  // namespace gbnfft
