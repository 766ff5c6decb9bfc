// Forward-path grid transform, fused: deconvolution, the unnormalised inverse
// DFT of the oversampled grid and the ghost-padded layout the column gathers
// read, for power-of-two grid sizes (16 <= n_d <= 2048).
//
//   g_l = sum_{k in I_N} c_k D1[k1] D2[k2] D3[k3] exp(+2 pi i k.l / n)
//
// computed as three passes of 1D DFTs over the nonzero band only:
//   rows   (along l3): one line per in-band (k1, k2), input c deconvolved;
//   cols2  (along l2): one line per (k1, l3);
//   out    (along l1): one line per (l2, l3), written to every padded
//                      position p = l + shift + t n in [0, n + 2m) (t = -1, 0, 1).
// Each line is transformed in shared memory by radix-8 (then 4 or 2) Stockham
// passes.  The FP64 family computes in double-float on the FP32 pipe (the
// grid values enter as FP64 products and are split into float pairs), and
// the mixed family in FP32; the padded output is what the gathers expect
// (float4 re_hi, re_lo, im_hi, im_lo, or float2).
// With ng = 4 the same passes also produce the gradient grids 2 pi i k_d g.
#include "fastdiv.cuh"
#include "internal.cuh"

#ifndef GBNFFT_DF_LINE_ELEMS
#define GBNFFT_DF_LINE_ELEMS 2048    // double-float passes: elements per block (4096: 3.27 / 3.87 ms
                                     // forward / adjoint at n = 512^3, 2048: 3.09 / 3.37 ms)
#endif
#ifndef GBNFFT_DF_EPT
#define GBNFFT_DF_EPT 8              // double-float passes: elements per thread
#endif
#ifndef GBNFFT_F32_LINE_ELEMS
#define GBNFFT_F32_LINE_ELEMS 4096   // FP32 passes: elements per block (2048 and 8192 measured slower at 8 a thread)
#endif
#ifndef GBNFFT_F32_EPT
#define GBNFFT_F32_EPT 8             // FP32 adjoint passes: elements per thread (8: one radix-8 butterfly a pass)
#endif
#ifndef GBNFFT_F32_FWD_ELEMS
#define GBNFFT_F32_FWD_ELEMS 4096    // FP32 forward passes: elements per block
#endif
#ifndef GBNFFT_F32_FWD_EPT
#define GBNFFT_F32_FWD_EPT 16        // FP32 forward passes: elements per thread (16: 1.09 -> 0.96 ms at n = 512^3)
#endif

namespace gbnfft {
namespace {

// Line elements per block (lines x length) are A::kElems (at least the
// longest line, 2^11); a block has
// A::kThreads = kElems / kEPT threads, each holding kEPT elements of a line
// (kEPT / 8 radix-8 butterflies per pass).

// ---- double-float arithmetic (FP64-accurate on the FP32 pipe) ---------------
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}
__device__ __forceinline__ void dd_add(float ah, float al, float bh, float bl, float &h, float &l) {
    float s, e;
    two_sum(ah, bh, s, e);
    e = __fadd_rn(e, __fadd_rn(al, bl));
    fast_two_sum(s, e, h, l);
}
__device__ __forceinline__ void dd_mul(float ah, float al, float bh, float bl, float &h, float &l) {
    const float p = __fmul_rn(ah, bh);
    float e = __fmaf_rn(ah, bh, -p);
    e = __fmaf_rn(ah, bl, e);
    e = __fmaf_rn(al, bh, e);
    fast_two_sum(p, e, h, l);
}

struct ArithDF {
    struct C {
        float rh, rl, ih, il;
    };
    using S = float4;
    static constexpr int kPadShift = 3;   // 16-byte elements: one pad per 8
    static constexpr int kElems = GBNFFT_DF_LINE_ELEMS;
    static constexpr int kEPT = GBNFFT_DF_EPT, kThreads = kElems / kEPT;
    static __device__ __forceinline__ C ld(const S &s) { return C{s.x, s.y, s.z, s.w}; }
    static __device__ __forceinline__ S st(const C &c) { return make_float4(c.rh, c.rl, c.ih, c.il); }
    static __device__ __forceinline__ C zero() { return C{0.f, 0.f, 0.f, 0.f}; }
    static __device__ __forceinline__ C add(const C &a, const C &b) {
        C o;
        dd_add(a.rh, a.rl, b.rh, b.rl, o.rh, o.rl);
        dd_add(a.ih, a.il, b.ih, b.il, o.ih, o.il);
        return o;
    }
    static __device__ __forceinline__ C sub(const C &a, const C &b) {
        C o;
        dd_add(a.rh, a.rl, -b.rh, -b.rl, o.rh, o.rl);
        dd_add(a.ih, a.il, -b.ih, -b.il, o.ih, o.il);
        return o;
    }
    // a * w (w a table twiddle)
    static __device__ __forceinline__ C mul(const C &a, const S &w) {
        float t1h, t1l, t2h, t2l, t3h, t3l, t4h, t4l;
        dd_mul(a.rh, a.rl, w.x, w.y, t1h, t1l);   // ar wr
        dd_mul(a.ih, a.il, w.z, w.w, t2h, t2l);   // ai wi
        dd_mul(a.rh, a.rl, w.z, w.w, t3h, t3l);   // ar wi
        dd_mul(a.ih, a.il, w.x, w.y, t4h, t4l);   // ai wr
        C o;
        dd_add(t1h, t1l, -t2h, -t2l, o.rh, o.rl);
        dd_add(t3h, t3l, t4h, t4l, o.ih, o.il);
        return o;
    }
    static __device__ __forceinline__ C mul_i(const C &a) { return C{-a.ih, -a.il, a.rh, a.rl}; }
    static __device__ __forceinline__ C conj(const C &a) { return C{a.rh, a.rl, -a.ih, -a.il}; }
    // a grid value of the adjoint (FP64), split into float pairs
    static __device__ __forceinline__ C from(double2 v) {
        C o;
        split_df(v.x, o.rh, o.rl);
        split_df(v.y, o.ih, o.il);
        return o;
    }
    // a * (1 + i) / sqrt 2 and a * (-1 + i) / sqrt 2
    static __device__ __forceinline__ C mul_w8(const C &a) {
        float dh, dl, sh, sl;
        dd_add(a.rh, a.rl, -a.ih, -a.il, dh, dl);
        dd_add(a.rh, a.rl, a.ih, a.il, sh, sl);
        C o;
        dd_mul(dh, dl, kR2h, kR2l, o.rh, o.rl);
        dd_mul(sh, sl, kR2h, kR2l, o.ih, o.il);
        return o;
    }
    static __device__ __forceinline__ C mul_w83(const C &a) {
        float dh, dl, sh, sl;
        dd_add(a.rh, a.rl, -a.ih, -a.il, dh, dl);
        dd_add(a.rh, a.rl, a.ih, a.il, sh, sl);
        C o;
        dd_mul(-sh, -sl, kR2h, kR2l, o.rh, o.rl);
        dd_mul(dh, dl, kR2h, kR2l, o.ih, o.il);
        return o;
    }
    static constexpr double kR2 = 0.70710678118654752440;
    static constexpr float kR2h = (float)kR2;
    static constexpr float kR2l = (float)(kR2 - (double)(float)kR2);
};

struct ArithF32 {
    struct C {
        float r, i;
    };
    using S = float2;
    static constexpr int kPadShift = 4;   // 8-byte elements: one pad per 16
    static constexpr int kElems = GBNFFT_F32_LINE_ELEMS;
    static constexpr int kEPT = GBNFFT_F32_EPT, kThreads = kElems / kEPT;
    static __device__ __forceinline__ C ld(const S &s) { return C{s.x, s.y}; }
    static __device__ __forceinline__ S st(const C &c) { return make_float2(c.r, c.i); }
    static __device__ __forceinline__ C zero() { return C{0.f, 0.f}; }
    static __device__ __forceinline__ C add(const C &a, const C &b) { return C{a.r + b.r, a.i + b.i}; }
    static __device__ __forceinline__ C sub(const C &a, const C &b) { return C{a.r - b.r, a.i - b.i}; }
    static __device__ __forceinline__ C mul(const C &a, const S &w) {
        return C{fmaf(a.r, w.x, -a.i * w.y), fmaf(a.r, w.y, a.i * w.x)};
    }
    static __device__ __forceinline__ C mul_i(const C &a) { return C{-a.i, a.r}; }
    static __device__ __forceinline__ C conj(const C &a) { return C{a.r, -a.i}; }
    static __device__ __forceinline__ C from(float2 v) { return C{v.x, v.y}; }
    static __device__ __forceinline__ C mul_w8(const C &a) {
        constexpr float r2 = 0.70710678118654752440f;
        return C{(a.r - a.i) * r2, (a.r + a.i) * r2};
    }
    static __device__ __forceinline__ C mul_w83(const C &a) {
        constexpr float r2 = 0.70710678118654752440f;
        return C{-(a.r + a.i) * r2, (a.r - a.i) * r2};
    }
};

// The forward (series to padded grid) FP32 passes: the same arithmetic with
// their own block shape (two radix-8 butterflies per thread and pass measured
// faster there, slower in the adjoint passes)
struct ArithF32Fwd : ArithF32 {
    static constexpr int kElems = GBNFFT_F32_FWD_ELEMS;
    static constexpr int kEPT = GBNFFT_F32_FWD_EPT, kThreads = kElems / kEPT;
};
#ifndef GBNFFT_F32_ROWS_ELEMS
#define GBNFFT_F32_ROWS_ELEMS 2048   // 0.963 -> 0.944 ms for the three passes at n = 512^3
#endif
#ifndef GBNFFT_F32_ROWS_EPT
#define GBNFFT_F32_ROWS_EPT 8
#endif
// the first forward pass (rows along l3) may take its own block shape
struct ArithF32Rows : ArithF32 {
    static constexpr int kElems = GBNFFT_F32_ROWS_ELEMS;
    static constexpr int kEPT = GBNFFT_F32_ROWS_EPT, kThreads = kElems / kEPT;
};
template <class A> struct RowsArith { using T = A; };
template <> struct RowsArith<ArithF32Fwd> { using T = ArithF32Rows; };

// ---- radix-R DFTs with the inverse sign: X_k = sum_a x_a exp(+2 pi i a k / R) --
template <class A> __device__ __forceinline__ void dft2(typename A::C &x0, typename A::C &x1) {
    const typename A::C s = A::add(x0, x1), d = A::sub(x0, x1);
    x0 = s;
    x1 = d;
}
template <class A>
__device__ __forceinline__ void dft4(typename A::C &y0, typename A::C &y1, typename A::C &y2,
                                     typename A::C &y3) {
    const typename A::C s0 = A::add(y0, y2), s1 = A::sub(y0, y2), s2 = A::add(y1, y3),
                        s3 = A::mul_i(A::sub(y1, y3));
    y0 = A::add(s0, s2);
    y1 = A::add(s1, s3);
    y2 = A::sub(s0, s2);
    y3 = A::sub(s1, s3);
}
// X_{2k} = DFT4(x_a + x_{a+4}), X_{2k+1} = DFT4((x_a - x_{a+4}) w8^a)
template <class A> __device__ __forceinline__ void dft8(typename A::C *x) {
    using C = typename A::C;
    C u[4], v[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        u[a] = A::add(x[a], x[a + 4]);
        v[a] = A::sub(x[a], x[a + 4]);
    }
    v[1] = A::mul_w8(v[1]);
    v[2] = A::mul_i(v[2]);
    v[3] = A::mul_w83(v[3]);
    dft4<A>(u[0], u[1], u[2], u[3]);
    dft4<A>(v[0], v[1], v[2], v[3]);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        x[2 * k] = u[k];
        x[2 * k + 1] = v[k];
    }
}

template <class A> __device__ __forceinline__ int pidx(int i) { return i + (i >> A::kPadShift); }

// One Stockham pass of radix R = 2^LOGR over a line x of length L = 2^LOGL
// (element i at pidx(i)), by the line's T = L/8 threads, each taking 8/R
// butterflies: butterfly j reads x[j + r L/R], applies w_{Ns R}^{r (j mod Ns)}
// (w_n = exp(2 pi i / n), table tw[i] = w_L^i), and writes
// x'[(j / Ns) Ns R + j mod Ns + r Ns], Ns = 2^LOGNS.  In place: all reads, a
// barrier, all writes.  Sizes are compile-time, so strides and pads fold.
template <class A, int LOGL, int LOGNS, int LOGR>
__device__ __forceinline__ void stockham_pass(typename A::S *x, const typename A::S *tw, int u, int bh) {
    using C = typename A::C;
    constexpr int R = 1 << LOGR, PER = A::kEPT / R;
    constexpr int T = (1 << LOGL) / A::kEPT;
    constexpr int NB = 1 << (LOGL - LOGR);
    constexpr int NS = 1 << LOGNS;
    constexpr int TWS = LOGL - LOGNS - LOGR;   // twiddle index shift
    constexpr int PS = A::kPadShift;
    C v[A::kEPT];
#pragma unroll
    for (int b = 0; b < PER; ++b) {
        const int j = u + b * T;
        const int k = j & (NS - 1);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            int idx;
            if constexpr ((NB & ((1 << PS) - 1)) == 0)
                idx = pidx<A>(j) + r * (NB + (NB >> PS));
            else
                idx = pidx<A>(j + r * NB);
            C t;
            if constexpr (LOGNS == 0) {
                // first pass: only the band l < bh or l >= L - bh holds input;
                // the rest of the line buffer is never written and reads as zero
                const int l = j + r * NB;
                t = (l < bh || l >= (1 << LOGL) - bh) ? A::ld(x[idx]) : A::zero();
            } else {
                t = A::ld(x[idx]);
                if (r > 0) t = A::mul(t, tw[(r * k) << TWS]);
            }
            v[b * R + r] = t;
        }
    }
#pragma unroll
    for (int b = 0; b < PER; ++b) {
        if constexpr (R == 8)
            dft8<A>(v + 8 * b);
        else if constexpr (R == 4)
            dft4<A>(v[4 * b], v[4 * b + 1], v[4 * b + 2], v[4 * b + 3]);
        else
            dft2<A>(v[2 * b], v[2 * b + 1]);
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < PER; ++b) {
        const int j = u + b * T;
        const int d = ((j >> LOGNS) << (LOGNS + LOGR)) + (j & (NS - 1));
#pragma unroll
        for (int r = 0; r < R; ++r) {
            int idx;
            if constexpr ((NS & ((1 << PS) - 1)) == 0)
                idx = pidx<A>(d) + r * (NS + (NS >> PS));
            else
                idx = pidx<A>(d + r * NS);
            x[idx] = A::st(v[b * R + r]);
        }
    }
    __syncthreads();
}

template <class A, int LOGL, int LOGNS>
__device__ __forceinline__ void stockham_from(typename A::S *x, const typename A::S *tw, int u, int bh) {
    if constexpr (LOGL - LOGNS >= 3) {
        stockham_pass<A, LOGL, LOGNS, 3>(x, tw, u, bh);
        stockham_from<A, LOGL, LOGNS + 3>(x, tw, u, bh);
    } else if constexpr (LOGL - LOGNS == 2) {
        stockham_pass<A, LOGL, LOGNS, 2>(x, tw, u, bh);
    } else if constexpr (LOGL - LOGNS == 1) {
        stockham_pass<A, LOGL, LOGNS, 1>(x, tw, u, bh);
    }
}

// In-place DFT of the block's lines in shared memory: line `line` of length
// L = 2^LOGL starts at sm + line * LS, T = L/kEPT threads per line, radix-8
// passes then one radix-4 or radix-2 pass for the remaining factor.
template <class A, int LOGL>
__device__ __forceinline__ void line_dft(typename A::S *sm, const typename A::S *__restrict__ tw, int LS,
                                         int bh) {
    constexpr int T = (1 << LOGL) / A::kEPT;
    const int line = threadIdx.x / T, u = threadIdx.x - line * T;
    stockham_from<A, LOGL, 0>(sm + line * LS, tw, u, bh);
}

template <class A> __device__ __forceinline__ void load_twiddles(typename A::S *dst, const typename A::S *src, int L) {
    for (int i = threadIdx.x; i < L; i += blockDim.x) dst[i] = src[i];
}

// deconvolved input value of grid q (0: c_k D; d = 1..3: 2 pi i k_d c_k D);
// the FP64 family's c enters scaled by 2^vs (range scaling, internal.cuh)
__device__ __forceinline__ ArithDF::C series_value(ArithDF, double2 c, double d, int q, int kq, int vs) {
    c = scale_value(c, vs);
    double re = c.x * d, im = c.y * d;
    if (q > 0) {
        const double f = 6.283185307179586476925286766559 * (double)kq;
        const double t = re;
        re = -f * im;
        im = f * t;
    }
    ArithDF::C o;
    split_df(re, o.rh, o.rl);
    split_df(im, o.ih, o.il);
    return o;
}
__device__ __forceinline__ ArithF32::C series_value(ArithF32, float2 c, float d, int q, int kq, int) {
    float re = c.x * d, im = c.y * d;
    if (q > 0) {
        const float f = 6.283185307179586476925286766559f * (float)kq;
        const float t = re;
        re = -f * im;
        im = f * t;
    }
    return ArithF32::C{re, im};
}

// padded ghost copy of primary position p (or -1), for 2m <= n
__device__ __forceinline__ int ghost_of(int p, int n, int m2) { return p < m2 ? p + n : (p >= n ? p - n : -1); }

__device__ __forceinline__ int band_pos(int i, int N, int n) {   // k = i - N/2 -> l = k mod n
    const int k = i - N / 2;
    return k < 0 ? k + n : k;
}

struct FusedArgs {
    int N1, N2, N3, n1, n2, n3;
    int logn1, logn2, logn3;
    int m, shift, ng;
    FastDiv divN2, divN3;
    const int *vexp;   // FP64 family's range word (nullptr: no scaling)
};

// Pass 1: rows along l3 for the in-band (k1, k2); input c deconvolved.
// A[q][i1 N2 + i2][l3].
template <class A, typename R, int LOGL>
__global__ void __launch_bounds__(A::kThreads) fused_rows_kernel(
    const typename Cplx<R>::T *__restrict__ c, const R *__restrict__ D1, const R *__restrict__ D2,
    const R *__restrict__ D3, const typename A::S *__restrict__ tw3, typename A::S *__restrict__ out,
    FusedArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using S = typename A::S;
    constexpr int L = 1 << LOGL, LPB = A::kElems / L;
    constexpr int LS = L + (L >> A::kPadShift) + 1;
    S *sm = reinterpret_cast<S *>(smem_raw);
    S *tws = sm + LPB * LS;
    const int q = blockIdx.y;
    const int64_t nrows = (int64_t)a.N1 * a.N2;
    const int64_t row0 = (int64_t)blockIdx.x * LPB;
    load_twiddles<A>(tws, tw3, L);
    const int vs = value_shift(a.vexp);
    // the N3 deconvolved coefficients of each row, at their band positions
    // (the first pass reads the rest of the line as zero)
    for (int e = threadIdx.x; e < LPB * a.N3; e += blockDim.x) {
        const int line = (int)a.divN3.div((unsigned)e), i3 = e - line * a.N3;
        const int64_t row = row0 + line;
        if (row >= nrows) continue;
        const int i1 = (int)a.divN2.div((unsigned)row), i2 = (int)(row - (int64_t)i1 * a.N2);
        // frequency k_q of the gradient grid q (unused for q = 0)
        const int kq = q == 1 ? i1 - a.N1 / 2 : q == 2 ? i2 - a.N2 / 2 : i3 - a.N3 / 2;
        const R d = D1[i1] * D2[i2] * D3[i3];
        sm[line * LS + pidx<A>(band_pos(i3, a.N3, a.n3))] =
            A::st(series_value(A{}, c[row * a.N3 + i3], d, q, kq, vs));
    }
    __syncthreads();
    line_dft<A, LOGL>(sm, tws, LS, a.N3 / 2);
    S *o = out + (int64_t)q * nrows * L;
    for (int e = threadIdx.x; e < LPB * L; e += blockDim.x) {
        const int line = e / L, l3 = e - line * L;
        const int64_t row = row0 + line;
        if (row < nrows) o[row * L + l3] = sm[line * LS + pidx<A>(l3)];
    }
}

// Pass 2: lines along l2 for each (k1, l3).  in A[q][i1 N2 + i2][l3],
// out B[q][i1][l2][l3].  A block takes LPB consecutive l3 of one i1.
template <class A, int LOGL>
__global__ void __launch_bounds__(A::kThreads) fused_cols_kernel(const typename A::S *__restrict__ in,
                                                                  const typename A::S *__restrict__ tw2,
                                                                  typename A::S *__restrict__ out,
                                                                  FusedArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using S = typename A::S;
    constexpr int L = 1 << LOGL, LPB = A::kElems / L;
    constexpr int LS = L + (L >> A::kPadShift) + 1;
    S *sm = reinterpret_cast<S *>(smem_raw);
    S *tws = sm + LPB * LS;
    const int q = blockIdx.y;
    const int nblk3 = (a.n3 + LPB - 1) / LPB;
    const int i1 = blockIdx.x / nblk3;
    const int l30 = (blockIdx.x - i1 * nblk3) * LPB;
    const int nl = a.n3 - l30 < LPB ? a.n3 - l30 : LPB;
    load_twiddles<A>(tws, tw2, L);
    // each thread keeps one line (l3) and walks i2 / l2 with a constant stride
    constexpr int STEP = A::kThreads / LPB;
    const int line = threadIdx.x & (LPB - 1), r0 = threadIdx.x / LPB;
    S *sl = sm + line * LS;
    if (line < nl) {
        const S *src = in + ((int64_t)q * a.N1 + i1) * a.N2 * a.n3 + l30 + line + (int64_t)r0 * a.n3;
        const int64_t sstep = (int64_t)STEP * a.n3;
        for (int i2 = r0; i2 < a.N2; i2 += STEP, src += sstep) sl[pidx<A>(band_pos(i2, a.N2, a.n2))] = *src;
    }
    __syncthreads();
    line_dft<A, LOGL>(sm, tws, LS, a.N2 / 2);
    if (line < nl) {
        S *dst = out + ((int64_t)q * a.N1 + i1) * a.n2 * a.n3 + l30 + line + (int64_t)r0 * a.n3;
        const int64_t dstep = (int64_t)STEP * a.n3;
#pragma unroll 4
        for (int l2 = r0; l2 < L; l2 += STEP, dst += dstep) *dst = sl[pidx<A>(l2)];
    }
}

// Pass 3: lines along l1 for each (l2, l3); in B[q][i1][l2][l3]; out the
// padded grid P[q][p1][p2][p3], p = l + shift + t n in [0, n + 2m).
template <class A, int LOGL>
__global__ void __launch_bounds__(A::kThreads) fused_out_kernel(const typename A::S *__restrict__ in,
                                                                 const typename A::S *__restrict__ tw1,
                                                                 typename A::S *__restrict__ P,
                                                                 FusedArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using S = typename A::S;
    constexpr int L = 1 << LOGL, LPB = A::kElems / L;
    constexpr int LS = L + (L >> A::kPadShift) + 1;
    S *sm = reinterpret_cast<S *>(smem_raw);
    S *tws = sm + LPB * LS;
    const int q = blockIdx.y;
    const int nblk3 = (a.n3 + LPB - 1) / LPB;
    const int l2 = blockIdx.x / nblk3;
    const int l30 = (blockIdx.x - l2 * nblk3) * LPB;
    const int nl = a.n3 - l30 < LPB ? a.n3 - l30 : LPB;
    load_twiddles<A>(tws, tw1, L);
    // each thread keeps one line (l3) and walks i1 / l1 with a constant stride
    constexpr int STEP = A::kThreads / LPB;
    const int line = threadIdx.x & (LPB - 1), r0 = threadIdx.x / LPB;
    S *sl = sm + line * LS;
    if (line < nl) {
        const int64_t sstep = (int64_t)a.n2 * a.n3;
        const S *src = in + (int64_t)q * a.N1 * sstep + (int64_t)l2 * a.n3 + l30 + line + r0 * sstep;
        for (int i1 = r0; i1 < a.N1; i1 += STEP, src += STEP * sstep) sl[pidx<A>(band_pos(i1, a.N1, a.n1))] = *src;
    }
    __syncthreads();
    line_dft<A, LOGL>(sm, tws, LS, a.N1 / 2);
    if (line >= nl) return;
    const int m2 = 2 * a.m;
    const int pn2 = a.n2 + m2, pn3 = a.n3 + m2;
    const int64_t plane = (int64_t)pn2 * pn3;
    // every l has its primary position p = l + shift in [0, n + 2m) and at most
    // one ghost copy (2m <= n): p + n if p < 2m, p - n if p >= n.  Along l2
    // and l3 the copies are fixed offsets from the primary element.
    const int p2 = l2 + a.shift, g2 = ghost_of(p2, a.n2, m2);
    const int p3 = l30 + line + a.shift, g3 = ghost_of(p3, a.n3, m2);
    const int64_t d2 = g2 >= 0 ? (int64_t)(g2 - p2) * pn3 : 0;
    const int d3 = g3 >= 0 ? g3 - p3 : 0;
    const int64_t d1 = (int64_t)a.n1 * plane;
    S *r = P + (int64_t)q * (a.n1 + m2) * plane + (int64_t)(r0 + a.shift) * plane + (int64_t)p2 * pn3 + p3;
    const int64_t rstep = (int64_t)STEP * plane;
    for (int l1 = r0; l1 < L; l1 += STEP, r += rstep) {
        const S v = sl[pidx<A>(l1)];
        const int p1 = l1 + a.shift;
        r[0] = v;
        if (g3 >= 0) r[d3] = v;
        if (g2 >= 0) {
            r[d2] = v;
            if (g3 >= 0) r[d2 + d3] = v;
        }
        if (p1 < m2 || p1 >= a.n1) {
            S *rg = r + (p1 < m2 ? d1 : -d1);
            rg[0] = v;
            if (g3 >= 0) rg[d3] = v;
            if (g2 >= 0) {
                rg[d2] = v;
                if (g3 >= 0) rg[d2 + d3] = v;
            }
        }
    }
}

// ---- adjoint direction: forward DFT of the oversampled grid, band only -------
// h_k = D1 D2 D3 sum_l H_l exp(-2 pi i k.l / n) for k in the band, as three
// passes of line DFTs: along l1 (all n2 n3 lines, N1 band outputs kept),
// along l2 (N1 n3 lines, N2 kept), along l3 (N1 N2 lines, N3 kept, then
// deconvolved).  The forward sign comes from conjugation: the input is
// conjugated once, the passes run the inverse-sign line DFT, and the output
// is conjugated back.
// deconvolved adjoint output of the FP64 family (range scaled back) / mixed
template <typename R> struct AdjOut;
template <> struct AdjOut<double> {
    static __device__ __forceinline__ double2 get(const ArithDF::C &v, double d, int vs) {
        return scale_value(make_double2(((double)v.rh + (double)v.rl) * d, ((double)v.ih + (double)v.il) * d), vs);
    }
};
template <> struct AdjOut<float> {
    static __device__ __forceinline__ float2 get(const ArithF32::C &v, float d, int) {
        return make_float2(v.r * d, v.i * d);
    }
};

// Pass 1: along l1 for each (l2, l3); in H[l1][l2][l3] (family type),
// out A[i1][l2][l3] (N1 n2 n3).  A block takes LPB consecutive l3 of one l2.
template <class A, typename R, int LOGL>
__global__ void __launch_bounds__(A::kThreads) adj_first_kernel(const typename Cplx<R>::T *__restrict__ H,
                                                                 const typename A::S *__restrict__ tw1,
                                                                 typename A::S *__restrict__ out, FusedArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using S = typename A::S;
    constexpr int L = 1 << LOGL, LPB = A::kElems / L;
    constexpr int LS = L + (L >> A::kPadShift) + 1;
    S *sm = reinterpret_cast<S *>(smem_raw);
    S *tws = sm + LPB * LS;
    const int nblk3 = (a.n3 + LPB - 1) / LPB;
    const int l2 = blockIdx.x / nblk3;
    const int l30 = (blockIdx.x - l2 * nblk3) * LPB;
    const int nl = a.n3 - l30 < LPB ? a.n3 - l30 : LPB;
    load_twiddles<A>(tws, tw1, L);
    constexpr int STEP = A::kThreads / LPB;
    const int line = threadIdx.x & (LPB - 1), r0 = threadIdx.x / LPB;
    S *sl = sm + line * LS;
    const int64_t plane = (int64_t)a.n2 * a.n3;
    if (line < nl) {
        const typename Cplx<R>::T *src = H + (int64_t)r0 * plane + (int64_t)l2 * a.n3 + l30 + line;
        for (int l1 = r0; l1 < L; l1 += STEP, src += STEP * plane) sl[pidx<A>(l1)] = A::st(A::conj(A::from(*src)));
    }
    __syncthreads();
    line_dft<A, LOGL>(sm, tws, LS, L / 2);
    if (line < nl) {
        S *dst = out + ((int64_t)r0 * a.n2 + l2) * a.n3 + l30 + line;
        for (int i1 = r0; i1 < a.N1; i1 += STEP, dst += STEP * plane) *dst = sl[pidx<A>(band_pos(i1, a.N1, a.n1))];
    }
}

// Pass 2: along l2 for each (i1, l3); in A[i1][l2][l3], out B[i1][i2][l3]
// (N1 N2 n3).  A block takes LPB consecutive l3 of one i1.
template <class A, int LOGL>
__global__ void __launch_bounds__(A::kThreads) adj_mid_kernel(const typename A::S *__restrict__ in,
                                                               const typename A::S *__restrict__ tw2,
                                                               typename A::S *__restrict__ out, FusedArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using S = typename A::S;
    constexpr int L = 1 << LOGL, LPB = A::kElems / L;
    constexpr int LS = L + (L >> A::kPadShift) + 1;
    S *sm = reinterpret_cast<S *>(smem_raw);
    S *tws = sm + LPB * LS;
    const int nblk3 = (a.n3 + LPB - 1) / LPB;
    const int i1 = blockIdx.x / nblk3;
    const int l30 = (blockIdx.x - i1 * nblk3) * LPB;
    const int nl = a.n3 - l30 < LPB ? a.n3 - l30 : LPB;
    load_twiddles<A>(tws, tw2, L);
    constexpr int STEP = A::kThreads / LPB;
    const int line = threadIdx.x & (LPB - 1), r0 = threadIdx.x / LPB;
    S *sl = sm + line * LS;
    if (line < nl) {
        const S *src = in + (int64_t)i1 * a.n2 * a.n3 + l30 + line + (int64_t)r0 * a.n3;
        for (int l2 = r0; l2 < L; l2 += STEP, src += (int64_t)STEP * a.n3) sl[pidx<A>(l2)] = *src;
    }
    __syncthreads();
    line_dft<A, LOGL>(sm, tws, LS, L / 2);
    if (line < nl) {
        S *dst = out + (int64_t)i1 * a.N2 * a.n3 + l30 + line + (int64_t)r0 * a.n3;
        for (int i2 = r0; i2 < a.N2; i2 += STEP, dst += (int64_t)STEP * a.n3)
            *dst = sl[pidx<A>(band_pos(i2, a.N2, a.n2))];
    }
}

// Pass 3: along l3 for each (i1, i2); in B[i1][i2][l3], out the deconvolved
// band c[i1][i2][i3] (family type, conjugated back, range scaled back).
template <class A, typename R, int LOGL>
__global__ void __launch_bounds__(A::kThreads) adj_last_kernel(const typename A::S *__restrict__ in,
                                                                const R *__restrict__ D1, const R *__restrict__ D2,
                                                                const R *__restrict__ D3,
                                                                const typename A::S *__restrict__ tw3,
                                                                typename Cplx<R>::T *__restrict__ c, FusedArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using S = typename A::S;
    constexpr int L = 1 << LOGL, LPB = A::kElems / L;
    constexpr int LS = L + (L >> A::kPadShift) + 1;
    S *sm = reinterpret_cast<S *>(smem_raw);
    S *tws = sm + LPB * LS;
    const int64_t nrows = (int64_t)a.N1 * a.N2;
    const int64_t row0 = (int64_t)blockIdx.x * LPB;
    load_twiddles<A>(tws, tw3, L);
    for (int e = threadIdx.x; e < LPB * L; e += blockDim.x) {
        const int line = e / L, l3 = e - line * L;
        const int64_t row = row0 + line;
        if (row < nrows) sm[line * LS + pidx<A>(l3)] = in[row * L + l3];
    }
    __syncthreads();
    line_dft<A, LOGL>(sm, tws, LS, L / 2);
    const int vs = -value_shift(a.vexp);
    for (int e = threadIdx.x; e < LPB * a.N3; e += blockDim.x) {
        const int line = (int)a.divN3.div((unsigned)e), i3 = e - line * a.N3;
        const int64_t row = row0 + line;
        if (row >= nrows) continue;
        const int i1 = (int)a.divN2.div((unsigned)row), i2 = (int)(row - (int64_t)i1 * a.N2);
        const R d = D1[i1] * D2[i2] * D3[i3];
        const typename A::C v = A::conj(A::ld(sm[line * LS + pidx<A>(band_pos(i3, a.N3, a.n3))]));
        c[row * a.N3 + i3] = AdjOut<R>::get(v, d, vs);
    }
}

int ilog2(int v) {
    int r = 0;
    while ((1 << r) < v) ++r;
    return r;
}

template <class A>
size_t line_smem(int L) {
    const int LPB = A::kElems / L;
    const int LS = L + (L >> A::kPadShift) + 1;
    return sizeof(typename A::S) * ((size_t)LPB * LS + L);
}

template <class A, typename R, int LOGL>
cudaError_t launch_rows(const typename Cplx<R>::T *c, const R *D1, const R *D2, const R *D3,
                        const typename A::S *tw, typename A::S *out, const FusedArgs &a, cudaStream_t st) {
    const size_t sm = line_smem<A>(1 << LOGL);
    cudaError_t e = cudaFuncSetAttribute(fused_rows_kernel<A, R, LOGL>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const int64_t rows = (int64_t)a.N1 * a.N2, lpb = A::kElems >> LOGL;
    dim3 g((unsigned)((rows + lpb - 1) / lpb), (unsigned)a.ng);
    fused_rows_kernel<A, R, LOGL><<<g, A::kThreads, sm, st>>>(c, D1, D2, D3, tw, out, a);
    return cudaGetLastError();
}

template <class A, int LOGL>
cudaError_t launch_cols(const typename A::S *in, const typename A::S *tw, typename A::S *out,
                        const FusedArgs &a, cudaStream_t st) {
    const size_t sm = line_smem<A>(1 << LOGL);
    cudaError_t e =
        cudaFuncSetAttribute(fused_cols_kernel<A, LOGL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const int lpb = A::kElems >> LOGL;
    dim3 g((unsigned)(a.N1 * ((a.n3 + lpb - 1) / lpb)), (unsigned)a.ng);
    fused_cols_kernel<A, LOGL><<<g, A::kThreads, sm, st>>>(in, tw, out, a);
    return cudaGetLastError();
}

template <class A, int LOGL>
cudaError_t launch_out(const typename A::S *in, const typename A::S *tw, typename A::S *P,
                       const FusedArgs &a, cudaStream_t st) {
    const size_t sm = line_smem<A>(1 << LOGL);
    cudaError_t e =
        cudaFuncSetAttribute(fused_out_kernel<A, LOGL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const int lpb = A::kElems >> LOGL;
    dim3 g((unsigned)(a.n2 * ((a.n3 + lpb - 1) / lpb)), (unsigned)a.ng);
    fused_out_kernel<A, LOGL><<<g, A::kThreads, sm, st>>>(in, tw, P, a);
    return cudaGetLastError();
}

// Line lengths 2^4 .. 2^11.
#define GBNFFT_LOGL_SWITCH(logl, CALL)          \
    switch (logl) {                            \
        case 4: return CALL(4);                \
        case 5: return CALL(5);                \
        case 6: return CALL(6);                \
        case 7: return CALL(7);                \
        case 8: return CALL(8);                \
        case 9: return CALL(9);                \
        case 10: return CALL(10);              \
        case 11: return CALL(11);              \
        default: return cudaErrorInvalidValue; \
    }

template <class A, typename R>
cudaError_t run_rows(const typename Cplx<R>::T *c, const R *D1, const R *D2, const R *D3,
                     const typename A::S *tw, typename A::S *out, const FusedArgs &a, cudaStream_t st) {
#define GBNFFT_CALL(L) launch_rows<A, R, L>(c, D1, D2, D3, tw, out, a, st)
    GBNFFT_LOGL_SWITCH(a.logn3, GBNFFT_CALL)
#undef GBNFFT_CALL
}
template <class A>
cudaError_t run_cols(const typename A::S *in, const typename A::S *tw, typename A::S *out, const FusedArgs &a,
                     cudaStream_t st) {
#define GBNFFT_CALL(L) launch_cols<A, L>(in, tw, out, a, st)
    GBNFFT_LOGL_SWITCH(a.logn2, GBNFFT_CALL)
#undef GBNFFT_CALL
}
template <class A>
cudaError_t run_out(const typename A::S *in, const typename A::S *tw, typename A::S *P, const FusedArgs &a,
                    cudaStream_t st) {
#define GBNFFT_CALL(L) launch_out<A, L>(in, tw, P, a, st)
    GBNFFT_LOGL_SWITCH(a.logn1, GBNFFT_CALL)
#undef GBNFFT_CALL
}

template <class A, typename R>
cudaError_t run_fused(const typename Cplx<R>::T *c, const R *D1, const R *D2, const R *D3,
                      const void *const tw[3], void *scratch, void *P, const FusedArgs &a,
                      cudaStream_t st) {
    using S = typename A::S;
    S *Abuf = (S *)scratch;
    S *Bbuf = Abuf + (int64_t)a.ng * a.N1 * a.N2 * a.n3;
    cudaError_t e = run_rows<typename RowsArith<A>::T, R>(c, D1, D2, D3, (const S *)tw[2], Abuf, a, st);
    if (e == cudaSuccess) e = run_cols<A>(Abuf, (const S *)tw[1], Bbuf, a, st);
    if (e == cudaSuccess) e = run_out<A>(Bbuf, (const S *)tw[0], (S *)P, a, st);
    return e;
}

template <class A, typename R, int LOGL>
cudaError_t launch_adj_first(const typename Cplx<R>::T *H, const typename A::S *tw, typename A::S *out,
                             const FusedArgs &a, cudaStream_t st) {
    const size_t sm = line_smem<A>(1 << LOGL);
    cudaError_t e = cudaFuncSetAttribute(adj_first_kernel<A, R, LOGL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm);
    if (e != cudaSuccess) return e;
    const int lpb = A::kElems >> LOGL;
    adj_first_kernel<A, R, LOGL><<<(unsigned)(a.n2 * ((a.n3 + lpb - 1) / lpb)), A::kThreads, sm, st>>>(H, tw, out,
                                                                                                         a);
    return cudaGetLastError();
}

template <class A, int LOGL>
cudaError_t launch_adj_mid(const typename A::S *in, const typename A::S *tw, typename A::S *out, const FusedArgs &a,
                           cudaStream_t st) {
    const size_t sm = line_smem<A>(1 << LOGL);
    cudaError_t e =
        cudaFuncSetAttribute(adj_mid_kernel<A, LOGL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const int lpb = A::kElems >> LOGL;
    adj_mid_kernel<A, LOGL><<<(unsigned)(a.N1 * ((a.n3 + lpb - 1) / lpb)), A::kThreads, sm, st>>>(in, tw, out, a);
    return cudaGetLastError();
}

template <class A, typename R, int LOGL>
cudaError_t launch_adj_last(const typename A::S *in, const R *D1, const R *D2, const R *D3, const typename A::S *tw,
                            typename Cplx<R>::T *c, const FusedArgs &a, cudaStream_t st) {
    const size_t sm = line_smem<A>(1 << LOGL);
    cudaError_t e = cudaFuncSetAttribute(adj_last_kernel<A, R, LOGL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm);
    if (e != cudaSuccess) return e;
    const int64_t rows = (int64_t)a.N1 * a.N2, lpb = A::kElems >> LOGL;
    adj_last_kernel<A, R, LOGL><<<(unsigned)((rows + lpb - 1) / lpb), A::kThreads, sm, st>>>(in, D1, D2, D3, tw,
                                                                                              c, a);
    return cudaGetLastError();
}

template <class A, typename R>
cudaError_t run_adjoint(const typename Cplx<R>::T *H, const R *D1, const R *D2, const R *D3, const void *const tw[3],
                        void *scratch, typename Cplx<R>::T *c, const FusedArgs &a, cudaStream_t st) {
    using S = typename A::S;
    S *Abuf = (S *)scratch;                                   // N1 n2 n3
    S *Bbuf = Abuf + (int64_t)a.N1 * a.n2 * a.n3;             // N1 N2 n3
    cudaError_t e;
    {
#define GBNFFT_CALL(L) launch_adj_first<A, R, L>(H, (const S *)tw[0], Abuf, a, st)
        e = [&]() -> cudaError_t { GBNFFT_LOGL_SWITCH(a.logn1, GBNFFT_CALL) }();
#undef GBNFFT_CALL
    }
    if (e != cudaSuccess) return e;
    {
#define GBNFFT_CALL(L) launch_adj_mid<A, L>(Abuf, (const S *)tw[1], Bbuf, a, st)
        e = [&]() -> cudaError_t { GBNFFT_LOGL_SWITCH(a.logn2, GBNFFT_CALL) }();
#undef GBNFFT_CALL
    }
    if (e != cudaSuccess) return e;
#define GBNFFT_CALL(L) launch_adj_last<A, R, L>(Bbuf, D1, D2, D3, (const S *)tw[2], c, a, st)
    GBNFFT_LOGL_SWITCH(a.logn3, GBNFFT_CALL)
#undef GBNFFT_CALL
}

FusedArgs make_args(const int N[3], const int n[3], int m, int shift, int ng, const int *vexp) {
    FusedArgs a;
    a.vexp = vexp;
    a.N1 = N[0];
    a.N2 = N[1];
    a.N3 = N[2];
    a.n1 = n[0];
    a.n2 = n[1];
    a.n3 = n[2];
    a.logn1 = ilog2(n[0]);
    a.logn2 = ilog2(n[1]);
    a.logn3 = ilog2(n[2]);
    a.m = m;
    a.shift = shift;
    a.ng = ng;
    a.divN2 = make_fastdiv((unsigned)N[1]);
    a.divN3 = make_fastdiv((unsigned)N[2]);
    return a;
}

}  // namespace

template <typename R>
cudaError_t launch_fused_adjoint(const typename Cplx<R>::T *H, const int N[3], const int n[3], const R *D1,
                                 const R *D2, const R *D3, const void *const tw[3], void *scratch,
                                 typename Cplx<R>::T *c, const int *vexp, cudaStream_t st) {
    const FusedArgs a = make_args(N, n, 0, 0, 1, vexp);
    if constexpr (sizeof(R) == 8)
        return run_adjoint<ArithDF, R>(H, D1, D2, D3, tw, scratch, c, a, st);
    else
        return run_adjoint<ArithF32, R>(H, D1, D2, D3, tw, scratch, c, a, st);
}

template cudaError_t launch_fused_adjoint<double>(const double2 *, const int[3], const int[3], const double *,
                                                  const double *, const double *, const void *const[3], void *,
                                                  double2 *, const int *, cudaStream_t);
template cudaError_t launch_fused_adjoint<float>(const float2 *, const int[3], const int[3], const float *,
                                                 const float *, const float *, const void *const[3], void *,
                                                 float2 *, const int *, cudaStream_t);

bool fused_supported(const int n[3]) {
    for (int d = 0; d < 3; ++d)
        if (n[d] < 16 || n[d] > 2048 || (n[d] & (n[d] - 1))) return false;
    return true;
}

size_t fused_scratch_bytes(const int N[3], const int n[3], int ng, int prec) {
    const size_t elem = prec == 64 ? 16 : 8;
    return elem * (size_t)ng * ((size_t)N[0] * N[1] * n[2] + (size_t)N[0] * n[1] * n[2]);
}

template <typename R>
cudaError_t launch_fused_series(const typename Cplx<R>::T *c, const int N[3], const int n[3], const R *D1,
                                const R *D2, const R *D3, const void *const tw[3], void *scratch,
                                void *P, int m, int shift, int ng, const int *vexp, cudaStream_t st) {
    const FusedArgs a = make_args(N, n, m, shift, ng, vexp);
    if constexpr (sizeof(R) == 8)
        return run_fused<ArithDF, R>(c, D1, D2, D3, tw, scratch, P, a, st);
    else
        return run_fused<ArithF32Fwd, R>(c, D1, D2, D3, tw, scratch, P, a, st);
}

template cudaError_t launch_fused_series<double>(const double2 *, const int[3], const int[3],
                                                 const double *, const double *, const double *,
                                                 const void *const[3], void *, void *, int, int, int,
                                                 const int *, cudaStream_t);
template cudaError_t launch_fused_series<float>(const float2 *, const int[3], const int[3], const float *,
                                                const float *, const float *, const void *const[3],
                                                void *, void *, int, int, int, const int *, cudaStream_t);

}  // namespace gbnfft
