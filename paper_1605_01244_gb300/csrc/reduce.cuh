// Reduction of a coordinate to its stencil origin and offset, with the
// results of FP64 round-to-nearest arithmetic (mostly computed on the integer
// pipe for n = 2^L), shared by set_points (points.cu) and the one- and
// two-dimensional NFFT (nfft_low.cu).
#pragma once
#include <cstring>

#include "internal.cuh"

namespace gbnfft {
namespace {

// Reduction of one coordinate (each step rounded as in FP64):
//   xw = x - floor(x + 1/2)                 (wrap onto [-1/2, 1/2); the series is periodic)
//   u  = n (xw + 1/2)                       (grid units; grid node l sits at x = -1/2 + l/n)
//   v  = u - alpha, l0 = ceil(v), s = l0 - v in [0, 1)
// The stencil l0 + {0..2m} holds exactly the nodes l with -alpha < u - l <= alpha.
// l0 is returned wrapped into [0, n).  Non-finite x is replaced by 0 and flagged.
struct Reduced {
    int l0;
    double s;
};

// The value of an integral double v with |v| < 2^31, from its bits (no FP64
// conversion instruction).
__device__ __forceinline__ int int_of_integral(double v) {
    const long long b = __double_as_longlong(v);
    const int e = (int)((b >> 52) & 0x7ff) - 1023;   // |v| = 1.f * 2^e, or v = +-0
    if (e < 0) return 0;
    const unsigned long long mant = ((unsigned long long)b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int mag = (int)(mant >> (52 - (e < 30 ? e : 30)));
    return b < 0 ? -mag : mag;
}

// Offset s in [0, 1) as the family's real type: FP64 unchanged; FP32 by
// truncating the significand from the bits (at most one unit in the last
// place below round-to-nearest, no FP64 conversion instruction).
template <typename R> __device__ __forceinline__ R offset_as(double s);
template <> __device__ __forceinline__ double offset_as<double>(double s) { return s; }
template <> __device__ __forceinline__ float offset_as<float>(double s) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(s);
    const int e = (int)(b >> 52) - 1023;   // s >= 0
    if (e < -126) return 0.f;
    return __int_as_float(((e + 127) << 23) | (int)((b >> 29) & 0x7FFFFF));
}

// Bit casts and count-leading-zeros for the integer path below, which is also
// compiled for the host by a CPU test of its exactness (same arithmetic).
__host__ __device__ __forceinline__ long long bits_of(double v) {
#ifdef __CUDA_ARCH__
    return __double_as_longlong(v);
#else
    long long b;
    std::memcpy(&b, &v, sizeof b);
    return b;
#endif
}
__host__ __device__ __forceinline__ double double_of(long long b) {
#ifdef __CUDA_ARCH__
    return __longlong_as_double(b);
#else
    double v;
    std::memcpy(&v, &b, sizeof v);
    return v;
#endif
}
__host__ __device__ __forceinline__ int clz64(long long v) {
#ifdef __CUDA_ARCH__
    return __clzll(v);
#else
    return v == 0 ? 64 : __builtin_clzll((unsigned long long)v);
#endif
}

// Per-dimension constants of the reduction (hoisted out of the point loops).
// For n = 2^L the steps after t = x_w + 1/2 can run on fixed-point integers in
// units of 2^-F grid cells, F = 62 - L: u = n t is U = t 2^62 (exact for
// t >= 2^-10, whose 53-bit significand then sits at or above bit 0) and
// alpha is A = (2m + 1) 2^(F - 1).  F = 0 marks n without that path.
struct CoordParams {
    int n;
    double nd, alpha;
    int F;
    int Et_min;                  // smallest biased exponent of t the path takes
    long long A, A_half, mask;   // A, A / 2, 2^F - 1
};

__host__ __device__ __forceinline__ CoordParams coord_params(int n, int m) {
    CoordParams c;
    c.n = n;
    c.nd = (double)n;
    c.alpha = (double)m + 0.5;
    c.F = 0;
    c.Et_min = 0;
    c.A = c.A_half = c.mask = 0;
    // 8 <= n <= 2^30 keeps A = (2m + 1) 2^(61 - L) below 2^63
    if (n >= 8 && n <= (1 << 30) && (n & (n - 1)) == 0) {
        int L = 0;
        while ((1 << L) < n) ++L;
        c.F = 62 - L;
        // t >= 2^(Et_min - 1023): U is a multiple of 2^(Et - 1013) and so are
        // V and the offset S < 2^F, which then has at most 53 significant
        // bits when Et - 1013 >= F - 53
        c.Et_min = 1013 + (c.F > 53 ? c.F - 53 : 0);
        c.A = (long long)(2 * m + 1) << (c.F - 1);
        c.A_half = c.A >> 1;
        c.mask = (1ll << c.F) - 1;
    }
    return c;
}

// The double S 2^-F for 0 <= S < 2^63 holding at most 53 significant bits.
__host__ __device__ __forceinline__ double fixed_to_double(unsigned long long S, int F) {
    if (S == 0) return 0.0;
    const int p = 63 - clz64((long long)S);
    const unsigned long long mant = p <= 52 ? S << (52 - p) : S >> (p - 52);
    return double_of((long long)(((unsigned long long)(p - F + 1023) << 52) | (mant & 0xFFFFFFFFFFFFFull)));
}

// The fixed-point path for u >= alpha / 2 (all but a sliver next to
// x = -1/2).  There V = U - A is a multiple of U's lowest significand bit
// with |V| <= U, so it has at most 53 significant bits: the FP64 difference
// u - alpha is exactly v = V 2^-F.  Then l0 = ceil(v) is a shift, and
// l0 - v is S = (-V) mod 2^F, exact too (CoordParams::Et_min).  Returns false
// (nothing written) for t below that bound or u < alpha / 2, which take the
// FP64 sequence.
__host__ __device__ __forceinline__ bool reduce_fixed(double t, const CoordParams &c, long long &l0, double &s) {
    const unsigned long long tb = (unsigned long long)bits_of(t);   // 0 <= t <= 1
    const int Et = (int)(tb >> 52);
    if (Et < c.Et_min) return false;
    const long long U = (long long)(((tb & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << (Et - 1013));
    if (U < c.A_half) return false;
    const long long V = U - c.A;
    l0 = (V + c.mask) >> c.F;                                                  // ceil(v), arithmetic shift
    s = fixed_to_double((unsigned long long)(-V) & (unsigned long long)c.mask, c.F);
    return true;
}

// The rare paths of reduce_coord, kept out of line: inlined, the compiler
// turns them into predicated FP64 instructions that every lane issues.
// Wrap of |x| >= 1/2 onto [-1/2, 1/2].
__device__ __noinline__ double wrap_coord(double x) { return __dsub_rn(x, floor(__dadd_rn(x, 0.5))); }

// i mod n in [0, n) for any int i (grids smaller than the stencil).
__device__ __noinline__ int wrap_index(int i, int n) {
    const int r = i % n;
    return r < 0 ? r + n : r;
}

// The FP64 sequence after t = x_w + 1/2 (any n): l0 (not yet wrapped) and s.
__device__ __noinline__ Reduced reduce_fp64(double t, double nd, double alpha) {
    const double u = __dmul_rn(nd, t);
    const double v = __dsub_rn(u, alpha);
    const double l0 = ceil(v);
    Reduced r;
    r.s = __dsub_rn(l0, v);
    r.l0 = int_of_integral(l0);
    return r;
}

// The finiteness and range tests work on the bits; x_w + 1/2 is the one
// step always on the FP64 pipe (the bound of this kernel on GB300), the rest
// runs on integers where CoordParams allows it.
__device__ __forceinline__ Reduced reduce_coord(double x, const CoordParams &c, int *status) {
    unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    if ((bits & 0x7FF0000000000000ull) == 0x7FF0000000000000ull) {
        atomicOr(status, 1);
        x = 0.0;
        bits = 0;
    }
    // explicit round-to-nearest steps: no contraction into FMAs, so that the
    // stencil choice at exact half-integer u is reproducible.  Coordinates
    // already in [-1/2, 1/2) (|x| < 1/2, or x = -1/2) skip the wrap, whose
    // result they equal.
    const unsigned long long mag = bits & 0x7FFFFFFFFFFFFFFFull;
    const bool in_range = mag < 0x3FE0000000000000ull || bits == 0xBFE0000000000000ull;
    const double xw = in_range ? x : wrap_coord(x);
    const double t = __dadd_rn(xw, 0.5);
    Reduced r;
    long long l0i;
    if (!(c.F > 0 && reduce_fixed(t, c, l0i, r.s))) {
        r = reduce_fp64(t, c.nd, c.alpha);
        l0i = r.l0;
    }
    // s >= 1 cannot happen for finite v; the bit test keeps s in [0, 1) regardless
    if (__double_as_longlong(r.s) >= 0x3FF0000000000000ll) r.s = 0.0;
    // xw lies in [-1/2, 1/2], so u in [0, n] and l0 in [-m, n - m]: one
    // add wraps it unless n < m
    int li = (int)l0i;
    li += li < 0 ? c.n : 0;
    if ((unsigned)li >= (unsigned)c.n) li = wrap_index(li, c.n);
    r.l0 = li;
    return r;
}

}  // namespace
}  // namespace gbnfft
