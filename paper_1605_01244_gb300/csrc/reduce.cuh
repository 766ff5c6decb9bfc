// FP64 reduction of a coordinate to its stencil origin and offset, shared by
// set_points (points.cu) and the one- and two-dimensional NFFT (nfft_low.cu).
#pragma once
#include "internal.cuh"

namespace gbnfft {
namespace {

// Reduction of one coordinate (FP64):
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

// Round-to-nearest-even of a magnitude 0 < a < 2^63 to 53 significant bits
// (the rounding of an FP64 result whose exact value is the integer a times a
// power of two).
__device__ __forceinline__ unsigned long long round53(unsigned long long a) {
    const int p = 63 - __clzll((long long)a);
    if (p <= 52) return a;
    const int d = p - 52;
    const unsigned long long q = a >> d, rem = a & ((1ull << d) - 1), half = 1ull << (d - 1);
    return (q + ((rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull)) << d;
}

// The double S 2^-F for 0 <= S < 2^63 holding at most 53 significant bits.
__device__ __forceinline__ double fixed_to_double(unsigned long long S, int F) {
    if (S == 0) return 0.0;
    const int p = 63 - __clzll((long long)S);
    const unsigned long long mant = p <= 52 ? S << (52 - p) : S >> (p - 52);
    return __longlong_as_double((long long)(((unsigned long long)(p - F + 1023) << 52) |
                                            (mant & 0xFFFFFFFFFFFFFull)));
}

// The steps after t = x_w + 1/2 for n = 2^L, on the integer pipe.  With
// F = 62 - L, every quantity is an integer in units of 2^-F grid cells:
// u = n t is U = t 2^62 (exact for t >= 2^-10, whose 53-bit significand
// then sits at or above bit 0), alpha is (2m + 1) 2^(F - 1), and the two
// FP64 subtractions u - alpha and l0 - v are the exact integer differences
// rounded to 53 significant bits (ties to even), i.e. the same doubles as the
// FP64 sequence; ceil is a shift.  Returns false (nothing written) for
// t < 2^-10, which takes the FP64 sequence.
__device__ __forceinline__ bool reduce_fixed(double t, int L, int width, long long &l0, double &s) {
    const unsigned long long tb = (unsigned long long)__double_as_longlong(t);   // 0 <= t <= 1
    const int Et = (int)(tb >> 52);
    if (Et < 1013) return false;
    const int F = 62 - L;
    const long long U = (long long)(((tb & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << (Et - 1013));
    long long V = U - ((long long)width << (F - 1));   // |V| < 2^62
    if (V > 0) V = (long long)round53((unsigned long long)V);
    else if (V < 0) V = -(long long)round53((unsigned long long)(-V));
    l0 = (V + ((1ll << F) - 1)) >> F;                               // ceil(v), arithmetic shift
    const unsigned long long S = (unsigned long long)(l0 * (1ll << F) - V);   // (l0 - v) 2^F in [0, 2^F)
    s = fixed_to_double(S == 0 ? 0ull : round53(S), F);
    return true;
}

// nd = (double)n and alpha = m + 1/2 (width = 2m + 1) are passed in (hoisted
// by the caller); log2n = log2(n) when n is a power of two, else -1.  The
// finiteness and range tests work on the bits; for n = 2^L only x_w + 1/2
// runs on the FP64 pipe (the bound of this kernel on GB300), for other n the
// whole sequence does.
__device__ __forceinline__ Reduced reduce_coord(double x, int n, double nd, double alpha, int log2n, int width,
                                                int *status) {
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
    const double xw = in_range ? x : __dsub_rn(x, floor(__dadd_rn(x, 0.5)));
    const double t = __dadd_rn(xw, 0.5);
    Reduced r;
    long long l0i;
    if (!(log2n >= 0 && reduce_fixed(t, log2n, width, l0i, r.s))) {
        const double u = __dmul_rn(nd, t);
        const double v = __dsub_rn(u, alpha);
        const double l0 = ceil(v);
        r.s = __dsub_rn(l0, v);
        l0i = int_of_integral(l0);
    }
    // s >= 1 cannot happen for finite v; the bit test keeps s in [0, 1) regardless
    if (__double_as_longlong(r.s) >= 0x3FF0000000000000ll) r.s = 0.0;
    // xw lies in [-1/2, 1/2], so u in [0, n] and l0 in [-m, n - m]: one
    // add wraps it unless n < m (small grids loop a few times)
    int li = (int)l0i;
    while (li < 0) li += n;
    while (li >= n) li -= n;
    r.l0 = li;
    return r;
}

// log2(n) for a power of two 8 <= n <= 2^30 (the range in which the
// fixed-point integers of reduce_fixed stay below 2^63), else -1
__host__ __device__ __forceinline__ int log2_if_pow2(int n) {
    if (n < 8 || n > (1 << 30) || (n & (n - 1))) return -1;
    int L = 0;
    while ((1 << L) < n) ++L;
    return L;
}

}  // namespace
}  // namespace gbnfft
