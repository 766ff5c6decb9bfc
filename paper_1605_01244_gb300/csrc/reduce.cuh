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

// nd = (double)n and alpha = m + 1/2 are passed in (hoisted by the caller);
// the finiteness and range tests work on the bits, so the FP64 pipe (the
// bound of this kernel on GB300) only does the arithmetic of the reduction.
__device__ __forceinline__ Reduced reduce_coord(double x, int n, double nd, double alpha, int *status) {
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
    const double u = __dmul_rn(nd, __dadd_rn(xw, 0.5));
    const double v = __dsub_rn(u, alpha);
    const double l0 = ceil(v);
    Reduced r;
    r.s = __dsub_rn(l0, v);
    // s >= 1 cannot happen for finite v; the bit test keeps s in [0, 1) regardless
    if (__double_as_longlong(r.s) >= 0x3FF0000000000000ll) r.s = 0.0;
    // xw lies in [-1/2, 1/2], so u in [0, n] and l0 in [-m, n - m]: one
    // add wraps it unless n < m (small grids loop a few times)
    int li = int_of_integral(l0);
    while (li < 0) li += n;
    while (li >= n) li -= n;
    r.l0 = li;
    return r;
}

}  // namespace
}  // namespace gbnfft
