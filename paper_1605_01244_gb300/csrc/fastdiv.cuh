// Exact unsigned division by a runtime divisor d >= 1 for 32-bit dividends,
// by multiply-high and shift (Granlund-Montgomery):
//     q = (umulhi(M, x) + x) >> s,  s = ceil(log2 d),  M = floor(2^32 (2^s - d) / d) + 1.
// Used by the fused transform's index arithmetic; host-compilable so that a
// CPU test can check it against division.
#pragma once

namespace gbnfft {

struct FastDiv {
    unsigned M;
    int s;
    __host__ __device__ __forceinline__ unsigned div(unsigned x) const {
#ifdef __CUDA_ARCH__
        const unsigned hi = __umulhi(M, x);
#else
        const unsigned hi = (unsigned)(((unsigned long long)M * x) >> 32);
#endif
        return (unsigned)(((unsigned long long)hi + x) >> s);
    }
};

inline FastDiv make_fastdiv(unsigned d) {
    FastDiv f;
    f.s = 0;
    while ((1ull << f.s) < d) ++f.s;
    f.M = (unsigned)((((1ull << f.s) - d) << 32) / d + 1);
    return f;
}

}  // namespace gbnfft
