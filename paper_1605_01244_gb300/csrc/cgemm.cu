// Complex matrix products for the rectilinear-grid evaluation (grid_eval.cu):
//     C[b] = A[b] B[b],   A (M x K), B (K x N), C (M x N), b < batch,
// element (r, c) of a row-major X at X[r ldx + c]; with TRANSB, B(k, n) is
// read at B[n ldb + k].  Three arithmetic variants:
//   * FP32 (mixed family): complex float, FP32 FMAs;
//   * FP64 (FP64 family, default): complex double, FP64 FMAs;
//   * double-float (FP64 family, option): complex double in and out, each
//     value split into a float pair when a tile is staged, products and sums
//     in double-float on the FP32 pipe (GB300's FP64 pipe is 64x slower),
//     about 48 significant bits as in the NFFT's FP64 family -- faster, but
//     ~30x the FP64 rounding error.
// Tiling: a block computes a BM x BN tile of C from K-slices of BK staged in
// shared memory; thread (tx, ty) of a 16 x 16 block owns the 4 x 4 outputs
// (ty + 16 i, tx + 16 j).  Range: with vexp given, A is scaled by 2^s on
// load (s from the range word, see internal.cuh) or C is scaled by 2^-s on
// store, so that the double-float products stay within FP32's exponents.
#include "col_common.cuh"

namespace gbnfft {
namespace {

constexpr int kBM = 64, kBN = 64, kTM = 4, kTN = 4, kThreads = 256;

struct F32 {
    using In = float2;
    using S = float2;       // staged value
    static constexpr int BK = 16;
    struct Acc {
        float re, im;
    };
    static __device__ __forceinline__ S stage(In v, int) { return v; }
    static __device__ __forceinline__ S zero() { return make_float2(0.f, 0.f); }
    static __device__ __forceinline__ void init(Acc &a) { a.re = a.im = 0.f; }
    static __device__ __forceinline__ void mac(Acc &c, S a, S b) {
        c.re = fmaf(a.x, b.x, fmaf(-a.y, b.y, c.re));
        c.im = fmaf(a.x, b.y, fmaf(a.y, b.x, c.im));
    }
    static __device__ __forceinline__ In out(const Acc &c, int) { return make_float2(c.re, c.im); }
};

struct F64 {
    using In = double2;
    using S = double2;
    static constexpr int BK = 8;
    struct Acc {
        double re, im;
    };
    static __device__ __forceinline__ S stage(In v, int shift) { return scale_value(v, shift); }
    static __device__ __forceinline__ S zero() { return make_double2(0.0, 0.0); }
    static __device__ __forceinline__ void init(Acc &a) { a.re = a.im = 0.0; }
    static __device__ __forceinline__ void mac(Acc &c, S a, S b) {
        c.re = fma(a.x, b.x, fma(-a.y, b.y, c.re));
        c.im = fma(a.x, b.y, fma(a.y, b.x, c.im));
    }
    static __device__ __forceinline__ In out(const Acc &c, int shift) {
        return scale_value(make_double2(c.re, c.im), shift);
    }
};

struct DF {
    using In = double2;
    using S = float4;       // (re_hi, re_lo, im_hi, im_lo)
    static constexpr int BK = 8;
    struct Acc {
        float rh, rl, ih, il;
    };
    static __device__ __forceinline__ S stage(In v, int shift) {
        v = scale_value(v, shift);
        S o;
        split_df(v.x, o.x, o.y);
        split_df(v.y, o.z, o.w);
        return o;
    }
    static __device__ __forceinline__ S zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
    static __device__ __forceinline__ void init(Acc &a) { a.rh = a.rl = a.ih = a.il = 0.f; }
    static __device__ __forceinline__ void mac(Acc &c, S a, S b) {
        df_mac(c.rh, c.rl, a.x, a.y, b.x, b.y);
        df_mac(c.rh, c.rl, -a.z, -a.w, b.z, b.w);
        df_mac(c.ih, c.il, a.x, a.y, b.z, b.w);
        df_mac(c.ih, c.il, a.z, a.w, b.x, b.y);
    }
    static __device__ __forceinline__ In out(const Acc &c, int shift) {
        return scale_value(make_double2((double)c.rh + (double)c.rl, (double)c.ih + (double)c.il), shift);
    }
};

template <class Ar, bool TRANSB>
__global__ void __launch_bounds__(kThreads) cgemm_kernel(const typename Ar::In *__restrict__ A, int64_t lda,
                                                          int64_t sA, const typename Ar::In *__restrict__ B,
                                                          int64_t ldb, int64_t sB, typename Ar::In *__restrict__ C,
                                                          int64_t ldc, int64_t sC, int M, int N, int K,
                                                          const int *__restrict__ vexp, int scale_a, int scale_c) {
    using S = typename Ar::S;
    constexpr int BK = Ar::BK;
    __shared__ S As[BK][kBM];
    __shared__ S Bs[BK][kBN];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
    const int64_t b = blockIdx.z;
    A += b * sA;
    B += b * sB;
    C += b * sC;
    const int vs = value_shift(vexp);
    const int sa = scale_a ? vs : 0, sc = scale_c ? -vs : 0;
    typename Ar::Acc acc[kTM][kTN];
#pragma unroll
    for (int i = 0; i < kTM; ++i)
#pragma unroll
        for (int j = 0; j < kTN; ++j) Ar::init(acc[i][j]);
    for (int k0 = 0; k0 < K; k0 += BK) {
        // stage A (BM x BK, k fastest in memory) and B (BK x BN)
        for (int e = tid; e < kBM * BK; e += kThreads) {
            const int mm = e / BK, kk = e - mm * BK;
            const int m = m0 + mm, k = k0 + kk;
            As[kk][mm] = (m < M && k < K) ? Ar::stage(A[(int64_t)m * lda + k], sa) : Ar::zero();
        }
        for (int e = tid; e < kBN * BK; e += kThreads) {
            int kk, nn;
            if (TRANSB) {
                nn = e / BK;
                kk = e - nn * BK;
            } else {
                kk = e / kBN;
                nn = e - kk * kBN;
            }
            const int n = n0 + nn, k = k0 + kk;
            const int64_t off = TRANSB ? (int64_t)n * ldb + k : (int64_t)k * ldb + n;
            Bs[kk][nn] = (n < N && k < K) ? Ar::stage(B[off], 0) : Ar::zero();
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            S a[kTM], bv[kTN];
#pragma unroll
            for (int i = 0; i < kTM; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < kTN; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < kTM; ++i)
#pragma unroll
                for (int j = 0; j < kTN; ++j) Ar::mac(acc[i][j], a[i], bv[j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < kTM; ++i) {
        const int m = m0 + ty + 16 * i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < kTN; ++j) {
            const int n = n0 + tx + 16 * j;
            if (n < N) C[(int64_t)m * ldc + n] = Ar::out(acc[i][j], sc);
        }
    }
}

template <class Ar>
cudaError_t run(const void *A, int64_t lda, int64_t sA, const void *B, int64_t ldb, int64_t sB, bool transb,
                void *C, int64_t ldc, int64_t sC, int M, int N, int K, int batch, const int *vexp, int scale_a,
                int scale_c, cudaStream_t st) {
    if (M <= 0 || N <= 0 || batch <= 0) return cudaSuccess;
    using In = typename Ar::In;
    const dim3 grid((N + kBN - 1) / kBN, (M + kBM - 1) / kBM, batch);
    if (grid.y > 65535 || grid.z > 65535) return cudaErrorInvalidValue;
    if (transb)
        cgemm_kernel<Ar, true><<<grid, kThreads, 0, st>>>((const In *)A, lda, sA, (const In *)B, ldb, sB, (In *)C,
                                                          ldc, sC, M, N, K, vexp, scale_a, scale_c);
    else
        cgemm_kernel<Ar, false><<<grid, kThreads, 0, st>>>((const In *)A, lda, sA, (const In *)B, ldb, sB,
                                                           (In *)C, ldc, sC, M, N, K, vexp, scale_a, scale_c);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_cgemm(int arith, const void *A, int64_t lda, int64_t sA, const void *B, int64_t ldb, int64_t sB,
                         bool transb, void *C, int64_t ldc, int64_t sC, int M, int N, int K, int batch,
                         const int *vexp, int scale_a, int scale_c, cudaStream_t st) {
    if (arith == kGemmDF)
        return run<DF>(A, lda, sA, B, ldb, sB, transb, C, ldc, sC, M, N, K, batch, vexp, scale_a, scale_c, st);
    if (arith == kGemmF64)
        return run<F64>(A, lda, sA, B, ldb, sB, transb, C, ldc, sC, M, N, K, batch, nullptr, 0, 0, st);
    return run<F32>(A, lda, sA, B, ldb, sB, transb, C, ldc, sC, M, N, K, batch, nullptr, 0, 0, st);
}

}  // namespace gbnfft
