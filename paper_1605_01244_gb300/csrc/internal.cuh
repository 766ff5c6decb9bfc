// Internal declarations shared by the gbnfft translation units.
#pragma once

#include <cuda_runtime.h>
#include <cufft.h>
#include <stdint.h>

#include "gbnfft.h"

namespace gbnfft {

constexpr int kMaxM = 8;       // largest window cutoff compiled in (2m+1 = 17 taps)
constexpr int kTile = 8;       // grid tile edge (cells) used to bucket points

template <typename R> struct Cplx;
template <> struct Cplx<double> { using T = double2; };
template <> struct Cplx<float> { using T = float2; };

// Window weights.  The window is the Kaiser-Bessel function in grid units
// with half-width alpha = m + 1/2,
//   phi(tau) = sinh(b sqrt(alpha^2 - tau^2)) / (pi sqrt(alpha^2 - tau^2)),
// on the support -alpha < tau <= alpha, normalised to phi(0) = 1 (the
// normalisation is folded into the deconvolution tables).  A point with
// offset s in [0,1) has taps tau_a = alpha - s - a, a = 0..2m; each tap's
// weight w_a(s) is an entire function of s and is evaluated as a polynomial
// in t = 2s - 1 of degree kPolyDeg<R> (Horner), with coefficients fitted on
// the host at plan creation (Chebyshev interpolation in long double).
template <typename R> struct PolyDeg;
template <> struct PolyDeg<double> { static constexpr int value = 16; };
template <> struct PolyDeg<float> { static constexpr int value = 10; };

constexpr int kMaxTaps = 2 * kMaxM + 1;
constexpr int kMaxCoef = 17;   // >= PolyDeg<R>::value + 1

// Host-side coefficient table of a plan: coef[d][a][k], k = power of t.
template <typename R> struct WinTable {
    R coef[3][kMaxTaps][kMaxCoef];
};

// Kernel-parameter copy sized for one m (lives in the constant bank).
template <typename R, int MM> struct Poly {
    static constexpr int W = 2 * MM + 1;
    static constexpr int D = PolyDeg<R>::value;
    R c[3][W][D + 1];
};

template <typename R, int MM> Poly<R, MM> make_poly(const WinTable<R> &t) {
    Poly<R, MM> p;
    for (int d = 0; d < 3; ++d)
        for (int a = 0; a < Poly<R, MM>::W; ++a)
            for (int k = 0; k <= Poly<R, MM>::D; ++k) p.c[d][a][k] = t.coef[d][a][k];
    return p;
}

// Sorted point data written by set_points.
//   key[j] = (l0_1, l0_2, l0_3, original index); l0_d in [0, n_d) is the
//   first stencil node (wrapped), the stencil is l0_d + {0..2m} mod n_d.
//   s_d[j] in [0,1): tau of tap a is alpha - s_d - a.
//   vexp: FP64 family only (nullptr otherwise): device word holding the
//   exponent rank (value_rank) of the largest input magnitude of the call;
//   the inputs entered the arithmetic scaled by 2^value_shift(vexp) and the
//   results leave scaled back (see the range scaling below).
template <typename R> struct PointsView {
    const int4 *key;
    const R *s1, *s2, *s3;
    int64_t M;
    const int *vexp;
};

struct Grid3 {
    int n1, n2, n3;
};

// Double-float window polynomials for the FP64 family's FP32-pipe gather:
// each coefficient is hi + lo (two floats), degree kPolyDegDF in t.
constexpr int kPolyDegDF = 16;
struct WinTableDF {
    float ch[3][kMaxTaps][kMaxCoef];
    float cl[3][kMaxTaps][kMaxCoef];
};
template <int MM> struct PolyDF {
    static constexpr int W = 2 * MM + 1;
    float ch[3][W][kPolyDegDF + 1];
    float cl[3][W][kPolyDegDF + 1];
};
template <int MM> PolyDF<MM> make_poly_df(const WinTableDF &t) {
    PolyDF<MM> p;
    for (int d = 0; d < 3; ++d)
        for (int a = 0; a < PolyDF<MM>::W; ++a)
            for (int k = 0; k <= kPolyDegDF; ++k) {
                p.ch[d][a][k] = t.ch[d][a][k];
                p.cl[d][a][k] = t.cl[d][a][k];
            }
    return p;
}

// Half-interval window tables of the FP64 family's value gather.  The window
// is even, so tap 2m - a at offset s weighs what tap a weighs at 1 - s:
// w_{2m-a}(s) = w_a(1 - s).  A table of each tap on s in [1/2, 1] alone, as a
// polynomial in u = 4s - 3, therefore serves every s: tap a at s >= 1/2 is row
// a at u = 4s - 3, at s < 1/2 it is row 2m - a at u = 1 - 4s.  On the shorter
// interval degree kPolyDegHalf reaches the accuracy that degree 16 gives on
// the whole interval for m >= 4 (Chebyshev interpolation of the entire
// window function; below m = 4 it falls short and the whole-interval table
// serves).
constexpr int kPolyDegHalf = 11;
struct HalfTables {
    WinTable<double> w64;   // FP64 coefficients, degree kPolyDegHalf in u
    WinTableDF wdf;         // the same as float pairs (hi + lo)
    int mode;               // 0: whole-interval FP64 table, 1: half table in FP64, 2: half table in double-float
};
template <typename R, int MM, int DD> struct PolyN {
    static constexpr int W = 2 * MM + 1, D = DD;
    R c[3][W][DD + 1];
};
template <typename R, int MM, int DD> PolyN<R, MM, DD> make_poly_n(const WinTable<R> &t) {
    PolyN<R, MM, DD> p;
    for (int d = 0; d < 3; ++d)
        for (int a = 0; a < PolyN<R, MM, DD>::W; ++a)
            for (int k = 0; k <= DD; ++k) p.c[d][a][k] = t.coef[d][a][k];
    return p;
}
template <int MM, int DD> struct PolyDFN {
    static constexpr int W = 2 * MM + 1, D = DD;
    float ch[3][W][DD + 1];
    float cl[3][W][DD + 1];
};
template <int MM, int DD> PolyDFN<MM, DD> make_poly_dfn(const WinTableDF &t) {
    PolyDFN<MM, DD> p;
    for (int d = 0; d < 3; ++d)
        for (int a = 0; a < PolyDFN<MM, DD>::W; ++a)
            for (int k = 0; k <= DD; ++k) {
                p.ch[d][a][k] = t.ch[d][a][k];
                p.cl[d][a][k] = t.cl[d][a][k];
            }
    return p;
}

// ---- range scaling of the FP64 family ---------------------------------------
// The FP64 family computes its window sums, transform and adjoint spread in
// double-float (float pairs), whose exponent range is FP32's.  So that any
// finite FP64 input is served, each call first finds the largest magnitude
// among its input values (the coefficients c of eval / eval_grad /
// precompute, the values f of adjoint) and scales every input by the exact
// power of two 2^s that brings that magnitude into [1, 2); the results are
// scaled back by 2^-s when they are written as FP64.  Scaling by a power of
// two is exact, so an input already of order one gives the same bits as
// without it.  After scaling, entries below 2^-100 of the largest are
// dropped by split_df (their share of any result is below 2^-100 of the
// result's scale), and no double-float intermediate comes near FP32's
// overflow: for every plan the library accepts (N_d <= 4096, sigma >= 1.25,
// m <= 8) the grid values are bounded by sum_k |c_k D(k)| 2 pi |k| < 2^64
// and the window sums by 2^76.
//
// value_rank(bits of |v|) = floor(log2 |v|) + 1100 for finite nonzero v
// (subnormals included), 0 for zero and kRankNonFinite for inf / NaN.
constexpr int kRankNonFinite = 4000;
__device__ __forceinline__ int value_rank(unsigned long long b) {
    b &= 0x7FFFFFFFFFFFFFFFull;
    const int e = (int)(b >> 52);
    if (e == 0x7ff) return kRankNonFinite;
    if (e > 0) return e + 77;                         // (e - 1023) + 1100
    const unsigned long long mant = b & 0xFFFFFFFFFFFFFull;
    return mant ? 89 - __clzll((long long)mant) : 0;  // (63 - clz) - 1074 + 1100
}
// the shift s of a call from its stored rank (0 when all inputs are zero or
// one is not finite: those pass through unscaled)
__device__ __forceinline__ int value_shift(const int *vexp) {
    if (!vexp) return 0;
    const int r = *vexp;
    return (r == 0 || r >= kRankNonFinite) ? 0 : 1100 - r;
}
__device__ __forceinline__ double2 scale_value(double2 v, int s) {
    return s ? make_double2(scalbn(v.x, s), scalbn(v.y, s)) : v;
}
__device__ __forceinline__ float2 scale_value(float2 v, int) { return v; }

// Split an FP64 value into floats hi + lo without FP64 arithmetic: hi keeps
// the leading 24 significant bits (exact truncation), lo is the remaining 29
// bits rounded to a float, so hi + lo carries ~48 bits.  Values below 2^-100
// in magnitude are flushed to zero; callers pass values scaled as above, so
// the largest is of order one and nothing reaches FP32's overflow.
__device__ __forceinline__ void split_df(double v, float &hi, float &lo) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const unsigned int sign = (unsigned int)(b >> 63) << 31;
    const int e = (int)((b >> 52) & 0x7ff);
    if (e < 1023 - 100) {
        hi = __int_as_float(sign);
        lo = hi;
        return;
    }
    const unsigned long long mant = b & 0xFFFFFFFFFFFFFull;
    hi = __int_as_float((int)(sign | ((unsigned int)(e - 1023 + 127) << 23) | (unsigned int)(mant >> 29)));
    const int low = (int)(mant & 0x1FFFFFFFull);
    // low * 2^(e - 1023 - 52), with the sign of v
    const float lf = ldexpf(__int2float_rn(low), e - 1075);
    lo = sign ? -lf : lf;
}

// ---- window-derivative gradient gathers (gather_wd.cu) --------------------------
// f and grad[3j + d] from one padded grid (origin layout): the window sum with
// phi replaced by n_d phi' in dimension d.  n: oversampled sizes.
cudaError_t launch_gather_wd_df(const float4 *G, Grid3 pg, int m, PointsView<double> pts,
                                const WinTable<double> &w, const int n[3], double2 *f, double2 *grad,
                                cudaStream_t st);
cudaError_t launch_gather_wd_f32(const float2 *G, Grid3 pg, int m, PointsView<float> pts,
                                 const WinTable<float> &w, const int n[3], float2 *f, float2 *grad,
                                 cudaStream_t st);

// ---- fused forward transform (fft_fused.cu) -----------------------------------
// Deconvolve + inverse DFT of the oversampled grid + ghost-padded output
// P[q][p] = g_q[(p - shift) mod n] for ng grids (q > 0: 2 pi i k_q c_k D), in
// double-float (R = double) or FP32.  tw[d]: table of exp(2 pi i j / n_d).
bool fused_supported(const int n[3]);
size_t fused_scratch_bytes(const int N[3], const int n[3], int ng, int prec);
template <typename R>
cudaError_t launch_fused_series(const typename Cplx<R>::T *c, const int N[3], const int n[3], const R *D1,
                                const R *D2, const R *D3, const void *const tw[3], void *scratch,
                                void *P, int m, int shift, int ng, const int *vexp, cudaStream_t st);

// Adjoint direction of the same passes: c_out[k] = D1 D2 D3 sum_l H_l
// exp(-2 pi i k.l / n) for k in the band (FP64 family: double-float passes,
// output scaled by 2^-s; the scratch of fused_scratch_bytes(N, n, 1, prec)).
template <typename R>
cudaError_t launch_fused_adjoint(const typename Cplx<R>::T *H, const int N[3], const int n[3], const R *D1,
                                 const R *D2, const R *D3, const void *const tw[3], void *scratch,
                                 typename Cplx<R>::T *c, const int *vexp, cudaStream_t st);

// ---- range scaling (range.cu) -----------------------------------------------
// *rank = max(*rank, value_rank of each of the count doubles at v); the caller
// zeroes *rank first.
cudaError_t launch_value_rank(const double *v, int64_t count, int *rank, cudaStream_t st);
// gx[3 j + d] = Re(conj(G_j) grad[3 j + d]) for j < M (chain.cu).
template <typename R>
cudaError_t launch_chain_x(const R *G, const R *grad, double *gx, int64_t M, cudaStream_t st);

// ---- complex matrix products (cgemm.cu) -------------------------------------
// C[b] = A[b] B[b] for b < batch (strides sA, sB, sC elements), A (M x K),
// B (K x N) or, with transb, B(k, n) at B[n ldb + k]; row-major, complex
// (float2 for kGemmF32, double2 otherwise).  kGemmDF: A scaled by 2^s on load
// (scale_a) or C by 2^-s on store (scale_c), s = value_shift(vexp).
enum { kGemmF32 = 0, kGemmF64 = 1, kGemmDF = 2 };
cudaError_t launch_cgemm(int arith, const void *A, int64_t lda, int64_t sA, const void *B, int64_t ldb, int64_t sB,
                         bool transb, void *C, int64_t ldc, int64_t sC, int M, int N, int K, int batch,
                         const int *vexp, int scale_a, int scale_c, cudaStream_t st);

// ---- launchers implemented in gather_df.cu ---------------------------------
cudaError_t launch_grid_to_df(double2 *G, int64_t total, cudaStream_t st);
cudaError_t launch_gather_df(const float4 *G, Grid3 g, int m, PointsView<double> pts,
                             const WinTableDF &w, double2 *f, cudaStream_t st);
cudaError_t launch_gather_grad_df(const float4 *G4, Grid3 g, int m, PointsView<double> pts,
                                  const WinTableDF &w, double2 *f, double2 *grad, cudaStream_t st);

// ---- launchers implemented in gather_col.cu (ng = 1: value, 4: value+gradient)
// Padded copy P (dims pg = n + 2m) of ng grids: P[p] = g[(p - shift) mod n]
// (shift 0: column kernels; shift m: tile-staged kernel); the _df variant also
// splits FP64 values into double-float (re_hi, re_lo, im_hi, im_lo).
cudaError_t launch_pad_grid_f32(const float2 *G, Grid3 g, float2 *P, Grid3 pg, int ng, int shift,
                                cudaStream_t st);
cudaError_t launch_pad_grid_df(const double2 *G, Grid3 g, float4 *P, Grid3 pg, int ng, int shift,
                               cudaStream_t st);
// Column-parallel gathers over the padded grid (G = P, g = pg).
cudaError_t launch_gather_col_f32(const float2 *G, Grid3 g, int m, PointsView<float> pts,
                                  const WinTable<float> &w, float2 *f, float2 *grad, int ng,
                                  cudaStream_t st);
// half: the half-interval tables and their mode for the value gather (ng = 1;
// nullptr or mode 0: the whole-interval FP64 table)
cudaError_t launch_gather_col_df(const float4 *G, Grid3 g, int m, PointsView<double> pts,
                                 const WinTableDF &w, const WinTable<double> &w64, bool fp64_weights,
                                 double2 *f, double2 *grad, int ng, cudaStream_t st,
                                 const HalfTables *half = nullptr);

// ---- launchers implemented in kernels.cu (all enqueue on `st`) ------------

// vexp (here and in launch_deconv_gather, launch_fused_series): the call's
// range word; c enters scaled by 2^s, the adjoint's output leaves scaled by
// 2^-s (nullptr: no scaling, the mixed family and the FP64-pipe paths).
template <typename R>
cudaError_t launch_deconv_scatter(const typename Cplx<R>::T *c, int N1, int N2, int N3,
                                  const R *D1, const R *D2, const R *D3, typename Cplx<R>::T *G,
                                  Grid3 g, int with_grad, const int *vexp, cudaStream_t st);

// Force-load the deconvolve + scatter kernel and the 4-grid gather of cutoff
// m on the current device (modules load lazily on first use otherwise).
template <typename R> cudaError_t preload_grad_kernels(int m);

template <typename R>
cudaError_t launch_gather(const typename Cplx<R>::T *G, Grid3 g, int m, PointsView<R> pts,
                          const WinTable<R> &w, typename Cplx<R>::T *f, cudaStream_t st);

template <typename R>
cudaError_t launch_gather_grad(const typename Cplx<R>::T *G4, Grid3 g, int m, PointsView<R> pts,
                               const WinTable<R> &w, typename Cplx<R>::T *f,
                               typename Cplx<R>::T *grad, cudaStream_t st);

template <typename R>
cudaError_t launch_spread(const typename Cplx<R>::T *f, Grid3 g, int m, PointsView<R> pts,
                          const WinTable<R> &w, typename Cplx<R>::T *H, cudaStream_t st);
// Adjoint spread through shared-memory tile boxes (spread_tile.cu): one block
// per chunk of the set_points chunk list.
// Hq non-null (FP64 family, m <= 7): the boxes are flushed as exact
// fixed-point sums into Hq (four int64 limbs per node, zeroed by the caller)
// instead of FP64 atomics into H; launch_fixed_to_grid then writes H.
// wdf_dev: the FP64 family's table wdf in device memory (16-byte aligned H).
template <typename R>
cudaError_t launch_spread_tiles(const typename Cplx<R>::T *f, Grid3 g, int m, PointsView<R> pts,
                                const WinTable<R> &w, const WinTableDF *wdf, const WinTableDF *wdf_dev,
                                const int4 *chunks, int nchunks, int nt2, int nt3, typename Cplx<R>::T *H,
                                unsigned long long *Hq, cudaStream_t st);
cudaError_t launch_fixed_to_grid(const unsigned long long *Hq, double2 *H, int64_t total, cudaStream_t st);

template <typename R>
cudaError_t launch_deconv_gather(const typename Cplx<R>::T *H, Grid3 g, const R *D1, const R *D2,
                                 const R *D3, int N1, int N2, int N3, typename Cplx<R>::T *c,
                                 const int *vexp, cudaStream_t st);

// ---- launchers implemented in points.cu ------------------------------------

// One reduced point before sorting: stencil origin and original index (key.w), offsets.
template <typename R> struct alignas(16) PointRec {
    int4 key;
    R s[3];
};
// scratch bytes set_points needs for capacity M
inline size_t points_scratch_bytes(int64_t M, int prec) {
    return (prec == 64 ? sizeof(PointRec<double>) : sizeof(PointRec<float>)) * (size_t)(M + 1) +
           sizeof(int) * (size_t)(M + 1);
}

struct PointsBuild {
    int m;
    Grid3 g;
    int nt1, nt2, nt3;      // tiles per dimension
    int64_t ntile;
    int64_t M;
    // sort keys: tile x nsub + the stencil centre's (x, y) cell inside the
    // tile (nsub = 64, mixed family), so points reading the same grid rows are
    // neighbours in the sorted order; nsub = 1 (tile only) for the FP64 family
    // or when ntile x 64 would be too large
    int nsub;
    int64_t nkey;           // ntile * nsub
    int *key_count;         // nkey + 1 (last entry stays 0)
    int *key_start;         // nkey + 1 (exclusive scan)
    int *tile_start;        // ntile + 1: key_start[t * nsub]
    int2 *key_rank;         // M: (sort key, rank among the points of that key)
    int *scan_tmp;          // scan partials
    int *status;            // device status word (bit 0: non-finite coordinate)
    void *scratch;          // unsorted reduced points: (M_cap + 1) PointRec + M_cap ints (inverse permutation)
    int64_t M_cap;
    // work list of the tile-staged gather: chunks of <= kChunk points of one tile
    int *chunk_count;       // ntile + 1 (chunks per tile; last entry 0)
    int *chunk_start;       // ntile + 1 (exclusive scan; last entry = number of chunks)
    int4 *chunks;           // (tile, first sorted point, count, 0), chunk_cap entries
    int64_t chunk_cap;
    // split of the mixed family's value gather (nsub > 1 only): sort keys
    // holding at least dense_min points are "dense" and gathered in batches
    // of <= 32 points that share their first two stencil nodes (one point per
    // lane); the points of the other keys are "sparse" and gathered by the
    // column kernel through an index list.  Counts and starts are per tile.
    int dense_min;          // 0: no split
    int *tile_dense;        // ntile + 1: batches per tile
    int *tile_dense_start;  // ntile + 1: exclusive scan
    int *tile_sparse;       // ntile + 1: sparse points per tile
    int *tile_sparse_start; // ntile + 1
    int2 *batches;          // (first sorted point, count <= 32), batch_cap entries
    int64_t batch_cap;
    int *sparse_idx;        // sorted indices of the sparse points, M_cap entries
};

constexpr int kDenseBatch = 32;       // points per batch of the dense gather (one per lane)
constexpr int kDenseMinDefault = 12;  // points a sort key needs to go to the dense gather

constexpr int kChunk = 128;   // points per chunk of the tile-staged gather

// Tile-staged FP32 gather (gather_tma.cu).  tmap: a CUtensorMap (128 bytes)
// from encode_padded_tmap for the padded grid.
int encode_padded_tmap(void *tmap_out, const void *P, Grid3 pg, int m);
// first_wait_limit: polls of the first mbarrier wait before the kernel gives
// up (clamped to the normal limit); lowered only by the failure-detection test.
cudaError_t launch_gather_tma_f32(const void *tmap, const int4 *chunks, int nchunks, int nt2, int nt3,
                                  Grid3 g, int m, PointsView<float> pts, const WinTable<float> &w,
                                  float2 *f, int *status, unsigned first_wait_limit, cudaStream_t st);

// Buffers of the stable (deterministic) point order: a second permutation
// buffer (M_cap ints), per-pass digit counts and offsets
// (stable_sort_count_ints each) and the scan's temporary.
struct StableSort {
    int *buf;
    int *counts;
    int *offsets;
    int *scan_tmp;
};
size_t stable_sort_count_ints(int64_t M_cap);
// kernels launch_points adds with a stable sort, in place of one
int stable_sort_launches(const PointsBuild &pb);

// stable: nullptr for the default order (by key; the order within a key
// follows the count pass's atomics), else points within a key keep their
// original order.  split, second: with 0 < split < M and an event, the
// first pass takes points [0, split) at once and points [split, M) after
// `second` (x's second part arriving by a copy that records it).
template <typename R>
cudaError_t launch_points(const double *x, PointsBuild &pb, int4 *key, R *s1, R *s2, R *s3,
                          cudaStream_t st, const StableSort *stable, int64_t split = 0,
                          cudaEvent_t second = nullptr);

// Chunk list from tile_start (after launch_points); the number of chunks is
// left in chunk_start[ntile].
cudaError_t launch_chunks(PointsBuild &pb, cudaStream_t st);
// Dense batches and sparse index list of the split gather (after
// launch_points, nsub > 1 and dense_min > 0); their numbers are left in
// tile_dense_start[ntile] and tile_sparse_start[ntile].
cudaError_t launch_split_lists(PointsBuild &pb, cudaStream_t st);
int split_list_launches(const PointsBuild &pb);

// Split value gather of the mixed family over the padded grid (G = P, g = pg):
// dense batches (one point per lane, shared first two stencil nodes) and the
// sparse points through the column kernel.
cudaError_t launch_gather_split_f32(const float2 *G, Grid3 g, int m, PointsView<float> pts,
                                    const WinTable<float> &w, const int2 *batches, int nbatch,
                                    const int *sparse_idx, int nsparse, float2 *f, cudaStream_t st);

size_t scan_tmp_ints(int64_t n);
// Exclusive scan of n ints on the stream; tmp must hold scan_tmp_ints(n) ints.
cudaError_t exclusive_scan(const int *in, int *out, int64_t n, int *tmp, cudaStream_t st);
int scan_launches(int64_t n);   // kernels exclusive_scan enqueues for n entries

}  // namespace gbnfft
