// set_points: FP64 coordinate reduction and counting sort of the points by
// grid tile.
#include "reduce.cuh"

namespace gbnfft {
namespace {

// centre node l0 + m (mod n) of a stencil; its tile is centre / kTile
__device__ __forceinline__ int centre_node(int l0, int m, int n) {
    int c = l0 + m;
    while (c >= n) c -= n;
    return c;
}

// Pass 1: reduce every point once (FP64 results, integer pipe for n = 2^L),
// store the result unsorted as one aligned record per point (stencil origin,
// tile, offsets), and count the points per tile; the returned count is the
// point's rank within its tile.
template <typename R>
__global__ void points_count_kernel(const double *__restrict__ x, PointsBuild pb,
                                    PointRec<R> *__restrict__ rec) {
    const double alpha = (double)pb.m + 0.5;
    const double nd1 = (double)pb.g.n1, nd2 = (double)pb.g.n2, nd3 = (double)pb.g.n3;
    const int L1 = log2_if_pow2(pb.g.n1), L2 = log2_if_pow2(pb.g.n2), L3 = log2_if_pow2(pb.g.n3);
    const int width = 2 * pb.m + 1;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < pb.M;
         j += (int64_t)gridDim.x * blockDim.x) {
        const Reduced r1 = reduce_coord(x[3 * j + 0], pb.g.n1, nd1, alpha, L1, width, pb.status);
        const Reduced r2 = reduce_coord(x[3 * j + 1], pb.g.n2, nd2, alpha, L2, width, pb.status);
        const Reduced r3 = reduce_coord(x[3 * j + 2], pb.g.n3, nd3, alpha, L3, width, pb.status);
        const int c1 = centre_node(r1.l0, pb.m, pb.g.n1);
        const int c2 = centre_node(r2.l0, pb.m, pb.g.n2);
        const int c3 = centre_node(r3.l0, pb.m, pb.g.n3);
        const int64_t t = ((int64_t)(c1 / kTile) * pb.nt2 + c2 / kTile) * pb.nt3 + c3 / kTile;
        const int sub = pb.nsub == 1 ? 0 : (c1 % kTile) * kTile + c2 % kTile;
        const int64_t k = t * pb.nsub + sub;
        pb.rank[j] = atomicAdd(&pb.key_count[k], 1);
        PointRec<R> o;
        o.key = make_int4(r1.l0, r2.l0, r3.l0, (int)k);
        o.s[0] = offset_as<R>(r1.s);
        o.s[1] = offset_as<R>(r2.s);
        o.s[2] = offset_as<R>(r3.s);
        rec[j] = o;
    }
}

// Pass 2a: the inverse permutation, perm[tile_start[tile] + rank] = j (one
// 4-byte store per point at its sorted position).
template <typename R>
__global__ void points_perm_kernel(PointsBuild pb, const PointRec<R> *__restrict__ rec, int *__restrict__ perm) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < pb.M;
         j += (int64_t)gridDim.x * blockDim.x)
        perm[(int64_t)pb.key_start[rec[j].key.w] + pb.rank[j]] = (int)j;
}

// Pass 2b: write the sorted arrays in order: position p takes record perm[p]
// (one aligned record read per point, all stores contiguous).
template <typename R>
__global__ void points_gather_kernel(PointsBuild pb, const PointRec<R> *__restrict__ rec,
                                     const int *__restrict__ perm, int4 *__restrict__ key, R *__restrict__ s1,
                                     R *__restrict__ s2, R *__restrict__ s3) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < pb.M;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int j = perm[p];
        const PointRec<R> r = rec[j];
        key[p] = make_int4(r.key.x, r.key.y, r.key.z, j);
        s1[p] = r.s[0];
        s2[p] = r.s[1];
        s3[p] = r.s[2];
    }
}

__global__ void tile_start_kernel(PointsBuild pb) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t <= pb.ntile;
         t += (int64_t)gridDim.x * blockDim.x)
        pb.tile_start[t] = pb.key_start[t * pb.nsub];
}

// ---- exclusive scan (three phases, recursive over block sums) -------------

constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanChunk = kScanThreads * kScanItems;

__device__ __forceinline__ int warp_incl_scan(int v) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) >= o) v += t;
    }
    return v;
}

// exclusive scan of `in` (n entries) into `out` per chunk of kScanChunk;
// chunk totals go to bsum (if non-null).
__global__ void __launch_bounds__(kScanThreads) scan_chunk_kernel(const int *__restrict__ in,
                                                                  int *__restrict__ out, int64_t n,
                                                                  int *__restrict__ bsum) {
    __shared__ int warp_tot[kScanThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanChunk + (int64_t)threadIdx.x * kScanItems;
    int v[kScanItems];
    int local = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const int64_t idx = base + i;
        v[i] = idx < n ? in[idx] : 0;
        local += v[i];
    }
    const int incl = warp_incl_scan(local);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int t = lane < kScanThreads / 32 ? warp_tot[lane] : 0;
        t = warp_incl_scan(t);
        if (lane < kScanThreads / 32) warp_tot[lane] = t;
    }
    __syncthreads();
    int run = incl - local + (wid > 0 ? warp_tot[wid - 1] : 0);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const int64_t idx = base + i;
        if (idx < n) out[idx] = run;
        run += v[i];
    }
    if (bsum && threadIdx.x == kScanThreads - 1) bsum[blockIdx.x] = run;
}

__global__ void scan_add_kernel(int *__restrict__ out, int64_t n, const int *__restrict__ boff) {
    const int64_t base = (int64_t)blockIdx.x * kScanChunk;
    const int add = boff[blockIdx.x];
    for (int i = threadIdx.x; i < kScanChunk; i += blockDim.x) {
        const int64_t idx = base + i;
        if (idx < n) out[idx] += add;
    }
}

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

__global__ void chunk_count_kernel(PointsBuild pb) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t <= pb.ntile;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int cnt = t < pb.ntile ? pb.tile_start[t + 1] - pb.tile_start[t] : 0;
        pb.chunk_count[t] = (cnt + kChunk - 1) / kChunk;
    }
}

__global__ void chunk_fill_kernel(PointsBuild pb) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < pb.ntile;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int first = pb.tile_start[t], cnt = pb.tile_start[t + 1] - first;
        const int base = pb.chunk_start[t];
        for (int k = 0; k * kChunk < cnt; ++k) {
            const int n = cnt - k * kChunk < kChunk ? cnt - k * kChunk : kChunk;
            if (base + k < pb.chunk_cap) pb.chunks[base + k] = make_int4((int)t, first + k * kChunk, n, 0);
        }
    }
}

int point_blocks(int64_t M) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t want = ceil_div(M, 256);
    int64_t cap = (int64_t)sms * 8;
    return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

}  // namespace

// Exclusive scan of n ints; tmp must hold scan_tmp_ints(n) ints.
cudaError_t exclusive_scan(const int *in, int *out, int64_t n, int *tmp, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int64_t nb = ceil_div(n, kScanChunk);
    if (nb == 1) {
        scan_chunk_kernel<<<1, kScanThreads, 0, st>>>(in, out, n, nullptr);
        return cudaGetLastError();
    }
    int *bsum = tmp;
    int *boff = tmp + nb;
    scan_chunk_kernel<<<(unsigned)nb, kScanThreads, 0, st>>>(in, out, n, bsum);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = exclusive_scan(bsum, boff, nb, tmp + 2 * nb, st);
    if (e != cudaSuccess) return e;
    scan_add_kernel<<<(unsigned)nb, kScanThreads, 0, st>>>(out, n, boff);
    return cudaGetLastError();
}

size_t scan_tmp_ints(int64_t n) {
    size_t tot = 0;
    while (n > kScanChunk) {
        const int64_t nb = ceil_div(n, kScanChunk);
        tot += 2 * nb;
        n = nb;
    }
    return tot + 1;
}

int scan_launches(int64_t n) {
    if (n <= 0) return 0;
    const int64_t nb = ceil_div(n, kScanChunk);
    return nb == 1 ? 1 : 2 + scan_launches(nb);
}

template <typename R>
cudaError_t launch_points(const double *x, PointsBuild &pb, int4 *key, R *s1, R *s2, R *s3,
                          cudaStream_t st) {
    // key_count has nkey + 1 entries; the extra zero makes key_start[nkey] = M.
    cudaError_t e = cudaMemsetAsync(pb.key_count, 0, sizeof(int) * (pb.nkey + 1), st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(pb.status, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    PointRec<R> *rec = (PointRec<R> *)pb.scratch;
    int *perm = (int *)((char *)pb.scratch + sizeof(PointRec<R>) * (pb.M_cap + 1));
    if (pb.M > 0) {
        points_count_kernel<R><<<point_blocks(pb.M), 256, 0, st>>>(x, pb, rec);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    e = exclusive_scan(pb.key_count, pb.key_start, pb.nkey + 1, pb.scan_tmp, st);
    if (e != cudaSuccess) return e;
    tile_start_kernel<<<point_blocks(pb.ntile + 1), 256, 0, st>>>(pb);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (pb.M > 0) {
        points_perm_kernel<R><<<point_blocks(pb.M), 256, 0, st>>>(pb, rec, perm);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        points_gather_kernel<R><<<point_blocks(pb.M), 256, 0, st>>>(pb, rec, perm, key, s1, s2, s3);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_chunks(PointsBuild &pb, cudaStream_t st) {
    const int64_t n = pb.ntile + 1;
    chunk_count_kernel<<<point_blocks(n), 256, 0, st>>>(pb);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = exclusive_scan(pb.chunk_count, pb.chunk_start, n, pb.scan_tmp, st);
    if (e != cudaSuccess) return e;
    chunk_fill_kernel<<<point_blocks(pb.ntile), 256, 0, st>>>(pb);
    return cudaGetLastError();
}

template cudaError_t launch_points<double>(const double *, PointsBuild &, int4 *, double *,
                                           double *, double *, cudaStream_t);
template cudaError_t launch_points<float>(const double *, PointsBuild &, int4 *, float *, float *,
                                          float *, cudaStream_t);

}  // namespace gbnfft

namespace gbnfft {
namespace {

__global__ void reduce_coords_kernel(const double *__restrict__ x, int64_t M, int n, int m, int *__restrict__ l0,
                                     double *__restrict__ s, float *__restrict__ s32, int *__restrict__ status) {
    const double alpha = (double)m + 0.5, nd = (double)n;
    const int L = log2_if_pow2(n);
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < M; j += (int64_t)gridDim.x * blockDim.x) {
        const Reduced r = reduce_coord(x[j], n, nd, alpha, L, 2 * m + 1, status);
        if (l0) l0[j] = r.l0;
        if (s) s[j] = offset_as<double>(r.s);
        if (s32) s32[j] = offset_as<float>(r.s);
    }
}

}  // namespace
}  // namespace gbnfft

extern "C" int nfft3_reduce_coords(int n, int m, const double *x, int64_t M, int *l0, double *s, float *s32,
                                   int *status, void *stream) {
    using namespace gbnfft;
    if (n < 2 || m < 1 || m > kMaxM || M < 0 || !status) return NFFT3_ERR_ARG;
    if (M > 0 && !x) return NFFT3_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return NFFT3_ERR_CUDA;
    if (M == 0) return NFFT3_OK;
    reduce_coords_kernel<<<point_blocks(M), 256, 0, st>>>(x, M, n, m, l0, s, s32, status);
    return cudaGetLastError() == cudaSuccess ? NFFT3_OK : NFFT3_ERR_CUDA;
}
