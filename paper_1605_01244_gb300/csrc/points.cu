// set_points: FP64 coordinate reduction and counting sort of the points by
// grid tile.
#include "reduce.cuh"

namespace gbnfft {
namespace {

// centre node l0 + m (mod n) of a stencil (l0 in [0, n)); its tile is centre / kTile
__device__ __forceinline__ int centre_node(int l0, int m, int n) {
    int c = l0 + m;
    c -= c >= n ? n : 0;
    if (c >= n) c = wrap_index(c, n);   // n < m only
    return c;
}

// Points per thread per loop trip in the set_points passes: their loads are
// issued together, so each thread keeps several HBM requests in flight.
#ifndef GBNFFT_PTS_ILP
#define GBNFFT_PTS_ILP 4
#endif
#ifndef GBNFFT_PTS_BLOCKS_PER_SM
#define GBNFFT_PTS_BLOCKS_PER_SM 8
#endif
constexpr int kPtsILP = GBNFFT_PTS_ILP;

// Pass 1: reduce every point once (FP64 results, integer pipe for n = 2^L),
// store the result unsorted as one aligned record per point (stencil origin,
// original index, offsets) plus its (key, rank) pair, where rank counts the
// points of the key before it.
template <typename R>
__global__ void __launch_bounds__(256) points_count_kernel(const double *__restrict__ x, PointsBuild pb,
                                                           PointRec<R> *__restrict__ rec, int64_t j_begin,
                                                           int64_t j_end) {
    const CoordParams cp1 = coord_params(pb.g.n1, pb.m), cp2 = coord_params(pb.g.n2, pb.m),
                      cp3 = coord_params(pb.g.n3, pb.m);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j0 = j_begin + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j0 < j_end;
         j0 += kPtsILP * stride) {
        double xs[kPtsILP][3];
#pragma unroll
        for (int q = 0; q < kPtsILP; ++q) {
            const int64_t j = j0 + q * stride;
#pragma unroll
            for (int d = 0; d < 3; ++d) xs[q][d] = j < j_end ? __ldcs(x + 3 * j + d) : 0.0;
        }
        // phase 1: reduce, store the records, and issue one atomic per
        // distinct key in the warp (clustered points share keys) for all
        // points of the trip before any result is needed
        int k[kPtsILP], base[kPtsILP];
        unsigned peers[kPtsILP];
        const int lane = threadIdx.x & 31;
#pragma unroll
        for (int q = 0; q < kPtsILP; ++q) {
            const int64_t j = j0 + q * stride;
            peers[q] = 0;
            base[q] = 0;
            k[q] = 0;
            if (j >= j_end) continue;
            const Reduced r1 = reduce_coord(xs[q][0], cp1, pb.status);
            const Reduced r2 = reduce_coord(xs[q][1], cp2, pb.status);
            const Reduced r3 = reduce_coord(xs[q][2], cp3, pb.status);
            PointRec<R> o;
            o.key = make_int4(r1.l0, r2.l0, r3.l0, (int)j);
            o.s[0] = offset_as<R>(r1.s);
            o.s[1] = offset_as<R>(r2.s);
            o.s[2] = offset_as<R>(r3.s);
            rec[j] = o;
            const int c1 = centre_node(r1.l0, pb.m, pb.g.n1);
            const int c2 = centre_node(r2.l0, pb.m, pb.g.n2);
            const int c3 = centre_node(r3.l0, pb.m, pb.g.n3);
            // nkey = ntile nsub < 2^31 (checked at plan creation)
            const int t = ((c1 / kTile) * pb.nt2 + c2 / kTile) * pb.nt3 + c3 / kTile;
            k[q] = pb.nsub == 1 ? t : t * pb.nsub + (c1 % kTile) * kTile + c2 % kTile;
            peers[q] = __match_any_sync(__activemask(), k[q]);
            if (lane == __ffs(peers[q]) - 1) base[q] = atomicAdd(&pb.key_count[k[q]], __popc(peers[q]));
        }
        // phase 2: each lane's rank is its leader's base plus its place among
        // the lanes with the same key
#pragma unroll
        for (int q = 0; q < kPtsILP; ++q) {
            const int64_t j = j0 + q * stride;
            if (j >= j_end) continue;
            const int b = __shfl_sync(peers[q], base[q], __ffs(peers[q]) - 1);
            pb.key_rank[j] = make_int2(k[q], b + __popc(peers[q] & ((1u << lane) - 1u)));
        }
    }
}

// Pass 2a: the inverse permutation, perm[key_start[key] + rank] = j (one
// 4-byte store per point at its sorted position).
__global__ void __launch_bounds__(256) points_perm_kernel(PointsBuild pb, int *__restrict__ perm) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j0 < pb.M; j0 += kPtsILP * stride) {
        int2 kr[kPtsILP];
#pragma unroll
        for (int q = 0; q < kPtsILP; ++q) {
            const int64_t j = j0 + q * stride;
            kr[q] = j < pb.M ? pb.key_rank[j] : make_int2(0, 0);
        }
        int ks[kPtsILP];
#pragma unroll
        for (int q = 0; q < kPtsILP; ++q) ks[q] = j0 + q * stride < pb.M ? pb.key_start[kr[q].x] : 0;
#pragma unroll
        for (int q = 0; q < kPtsILP; ++q) {
            const int64_t j = j0 + q * stride;
            if (j < pb.M) perm[(int64_t)ks[q] + kr[q].y] = (int)j;
        }
    }
}

// Pass 2b: write the sorted arrays in order: position p takes record perm[p]
// (one aligned record read per point, all stores contiguous).
template <typename R>
__global__ void __launch_bounds__(256) points_gather_kernel(PointsBuild pb, const PointRec<R> *__restrict__ rec,
                                                            const int *__restrict__ perm, int4 *__restrict__ key,
                                                            R *__restrict__ s1, R *__restrict__ s2,
                                                            R *__restrict__ s3) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p0 < pb.M; p0 += kPtsILP * stride) {
        int js[kPtsILP];
#pragma unroll
        for (int q = 0; q < kPtsILP; ++q) js[q] = p0 + q * stride < pb.M ? perm[p0 + q * stride] : 0;
        PointRec<R> r[kPtsILP];
#pragma unroll
        for (int q = 0; q < kPtsILP; ++q) r[q] = rec[js[q]];
#pragma unroll
        for (int q = 0; q < kPtsILP; ++q) {
            const int64_t p = p0 + q * stride;
            if (p >= pb.M) break;
            key[p] = r[q].key;
            s1[p] = r[q].s[0];
            s2[p] = r[q].s[1];
            s3[p] = r[q].s[2];
        }
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

// Split lists of the mixed family's gather, one warp per tile: each lane
// takes two of the tile's nsub = 64 sort keys; a key with at least dense_min
// points contributes ceil(count / 32) batches, any other key its points to
// the sparse list.
__device__ __forceinline__ void key_split(const PointsBuild &pb, int64_t k, int &nb, int &ns, int &first,
                                          int &cnt) {
    first = pb.key_start[k];
    cnt = pb.key_start[k + 1] - first;
    const bool dense = cnt >= pb.dense_min;
    nb = dense ? (cnt + kDenseBatch - 1) / kDenseBatch : 0;
    ns = dense ? 0 : cnt;
}

__global__ void __launch_bounds__(256) split_count_kernel(PointsBuild pb) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t <= pb.ntile; t += nw) {
        int nb = 0, ns = 0;
        if (t < pb.ntile) {
            for (int h = 0; h < 2; ++h) {
                int b, s, first, cnt;
                key_split(pb, t * pb.nsub + h * 32 + lane, b, s, first, cnt);
                nb += b;
                ns += s;
            }
        }
        nb = __reduce_add_sync(0xffffffffu, nb);
        ns = __reduce_add_sync(0xffffffffu, ns);
        if (lane == 0) {
            pb.tile_dense[t] = nb;
            pb.tile_sparse[t] = ns;
        }
    }
}

__global__ void __launch_bounds__(256) split_fill_kernel(PointsBuild pb) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < pb.ntile; t += nw) {
        int nb[2], ns[2], first[2], cnt[2];
        for (int h = 0; h < 2; ++h) key_split(pb, t * pb.nsub + h * 32 + lane, nb[h], ns[h], first[h], cnt[h]);
        // positions: keys in order h = 0 (lanes 0..31), then h = 1
        int ob = pb.tile_dense_start[t], os = pb.tile_sparse_start[t];
        for (int h = 0; h < 2; ++h) {
            const int ib = warp_incl_scan(nb[h]), is = warp_incl_scan(ns[h]);
            const int pb0 = ob + ib - nb[h], ps0 = os + is - ns[h];
            // the batches of each dense key, written by the whole warp (a key
            // can hold millions of points: a lattice inside one cell)
            for (unsigned dense = __ballot_sync(0xffffffffu, nb[h] > 0); dense; dense &= dense - 1) {
                const int src = __ffs(dense) - 1;
                const int kb = __shfl_sync(0xffffffffu, nb[h], src), kp = __shfl_sync(0xffffffffu, pb0, src);
                const int kf = __shfl_sync(0xffffffffu, first[h], src), kc = __shfl_sync(0xffffffffu, cnt[h], src);
                for (int b = lane; b < kb; b += 32) {
                    const int n = kc - b * kDenseBatch < kDenseBatch ? kc - b * kDenseBatch : kDenseBatch;
                    if (kp + b < pb.batch_cap) pb.batches[kp + b] = make_int2(kf + b * kDenseBatch, n);
                }
            }
            for (int i = 0; i < ns[h]; ++i)
                if (ps0 + i < pb.M_cap) pb.sparse_idx[ps0 + i] = first[h] + i;
            ob += __shfl_sync(0xffffffffu, ib, 31);
            os += __shfl_sync(0xffffffffu, is, 31);
        }
    }
}

// ---- stable order (deterministic mode) --------------------------------------
// An LSD radix sort of the point indices by sort key, kRadixBits per pass:
// each pass is a stable counting sort (per-block digit histograms, a scan
// over (digit, block), then a scatter that ranks every block's elements in
// their order), so the result lists the points by key and, within a key, by
// original index -- independent of scheduling.
constexpr int kRadixBits = 8, kRadixBins = 1 << kRadixBits, kRadixThreads = 256, kRadixBlock = 4096;

__device__ __forceinline__ int radix_digit(const int2 *key_rank, const int *vin, int64_t e, int shift, int &j) {
    j = vin ? vin[e] : (int)e;
    return (key_rank[j].x >> shift) & (kRadixBins - 1);
}

__global__ void __launch_bounds__(kRadixThreads) radix_hist_kernel(const int2 *__restrict__ key_rank,
                                                                   const int *__restrict__ vin, int64_t M,
                                                                   int shift, int *__restrict__ counts,
                                                                   int nblocks) {
    __shared__ int h[kRadixBins];
    for (int d = threadIdx.x; d < kRadixBins; d += blockDim.x) h[d] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRadixBlock;
    for (int i = threadIdx.x; i < kRadixBlock; i += blockDim.x) {
        const int64_t e = base + i;
        if (e >= M) break;
        int j;
        atomicAdd(&h[radix_digit(key_rank, vin, e, shift, j)], 1);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadixBins; d += blockDim.x) counts[(int64_t)d * nblocks + blockIdx.x] = h[d];
}

__global__ void __launch_bounds__(kRadixThreads) radix_scatter_kernel(const int2 *__restrict__ key_rank,
                                                                      const int *__restrict__ vin,
                                                                      int *__restrict__ vout, int64_t M, int shift,
                                                                      const int *__restrict__ offsets, int nblocks) {
    constexpr int NW = kRadixThreads / 32;
    __shared__ int running[kRadixBins];
    __shared__ int wcount[NW][kRadixBins];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < kRadixBins; d += blockDim.x) {
        running[d] = offsets[(int64_t)d * nblocks + blockIdx.x];
        for (int w = 0; w < NW; ++w) wcount[w][d] = 0;
    }
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRadixBlock;
    for (int r = 0; r < kRadixBlock / kRadixThreads; ++r) {
        // element e of this round: its rank among the block's earlier elements
        // of the same digit = the running count + the earlier warps' counts in
        // this round + the lower lanes of its own warp with the same digit
        const int64_t e = base + (int64_t)r * kRadixThreads + threadIdx.x;
        const bool valid = e < M;
        int j = 0, d = kRadixBins;   // invalid lanes match each other only
        if (valid) d = radix_digit(key_rank, vin, e, shift, j);
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int leader = __ffs(peers) - 1;
        if (valid && lane == leader) wcount[warp][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            int pos = running[d] + __popc(peers & ((1u << lane) - 1u));
            for (int w = 0; w < warp; ++w) pos += wcount[w][d];
            vout[pos] = j;
        }
        __syncthreads();
        if (valid && lane == leader) {
            atomicAdd(&running[d], __popc(peers));
            wcount[warp][d] = 0;
        }
        __syncthreads();
    }
}

int point_blocks(int64_t M) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t want = ceil_div(M, 256);
    int64_t cap = (int64_t)sms * GBNFFT_PTS_BLOCKS_PER_SM;
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

int64_t radix_blocks(int64_t M) { return ceil_div(M > 0 ? M : 1, kRadixBlock); }
int radix_passes(int64_t nkey) {
    int bits = 1;
    while (bits < 31 && ((int64_t)1 << bits) < nkey) ++bits;
    return (bits + kRadixBits - 1) / kRadixBits;
}

// The stable permutation (sorted position -> original index) into one of the
// two buffers; returns it in *perm_out.
cudaError_t stable_perm(PointsBuild &pb, int *bufA, int *bufB, const StableSort &ss, int **perm_out,
                        cudaStream_t st) {
    const int64_t nb = radix_blocks(pb.M);
    const int passes = radix_passes(pb.nkey);
    const int *vin = nullptr;
    int *vout = bufA;
    for (int ps = 0; ps < passes; ++ps) {
        const int shift = ps * kRadixBits;
        radix_hist_kernel<<<(unsigned)nb, kRadixThreads, 0, st>>>(pb.key_rank, vin, pb.M, shift, ss.counts, (int)nb);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        e = exclusive_scan(ss.counts, ss.offsets, (int64_t)kRadixBins * nb, ss.scan_tmp, st);
        if (e != cudaSuccess) return e;
        radix_scatter_kernel<<<(unsigned)nb, kRadixThreads, 0, st>>>(pb.key_rank, vin, vout, pb.M, shift, ss.offsets,
                                                                     (int)nb);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        vin = vout;
        vout = vout == bufA ? bufB : bufA;
    }
    *perm_out = const_cast<int *>(vin);
    return cudaSuccess;
}

template <typename R>
cudaError_t launch_points(const double *x, PointsBuild &pb, int4 *key, R *s1, R *s2, R *s3,
                          cudaStream_t st, const StableSort *stable, int64_t split, cudaEvent_t second) {
    // key_count has nkey + 1 entries; the extra zero makes key_start[nkey] = M.
    cudaError_t e = cudaMemsetAsync(pb.key_count, 0, sizeof(int) * (pb.nkey + 1), st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(pb.status, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    PointRec<R> *rec = (PointRec<R> *)pb.scratch;
    int *perm = (int *)((char *)pb.scratch + sizeof(PointRec<R>) * (pb.M_cap + 1));
    if (pb.M > 0) {
        // points [split, M) only after `second` (their coordinates may still
        // be arriving); ranks come from the same atomic counts either way
        const int64_t j1 = second && split > 0 && split < pb.M ? split : pb.M;
        points_count_kernel<R><<<point_blocks(j1), 256, 0, st>>>(x, pb, rec, 0, j1);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (j1 < pb.M) {
            if ((e = cudaStreamWaitEvent(st, second, 0)) != cudaSuccess) return e;
            points_count_kernel<R><<<point_blocks(pb.M - j1), 256, 0, st>>>(x, pb, rec, j1, pb.M);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
    }
    e = exclusive_scan(pb.key_count, pb.key_start, pb.nkey + 1, pb.scan_tmp, st);
    if (e != cudaSuccess) return e;
    tile_start_kernel<<<point_blocks(pb.ntile + 1), 256, 0, st>>>(pb);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (pb.M > 0) {
        if (stable) {
            // deterministic order: by key, then by original index
            int *sorted = nullptr;
            if ((e = stable_perm(pb, perm, stable->buf, *stable, &sorted, st)) != cudaSuccess) return e;
            perm = sorted;
        } else {
            points_perm_kernel<<<point_blocks(pb.M), 256, 0, st>>>(pb, perm);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        points_gather_kernel<R><<<point_blocks(pb.M), 256, 0, st>>>(pb, rec, perm, key, s1, s2, s3);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

size_t stable_sort_count_ints(int64_t M_cap) { return (size_t)kRadixBins * (size_t)radix_blocks(M_cap); }

int stable_sort_launches(const PointsBuild &pb) {
    if (pb.M <= 0) return 0;
    return radix_passes(pb.nkey) * (2 + scan_launches((int64_t)kRadixBins * radix_blocks(pb.M))) - 1;
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

cudaError_t launch_split_lists(PointsBuild &pb, cudaStream_t st) {
    if (pb.nsub != 64 || pb.dense_min <= 0) return cudaErrorInvalidValue;
    const int64_t n = pb.ntile + 1;
    const int blocks = point_blocks(n * 32);
    split_count_kernel<<<blocks, 256, 0, st>>>(pb);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = exclusive_scan(pb.tile_dense, pb.tile_dense_start, n, pb.scan_tmp, st);
    if (e != cudaSuccess) return e;
    e = exclusive_scan(pb.tile_sparse, pb.tile_sparse_start, n, pb.scan_tmp, st);
    if (e != cudaSuccess) return e;
    split_fill_kernel<<<blocks, 256, 0, st>>>(pb);
    return cudaGetLastError();
}

int split_list_launches(const PointsBuild &pb) { return 2 + 2 * scan_launches(pb.ntile + 1); }

template cudaError_t launch_points<double>(const double *, PointsBuild &, int4 *, double *,
                                           double *, double *, cudaStream_t, const StableSort *, int64_t,
                                           cudaEvent_t);
template cudaError_t launch_points<float>(const double *, PointsBuild &, int4 *, float *, float *,
                                          float *, cudaStream_t, const StableSort *, int64_t, cudaEvent_t);

}  // namespace gbnfft

namespace gbnfft {
namespace {

__global__ void reduce_coords_kernel(const double *__restrict__ x, int64_t M, int n, int m, int *__restrict__ l0,
                                     double *__restrict__ s, float *__restrict__ s32, int *__restrict__ status) {
    const CoordParams cp = coord_params(n, m);
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < M; j += (int64_t)gridDim.x * blockDim.x) {
        const Reduced r = reduce_coord(x[j], cp, status);
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
