// Tile-staged window gather for the mixed family: the points of one 8^3 tile
// of stencil centres are evaluated from a (8 + 2m)^3 box of the padded grid
// that one TMA bulk-tensor copy (cp.async.bulk.tensor.3d) brings into shared
// memory, instead of every lane reading its rows through L1.
//
// Work items are chunks of at most kChunk sorted points of one tile (built
// by set_points).  Persistent CTAs (as many as fit on the GPU) walk the chunk
// list with two box buffers: the copy of chunk i + 2's box (armed on an
// mbarrier with the box's byte count) overlaps the evaluation of chunk i.
// Waits are bounded: after kWaitLimit polls the CTA records an error bit in
// the plan's status word, waits (again bounded) for every copy it issued that
// may still be in flight -- the late one and the other buffer's -- and
// returns without touching shared memory again.  The first wait's limit is a
// launch parameter (normally kWaitLimit), so that a test can make it run out.
// Evaluation uses the column-group mapping of gather_col.cu on shared memory.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>

#include "internal.cuh"

namespace gbnfft {
namespace {

constexpr unsigned kWaitLimit = 1u << 24;

template <int W> struct GS {
    static constexpr int value = W <= 2 ? 2 : W <= 4 ? 4 : W <= 8 ? 8 : W <= 16 ? 16 : 32;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int x,
                                            int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"((unsigned long long)map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

template <int MM>
__global__ void __launch_bounds__(256) gather_tma_f32_kernel(const __grid_constant__ CUtensorMap tmap,
                                                             const int4 *__restrict__ chunks, int nchunks,
                                                             int nt2, int nt3, Grid3 g,
                                                             PointsView<float> pts,
                                                             const __grid_constant__ Poly<float, MM> P,
                                                             float2 *__restrict__ f,
                                                             int *__restrict__ status,
                                                             unsigned first_wait_limit) {
    constexpr int W = 2 * MM + 1;
    constexpr int G = GS<W>::value;
    constexpr int B = kTile + 2 * MM;           // box edge
    constexpr int D = PolyDeg<float>::value;
    constexpr uint32_t kBoxBytes = B * B * B * sizeof(float2);
    constexpr uint32_t kBoxStride = ((kBoxBytes + 127) / 128) * 128;
    extern __shared__ __align__(128) unsigned char smem[];
    float2 *box[2] = {reinterpret_cast<float2 *>(smem), reinterpret_cast<float2 *>(smem + kBoxStride)};
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 2 * kBoxStride);
    float *coef = reinterpret_cast<float *>(bar + 2);

    // issue the copy of chunk c's tile box into buffer b (thread 0 only)
    auto issue = [&](int c, int b) {
        const int tile = chunks[c].x;
        const int t3 = tile % nt3, t2 = (tile / nt3) % nt2, t1 = tile / (nt3 * nt2);
        mbar_expect_tx(&bar[b], kBoxBytes);
        tma_load_3d(box[b], &tmap, &bar[b], kTile * t3, kTile * t2, kTile * t1);
    };
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_fence_init();
        if ((int)blockIdx.x < nchunks) issue(blockIdx.x, 0);
        if ((int)(blockIdx.x + gridDim.x) < nchunks) issue(blockIdx.x + gridDim.x, 1);
    }
    for (int i = threadIdx.x; i < 3 * W * (D + 1); i += blockDim.x) coef[i] = (&P.c[0][0][0])[i];
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int sub = lane & (G - 1);
    const int gbase = lane & ~(G - 1);
    const int tap = sub < W ? sub : 0;
    const int groups = blockDim.x / G;
    const int grp = threadIdx.x / G;
    uint32_t phase[2] = {0u, 0u};
    int it = 0;
    for (int c = blockIdx.x; c < nchunks; c += gridDim.x, ++it) {
        const int b = it & 1;
        bool ready = false;
        const unsigned limit = it == 0 ? first_wait_limit : kWaitLimit;
        for (unsigned k = 0; k < limit; ++k)
            if ((ready = mbar_try_wait(&bar[b], phase[b]))) break;
        // the decision is taken by the whole block, so that no thread is left
        // waiting at a later barrier
        if (!__syncthreads_and(ready)) {
            if (threadIdx.x == 0) {
                atomicOr(status, 2);
                // let the copies still in flight land before the block's shared
                // memory is released: this buffer's, and the other buffer's if
                // one was issued for the next chunk
                for (unsigned k = 0; k < kWaitLimit; ++k)
                    if (mbar_try_wait(&bar[b], phase[b])) break;
                if (c + (int)gridDim.x < nchunks)
                    for (unsigned k = 0; k < kWaitLimit; ++k)
                        if (mbar_try_wait(&bar[b ^ 1], phase[b ^ 1])) break;
            }
            return;
        }
        phase[b] ^= 1u;
        const int4 ch = chunks[c];
        const int tile = ch.x;
        const int t3 = tile % nt3, t2 = (tile / nt3) % nt2, t1 = tile / (nt3 * nt2);
        const float2 *bx = box[b];
        for (int p0 = 0; p0 < ch.z; p0 += groups) {
            const bool valid = p0 + grp < ch.z;
            const int64_t j = ch.y + (valid ? p0 + grp : 0);
            const int4 key = pts.key[j];
            float myw[3];
            {
                const float s[3] = {pts.s1[j], pts.s2[j], pts.s3[j]};
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    const float t = 2.f * s[d] - 1.f;
                    const float *cd = coef + (d * W + tap) * (D + 1);
                    float v = cd[D];
#pragma unroll
                    for (int k = D - 1; k >= 0; --k) v = fmaf(v, t, cd[k]);
                    myw[d] = sub < W ? v : 0.f;
                }
            }
            float w1[W], w2[W];
#pragma unroll
            for (int a = 0; a < W; ++a) {
                w1[a] = __shfl_sync(0xffffffffu, myw[0], gbase + a);
                w2[a] = __shfl_sync(0xffffffffu, myw[1], gbase + a);
            }
            // stencil centre relative to the box origin, in [0, kTile)
            int c1 = key.x + MM, c2 = key.y + MM, c3 = key.z + MM;
            while (c1 >= g.n1) c1 -= g.n1;
            while (c2 >= g.n2) c2 -= g.n2;
            while (c3 >= g.n3) c3 -= g.n3;
            const int b1 = c1 - kTile * t1, b2 = c2 - kTile * t2, b3 = c3 - kTile * t3;
            const float2 *base = bx + (b1 * B + b2) * B + b3 + tap;
            float T0 = 0.f, T1 = 0.f;
#pragma unroll 1
            for (int a = 0; a < W; ++a) {
                float S0 = 0.f, S1 = 0.f;
#pragma unroll
                for (int bb = 0; bb < W; ++bb) {
                    const float2 v = base[bb * B];
                    S0 = fmaf(w2[bb], v.x, S0);
                    S1 = fmaf(w2[bb], v.y, S1);
                }
                T0 = fmaf(w1[0], S0, T0);
                T1 = fmaf(w1[0], S1, T1);
#pragma unroll
                for (int k = 0; k < W - 1; ++k) w1[k] = w1[k + 1];
                base += B * B;
            }
            float re = myw[2] * T0, im = myw[2] * T1;
#pragma unroll
            for (int off = G / 2; off > 0; off >>= 1) {
                re += __shfl_xor_sync(0xffffffffu, re, off, G);
                im += __shfl_xor_sync(0xffffffffu, im, off, G);
            }
            if (valid && sub == 0) f[key.w] = make_float2(re, im);
        }
        __syncthreads();  // every thread is done with buffer b
        if (threadIdx.x == 0 && c + 2 * (int)gridDim.x < nchunks) issue(c + 2 * gridDim.x, b);
    }
}

template <int MM> size_t tma_smem_bytes() {
    constexpr int W = 2 * MM + 1, B = kTile + 2 * MM, D = PolyDeg<float>::value;
    const size_t box = ((B * B * B * sizeof(float2) + 127) / 128) * 128;
    return 2 * box + 2 * sizeof(uint64_t) + sizeof(float) * 3 * W * (D + 1);
}

template <int MM>
cudaError_t tma_dispatch(const CUtensorMap &map, const int4 *chunks, int nchunks, int nt2, int nt3,
                         Grid3 g, PointsView<float> pts, const WinTable<float> &w, float2 *f,
                         int *status, unsigned first_wait_limit, cudaStream_t st) {
    const size_t sm = tma_smem_bytes<MM>();
    static int blocks_per_sm = 0;  // per process; the attribute and occupancy are per function
    if (!blocks_per_sm) {
        cudaFuncSetAttribute(gather_tma_f32_kernel<MM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, gather_tma_f32_kernel<MM>, 256, sm);
        if (blocks_per_sm < 1) blocks_per_sm = 1;
    }
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = nchunks < sms * blocks_per_sm ? nchunks : sms * blocks_per_sm;
    gather_tma_f32_kernel<MM><<<grid, 256, sm, st>>>(map, chunks, nchunks, nt2, nt3, g, pts,
                                                     make_poly<float, MM>(w), f, status, first_wait_limit);
    return cudaGetLastError();
}

}  // namespace

// Encode the 3D tensor map of a padded FP32 grid (element = one complex, 8 bytes):
// dims (p3, p2, p1) innermost first, box (8 + 2m)^3.  Returns 0 on success.
int encode_padded_tmap(void *tmap_out, const void *P, Grid3 pg, int m) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return -1;
        encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
    const int B = kTile + 2 * m;
    cuuint64_t dims[3] = {(cuuint64_t)pg.n3, (cuuint64_t)pg.n2, (cuuint64_t)pg.n1};
    cuuint64_t strides[2] = {(cuuint64_t)pg.n3 * 8, (cuuint64_t)pg.n3 * pg.n2 * 8};
    cuuint32_t box[3] = {(cuuint32_t)B, (cuuint32_t)B, (cuuint32_t)B};
    cuuint32_t estr[3] = {1, 1, 1};
    CUtensorMap map;
    std::memset(&map, 0, sizeof(map));
    const CUresult r = encode(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, const_cast<void *>(P), dims, strides,
                              box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return -1;
    std::memcpy(tmap_out, &map, sizeof(map));
    return 0;
}

cudaError_t launch_gather_tma_f32(const void *tmap, const int4 *chunks, int nchunks, int nt2, int nt3,
                                  Grid3 g, int m, PointsView<float> pts, const WinTable<float> &w,
                                  float2 *f, int *status, unsigned first_wait_limit, cudaStream_t st) {
    if (nchunks <= 0 || pts.M == 0) return cudaSuccess;
    const CUtensorMap &map = *reinterpret_cast<const CUtensorMap *>(tmap);
    if (first_wait_limit > kWaitLimit) first_wait_limit = kWaitLimit;
    switch (m) {
        case 1: return tma_dispatch<1>(map, chunks, nchunks, nt2, nt3, g, pts, w, f, status, first_wait_limit, st);
        case 2: return tma_dispatch<2>(map, chunks, nchunks, nt2, nt3, g, pts, w, f, status, first_wait_limit, st);
        case 3: return tma_dispatch<3>(map, chunks, nchunks, nt2, nt3, g, pts, w, f, status, first_wait_limit, st);
        case 4: return tma_dispatch<4>(map, chunks, nchunks, nt2, nt3, g, pts, w, f, status, first_wait_limit, st);
        case 5: return tma_dispatch<5>(map, chunks, nchunks, nt2, nt3, g, pts, w, f, status, first_wait_limit, st);
        case 6: return tma_dispatch<6>(map, chunks, nchunks, nt2, nt3, g, pts, w, f, status, first_wait_limit, st);
        case 7: return tma_dispatch<7>(map, chunks, nchunks, nt2, nt3, g, pts, w, f, status, first_wait_limit, st);
        case 8: return tma_dispatch<8>(map, chunks, nchunks, nt2, nt3, g, pts, w, f, status, first_wait_limit, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace gbnfft
