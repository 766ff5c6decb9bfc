// Kernels of the small 3D CNN that proposes vortex-core cells from coarse
// patches of psi: direct 3D convolution (forward, input gradient, weight
// gradient), the BCE + L1 loss, and Adam.  Weights and activations are BF16,
// every accumulation is FP32, the optimizer keeps FP32 master weights.
//
// Layouts (row-major): activations [B][C][D][D][D], weights
// [Cout][Cin][k][k][k] (k = 1 or 3, zero padding k/2: output size = input
// size), bias [Cout].  The paper has no learned component; this network is
// the proposal stage in front of the NFFT + Newton refinement.
#include <cuda_bf16.h>

#include <cstdlib>

#include "internal.cuh"

namespace {

__device__ __forceinline__ float bf(const __nv_bfloat16 v) { return __bfloat162float(v); }

struct ConvShape {
    int B, Cin, Cout, D, k;
};

// y[b, co, p] = bias[co] + sum_{ci, t} w[co, ci, t] x[b, ci, p + t - k/2]; optional ReLU.
// y is written as BF16 (activation) and/or FP32 (pre-activation logits).
__global__ void conv_fwd_kernel(const __nv_bfloat16 *__restrict__ x, const __nv_bfloat16 *__restrict__ w,
                                const float *__restrict__ bias, ConvShape s, int relu,
                                __nv_bfloat16 *__restrict__ ybf, float *__restrict__ yf) {
    const int D = s.D, D3 = D * D * D, h = s.k / 2;
    const int64_t total = (int64_t)s.B * s.Cout * D3;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int p = (int)(e % D3);
        const int co = (int)((e / D3) % s.Cout);
        const int b = (int)(e / ((int64_t)D3 * s.Cout));
        const int z = p / (D * D), yy = (p / D) % D, xx = p % D;
        float acc = bias ? bias[co] : 0.f;
        for (int ci = 0; ci < s.Cin; ++ci) {
            const __nv_bfloat16 *xin = x + ((int64_t)b * s.Cin + ci) * D3;
            const __nv_bfloat16 *wk = w + ((int64_t)co * s.Cin + ci) * s.k * s.k * s.k;
            for (int dz = 0; dz < s.k; ++dz) {
                const int zz = z + dz - h;
                if (zz < 0 || zz >= D) continue;
                for (int dy = 0; dy < s.k; ++dy) {
                    const int y2 = yy + dy - h;
                    if (y2 < 0 || y2 >= D) continue;
                    for (int dx = 0; dx < s.k; ++dx) {
                        const int x2 = xx + dx - h;
                        if (x2 < 0 || x2 >= D) continue;
                        acc = fmaf(bf(wk[(dz * s.k + dy) * s.k + dx]), bf(xin[(zz * D + y2) * D + x2]), acc);
                    }
                }
            }
        }
        if (relu && acc < 0.f) acc = 0.f;
        if (ybf) ybf[e] = __float2bfloat16_rn(acc);
        if (yf) yf[e] = acc;
    }
}

// dx[b, ci, q] = sum_{co, t} w[co, ci, t] dy[b, co, q - t + k/2]  (transpose of conv_fwd),
// then multiplied by the ReLU mask of the input activation when mask != NULL
// (mask = the forward activation: derivative 1 where it is > 0).
__global__ void conv_dgrad_kernel(const float *__restrict__ dy, const __nv_bfloat16 *__restrict__ w,
                                  ConvShape s, const __nv_bfloat16 *__restrict__ mask,
                                  float *__restrict__ dx) {
    const int D = s.D, D3 = D * D * D, h = s.k / 2;
    const int64_t total = (int64_t)s.B * s.Cin * D3;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int q = (int)(e % D3);
        const int ci = (int)((e / D3) % s.Cin);
        const int b = (int)(e / ((int64_t)D3 * s.Cin));
        if (mask && !(bf(mask[e]) > 0.f)) {
            dx[e] = 0.f;
            continue;
        }
        const int z = q / (D * D), yy = (q / D) % D, xx = q % D;
        float acc = 0.f;
        for (int co = 0; co < s.Cout; ++co) {
            const float *dyo = dy + ((int64_t)b * s.Cout + co) * D3;
            const __nv_bfloat16 *wk = w + ((int64_t)co * s.Cin + ci) * s.k * s.k * s.k;
            for (int dz = 0; dz < s.k; ++dz) {
                const int zz = z - dz + h;
                if (zz < 0 || zz >= D) continue;
                for (int dyy = 0; dyy < s.k; ++dyy) {
                    const int y2 = yy - dyy + h;
                    if (y2 < 0 || y2 >= D) continue;
                    for (int dx2 = 0; dx2 < s.k; ++dx2) {
                        const int x2 = xx - dx2 + h;
                        if (x2 < 0 || x2 >= D) continue;
                        acc = fmaf(bf(wk[(dz * s.k + dyy) * s.k + dx2]), dyo[(zz * D + y2) * D + x2], acc);
                    }
                }
            }
        }
        dx[e] = acc;
    }
}

// dw[co, ci, t] = sum_{b, p} dy[b, co, p] x[b, ci, p + t - k/2]; db[co] = sum dy[b, co, p].
// One block per weight (and one extra block row for the biases), block reduction.
__global__ void conv_wgrad_kernel(const float *__restrict__ dy, const __nv_bfloat16 *__restrict__ x,
                                  ConvShape s, float *__restrict__ dw, float *__restrict__ db) {
    const int K3 = s.k * s.k * s.k, D = s.D, D3 = D * D * D, h = s.k / 2;
    const int nw = s.Cout * s.Cin * K3;
    const int widx = blockIdx.x;
    __shared__ float red[256];
    float acc = 0.f;
    if (widx < nw) {
        const int t = widx % K3;
        const int ci = (widx / K3) % s.Cin;
        const int co = widx / (K3 * s.Cin);
        const int dz = t / (s.k * s.k) - h, dyy = (t / s.k) % s.k - h, dx2 = t % s.k - h;
        const int64_t npos = (int64_t)s.B * D3;
        for (int64_t i = threadIdx.x; i < npos; i += blockDim.x) {
            const int b = (int)(i / D3), p = (int)(i % D3);
            const int z = p / (D * D) + dz, yy = (p / D) % D + dyy, xx = p % D + dx2;
            if (z < 0 || z >= D || yy < 0 || yy >= D || xx < 0 || xx >= D) continue;
            acc = fmaf(dy[((int64_t)b * s.Cout + co) * D3 + p],
                       bf(x[((int64_t)b * s.Cin + ci) * D3 + (z * D + yy) * D + xx]), acc);
        }
    } else {
        const int co = widx - nw;
        const int64_t npos = (int64_t)s.B * D3;
        for (int64_t i = threadIdx.x; i < npos; i += blockDim.x) {
            const int b = (int)(i / D3), p = (int)(i % D3);
            acc += dy[((int64_t)b * s.Cout + co) * D3 + p];
        }
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (widx < nw)
            dw[widx] = red[0];
        else if (db)
            db[widx - nw] = red[0];
    }
}

// Loss over B x D^3 voxels of the 4-channel head y (channel 0 logit, 1..3 offset):
//   L = mean_v [ (1 + (pw - 1) t_v) BCE(logit_v, t_v) ] + lam * sum_v t_v |off_v - off*_v|_1 / max(1, sum t)
// (pw weights the rare positive voxels)
// dy receives dL/dy; loss[0] += L (atomic), loss[1] += positives.
__global__ void core_loss_kernel(const float *__restrict__ y, const float *__restrict__ target,
                                 const float *__restrict__ off_target, int B, int D, float lam,
                                 float pw, float npos, float *__restrict__ dy, float *__restrict__ loss) {
    const int D3 = D * D * D;
    const int64_t total = (int64_t)B * D3;
    const float inv_n = 1.f / (float)total, inv_pos = 1.f / fmaxf(npos, 1.f);
    float part = 0.f;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(e / D3), p = (int)(e % D3);
        const float l = y[((int64_t)b * 4 + 0) * D3 + p];
        const float t = target[e];
        const float wt = 1.f + (pw - 1.f) * t;
        part += wt * (fmaxf(l, 0.f) - l * t + log1pf(expf(-fabsf(l)))) * inv_n;
        dy[((int64_t)b * 4 + 0) * D3 + p] = wt * (1.f / (1.f + expf(-l)) - t) * inv_n;
        for (int c = 1; c < 4; ++c) {
            const float o = y[((int64_t)b * 4 + c) * D3 + p];
            const float d = o - off_target[e * 3 + (c - 1)];
            part += lam * t * fabsf(d) * inv_pos;
            dy[((int64_t)b * 4 + c) * D3 + p] = lam * t * (d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f)) * inv_pos;
        }
    }
    atomicAdd(loss, part);
}

// Adam on FP32 master weights, BF16 copy for the forward/backward kernels.
__global__ void adam_kernel(float *__restrict__ wm, __nv_bfloat16 *__restrict__ wbf,
                            const float *__restrict__ g, float *__restrict__ m1, float *__restrict__ m2,
                            int64_t n, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float a = b1 * m1[i] + (1.f - b1) * gi;
        const float v = b2 * m2[i] + (1.f - b2) * gi * gi;
        m1[i] = a;
        m2[i] = v;
        const float w = wm[i] - lr * (a / c1) / (sqrtf(v / c2) + eps);
        wm[i] = w;
        if (wbf) wbf[i] = __float2bfloat16_rn(w);
    }
}

// ---- shared-memory tiled versions (k = 1 or 3, at most kMaxC channels) -----
// A block covers a tile of kTX x kTY x kTZ voxels (one per thread) of one
// batch entry.  conv_tiled_kernel stages the tile's input with its halo (all
// input channels) and every weight in shared memory; each thread then forms
// all output channels of its voxel, each input value read once from shared
// memory for all of them and each weight read as a broadcast.  The same
// kernel computes the input gradient (dgrad) as the convolution of dy with
// the transposed, flipped weights.
constexpr int kTX = 8, kTY = 8, kTZ = 4, kTileVox = kTX * kTY * kTZ, kMaxC = 16;

template <int K> __host__ __device__ constexpr int halo_vol() {
    return (kTX + K - 1) * (kTY + K - 1) * (kTZ + K - 1);
}

template <int K> size_t conv_tiled_smem(int Cin, int Cout) {
    return sizeof(float) * ((size_t)Cin * halo_vol<K>() + (size_t)Cout * Cin * K * K * K);
}

// DGRAD = false: y[b, co] = bias + sum_ci,t w[co, ci, t] x[b, ci, p + t - h]
//   (x BF16; ReLU optional; output BF16 and/or FP32)
// DGRAD = true:  dx[b, ci] = sum_co,t w[co, ci, t] dy[b, co, q - t + h]
//   (dy FP32, Cin <-> Cout exchanged; masked by the ReLU of the input
//   activation when mask is given; output FP32)
template <int K, bool DGRAD>
__global__ void __launch_bounds__(kTileVox) conv_tiled_kernel(const void *__restrict__ xin,
                                                              const __nv_bfloat16 *__restrict__ w,
                                                              const float *__restrict__ bias, ConvShape s,
                                                              int relu, const __nv_bfloat16 *__restrict__ mask,
                                                              __nv_bfloat16 *__restrict__ ybf,
                                                              float *__restrict__ yf) {
    constexpr int K3 = K * K * K, h = K / 2;
    constexpr int HX = kTX + K - 1, HY = kTY + K - 1, HV = halo_vol<K>();
    extern __shared__ float sm[];
    // channels in and out of this convolution
    const int Ci = DGRAD ? s.Cout : s.Cin, Co = DGRAD ? s.Cin : s.Cout;
    float *xs = sm;                       // [Ci][HV]
    float *ws = sm + (size_t)Ci * HV;     // [Co][Ci][K3] (DGRAD: transposed and flipped)
    const int D = s.D;
    const int ntx = (D + kTX - 1) / kTX, nty = (D + kTY - 1) / kTY;
    int bt = blockIdx.x;
    const int tx0 = (bt % ntx) * kTX;
    bt /= ntx;
    const int ty0 = (bt % nty) * kTY;
    const int tz0 = (bt / nty) * kTZ;
    const int b = blockIdx.y;
    const int64_t D3 = (int64_t)D * D * D;
    for (int e = threadIdx.x; e < Co * Ci * K3; e += blockDim.x) {
        const int t = e % K3, c2 = (e / K3) % Ci, c1 = e / (K3 * Ci);
        // ws[c1][c2][t]: forward w[c1][c2][t]; dgrad w[c2][c1][K3 - 1 - t]
        ws[e] = DGRAD ? bf(w[((int64_t)c2 * s.Cin + c1) * K3 + (K3 - 1 - t)]) : bf(w[e]);
    }
    for (int e = threadIdx.x; e < Ci * HV; e += blockDim.x) {
        const int v = e % HV, c = e / HV;
        const int lx = v % HX, ly = (v / HX) % HY, lz = v / (HX * HY);
        const int gx = tx0 + lx - h, gy = ty0 + ly - h, gz = tz0 + lz - h;
        float val = 0.f;
        if (gx >= 0 && gx < D && gy >= 0 && gy < D && gz >= 0 && gz < D) {
            const int64_t gi = ((int64_t)b * Ci + c) * D3 + ((int64_t)gz * D + gy) * D + gx;
            val = DGRAD ? static_cast<const float *>(xin)[gi] : bf(static_cast<const __nv_bfloat16 *>(xin)[gi]);
        }
        xs[e] = val;
    }
    __syncthreads();
    const int lx = threadIdx.x % kTX, ly = (threadIdx.x / kTX) % kTY, lz = threadIdx.x / (kTX * kTY);
    const int x = tx0 + lx, y = ty0 + ly, z = tz0 + lz;
    if (x >= D || y >= D || z >= D) return;
    float acc[kMaxC];
#pragma unroll
    for (int c = 0; c < kMaxC; ++c) acc[c] = (!DGRAD && bias && c < Co) ? bias[c] : 0.f;
    for (int ci = 0; ci < Ci; ++ci) {
        const float *xc = xs + ci * HV + (lz * HY + ly) * HX + lx;
#pragma unroll
        for (int t = 0; t < K3; ++t) {
            const int dz = t / (K * K), dy = (t / K) % K, dx = t % K;
            const float xv = xc[(dz * HY + dy) * HX + dx];
            const float *wt = ws + ci * K3 + t;
#pragma unroll
            for (int c = 0; c < kMaxC; ++c)
                if (c < Co) acc[c] = fmaf(wt[(size_t)c * Ci * K3], xv, acc[c]);
        }
    }
    const int64_t p = ((int64_t)z * D + y) * D + x;
    for (int c = 0; c < Co; ++c) {
        const int64_t oi = ((int64_t)b * Co + c) * D3 + p;
        float v = acc[c];
        if (DGRAD) {
            if (mask && !(bf(mask[oi]) > 0.f)) v = 0.f;
            yf[oi] = v;
        } else {
            if (relu && v < 0.f) v = 0.f;
            if (ybf) ybf[oi] = __float2bfloat16_rn(v);
            if (yf) yf[oi] = v;
        }
    }
}

// dw[co, ci, t] = sum_{b, p} dy[b, co, p] x[b, ci, p + t - h]: block
// (pair, b) of the grid takes one (co, ci) pair (blockIdx.x < Cout Cin; the
// next Cout values of blockIdx.x sum db[co] = sum dy[b, co, p] instead) and
// one batch entry b (blockIdx.y), walks its tiles of kTX x kTY x kWZ voxels
// (staging the tile of x with its halo), each thread keeping the K^3 sums of
// its kWZ / kTZ voxel slots, and a fixed-order tree reduces them into
// part[b][pair][t]; wgrad_sum_kernel then adds the batch entries in order:
// deterministic.
constexpr int kWZ = 16, kWPer = kWZ / kTZ;   // voxels per thread along z

template <int K>
__global__ void __launch_bounds__(kTileVox) conv_wgrad_tiled_kernel(const float *__restrict__ dy,
                                                                    const __nv_bfloat16 *__restrict__ x,
                                                                    ConvShape s, float *__restrict__ part) {
    constexpr int K3 = K * K * K, h = K / 2;
    constexpr int HX = kTX + K - 1, HY = kTY + K - 1, HZ = kWZ + K - 1, HV = HX * HY * HZ;
    __shared__ float xs[HV];
    __shared__ float red[kTileVox];
    const int D = s.D;
    const int64_t D3 = (int64_t)D * D * D;
    const int ntx = (D + kTX - 1) / kTX, nty = (D + kTY - 1) / kTY, ntz = (D + kWZ - 1) / kWZ;
    const bool bias_block = (int)blockIdx.x >= s.Cout * s.Cin;
    const int co = bias_block ? (int)blockIdx.x - s.Cout * s.Cin : (int)blockIdx.x / s.Cin;
    const int ci = bias_block ? 0 : (int)blockIdx.x % s.Cin;
    const int lx = threadIdx.x % kTX, ly = (threadIdx.x / kTX) % kTY, lz0 = threadIdx.x / (kTX * kTY);
    const int b = blockIdx.y;
    float acc[K3];
#pragma unroll
    for (int t = 0; t < K3; ++t) acc[t] = 0.f;
    {
        for (int tz = 0; tz < ntz; ++tz)
            for (int ty = 0; ty < nty; ++ty)
                for (int tx = 0; tx < ntx; ++tx) {
                    const int tx0 = tx * kTX, ty0 = ty * kTY, tz0 = tz * kWZ;
                    if (!bias_block) {
                        for (int e = threadIdx.x; e < HV; e += blockDim.x) {
                            const int vx = e % HX, vy = (e / HX) % HY, vz = e / (HX * HY);
                            const int gx = tx0 + vx - h, gy = ty0 + vy - h, gz = tz0 + vz - h;
                            xs[e] = (gx >= 0 && gx < D && gy >= 0 && gy < D && gz >= 0 && gz < D)
                                        ? bf(x[((int64_t)b * s.Cin + ci) * D3 + ((int64_t)gz * D + gy) * D + gx])
                                        : 0.f;
                        }
                    }
                    __syncthreads();
                    const int gx = tx0 + lx, gy = ty0 + ly;
#pragma unroll
                    for (int q = 0; q < kWPer; ++q) {
                        const int lz = lz0 + kTZ * q, gz = tz0 + lz;
                        if (gx >= D || gy >= D || gz >= D) continue;
                        const float d = dy[((int64_t)b * s.Cout + co) * D3 + ((int64_t)gz * D + gy) * D + gx];
                        if (bias_block) {
                            acc[0] += d;
                        } else {
                            const float *xc = xs + (lz * HY + ly) * HX + lx;
#pragma unroll
                            for (int t = 0; t < K3; ++t)
                                acc[t] = fmaf(d, xc[((t / (K * K)) * HY + (t / K) % K) * HX + t % K], acc[t]);
                        }
                    }
                    __syncthreads();
                }
    }
    // partial sums of this batch entry: part[b][nw + Cout], weights then biases
    const int64_t nw = (int64_t)s.Cout * s.Cin * K3;
    float *pb = part + (int64_t)b * (nw + s.Cout);
    const int nt = bias_block ? 1 : K3;
    for (int t = 0; t < nt; ++t) {
        red[threadIdx.x] = acc[t];
        __syncthreads();
        for (int o = kTileVox / 2; o > 0; o >>= 1) {
            if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            if (bias_block)
                pb[nw + co] = red[0];
            else
                pb[((int64_t)co * s.Cin + ci) * K3 + t] = red[0];
        }
        __syncthreads();
    }
}

// dw / db = the batch entries' partial sums, added in batch order
__global__ void wgrad_sum_kernel(const float *__restrict__ part, int B, int64_t nw, int Cout,
                                 float *__restrict__ dw, float *__restrict__ db) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nw + Cout;
         i += (int64_t)gridDim.x * blockDim.x) {
        float acc = 0.f;
        for (int b = 0; b < B; ++b) acc += part[(int64_t)b * (nw + Cout) + i];
        if (i < nw)
            dw[i] = acc;
        else if (db)
            db[i - nw] = acc;
    }
}

int nblocks(int64_t n, int t) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (n + t - 1) / t, cap = (int64_t)sms * 32;
    return (int)(want < cap ? (want < 1 ? 1 : want) : cap);
}

bool shape_ok(int B, int Cin, int Cout, int D, int k) {
    return B > 0 && Cin > 0 && Cout > 0 && D > 0 && (k == 1 || k == 3);
}

int status_of(cudaError_t e) { return e == cudaSuccess ? NFFT3_OK : NFFT3_ERR_CUDA; }

template <bool DGRAD, int K>
cudaError_t launch_tiled_k(const void *x, const __nv_bfloat16 *w, const float *bias, const ConvShape &s, int relu,
                           const __nv_bfloat16 *mask, __nv_bfloat16 *ybf, float *yf, cudaStream_t st) {
    const int Ci = DGRAD ? s.Cout : s.Cin, Co = DGRAD ? s.Cin : s.Cout;
    const size_t sm = conv_tiled_smem<K>(Ci, Co);
    cudaError_t e = cudaFuncSetAttribute(conv_tiled_kernel<K, DGRAD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm);
    if (e != cudaSuccess) return e;
    const int ntx = (s.D + kTX - 1) / kTX, nty = (s.D + kTY - 1) / kTY, ntz = (s.D + kTZ - 1) / kTZ;
    const dim3 grid((unsigned)(ntx * nty * ntz), (unsigned)s.B);
    conv_tiled_kernel<K, DGRAD><<<grid, kTileVox, sm, st>>>(x, w, bias, s, relu, mask, ybf, yf);
    return cudaGetLastError();
}

template <bool DGRAD>
cudaError_t launch_tiled(const void *x, const __nv_bfloat16 *w, const float *bias, const ConvShape &s, int relu,
                         const __nv_bfloat16 *mask, __nv_bfloat16 *ybf, float *yf, cudaStream_t st) {
    if (s.B > 65535) return cudaErrorInvalidValue;
    return s.k == 3 ? launch_tiled_k<DGRAD, 3>(x, w, bias, s, relu, mask, ybf, yf, st)
                    : launch_tiled_k<DGRAD, 1>(x, w, bias, s, relu, mask, ybf, yf, st);
}

}  // namespace

extern "C" int cnn_conv3d_fwd(const void *x, const void *w, const float *bias, int B, int Cin,
                              int Cout, int D, int k, int relu, void *y_bf16, float *y_f32,
                              void *stream) {
    if (!x || !w || (!y_bf16 && !y_f32) || !shape_ok(B, Cin, Cout, D, k)) return NFFT3_ERR_ARG;
    const ConvShape s{B, Cin, Cout, D, k};
    if (Cin <= kMaxC && Cout <= kMaxC && !std::getenv("GBNFFT_CNN_NAIVE"))
        return status_of(launch_tiled<false>(x, (const __nv_bfloat16 *)w, bias, s, relu, nullptr,
                                             (__nv_bfloat16 *)y_bf16, y_f32, (cudaStream_t)stream));
    const int64_t total = (int64_t)B * Cout * D * D * D;
    conv_fwd_kernel<<<nblocks(total, 256), 256, 0, (cudaStream_t)stream>>>(
        (const __nv_bfloat16 *)x, (const __nv_bfloat16 *)w, bias, s, relu, (__nv_bfloat16 *)y_bf16, y_f32);
    return status_of(cudaGetLastError());
}

extern "C" int cnn_conv3d_dgrad(const float *dy, const void *w, int B, int Cin, int Cout, int D, int k,
                                const void *relu_mask, float *dx, void *stream) {
    if (!dy || !w || !dx || !shape_ok(B, Cin, Cout, D, k)) return NFFT3_ERR_ARG;
    const ConvShape s{B, Cin, Cout, D, k};
    if (Cin <= kMaxC && Cout <= kMaxC && !std::getenv("GBNFFT_CNN_NAIVE"))
        return status_of(launch_tiled<true>(dy, (const __nv_bfloat16 *)w, nullptr, s, 0,
                                            (const __nv_bfloat16 *)relu_mask, nullptr, dx, (cudaStream_t)stream));
    const int64_t total = (int64_t)B * Cin * D * D * D;
    conv_dgrad_kernel<<<nblocks(total, 256), 256, 0, (cudaStream_t)stream>>>(
        dy, (const __nv_bfloat16 *)w, s, (const __nv_bfloat16 *)relu_mask, dx);
    return status_of(cudaGetLastError());
}

extern "C" int cnn_conv3d_wgrad(const float *dy, const void *x, int B, int Cin, int Cout, int D, int k,
                                float *dw, float *db, void *stream) {
    if (!dy || !x || !dw || !shape_ok(B, Cin, Cout, D, k)) return NFFT3_ERR_ARG;
    const ConvShape s{B, Cin, Cout, D, k};
    if (!std::getenv("GBNFFT_CNN_NAIVE") && B <= 65535) {
        // per-batch-entry partial sums in stream-ordered scratch, then an ordered sum
        const cudaStream_t st = (cudaStream_t)stream;
        const int64_t nw = (int64_t)Cout * Cin * k * k * k;
        float *part = nullptr;
        if (cudaMallocAsync((void **)&part, sizeof(float) * (size_t)B * (nw + Cout), st) != cudaSuccess) {
            cudaGetLastError();
            return NFFT3_ERR_ALLOC;
        }
        const dim3 grid((unsigned)(Cout * Cin + Cout), (unsigned)B);
        if (k == 3)
            conv_wgrad_tiled_kernel<3><<<grid, kTileVox, 0, st>>>(dy, (const __nv_bfloat16 *)x, s, part);
        else
            conv_wgrad_tiled_kernel<1><<<grid, kTileVox, 0, st>>>(dy, (const __nv_bfloat16 *)x, s, part);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) {
            wgrad_sum_kernel<<<nblocks(nw + Cout, 256), 256, 0, st>>>(part, B, nw, Cout, dw, db);
            e = cudaGetLastError();
        }
        cudaFreeAsync(part, st);
        return status_of(e);
    }
    const int nw = Cout * Cin * k * k * k;
    conv_wgrad_kernel<<<nw + (db ? Cout : 0), 256, 0, (cudaStream_t)stream>>>(dy, (const __nv_bfloat16 *)x, s, dw, db);
    return status_of(cudaGetLastError());
}

extern "C" int cnn_core_loss(const float *y, const float *target, const float *off_target, int B, int D,
                             float lam, float pos_weight, float npos, float *dy, float *loss, void *stream) {
    if (!y || !target || !off_target || !dy || !loss || B <= 0 || D <= 0) return NFFT3_ERR_ARG;
    const int64_t total = (int64_t)B * D * D * D;
    core_loss_kernel<<<nblocks(total, 256), 256, 0, (cudaStream_t)stream>>>(y, target, off_target, B, D,
                                                                          lam, pos_weight, npos, dy, loss);
    return status_of(cudaGetLastError());
}

extern "C" int cnn_adam(float *w_master, void *w_bf16, const float *g, float *m1, float *m2, int64_t n,
                        float lr, float b1, float b2, float eps, int step, void *stream) {
    if (!w_master || !g || !m1 || !m2 || n < 0 || step < 1) return NFFT3_ERR_ARG;
    if (n == 0) return NFFT3_OK;
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    adam_kernel<<<nblocks(n, 256), 256, 0, (cudaStream_t)stream>>>(w_master, (__nv_bfloat16 *)w_bf16, g, m1,
                                                                  m2, n, lr, b1, b2, eps, c1, c2);
    return status_of(cudaGetLastError());
}
