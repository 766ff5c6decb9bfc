// Adjoint spread by tile boxes (the first step of the transposed NFFT:
// H[l] += f_j phi(x_j - l / n) over the 2m+1 stencil nodes per dimension),
// one block (or two) per chunk of at most kChunk sorted points of one
// kTile^3 tile.  The stencils of a tile's points lie in the box of
// (kTile + 2m)^3 nodes starting m nodes before the tile, so the block
// accumulates them there and then adds the box to the oversampled grid once
// (node indices wrapped mod n).
// spread_line_df_kernel (FP64, m <= 7): one thread per box line, the nodes
// in registers, rows added by bulk FP64 reductions.  spread_tile_df_kernel
// (FP64, m = 8; double-float half boxes in shared memory, rows of one parity
// in two planes per warp) and spread_tile_f32_kernel (mixed; one plane per
// warp) give each warp its own set of box nodes, so no node update needs an
// atomic, and add the box with global atomics.
#include <cstdint>

#include "col_common.cuh"

namespace gbnfft {
namespace {

// centre node l0 + m (mod n) of a stencil (l0 in [0, n))
__device__ __forceinline__ int tile_centre(int l0, int m, int n) {
    int c = l0 + m;
    while (c >= n) c -= n;
    return c;
}

__device__ __forceinline__ int wrap_node(int v, int n) {
    v %= n;
    return v < 0 ? v + n : v;
}

// wrap[d B + i] = the grid index (mod n_d) of box index i in dimension d; the
// box of tile (tt1, tt2, tt3) starts MM nodes before the tile.  The caller
// synchronises before the first read.
template <int B, int MM>
__device__ __forceinline__ void fill_wrap(int *wrap, int tt1, int tt2, int tt3, Grid3 g) {
    for (int e = threadIdx.x; e < 3 * B; e += blockDim.x) {
        const int d = e / B, i = e - d * B;
        const int tt = d == 0 ? tt1 : d == 1 ? tt2 : tt3, n = d == 0 ? g.n1 : d == 1 ? g.n2 : g.n3;
        wrap[e] = wrap_node(kTile * tt - MM + i, n);
    }
}

// ---- FP64 family: double-float accumulation without atomics ---------------
// GB300's FP64 pipe runs at 1/64 of the FP32 rate, and shared-memory FP64
// atomics add FP64 work of their own; the FP64 family therefore accumulates
// its box in double-float (hi + lo floats) on the FP32 pipe.  Phase 1: the
// block evaluates the tap weights of all the chunk's points by double-float
// Horner (the plan's hi + lo coefficient table, copied to shared memory) and
// stages them as float pairs.  Phase 2: the B warps own disjoint node sets
// and each walks every point of the chunk, adding the point's taps that fall
// in its set; the lanes of a warp take distinct nodes, so the node updates
// need no atomics.  Warp (q, h) owns the rows of parity h in the planes q and
// q + B/2.  A point's 2m+1 stencil planes start at one of the tile's kTile
// first planes, so the middle planes receive every point and the outer ones
// few: one plane per warp left most warps idle while the middle ones worked.
// Pairing plane q with plane q + B/2 evens the planes' loads (within about
// 10 %), and splitting rows by parity keeps the warp count at B.
__device__ __forceinline__ float2 df2_mul(float2 a, float2 b) {
    const float p = __fmul_rn(a.x, b.x);
    float e = __fmaf_rn(a.x, b.x, -p);
    e = __fmaf_rn(a.x, b.y, e);
    e = __fmaf_rn(a.y, b.x, e);
    const float h = __fadd_rn(p, e);
    return make_float2(h, __fsub_rn(e, __fsub_rn(h, p)));
}
__device__ __forceinline__ float2 df2_add(float2 a, float2 b) {
    const float s = __fadd_rn(a.x, b.x);
    const float bb = __fsub_rn(s, a.x);
    float e = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, bb)), __fsub_rn(b.x, bb));
    e = __fadd_rn(e, __fadd_rn(a.y, b.y));
    const float h = __fadd_rn(s, e);
    return make_float2(h, __fsub_rn(e, __fsub_rn(h, s)));
}
__device__ __forceinline__ float2 df2_split(double v) {
    const float h = __double2float_rn(v);
    return make_float2(h, __double2float_rn(v - (double)h));
}

// Each chunk is served by two blocks, one per half of its box (planes
// [0, B/2) and [B/2, B)): a half box and the chunk's staged weights fit twice
// in one SM's shared memory, so two blocks overlap one another's loads,
// barriers and flushes.  Warp (q, h) of a half owns the rows of parity h in
// the half's planes q and B/2 - 1 - q: a point's stencil planes start at one
// of the tile's first kTile planes, so the planes near the middle of the box
// receive every point and the outer ones few, and pairing an outer plane
// with an inner one evens the warps' loads.
//
// Layout of a half box in shared memory: in each plane the rows of even
// index come first, then the odd ones, each row padded to P nodes with
// P = 5 (mod 8).  A warp's lane slots cover consecutive rows of one parity,
// so the 8 lanes of a quarter warp (one 128-byte access of 16-byte nodes)
// take the end of one row and the start of the next; with P = 5 (mod 8)
// their nodes fall in 8 different bank groups.
template <int MM> struct SpreadDF {
    static constexpr int W = 2 * MM + 1, B = kTile + 2 * MM, HB = B / 2;   // HB: planes per half
    static constexpr int NPAIR = (HB + 1) / 2, THREADS = 64 * NPAIR;
    // NR: stencil rows of one parity (at most); NS2: lane slots covering them
    static constexpr int NR = (W + 1) / 2, NS2 = (NR * W + 31) / 32;
    static constexpr int P = B + ((13 - B % 8) % 8);   // row pitch: >= B, = 5 (mod 8)
    static constexpr int PLANE = B * P, NODES = HB * PLANE;   // + 1 spare node
    static_assert(B % 2 == 0, "two halves of B / 2 planes");
    static_assert(P % 8 == 5 && P >= B, "row pitch");
};

// shared memory of the double-float spread: the half box (float4 a node, and
// a spare node for lane slots outside the stencil), the staged weights,
// values and packed box offsets of up to kChunk points, the tap polynomials and the
// wrapped grid indices of the box
template <int MM> constexpr size_t spread_df_smem() {
    using S = SpreadDF<MM>;
    return sizeof(float4) * ((size_t)S::NODES + 1) + sizeof(float2) * (size_t)kChunk * 3 * S::W +
           sizeof(float4) * (size_t)kChunk + sizeof(int) * (size_t)kChunk + sizeof(PolyDF<MM>) +
           sizeof(int) * 3 * S::B;
}

// (double)h + (double)l of a normalised double-float pair (|l| <= ulp(h) / 2)
// with integer instructions (GB300's FP64 pipe is 1/64 of its FP32 rate):
// h's 24-bit significand T sits at bit 52 of an integer, l's is added at its
// binary point (bits of l below 2^-29 ulp(h) truncated), and T is brought
// back to [2^52, 2^53) by at most one shift -- within 2^-51 of the sum.
// Subnormal and non-finite h, and a pair that is not normalised, take the
// FP64 addition.
__device__ __forceinline__ double df_pair_to_double(float h, float l) {
    const unsigned uh = __float_as_uint(h), ul = __float_as_uint(l);
    const int eh = (int)((uh >> 23) & 0xFFu), el = (int)((ul >> 23) & 0xFFu);
    const int sh = el - eh + 29;   // l = ml 2^sh in units of 2^(eh - 179), h = T in those units
    if ((uh & 0x7FFFFFFFu) == 0u) return 0.0;   // h = 0: l = 0 in a normalised pair
    if (eh == 0 || eh == 0xFF || el == 0xFF || (el != 0 && sh > 5)) return (double)h + (double)l;
    long long T = (long long)((uh & 0x7FFFFFu) | 0x800000u) << 29;
    if (el != 0) {
        const long long ml = (long long)((ul & 0x7FFFFFu) | 0x800000u);
        const long long L = sh >= 0 ? (ml << sh) : (sh > -40 ? (ml >> -sh) : 0);
        T += ((uh ^ ul) >> 31) ? -L : L;
    }
    unsigned long long E = (unsigned long long)(eh + 896);   // T in [2^52, 2^53): exponent eh - 127
    if (T >= (1ll << 53)) {
        T >>= 1;
        ++E;
    } else if (T < (1ll << 52)) {
        T <<= 1;
        --E;
    }
    return __longlong_as_double((long long)(((unsigned long long)(uh & 0x80000000u) << 32) | (E << 52) |
                                            ((unsigned long long)T & ((1ull << 52) - 1))));
}

// ---- deterministic flush: exact fixed-point sums ----------------------------
// A float x = M 2^(E - 150) (normal, biased exponent E) as fixed point at
// resolution 2^-60 in two limbs, x ~ hi 2^-30 + lo 2^-60 with |lo| < 2^30,
// bits below 2^-60 dropped (zero and subnormal floats give 0).  Box values
// are below 2^9 in magnitude (f is scaled into [1, 2), at most kChunk points
// with weights <= 1), so hi < 2^39 and a node's sums of at most 2^24 flushes
// stay in int64.  Integer addition is exact and commutative, so the grid
// does not depend on the order of the flushes.
__device__ __forceinline__ void fixed_limbs(float x, long long &hi, long long &lo) {
    const unsigned u = __float_as_uint(x);
    const int E = (int)((u >> 23) & 0xFFu);
    if (E == 0) {
        hi = lo = 0;
        return;
    }
    const unsigned long long M = (u & 0x7FFFFFu) | 0x800000u;
    const int k = E - 90;   // x 2^60 = M 2^k
    unsigned long long h, l;
    if (k >= 30) {
        h = M << (k - 30 < 40 ? k - 30 : 40);
        l = 0;
    } else if (k >= 0) {
        const unsigned long long F = M << k;
        h = F >> 30;
        l = F & ((1ull << 30) - 1);
    } else {
        h = 0;
        l = -k < 32 ? M >> -k : 0;
    }
    const bool neg = (u >> 31) != 0;
    hi = neg ? -(long long)h : (long long)h;
    lo = neg ? -(long long)l : (long long)l;
}

// add the double-float value (h + l) to the node's two limbs
__device__ __forceinline__ void fixed_add(unsigned long long *q, float h, float l) {
    long long a1, b1, a2, b2;
    fixed_limbs(h, a1, b1);
    fixed_limbs(l, a2, b2);
    atomicAdd(q, (unsigned long long)(a1 + a2));
    atomicAdd(q + 1, (unsigned long long)(b1 + b2));
}

// FIXED: flush into the fixed-point grid Hq (four int64 limbs per node: re
// hi, re lo, im hi, im lo) instead of FP64 atomics into H (deterministic
// mode).  zero: a run-time zero for the packed arithmetic (x2_opaque).
template <int MM, bool FIXED>
__global__ void __launch_bounds__(SpreadDF<MM>::THREADS) spread_tile_df_kernel(
    const double2 *__restrict__ f, Grid3 g, PointsView<double> pts, const __grid_constant__ PolyDF<MM> Pt,
    const int4 *__restrict__ chunks, int nt2, int nt3, double2 *__restrict__ H, unsigned long long *__restrict__ Hq,
    f32x2 zero) {
    using S = SpreadDF<MM>;
    constexpr int W = S::W, B = S::B, HB = S::HB, D = kPolyDegDF, P = S::P, PLANE = S::PLANE;
    constexpr int NODES = S::NODES;   // box[NODES]: the spare node
    constexpr int THREADS = S::THREADS, NR = S::NR, NS2 = S::NS2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4 *box = reinterpret_cast<float4 *>(smem_raw);                 // (re hi, im hi, re lo, im lo); + 1 spare
    float2 *wts = reinterpret_cast<float2 *>(box + NODES + 1);            // [point][d][tap]
    float4 *fsm = reinterpret_cast<float4 *>(wts + kChunk * 3 * W);      // f_j as (re hi, im hi, re lo, im lo)
    int *osm = reinterpret_cast<int *>(fsm + kChunk);                    // first node's box indices, packed
    PolyDF<MM> *tab = reinterpret_cast<PolyDF<MM> *>(osm + kChunk);       // double-float tap polynomials
    int *wrap = reinterpret_cast<int *>(tab + 1);                         // grid index of box index i, per dimension
    const int part = blockIdx.x & 1;                                      // planes [part HB, part HB + HB)
    const int4 ch = chunks[blockIdx.x >> 1];
    const int t = ch.x;
    const int tt3 = t % nt3, tt2 = (t / nt3) % nt2, tt1 = t / (nt3 * nt2);
    for (int e = threadIdx.x; e < NODES; e += THREADS) box[e] = make_float4(0.f, 0.f, 0.f, 0.f);
    fill_wrap<B, MM>(wrap, tt1, tt2, tt3, g);
    {
        const float *src = &Pt.ch[0][0][0];
        float *dst = &tab->ch[0][0][0];
        constexpr int NC = 2 * 3 * W * (D + 1);   // ch then cl
        for (int e = threadIdx.x; e < NC; e += THREADS) dst[e] = src[e];
    }
    __syncthreads();
    // phase 1: tap weights by double-float Horner in t = 2s - 1 (FP32 pipe)
    for (int e = threadIdx.x; e < ch.z * 3 * W; e += THREADS) {
        const int i = e / (3 * W), r = e - i * (3 * W), d = r / W, tap = r - d * W;
        const int64_t j = (int64_t)ch.y + i;
        const double s = d == 0 ? pts.s1[j] : d == 1 ? pts.s2[j] : pts.s3[j];
        const float2 tv = df2_split(2.0 * s - 1.0);
        float2 v = make_float2(tab->ch[d][tap][D], tab->cl[d][tap][D]);
#pragma unroll
        for (int k = D - 1; k >= 0; --k)
            v = df2_add(df2_mul(v, tv), make_float2(tab->ch[d][tap][k], tab->cl[d][tap][k]));
        wts[e] = v;
    }
    for (int i = threadIdx.x; i < ch.z; i += THREADS) {
        const int4 key = pts.key[(int64_t)ch.y + i];
        // FP64 family: f enters scaled by 2^s, so the float pairs keep its range
        const double2 fv = scale_value(f[key.w], value_shift(pts.vexp));
        const float2 re = df2_split(fv.x), im = df2_split(fv.y);
        fsm[i] = make_float4(re.x, im.x, re.y, im.y);
        // box indices of the stencil's first node (plane relative to this
        // half, in [-HB, kTile)), packed with a bias of 32 into 6-bit fields
        const int ox = tile_centre(key.x, MM, g.n1) - kTile * tt1 - part * HB;
        const int oy = tile_centre(key.y, MM, g.n2) - kTile * tt2, oz = tile_centre(key.z, MM, g.n3) - kTile * tt3;
        osm[i] = (ox + 32) | (oy << 6) | (oz << 12);
    }
    __syncthreads();
    // phase 2: warp (q, h) owns local planes q and HB - 1 - q (one plane when
    // they coincide), rows of parity h.  Lane slot k covers stencil row
    // b = b0 + 2 r and column c (b0: the point's first row of parity h);
    // slots past the stencil update the spare node box[NODES], so the loop has
    // no branches.  Complex values are packed pairs: hi = (re hi, im hi),
    // lo = (re lo, im lo).
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, h = wid & 1, q0 = wid >> 1;
    const int plane_of[2] = {q0, HB - 1 - q0};
    const bool second = HB - 1 - q0 != q0;
    constexpr int kFar = 1 << 20;   // an offset that sends the slot to the spare node
    // slot k of a lane: stencil row b = b0 + 2 r lies r storage rows after
    // the point's first row of parity h
    int roff[2][NS2], w2o[2][NS2], w3o[NS2];
#pragma unroll
    for (int k = 0; k < NS2; ++k) {
        const int sl = lane + 32 * k;
        const int r = sl < NR * W ? sl / W : 0, c = sl < NR * W ? sl - (sl / W) * W : 0;
#pragma unroll
        for (int b0 = 0; b0 < 2; ++b0) {
            const int b = b0 + 2 * r;
            const bool ok = sl < NR * W && b < W;
            roff[b0][k] = ok ? r * P + c : kFar;
            w2o[b0][k] = ok ? W + b : W;
        }
        w3o[k] = 2 * W + c;
    }
    ulonglong2 *boxp = reinterpret_cast<ulonglong2 *>(box);
    for (int i = 0; i < ch.z; ++i) {
        const int op = osm[i];
        const int4 o = make_int4((op & 63) - 32, (op >> 6) & 63, op >> 12, 0);
        const int b0 = (h - o.y) & 1;   // first stencil row whose box row has parity h
        // storage row of box row o.y + b0 (parity h): h B/2 + (o.y + b0) / 2
        const int srow = h * (B / 2) + ((o.y + b0) >> 1);
        const float2 *wi = wts + i * 3 * W;
        const ulonglong2 fv = reinterpret_cast<const ulonglong2 *>(fsm)[i];
        // the point's nodes in this warp's set are distinct: all are loaded
        // before any is stored, so their updates overlap
        int idx[2][NS2];
        ulonglong2 nv[2][NS2];
#pragma unroll
        for (int pp = 0; pp < 2; ++pp) {
            const int plane = plane_of[pp], a = plane - o.x;
            const bool on = (pp == 0 || second) && a >= 0 && a < W;
            const int base = plane * PLANE + srow * P + o.z;
#pragma unroll
            for (int k = 0; k < NS2; ++k) {
                idx[pp][k] = min(base + (b0 ? roff[1][k] : roff[0][k]), NODES);
                if (on) nv[pp][k] = boxp[idx[pp][k]];
            }
        }
#pragma unroll
        for (int pp = 0; pp < 2; ++pp) {
            const int a = plane_of[pp] - o.x;
            if ((pp == 1 && !second) || a < 0 || a >= W) continue;
            // F = f w1 as packed double-float pairs
            const float2 w1 = wi[a];
            f32x2 fh = 0ull, fl = 0ull;
            x2_df_mac(fh, fl, fv.x, fv.y, x2_pack(w1.x, w1.x), x2_pack(w1.y, w1.y), zero);
            x2_df_norm(fh, fl);
#pragma unroll
            for (int k = 0; k < NS2; ++k) {
                // w2 w3 as an unnormalised pair (product, its error): the
                // multiply-add below only needs |low| within a few ulps
                const float2 u = wi[b0 ? w2o[1][k] : w2o[0][k]], v3 = wi[w3o[k]];
                const float wp = __fmul_rn(u.x, v3.x);
                float we = __fmaf_rn(u.x, v3.x, -wp);
                we = __fmaf_rn(u.x, v3.y, we);
                we = __fmaf_rn(u.y, v3.x, we);
                // node += F w2 w3: exact product, two-sum into the high part,
                // errors into the low part, renormalised so that the low part
                // stays below half an ulp of the high part
                ulonglong2 v = nv[pp][k];
                x2_df_mac(v.x, v.y, fh, fl, x2_pack(wp, wp), x2_pack(we, we), zero);
                x2_df_norm(v.x, v.y);
                boxp[idx[pp][k]] = v;
            }
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < NODES; e += THREADS) {
        const float4 v = box[e];   // (re hi, im hi, re lo, im lo); padding nodes stay zero
        if (v.x == 0.f && v.y == 0.f) continue;
        const int pl = e / PLANE, rem = e - pl * PLANE, sr = rem / P, i3 = rem - sr * P;
        if (i3 >= B) continue;
        const int i1 = pl + part * HB, i2 = sr < B / 2 ? 2 * sr : 2 * (sr - B / 2) + 1;
        const int64_t node = ((int64_t)wrap[i1] * g.n2 + wrap[B + i2]) * g.n3 + wrap[2 * B + i3];
        if (FIXED) {
            fixed_add(Hq + 4 * node, v.x, v.z);
            fixed_add(Hq + 4 * node + 2, v.y, v.w);
        } else {
            double *dst = reinterpret_cast<double *>(H + node);
            atomicAdd(dst, df_pair_to_double(v.x, v.z));
            atomicAdd(dst + 1, df_pair_to_double(v.y, v.w));
        }
    }
}

// ---- FP64 family, line-owned: the box in registers ----------------------------
// Thread (i1, i2) owns the box line of nodes (i1, i2, 0 .. B-1) and keeps
// them in registers as double-float pairs for the whole chunk.  For each
// point whose stencil crosses the line (i1 - ox and i2 - oy both within the
// 2m+1 taps), the thread forms F = f w1(i1 - ox) w2(i2 - oy) once and adds
// F w3(c) to its node oz + c for the 2m+1 taps c.  The chunk's points are
// the same for every thread, so the tap range along the line (oz) is the
// same across a warp and its test costs no divergence; no node is read or
// written in shared memory during the sums.  Lines are numbered i1-major, so
// a warp covers about 1.6 planes: for an average point 9 of the 13 warps
// have a line in its stencil, with 59 % of their lanes active.  After the
// last point each thread converts its line to FP64 in shared memory (lines
// at an odd pitch, which keeps a quarter warp's 16-byte stores in distinct
// banks) and adds it to the grid's row with bulk FP64 reductions by the
// tensor memory accelerator, one per contiguous piece of the row (two where
// the box wraps around the grid).  In deterministic mode the lines stay
// double-float pairs and the box is added in node order as exact fixed-point
// sums, as in the half-box kernel.
template <int MM> struct SpreadLine {
    static constexpr int W = 2 * MM + 1, B = kTile + 2 * MM, NL = B * B;
    static constexpr int THREADS = (NL + 31) / 32 * 32;
    static constexpr int LP = B + 1;   // line pitch of the flush box (nodes)
    // staging: f w1, w2 and w3 as 16-byte pairs per point and tap, f, the
    // packed offsets and the tap polynomials; the flush box reuses the bytes
    static constexpr size_t STAGE = sizeof(float4) * ((size_t)3 * kChunk * W + kChunk) +
                                    sizeof(int) * (size_t)kChunk + sizeof(PolyDF<MM>);
    static constexpr size_t BOX = sizeof(float4) * (size_t)NL * LP;
    static constexpr size_t UNION = ((STAGE > BOX ? STAGE : BOX) + 15) / 16 * 16;
    static constexpr size_t SMEM = UNION + sizeof(int) * 3 * B;
};

// node O + c += F w3(c) for the 2m+1 taps c, renormalised after each
// addition, for the point's first stencil node O = oz along the line: one
// straight run of independent updates per value of oz, so that the code
// generator can interleave their dependent chains (the node index must be a
// constant for the nodes to stay in registers)
template <int O, int B, int W>
__device__ __forceinline__ void line_taps(int oz, f32x2 (&acch)[B], f32x2 (&accl)[B], f32x2 Fh, f32x2 nFh,
                                          f32x2 nFl, const ulonglong2 *__restrict__ w3, f32x2 zero) {
    if constexpr (O + W <= B) {
        if (oz == O) {
#pragma unroll
            for (int c = 0; c < W; ++c) {
                const ulonglong2 wv = w3[c];
                x2_df_mac_neg(acch[O + c], accl[O + c], Fh, nFh, nFl, wv.x, wv.y, zero);
                x2_df_norm(acch[O + c], accl[O + c]);
            }
        } else {
            line_taps<O + 1, B, W>(oz, acch, accl, Fh, nFh, nFl, w3, zero);
        }
    }
}

// dst[0 .. bytes) += src[0 .. bytes) element by element in FP64, by the
// tensor memory accelerator (each element's addition is atomic); both
// addresses 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_add_f64(double *dst, const void *src, unsigned bytes) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(src);
    asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.f64 [%0], [%1], %2;"
                 :: "l"(dst), "r"(sa), "r"(bytes) : "memory");
}

template <int MM, bool FIXED>
__global__ void __launch_bounds__(SpreadLine<MM>::THREADS, 1) spread_line_df_kernel(
    const double2 *__restrict__ f, Grid3 g, PointsView<double> pts, const WinTableDF *__restrict__ wt,
    const int4 *__restrict__ chunks, int nt2, int nt3, double2 *__restrict__ H, unsigned long long *__restrict__ Hq,
    f32x2 zero) {
    using S = SpreadLine<MM>;
    constexpr int W = S::W, B = S::B, NL = S::NL, THREADS = S::THREADS, LP = S::LP, D = kPolyDegDF;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ulonglong2 *Gs = reinterpret_cast<ulonglong2 *>(smem_raw);     // [point][a] f w1: (re, im hi), (re, im lo)
    ulonglong2 *w2s = Gs + kChunk * W;                              // [point][b] w2: (hi, hi), (lo, lo)
    ulonglong2 *w3s = w2s + kChunk * W;                             // [point][c] w3: (hi, hi), (lo, lo)
    float4 *fsm = reinterpret_cast<float4 *>(w3s + kChunk * W);    // f: (re hi, im hi, re lo, im lo)
    int *osm = reinterpret_cast<int *>(fsm + kChunk);              // first stencil node's box indices, packed
    PolyDF<MM> *tab = reinterpret_cast<PolyDF<MM> *>(osm + kChunk);
    float4 *box = reinterpret_cast<float4 *>(smem_raw);            // flush: [line][i3], pitch LP
    int *wrap = reinterpret_cast<int *>(smem_raw + S::UNION);
    const int4 ch = chunks[blockIdx.x];
    const int t = ch.x;
    const int tt3 = t % nt3, tt2 = (t / nt3) % nt2, tt1 = t / (nt3 * nt2);
    fill_wrap<B, MM>(wrap, tt1, tt2, tt3, g);
    {
        // the plan's table in device memory (read by every block, so it stays
        // in L2): rows of D + 1 coefficients, consecutive threads on
        // consecutive addresses
        // (all of a thread's loads first, so that they wait on L2 once)
        constexpr int NR = 3 * W * (D + 1), PER = (2 * NR + THREADS - 1) / THREADS;
        float *dst = &tab->ch[0][0][0];   // ch then cl
        float v[PER];
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int e = threadIdx.x + q * THREADS, ee = e < 2 * NR ? e : 0;
            const int which = ee / NR, r = ee - which * NR, row = r / (D + 1), k = r - row * (D + 1);
            const int d = row / W, tap = row - d * W;
            v[q] = which ? wt->cl[d][tap][k] : wt->ch[d][tap][k];
        }
#pragma unroll
        for (int q = 0; q < PER; ++q)
            if (threadIdx.x + q * THREADS < 2 * NR) dst[threadIdx.x + q * THREADS] = v[q];
    }
    for (int i = threadIdx.x; i < ch.z; i += THREADS) {
        const int4 key = pts.key[(int64_t)ch.y + i];
        // f enters scaled by 2^s, so the float pairs keep its range
        const double2 fv = scale_value(f[key.w], value_shift(pts.vexp));
        const float2 re = df2_split(fv.x), im = df2_split(fv.y);
        fsm[i] = make_float4(re.x, im.x, re.y, im.y);
        // box indices of the stencil's first node, each in [0, kTile)
        const int ox = tile_centre(key.x, MM, g.n1) - kTile * tt1;
        const int oy = tile_centre(key.y, MM, g.n2) - kTile * tt2, oz = tile_centre(key.z, MM, g.n3) - kTile * tt3;
        osm[i] = ox | (oy << 6) | (oz << 12);
    }
    __syncthreads();
    // tap weights by double-float Horner in t = 2s - 1.  Item (i, d, g)
    // evaluates the taps g, g + TG, g + 2 TG, ... of dimension d of point i,
    // their Horner chains side by side (the steps of one chain depend on one
    // another, those of different taps do not).  The first dimension's
    // weights are multiplied by f here, once per point and tap.
    constexpr int TG = (W + 3) / 4, NT = (W + TG - 1) / TG;
    for (int e = threadIdx.x; e < ch.z * 3 * TG; e += THREADS) {
        const int i = e / (3 * TG), r = e - i * (3 * TG), d = r / TG, g0 = r - d * TG;
        const int64_t j = (int64_t)ch.y + i;
        const double s = d == 0 ? pts.s1[j] : d == 1 ? pts.s2[j] : pts.s3[j];
        const float2 tv = df2_split(2.0 * s - 1.0);
        float vh[NT], vl[NT];
#pragma unroll
        for (int q = 0; q < NT; ++q) {
            const int tap = min(g0 + TG * q, W - 1);   // a tap past W: computed, not stored
            vh[q] = tab->ch[d][tap][D];
            vl[q] = tab->cl[d][tap][D];
        }
#pragma unroll
        for (int k = D - 1; k >= 0; --k)
#pragma unroll
            for (int q = 0; q < NT; ++q) {
                const int tap = min(g0 + TG * q, W - 1);
                df_horner_step(vh[q], vl[q], tv.x, tv.y, tab->ch[d][tap][k], tab->cl[d][tap][k]);
            }
#pragma unroll
        for (int q = 0; q < NT; ++q) {
            const int tap = g0 + TG * q;
            if (tap >= W) break;
            if (d == 0) {
                const float4 fv = fsm[i];
                const float2 v = make_float2(vh[q], vl[q]);
                const float2 re = df2_mul(make_float2(fv.x, fv.z), v), im = df2_mul(make_float2(fv.y, fv.w), v);
                Gs[i * W + tap] = make_ulonglong2(x2_pack(re.x, im.x), x2_pack(re.y, im.y));
            } else {
                (d == 1 ? w2s : w3s)[i * W + tap] =
                    make_ulonglong2(x2_pack(vh[q], vh[q]), x2_pack(vl[q], vl[q]));
            }
        }
    }
    __syncthreads();
    const int line = threadIdx.x;
    const int i1 = line < NL ? line / B : B, i2 = line - (line / B) * B;   // i1 = B: a lane with no line
    f32x2 acch[B], accl[B];   // node (i1, i2, j): (re, im) hi and lo
#pragma unroll
    for (int j = 0; j < B; ++j) acch[j] = accl[j] = 0ull;
    for (int i = 0; i < ch.z; ++i) {
        const int op = osm[i];
        const int a = i1 - (op & 63), b = i2 - ((op >> 6) & 63);
        if ((unsigned)a >= (unsigned)W || (unsigned)b >= (unsigned)W) continue;
        const int oz = op >> 12;
        // F = f w1 w2 as packed double-float pairs
        const ulonglong2 G = Gs[i * W + a], w2 = w2s[i * W + b];
        f32x2 Fh, Fl;
        x2_df_mul(Fh, Fl, G.x, G.y, w2.x, w2.y, zero);
        // -F, made opaque so that no product of F is folded against it
        const f32x2 nFh = x2_opaque(x2_sub(0ull, Fh), zero), nFl = x2_opaque(x2_sub(0ull, Fl), zero);
        line_taps<0, B, W>(oz, acch, accl, Fh, nFh, nFl, w3s + i * W, zero);
    }
    __syncthreads();   // the staging bytes become the flush box
    if constexpr (!FIXED) {
        // each thread turns its line into FP64 and adds it to the grid row by
        // row with bulk reductions (split where the row wraps around the grid)
        if (line < NL) {
            double2 *row = reinterpret_cast<double2 *>(box) + line * LP;
            f32x2 any = 0ull;
#pragma unroll
            for (int j = 0; j < B; ++j) {
                float rh, ih, rl, il;
                x2_unpack(acch[j], rh, ih);
                x2_unpack(accl[j], rl, il);
                row[j] = make_double2(df_pair_to_double(rh, rl), df_pair_to_double(ih, il));
                any |= acch[j];
            }
            if (any != 0ull) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // the row, to the copy engine
                double *grow = reinterpret_cast<double *>(H + ((int64_t)wrap[i1] * g.n2 + wrap[B + i2]) * g.n3);
                for (int j = 0; j < B;) {
                    const int c3 = wrap[2 * B + j], run = min(B - j, g.n3 - c3);
                    bulk_add_f64(grow + 2 * (int64_t)c3, row + j, 16u * (unsigned)run);
                    j += run;
                }
            }
        }
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");   // the rows have been read
    } else {
        if (line < NL) {
            ulonglong2 *row = reinterpret_cast<ulonglong2 *>(box + line * LP);
#pragma unroll
            for (int j = 0; j < B; ++j) row[j] = make_ulonglong2(acch[j], accl[j]);
        }
        __syncthreads();
        // exact fixed-point sums, U nodes a thread at a time
        constexpr int NN = NL * B, U = 4;
        for (int e0 = threadIdx.x; e0 < NN; e0 += U * THREADS) {
            float4 v[U];
            int64_t node[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int e = e0 + u * THREADS, ee = e < NN ? e : NN - 1;
                const int ln = ee / B, i3 = ee - ln * B, l1 = ln / B, l2 = ln - l1 * B;
                v[u] = e < NN ? box[ln * LP + i3] : make_float4(0.f, 0.f, 0.f, 0.f);   // (re hi, im hi, re lo, im lo)
                node[u] = ((int64_t)wrap[l1] * g.n2 + wrap[B + l2]) * g.n3 + wrap[2 * B + i3];
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (v[u].x == 0.f && v[u].y == 0.f) continue;
                fixed_add(Hq + 4 * node[u], v[u].x, v[u].z);
                fixed_add(Hq + 4 * node[u] + 2, v[u].y, v[u].w);
            }
        }
    }
}

// H[node] = the fixed-point limbs as FP64 (deterministic mode)
__global__ void fixed_to_grid_kernel(const unsigned long long *__restrict__ Hq, double2 *__restrict__ H,
                                     int64_t total) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const long long *q = reinterpret_cast<const long long *>(Hq + 4 * e);
        H[e] = make_double2((double)q[0] * 0x1p-30 + (double)q[1] * 0x1p-60,
                            (double)q[2] * 0x1p-30 + (double)q[3] * 0x1p-60);
    }
}

// ---- mixed family: plane-owned FP32 box, no atomics in shared memory ------
// The block stages the chunk's tap weights (FP32 Horner), then warp p owns
// box plane p and adds every point's taps in that plane with plain
// shared-memory updates.  (Plane pairs with row parity, as in the FP64
// kernel, measured 9.1 against 8.4 ms here.)
template <int MM> constexpr size_t spread_f32_smem() {
    constexpr int W = 2 * MM + 1, B = kTile + 2 * MM;
    return sizeof(float2) * (size_t)B * B * B + sizeof(float) * (size_t)kChunk * 3 * W +
           sizeof(float2) * (size_t)kChunk + sizeof(int4) * (size_t)kChunk + sizeof(Poly<float, MM>) +
           sizeof(int) * 3 * B;
}

template <int MM>
__global__ void __launch_bounds__(32 * (kTile + 2 * MM)) spread_tile_f32_kernel(
    const float2 *__restrict__ f, Grid3 g, PointsView<float> pts, const __grid_constant__ Poly<float, MM> P,
    const int4 *__restrict__ chunks, int nt2, int nt3, float2 *__restrict__ H) {
    constexpr int W = 2 * MM + 1, B = kTile + 2 * MM, B3 = B * B * B, D = PolyDeg<float>::value;
    constexpr int THREADS = 32 * B, NSLOT = (W * W + 31) / 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *box = reinterpret_cast<float2 *>(smem_raw);                  // (re, im) per node
    float *wts = reinterpret_cast<float *>(box + B3);                     // [point][d][tap]
    float2 *fsm = reinterpret_cast<float2 *>(wts + kChunk * 3 * W);      // f_j
    int4 *osm = reinterpret_cast<int4 *>(fsm + kChunk);                  // box index of the first node
    Poly<float, MM> *tab = reinterpret_cast<Poly<float, MM> *>(osm + kChunk);
    int *wrap = reinterpret_cast<int *>(tab + 1);                         // grid index of box index i, per dimension
    const int4 ch = chunks[blockIdx.x];
    const int t = ch.x;
    const int tt3 = t % nt3, tt2 = (t / nt3) % nt2, tt1 = t / (nt3 * nt2);
    for (int e = threadIdx.x; e < B3; e += THREADS) box[e] = make_float2(0.f, 0.f);
    fill_wrap<B, MM>(wrap, tt1, tt2, tt3, g);
    {
        const float *src = &P.c[0][0][0];
        float *dst = &tab->c[0][0][0];
        for (int e = threadIdx.x; e < 3 * W * (D + 1); e += THREADS) dst[e] = src[e];
    }
    __syncthreads();
    // phase 1
    for (int e = threadIdx.x; e < ch.z * 3 * W; e += THREADS) {
        const int i = e / (3 * W), r = e - i * (3 * W), d = r / W, tap = r - d * W;
        const int64_t j = (int64_t)ch.y + i;
        const float s = d == 0 ? pts.s1[j] : d == 1 ? pts.s2[j] : pts.s3[j];
        const float tv = 2.f * s - 1.f;
        float v = tab->c[d][tap][D];
#pragma unroll
        for (int k = D - 1; k >= 0; --k) v = fmaf(v, tv, tab->c[d][tap][k]);
        wts[e] = v;
    }
    for (int i = threadIdx.x; i < ch.z; i += THREADS) {
        const int4 key = pts.key[(int64_t)ch.y + i];
        fsm[i] = f[key.w];
        osm[i] = make_int4(tile_centre(key.x, MM, g.n1) - kTile * tt1, tile_centre(key.y, MM, g.n2) - kTile * tt2,
                           tile_centre(key.z, MM, g.n3) - kTile * tt3, 0);
    }
    __syncthreads();
    // phase 2: warp p owns box plane p; a point's nodes in the plane are
    // distinct, so all are loaded before any is stored
    const int lane = threadIdx.x & 31, plane = threadIdx.x >> 5;
    for (int i = 0; i < ch.z; ++i) {
        const int4 o = osm[i];
        const int a = plane - o.x;
        if (a < 0 || a >= W) continue;
        const float *wi = wts + i * 3 * W;
        const float2 fv = fsm[i];
        const float w1 = wi[a];
        const float fr = fv.x * w1, fi = fv.y * w1;
        float2 *row = box + plane * B * B;
        int idx[NSLOT];
        float2 nv[NSLOT];
#pragma unroll
        for (int k = 0; k < NSLOT; ++k) {
            const int slot = lane + 32 * k;
            const int b = slot / W, c = slot - b * W;
            idx[k] = slot < W * W ? (o.y + b) * B + (o.z + c) : -1;
            if (idx[k] >= 0) nv[k] = row[idx[k]];
        }
#pragma unroll
        for (int k = 0; k < NSLOT; ++k) {
            if (idx[k] < 0) continue;
            const int slot = lane + 32 * k;
            const int b = slot / W, c = slot - b * W;
            const float w23 = wi[W + b] * wi[2 * W + c];
            row[idx[k]] = make_float2(fmaf(fr, w23, nv[k].x), fmaf(fi, w23, nv[k].y));
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < B3; e += THREADS) {
        const float2 v = box[e];
        if (v.x == 0.f && v.y == 0.f) continue;
        const int i1 = e / (B * B), i2 = (e / B) % B, i3 = e % B;
        const int64_t node = ((int64_t)wrap[i1] * g.n2 + wrap[B + i2]) * g.n3 + wrap[2 * B + i3];
        float *dst = reinterpret_cast<float *>(H + node);
        atomicAdd(dst, v.x);
        atomicAdd(dst + 1, v.y);
    }
}

// the line-owned FP64 kernel serves m <= 7
template <int MM> constexpr bool kLineSpread = MM <= 7;

template <typename R, int MM>
cudaError_t spread_tile_dispatch(const typename Cplx<R>::T *f, Grid3 g, PointsView<R> pts, const WinTable<R> &w,
                                 const WinTableDF *wdf, const WinTableDF *wdf_dev, const int4 *chunks, int nchunks,
                                 int nt2, int nt3, typename Cplx<R>::T *H, unsigned long long *Hq, cudaStream_t st) {
    constexpr int B = kTile + 2 * MM;
    if constexpr (sizeof(R) == 4) {
        if (Hq) return cudaErrorInvalidValue;   // deterministic mode: FP64 family only
        constexpr size_t smem_f = spread_f32_smem<MM>();
        auto kern = spread_tile_f32_kernel<MM>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_f);
        if (e != cudaSuccess) return e;
        kern<<<(unsigned)nchunks, 32 * B, smem_f, st>>>(f, g, pts, make_poly<float, MM>(w), chunks, nt2, nt3, H);
    } else {
        static_assert(spread_df_smem<MM>() <= 227 * 1024, "half box and staged weights fit one block");
        if (!wdf) return cudaErrorInvalidValue;
        if constexpr (kLineSpread<MM>) {
            // FP64 family, m <= 7: one thread per box line, nodes in registers
            constexpr size_t smem_l = SpreadLine<MM>::SMEM;
            static_assert(smem_l <= 227 * 1024, "flush box fits one block");
            if (!wdf_dev || (reinterpret_cast<uintptr_t>(H) & 15u)) return cudaErrorInvalidValue;
            auto kern = Hq ? spread_line_df_kernel<MM, true> : spread_line_df_kernel<MM, false>;
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_l);
            if (e != cudaSuccess) return e;
            kern<<<(unsigned)nchunks, SpreadLine<MM>::THREADS, smem_l, st>>>(f, g, pts, wdf_dev, chunks, nt2, nt3, H,
                                                                              Hq, 0ull);
            return cudaGetLastError();
        }
        // m = 8: the half-box kernel (a line of 24 nodes does not fit the
        // registers of 576 threads)
        constexpr size_t smem_df = spread_df_smem<MM>();
        auto kern = Hq ? spread_tile_df_kernel<MM, true> : spread_tile_df_kernel<MM, false>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_df);
        if (e != cudaSuccess) return e;
        // two blocks per chunk, one per half box
        kern<<<2u * (unsigned)nchunks, SpreadDF<MM>::THREADS, smem_df, st>>>(f, g, pts, make_poly_df<MM>(*wdf),
                                                                            chunks, nt2, nt3, H, Hq, 0ull);
    }
    return cudaGetLastError();
}

}  // namespace

template <typename R>
cudaError_t launch_spread_tiles(const typename Cplx<R>::T *f, Grid3 g, int m, PointsView<R> pts,
                                const WinTable<R> &w, const WinTableDF *wdf, const WinTableDF *wdf_dev,
                                const int4 *chunks, int nchunks, int nt2, int nt3, typename Cplx<R>::T *H,
                                unsigned long long *Hq, cudaStream_t st) {
    if (nchunks <= 0) return cudaSuccess;
    switch (m) {
        case 1: return spread_tile_dispatch<R, 1>(f, g, pts, w, wdf, wdf_dev, chunks, nchunks, nt2, nt3, H, Hq, st);
        case 2: return spread_tile_dispatch<R, 2>(f, g, pts, w, wdf, wdf_dev, chunks, nchunks, nt2, nt3, H, Hq, st);
        case 3: return spread_tile_dispatch<R, 3>(f, g, pts, w, wdf, wdf_dev, chunks, nchunks, nt2, nt3, H, Hq, st);
        case 4: return spread_tile_dispatch<R, 4>(f, g, pts, w, wdf, wdf_dev, chunks, nchunks, nt2, nt3, H, Hq, st);
        case 5: return spread_tile_dispatch<R, 5>(f, g, pts, w, wdf, wdf_dev, chunks, nchunks, nt2, nt3, H, Hq, st);
        case 6: return spread_tile_dispatch<R, 6>(f, g, pts, w, wdf, wdf_dev, chunks, nchunks, nt2, nt3, H, Hq, st);
        case 7: return spread_tile_dispatch<R, 7>(f, g, pts, w, wdf, wdf_dev, chunks, nchunks, nt2, nt3, H, Hq, st);
        case 8: return spread_tile_dispatch<R, 8>(f, g, pts, w, wdf, wdf_dev, chunks, nchunks, nt2, nt3, H, Hq, st);
        default: return cudaErrorInvalidValue;
    }
}

template cudaError_t launch_spread_tiles<double>(const double2 *, Grid3, int, PointsView<double>,
                                                 const WinTable<double> &, const WinTableDF *, const WinTableDF *,
                                                 const int4 *, int,
                                                 int, int, double2 *, unsigned long long *, cudaStream_t);
template cudaError_t launch_spread_tiles<float>(const float2 *, Grid3, int, PointsView<float>,
                                                const WinTable<float> &, const WinTableDF *, const WinTableDF *,
                                                const int4 *, int,
                                                int, int, float2 *, unsigned long long *, cudaStream_t);

cudaError_t launch_fixed_to_grid(const unsigned long long *Hq, double2 *H, int64_t total, cudaStream_t st) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (total + 255) / 256, cap = (int64_t)sms * 16;
    fixed_to_grid_kernel<<<(unsigned)(want < cap ? (want < 1 ? 1 : want) : cap), 256, 0, st>>>(Hq, H, total);
    return cudaGetLastError();
}

}  // namespace gbnfft
