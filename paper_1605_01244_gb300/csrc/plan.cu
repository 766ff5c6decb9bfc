// C ABI of gbnfft: plans, tables, cuFFT, and the eval / eval_grad / adjoint
// sequences.  Kernels live in kernels.cu and points.cu.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include "internal.cuh"
#include "plan_state.cuh"

using namespace gbnfft;

namespace {

int ensure_pgrid(nfft3_plan p, int ng);

enum { kFaultNone = 0, kFaultAlloc = 1, kFaultFftPlan = 2 };

int read_fault_env() {
    const char *v = std::getenv("GBNFFT_FAULT");
    if (!v) return kFaultNone;
    if (!std::strcmp(v, "alloc")) return kFaultAlloc;
    if (!std::strcmp(v, "fft_plan")) return kFaultFftPlan;
    return kFaultNone;
}

int dev_alloc(nfft3_plan p, void **ptr, size_t bytes) {
    *ptr = nullptr;
    if (p->fault == kFaultAlloc) return NFFT3_ERR_ALLOC;
    if (bytes == 0) bytes = 16;
    if (cudaMalloc(ptr, bytes) != cudaSuccess) {
        cudaGetLastError();  // clear the sticky-free allocation error
        *ptr = nullptr;
        return NFFT3_ERR_ALLOC;
    }
    return NFFT3_OK;
}

void dev_free(void *&ptr) {
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
}

int cuda_status(cudaError_t e) { return e == cudaSuccess ? NFFT3_OK : NFFT3_ERR_CUDA; }

void release_deterministic(nfft3_plan p) {
    void *v;
    v = p->ss.buf; dev_free(v);
    v = p->ss.counts; dev_free(v);
    v = p->ss.offsets; dev_free(v);
    v = p->ss.scan_tmp; dev_free(v);
    v = p->Hq; dev_free(v);
    p->ss = StableSort{nullptr, nullptr, nullptr, nullptr};
    p->Hq = nullptr;
    p->det = 0;
}

// Twiddle table exp(+2 pi i j / n_d), j in [0, n_d), from long double cos/sin:
// double-float (cos_hi, cos_lo, sin_hi, sin_lo) for the FP64 family, float2
// for the mixed family.
int make_twiddles(nfft3_plan p, int d) {
    const int L = p->n[d];
    const size_t elem = p->prec == 64 ? 4 * sizeof(float) : 2 * sizeof(float);
    float *h = (float *)std::malloc(elem * L);
    if (!h) return NFFT3_ERR_ALLOC;
    const long double two_pi = 6.283185307179586476925286766559005768L;
    for (int j = 0; j < L; ++j) {
        const long double a = two_pi * (long double)j / (long double)L;
        const long double cr = cosl(a), si = sinl(a);
        if (p->prec == 64) {
            const float ch = (float)cr, sh = (float)si;
            h[4 * j + 0] = ch;
            h[4 * j + 1] = (float)(cr - (long double)ch);
            h[4 * j + 2] = sh;
            h[4 * j + 3] = (float)(si - (long double)sh);
        } else {
            h[2 * j + 0] = (float)cr;
            h[2 * j + 1] = (float)si;
        }
    }
    int st = dev_alloc(p, &p->tw[d], elem * L);
    if (st == NFFT3_OK) st = cuda_status(cudaMemcpy(p->tw[d], h, elem * L, cudaMemcpyHostToDevice));
    std::free(h);
    return st;
}

// Line-pass buffers of the fused transform for ng grids.
int ensure_fscratch(nfft3_plan p, int ng) {
    if (p->fscratch && p->fscratch_ng >= ng) return NFFT3_OK;
    dev_free(p->fscratch);
    p->fscratch_ng = 0;
    const int st = dev_alloc(p, &p->fscratch, fused_scratch_bytes(p->N, p->n, ng, p->prec));
    if (st == NFFT3_OK) p->fscratch_ng = ng;
    return st;
}

// ---- stage timing ----------------------------------------------------------
// A record holds up to kTimingMarks events of one call; stage i of the call
// spans marks i..i+1.  Records are folded into stage_ms when the pool fills
// or when nfft3_timing_read is called.
enum { kRecSetPoints = 0, kRecEval = 1, kRecGrad = 2, kRecAdjoint = 3 };

void fold_records(nfft3_plan p) {
    // stages spanned by consecutive marks, per record kind (-1: unused span)
    static const int kSpans[4][kTimingMarks - 1] = {
        {NFFT3_STAGE_SET_POINTS, -1, -1, -1},
        {NFFT3_STAGE_DECONV, NFFT3_STAGE_FFT, NFFT3_STAGE_SPLIT, NFFT3_STAGE_GATHER},
        {NFFT3_STAGE_DECONV, NFFT3_STAGE_FFT, NFFT3_STAGE_SPLIT, NFFT3_STAGE_GATHER},
        {NFFT3_STAGE_SPREAD, NFFT3_STAGE_FFT_FWD, NFFT3_STAGE_DECONV_ADJ, -1}};
    for (int r = 0; r < p->nrec; ++r) {
        cudaEventSynchronize(p->ev[r][kTimingMarks - 1]);
        const int kind = p->rec_kind[r];
        for (int i = 0; i < kTimingMarks - 1; ++i) {
            const int st = kSpans[kind][i];
            if (st < 0) continue;
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, p->ev[r][i], p->ev[r][i + 1]) == cudaSuccess) {
                p->stage_ms[st] += ms;
                p->stage_calls[st] += 1;
            }
        }
    }
    p->nrec = 0;
    cudaGetLastError();
}

// start a record; returns its index or -1 when timing is off
int rec_begin(nfft3_plan p, int kind) {
    if (!p->timing) return -1;
    if (p->nrec == kTimingRecords) fold_records(p);
    const int r = p->nrec++;
    if (!p->ev_ready[r]) {
        for (int i = 0; i < kTimingMarks; ++i) cudaEventCreate(&p->ev[r][i]);
        p->ev_ready[r] = 1;
    }
    p->rec_kind[r] = kind;
    cudaEventRecord(p->ev[r][0], p->stream);
    return r;
}

void rec_mark(nfft3_plan p, int r, int i) {
    if (r >= 0) cudaEventRecord(p->ev[r][i], p->stream);
}

// fill the marks a call did not use, so that every record ends at mark kTimingMarks-1
void rec_end(nfft3_plan p, int r, int last_used) {
    if (r < 0) return;
    for (int i = last_used + 1; i < kTimingMarks; ++i) cudaEventRecord(p->ev[r][i], p->stream);
}

// Modified Bessel function I0 by its power series sum_k ((x/2)^{2k} / (k!)^2);
// all terms are positive, so the sum is accurate to rounding for the
// arguments used here (x < 60).
double bessel_i0(double x) {
    const double t = 0.25 * x * x;
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 1000; ++k) {
        term *= t / ((double)k * (double)k);
        sum += term;
        if (term < 1e-17 * sum) break;
    }
    return sum;
}

bool small_primes_only(int v) {
    for (int p : {2, 3, 5, 7})
        while (v % p == 0) v /= p;
    return v == 1;
}

int oversampled_size(int N, double sigma) {
    int n = (int)std::ceil(sigma * (double)N - 1e-9);
    if (n < N) n = N;
    if (n % 2) ++n;
    while (!small_primes_only(n)) n += 2;
    return n;
}

// relative l2 error estimate of the window at cutoff m and oversampling sigma
double error_estimate(int m, double sigma) {
    return 8.0 * std::exp(-2.0 * M_PI * std::sqrt(1.0 - 1.0 / sigma) * (m + 0.5));
}

// ---- window polynomials -----------------------------------------------------
// Exact normalised window weight of tap a at offset s (long double):
//   tau = alpha - s - a,  q^2 = alpha^2 - tau^2 = (s + a)(2m + 1 - s - a),
//   w = (alpha / q) sinh(b q) / sinh(b alpha)
//     = alpha / (1 - e^{-2 b alpha}) * exp(-b tau^2 / (q + alpha)) * (-expm1(-2 b q) / q),
// written so that no step cancels (q - alpha = -tau^2 / (q + alpha)); q = 0 gives 2b for the last factor.
long double exact_weight(long double s, int a, int m, long double b) {
    const long double al = (long double)m + 0.5L;
    const long double tau = al - s - (long double)a;
    const long double q2 = (s + (long double)a) * ((long double)(2 * m + 1) - s - (long double)a);
    const long double q = q2 > 0 ? sqrtl(q2) : 0.0L;
    const long double r = q > 0 ? -expm1l(-2.0L * b * q) / q : 2.0L * b;
    return al / (1.0L - expl(-2.0L * b * al)) * expl(-b * tau * tau / (q + al)) * r;
}

// Degree-D interpolant of w_a(s) for s in [s0, s1] at the Chebyshev nodes of
// t = (2s - s0 - s1) / (s1 - s0) in [-1, 1], returned as monomial
// coefficients in t (mono[k] multiplies t^k).  The whole interval [0, 1]
// gives t = 2s - 1; the upper half [1/2, 1] gives t = 4s - 3.
void fit_tap(int a, int m, long double b, int D, long double *mono, long double s0 = 0.0L,
             long double s1 = 1.0L) {
    const long double pi = acosl(-1.0L);
    long double f[kMaxCoef], cheb[kMaxCoef], Tm[kMaxCoef], T0[kMaxCoef], T1[kMaxCoef];
    for (int j = 0; j <= D; ++j) {
        const long double t = cosl(pi * ((long double)j + 0.5L) / (long double)(D + 1));
        f[j] = exact_weight(s0 + 0.5L * (s1 - s0) * (t + 1.0L), a, m, b);
    }
    for (int k = 0; k <= D; ++k) {
        long double acc = 0;
        for (int j = 0; j <= D; ++j)
            acc += f[j] * cosl(pi * (long double)k * ((long double)j + 0.5L) / (long double)(D + 1));
        cheb[k] = 2.0L * acc / (long double)(D + 1);
    }
    cheb[0] *= 0.5L;
    for (int k = 0; k < kMaxCoef; ++k) mono[k] = 0, T0[k] = 0, T1[k] = 0;
    T0[0] = 1;  // T_0
    T1[1] = 1;  // T_1
    for (int k = 0; k <= D; ++k) mono[k] += cheb[0] * T0[k];
    if (D >= 1)
        for (int k = 0; k <= D; ++k) mono[k] += cheb[1] * T1[k];
    for (int n = 2; n <= D; ++n) {
        // T_n = 2 t T_{n-1} - T_{n-2}
        for (int k = 0; k <= D; ++k) Tm[k] = (k > 0 ? 2.0L * T1[k - 1] : 0.0L) - T0[k];
        for (int k = 0; k <= D; ++k) {
            mono[k] += cheb[n] * Tm[k];
            T0[k] = T1[k];
            T1[k] = Tm[k];
        }
    }
}

template <typename R> R host_fma(R a, R b, R c);
template <> double host_fma<double>(double a, double b, double c) { return std::fma(a, b, c); }
template <> float host_fma<float>(float a, float b, float c) { return std::fmaf(a, b, c); }

constexpr int kWindowSamples = 400;  // points of s per tap at which the fits are checked

template <typename R> R horner(const R *c, int D, R t) {
    R v = c[D];
    for (int k = D - 1; k >= 0; --k) v = host_fma<R>(v, t, c[k]);
    return v;
}

// the double-float Horner of the FP64 family's FP32-pipe gather, step for
// step, at argument t (2s - 1 for the whole-interval table)
long double horner_df(const float *ch, const float *cl, int D, double t) {
    const float th = (float)t, tl = (float)(t - (double)th);
    float vh = ch[D], vl = cl[D];
    for (int k = D - 1; k >= 0; --k) {
        const float pp = vh * th;
        float e = std::fmaf(vh, th, -pp);
        e = std::fmaf(vh, tl, e);
        e = std::fmaf(vl, th, e);
        const float sm = pp + ch[k];
        const float bb = sm - pp;
        float err = (pp - (sm - bb)) + (ch[k] - bb);
        err = err + (e + cl[k]);
        vh = sm + err;
        vl = err - (vh - sm);
    }
    return (long double)vh + (long double)vl;
}

// Fit the window polynomials of a plan (FP64 family: FP64 and double-float
// tables; mixed family: FP32 table) and record the largest absolute error of
// each evaluation, as the kernels perform it, against the exact weight.
void build_window_tables(nfft3_plan p) {
    const int m = p->m;
    p->window_err = 0;
    p->window_err_df = 0;
    std::memset(&p->wt64, 0, sizeof(p->wt64));
    std::memset(&p->wt32, 0, sizeof(p->wt32));
    std::memset(&p->wtdf, 0, sizeof(p->wtdf));
    std::memset(&p->half.w64, 0, sizeof(p->half.w64));
    std::memset(&p->half.wdf, 0, sizeof(p->half.wdf));
    for (int d = 0; d < 3; ++d) {
        const long double b = (long double)p->b[d];
        for (int a = 0; a <= 2 * m; ++a) {
            long double mono[kMaxCoef];
            if (p->prec == 64) {
                fit_tap(a, m, b, PolyDeg<double>::value, mono);
                for (int k = 0; k <= PolyDeg<double>::value; ++k) p->wt64.coef[d][a][k] = (double)mono[k];
                fit_tap(a, m, b, kPolyDegDF, mono);
                for (int k = 0; k <= kPolyDegDF; ++k) {
                    p->wtdf.ch[d][a][k] = (float)mono[k];
                    p->wtdf.cl[d][a][k] = (float)(mono[k] - (long double)p->wtdf.ch[d][a][k]);
                }
                fit_tap(a, m, b, kPolyDegHalf, mono, 0.5L, 1.0L);
                for (int k = 0; k <= kPolyDegHalf; ++k) {
                    p->half.w64.coef[d][a][k] = (double)mono[k];
                    p->half.wdf.ch[d][a][k] = (float)mono[k];
                    p->half.wdf.cl[d][a][k] = (float)(mono[k] - (long double)p->half.wdf.ch[d][a][k]);
                }
            } else {
                fit_tap(a, m, b, PolyDeg<float>::value, mono);
                for (int k = 0; k <= PolyDeg<float>::value; ++k) p->wt32.coef[d][a][k] = (float)mono[k];
            }
            for (int i = 0; i <= kWindowSamples; ++i) {
                const double s = (double)i / kWindowSamples;
                const long double ex = exact_weight((long double)s, a, m, b);
                if (p->prec == 64) {
                    const double v = horner<double>(p->wt64.coef[d][a], PolyDeg<double>::value, 2.0 * s - 1.0);
                    const double e1 = (double)fabsl((long double)v - ex);
                    const double e2 = (double)fabsl(horner_df(p->wtdf.ch[d][a], p->wtdf.cl[d][a], kPolyDegDF, 2.0 * s - 1.0) - ex);
                    if (e1 > p->window_err) p->window_err = e1;
                    if (e2 > p->window_err_df) p->window_err_df = e2;
                } else {
                    const float v = horner<float>(p->wt32.coef[d][a], PolyDeg<float>::value, (float)(2.0 * s - 1.0));
                    const double e1 = (double)fabsl((long double)v - ex);
                    if (e1 > p->window_err) p->window_err = e1;
                }
            }
        }
    }
    if (p->prec != 64 || p->half.mode == 0) return;
    // the half-interval table in use, as the value gather evaluates it: tap a
    // at s >= 1/2 from row a at u = 4s - 3, below from row 2m - a at u = 1 - 4s
    for (int d = 0; d < 3; ++d) {
        const long double b = (long double)p->b[d];
        for (int a = 0; a <= 2 * m; ++a)
            for (int i = 0; i <= kWindowSamples; ++i) {
                const double s = (double)i / kWindowSamples;
                const bool up = s >= 0.5;
                const int row = up ? a : 2 * m - a;
                const double u = up ? std::fma(4.0, s, -3.0) : std::fma(-4.0, s, 1.0);
                const long double ex = exact_weight((long double)s, a, m, b);
                if (p->half.mode == 1) {
                    const double v = horner<double>(p->half.w64.coef[d][row], kPolyDegHalf, u);
                    const double e1 = (double)fabsl((long double)v - ex);
                    if (e1 > p->window_err) p->window_err = e1;
                } else {
                    const double e2 = (double)fabsl(
                        horner_df(p->half.wdf.ch[d][row], p->half.wdf.cl[d][row], kPolyDegHalf, u) - ex);
                    if (e2 > p->window_err_df) p->window_err_df = e2;
                }
            }
    }
}

template <typename R> const WinTable<R> &win_table(nfft3_plan p);
template <> const WinTable<double> &win_table<double>(nfft3_plan p) { return p->wt64; }
template <> const WinTable<float> &win_table<float>(nfft3_plan p) { return p->wt32; }

int finish(nfft3_plan p, int status) {
    if (status == NFFT3_OK && p && p->sync_check) {
        if (cudaStreamSynchronize(p->stream) != cudaSuccess) return NFFT3_ERR_CUDA;
        if (cudaGetLastError() != cudaSuccess) return NFFT3_ERR_CUDA;
    }
    return status;
}

void release(nfft3_plan p) {
    if (!p) return;
    for (int d = 0; d < 3; ++d) {
        dev_free(p->D[d]);
        dev_free(p->s[d]);
    }
    dev_free(p->grid);
    dev_free(p->pgrid);
    dev_free(p->wtdf_dev);
    {
        void *v = p->vexp;
        dev_free(v);
    }
    for (int d = 0; d < 3; ++d) dev_free(p->tw[d]);
    dev_free(p->fscratch);
    void *k = p->key;
    dev_free(k);
    void *v;
    v = p->pb.key_count; dev_free(v);
    v = p->pb.key_start; dev_free(v);
    v = p->pb.tile_start; dev_free(v);
    v = p->pb.key_rank; dev_free(v);
    v = p->pb.scan_tmp; dev_free(v);
    v = p->pb.status; dev_free(v);
    dev_free(p->pb.scratch);
    v = p->pb.chunk_count; dev_free(v);
    v = p->pb.chunk_start; dev_free(v);
    v = p->pb.chunks; dev_free(v);
    v = p->pb.tile_dense; dev_free(v);
    v = p->pb.tile_dense_start; dev_free(v);
    v = p->pb.tile_sparse; dev_free(v);
    v = p->pb.tile_sparse_start; dev_free(v);
    v = p->pb.batches; dev_free(v);
    v = p->pb.sparse_idx; dev_free(v);
    release_deterministic(p);
    v = p->x_dev; dev_free(v);
    dev_free(p->c_dev);
    dev_free(p->f_dev);
    if (p->aux_stream) {
        for (int i = 0; i < 5; ++i) cudaEventDestroy(p->aux_ev[i]);
        cudaStreamDestroy(p->aux_stream);
        cudaStreamDestroy(p->copy_stream);
    }
    if (p->fft1) cufftDestroy(p->fft1);
    if (p->have_fft4) cufftDestroy(p->fft4);
    if (p->fft2d) cufftDestroy(p->fft2d);
    if (p->fft1d) cufftDestroy(p->fft1d);
    for (int r = 0; r < kTimingRecords; ++r)
        if (p->ev_ready[r])
            for (int i = 0; i < kTimingMarks; ++i) cudaEventDestroy(p->ev[r][i]);
    delete p;
}

int make_plan(nfft3_plan *out, int prec, int N1, int N2, int N3, int64_t M, int m, double sigma,
              double eps, void *stream) {
    if (!out) return NFFT3_ERR_ARG;
    *out = nullptr;
    const int Ns[3] = {N1, N2, N3};
    for (int d = 0; d < 3; ++d) {
        if (Ns[d] < 2 || Ns[d] % 2) return NFFT3_ERR_ARG;
        if (Ns[d] > 4096) return NFFT3_ERR_TOO_LARGE;
    }
    if (M < 0) return NFFT3_ERR_ARG;
    if (M >= ((int64_t)1 << 31)) return NFFT3_ERR_TOO_LARGE;
    if (sigma <= 0) sigma = 2.0;
    if (!(sigma >= 1.25) || !(sigma <= 8.0)) return NFFT3_ERR_ARG;
    if (m > kMaxM) return NFFT3_ERR_ARG;
    int warn = NFFT3_OK;
    if (m <= 0) {
        if (!(eps > 0)) return NFFT3_ERR_ARG;
        m = nfft3_choose_m(eps, sigma);
        if (error_estimate(m, sigma) > eps) warn = NFFT3_WARN_EPS;
    } else if (eps > 0 && error_estimate(m, sigma) > eps) {
        warn = NFFT3_WARN_EPS;
    }

    nfft3_plan p = new (std::nothrow) nfft3_plan_s;
    if (!p) return NFFT3_ERR_ALLOC;
    std::memset(p, 0, sizeof(*p));
    p->prec = prec;
    p->m = m;
    p->M = M;
    p->M_cap = M;
    p->stream = (cudaStream_t)stream;
    p->fault = read_fault_env();
    p->sync_check = std::getenv("GBNFFT_SYNC_CHECK") != nullptr;
    cudaGetDevice(&p->device);
    for (int d = 0; d < 3; ++d) {
        p->N[d] = Ns[d];
        p->n[d] = oversampled_size(Ns[d], sigma);
        p->b[d] = M_PI * (2.0 - (double)Ns[d] / (double)p->n[d]);
    }
    {
        // FP64 value gather weights: half-interval table in double-float on
        // the FP32 pipe (default), "fp64": the same table on the FP64 pipe,
        // "full": the whole-interval FP64 table (read before the tables are
        // built and checked); below m = 4 the half table of degree
        // kPolyDegHalf is less accurate than the whole-interval one (2.9e-14
        // at m = 1 against 1.9e-16), so the whole-interval table serves
        const char *hw = std::getenv("GBNFFT_SLOT_WEIGHTS");
        p->half.mode = hw && !std::strcmp(hw, "full") ? 0 : hw && !std::strcmp(hw, "fp64") ? 1 : 2;
        if (p->m < 4) p->half.mode = 0;
    }
    build_window_tables(p);
    {
        // gather variant: default (col) = column-parallel groups over the
        // padded grid (FP32, or double-float for the FP64 family); tma = the
        // same, with mixed-family values read from TMA-staged shared-memory
        // tiles; thread = one thread per point (FP32 / double-float);
        // native = one thread per point in the family's own precision (FP64
        // on the FP64 pipe)
        const char *g = std::getenv("GBNFFT_GATHER");
        const char *wv = std::getenv("GBNFFT_DF_WEIGHTS");
        p->df_weights_fp64 = !(wv && !std::strcmp(wv, "df"));
        // adjoint spread: shared-memory tile boxes (default) or one thread per
        // point with global atomics only (GBNFFT_SPREAD=direct)
        const char *sp = std::getenv("GBNFFT_SPREAD");
        p->spread_direct = sp && !std::strcmp(sp, "direct");
        // GBNFFT_ADJ_FFT=cufft: the adjoint's forward FFT by cuFFT plus the
        // deconvolution kernel instead of the fused passes
        const char *af = std::getenv("GBNFFT_ADJ_FFT");
        p->adj_cufft = af && !std::strcmp(af, "cufft");
        // GBNFFT_TMA_FIRST_WAIT: polls of the tile-staged gather's first
        // mbarrier wait (failure-detection test only; default: the full limit)
        const char *fw = std::getenv("GBNFFT_TMA_FIRST_WAIT");
        p->tma_first_wait = fw ? (unsigned)std::strtoul(fw, nullptr, 10) : ~0u;
        p->gather_mode = !g                           ? 3
                         : !std::strcmp(g, "thread") ? 1
                         : !std::strcmp(g, "native") ? 2
                         : !std::strcmp(g, "tma")    ? 0
                                                     : 3;
    }
    const size_t rs = prec == 64 ? sizeof(double) : sizeof(float);
    int st = NFFT3_OK;

    // deconvolution tables: D_d[i] = (-1)^k phi(0) / Phi(k / n_d), k = i - N_d/2,
    // Phi(nu) = I0(alpha sqrt(b^2 - (2 pi nu)^2)), phi(0) = sinh(b alpha) / (pi alpha).
    const double al = m + 0.5;
    for (int d = 0; d < 3 && st == NFFT3_OK; ++d) {
        const int Nd = p->N[d];
        double *h = (double *)std::malloc(sizeof(double) * Nd);
        float *hf = (float *)std::malloc(sizeof(float) * Nd);
        if (!h || !hf) {
            std::free(h);
            std::free(hf);
            st = NFFT3_ERR_ALLOC;
            break;
        }
        const double b = p->b[d];
        const double phi0 = std::sinh(b * al) / (M_PI * al);
        for (int i = 0; i < Nd; ++i) {
            const int k = i - Nd / 2;
            const double nu = 2.0 * M_PI * (double)k / (double)p->n[d];
            const double Phi = bessel_i0(al * std::sqrt(b * b - nu * nu));
            h[i] = ((k & 1) ? -1.0 : 1.0) * phi0 / Phi;
            hf[i] = (float)h[i];
        }
        st = dev_alloc(p, &p->D[d], rs * Nd);
        if (st == NFFT3_OK)
            st = cuda_status(cudaMemcpy(p->D[d], prec == 64 ? (void *)h : (void *)hf, rs * Nd,
                                        cudaMemcpyHostToDevice));
        std::free(h);
        std::free(hf);
    }
    if (st == NFFT3_OK && prec == 64) {
        st = dev_alloc(p, &p->wtdf_dev, sizeof(WinTableDF));
        if (st == NFFT3_OK)
            st = cuda_status(cudaMemcpy(p->wtdf_dev, &p->wtdf, sizeof(WinTableDF), cudaMemcpyHostToDevice));
    }
    const int64_t nn = (int64_t)p->n[0] * p->n[1] * p->n[2];
    if (st == NFFT3_OK) {
        void *v = nullptr;
        st = dev_alloc(p, &v, 2 * sizeof(int));
        p->vexp = (int *)v;
    }
    if (st == NFFT3_OK) {
        p->grid_count = 1;
        st = dev_alloc(p, &p->grid, 2 * rs * nn);
    }
    if (st == NFFT3_OK && (p->gather_mode == 0 || p->gather_mode == 3)) st = ensure_pgrid(p, 1);
    if (st == NFFT3_OK) {
        if (p->fault == kFaultFftPlan) {
            st = NFFT3_ERR_CUFFT;
        } else if (cufftPlan3d(&p->fft1, p->n[0], p->n[1], p->n[2],
                               prec == 64 ? CUFFT_Z2Z : CUFFT_C2C) != CUFFT_SUCCESS) {
            p->fft1 = 0;
            st = NFFT3_ERR_CUFFT;
        } else if (cufftSetStream(p->fft1, p->stream) != CUFFT_SUCCESS) {
            st = NFFT3_ERR_CUFFT;
        }
    }
    if (st == NFFT3_OK) {
        const char *f = std::getenv("GBNFFT_FFT");
        p->fft_pruned = !(f && !std::strcmp(f, "full"));
        p->fused = !f && fused_supported(p->n) && (p->gather_mode == 0 || p->gather_mode == 3);
    }
    for (int d = 0; d < 3 && st == NFFT3_OK && p->fused; ++d) st = make_twiddles(p, d);
    if (st == NFFT3_OK && p->fft_pruned) {
        const cufftType ty = prec == 64 ? CUFFT_Z2Z : CUFFT_C2C;
        int n2d[2] = {p->n[1], p->n[2]};
        int n1d[1] = {p->n[0]};
        const int plane = p->n[1] * p->n[2];
        if (cufftPlanMany(&p->fft2d, 2, n2d, nullptr, 1, 0, nullptr, 1, 0, ty, p->N[0] / 2) !=
                CUFFT_SUCCESS ||
            cufftPlanMany(&p->fft1d, 1, n1d, n1d, plane, 1, n1d, plane, 1, ty, plane) != CUFFT_SUCCESS ||
            cufftSetStream(p->fft2d, p->stream) != CUFFT_SUCCESS ||
            cufftSetStream(p->fft1d, p->stream) != CUFFT_SUCCESS)
            st = NFFT3_ERR_CUFFT;
    }
    // points
    if (st == NFFT3_OK) {
        PointsBuild &pb = p->pb;
        pb.m = m;
        pb.g = Grid3{p->n[0], p->n[1], p->n[2]};
        pb.nt1 = (p->n[0] + kTile - 1) / kTile;
        pb.nt2 = (p->n[1] + kTile - 1) / kTile;
        pb.nt3 = (p->n[2] + kTile - 1) / kTile;
        pb.ntile = (int64_t)pb.nt1 * pb.nt2 * pb.nt3;
        pb.M = M;
        void *v = nullptr;
        // the finer key pays off where the gather is bound by L1 row reads (the
        // mixed family); the double-float gather is ALU-bound and keeps tile order
        pb.nsub = prec == 32 && pb.ntile * kTile * kTile <= ((int64_t)1 << 27) ? kTile * kTile : 1;
        pb.nkey = pb.ntile * pb.nsub;
        // sort keys and their offsets are int (a grid that large would not fit the device anyway)
        if (pb.nkey >= ((int64_t)1 << 31) - 1) st = NFFT3_ERR_TOO_LARGE;
        if (st == NFFT3_OK) st = dev_alloc(p, &v, sizeof(int) * (pb.nkey + 1));
        pb.key_count = (int *)v;
        if (st == NFFT3_OK) st = dev_alloc(p, &v, sizeof(int) * (pb.nkey + 1)), pb.key_start = (int *)v;
        if (st == NFFT3_OK) st = dev_alloc(p, &v, sizeof(int) * (pb.ntile + 1)), pb.tile_start = (int *)v;
        if (st == NFFT3_OK) st = dev_alloc(p, &v, sizeof(int2) * (M + 1)), pb.key_rank = (int2 *)v;
        if (st == NFFT3_OK) st = dev_alloc(p, &v, sizeof(int) * scan_tmp_ints(pb.nkey + 1)), pb.scan_tmp = (int *)v;
        if (st == NFFT3_OK) st = dev_alloc(p, &v, sizeof(int)), pb.status = (int *)v;
        pb.M_cap = M;
        if (st == NFFT3_OK) st = dev_alloc(p, &pb.scratch, points_scratch_bytes(M, prec));
        pb.chunk_cap = pb.ntile + M / kChunk + 1;
        if (st == NFFT3_OK) st = dev_alloc(p, &v, sizeof(int) * (pb.ntile + 1)), pb.chunk_count = (int *)v;
        if (st == NFFT3_OK) st = dev_alloc(p, &v, sizeof(int) * (pb.ntile + 1)), pb.chunk_start = (int *)v;
        if (st == NFFT3_OK) st = dev_alloc(p, &v, sizeof(int4) * pb.chunk_cap), pb.chunks = (int4 *)v;
        // split value gather of the mixed family (sort keys of one tile and
        // (x, y) cell): keys with at least dense_min points go to the dense
        // batches; GBNFFT_DENSE_MIN overrides the threshold, 0 disables the split
        pb.dense_min = 0;
        if (prec == 32 && pb.nsub == 64 && (p->gather_mode == 0 || p->gather_mode == 3)) {
            const char *dm = std::getenv("GBNFFT_DENSE_MIN");
            pb.dense_min = dm ? std::atoi(dm) : kDenseMinDefault;
            if (pb.dense_min > 0 && pb.dense_min < 4) pb.dense_min = 4;   // batch_cap below needs >= 4
        }
        if (pb.dense_min > 0) {
            // a dense key of cnt >= dense_min >= 4 points makes ceil(cnt / 32) <= cnt / 4 batches
            pb.batch_cap = M / 4 + 1;
            if (st == NFFT3_OK) st = dev_alloc(p, &v, sizeof(int) * (pb.ntile + 1)), pb.tile_dense = (int *)v;
            if (st == NFFT3_OK) st = dev_alloc(p, &v, sizeof(int) * (pb.ntile + 1)), pb.tile_dense_start = (int *)v;
            if (st == NFFT3_OK) st = dev_alloc(p, &v, sizeof(int) * (pb.ntile + 1)), pb.tile_sparse = (int *)v;
            if (st == NFFT3_OK) st = dev_alloc(p, &v, sizeof(int) * (pb.ntile + 1)), pb.tile_sparse_start = (int *)v;
            if (st == NFFT3_OK) st = dev_alloc(p, &v, sizeof(int2) * pb.batch_cap), pb.batches = (int2 *)v;
            if (st == NFFT3_OK) st = dev_alloc(p, &v, sizeof(int) * (M + 1)), pb.sparse_idx = (int *)v;
        }
        if (st == NFFT3_OK) st = dev_alloc(p, &v, sizeof(int4) * (M + 1)), p->key = (int4 *)v;
        for (int d = 0; d < 3 && st == NFFT3_OK; ++d) st = dev_alloc(p, &p->s[d], rs * (M + 1));
    }
    if (st == NFFT3_OK) st = noalloc_setup(p);
    if (st != NFFT3_OK) {
        release(p);
        return st;
    }
    *out = p;
    return warn;
}

// Range word of the forward calls (FP64 family; nullptr for the mixed family).
const int *fwd_vexp(nfft3_plan p) { return p->prec == 64 ? p->vexp : nullptr; }

// Points of the plan, with the forward range word; the adjoint substitutes its own.
template <typename R> PointsView<R> points_view(nfft3_plan p) {
    PointsView<R> v;
    v.key = p->key;
    v.s1 = (const R *)p->s[0];
    v.s2 = (const R *)p->s[1];
    v.s3 = (const R *)p->s[2];
    v.M = p->M;
    v.vexp = sizeof(R) == 8 ? fwd_vexp(p) : nullptr;
    return v;
}

// FP64 family: record the exponent rank of the largest of `count` complex
// input values in p->vexp[slot] (0: coefficients, 1: adjoint values), so the
// call's kernels can scale its double-float arithmetic into range.
int range_scan(nfft3_plan p, int slot, const void *values, int64_t count) {
    if (p->prec != 64) return NFFT3_OK;
    if (cudaMemsetAsync(p->vexp + slot, 0, sizeof(int), p->stream) != cudaSuccess) return NFFT3_ERR_CUDA;
    if (count <= 0) return NFFT3_OK;
    if (launch_value_rank((const double *)values, 2 * count, p->vexp + slot, p->stream) != cudaSuccess)
        return NFFT3_ERR_CUDA;
    p->launches += 1;
    return NFFT3_OK;
}

int64_t num_coeffs(nfft3_plan p) { return (int64_t)p->N[0] * p->N[1] * p->N[2]; }

int exec_fft(cufftHandle h, void *data, int prec, int direction) {
    cufftResult r;
    if (prec == 64)
        r = cufftExecZ2Z(h, (cufftDoubleComplex *)data, (cufftDoubleComplex *)data, direction);
    else
        r = cufftExecC2C(h, (cufftComplex *)data, (cufftComplex *)data, direction);
    return r == CUFFT_SUCCESS ? NFFT3_OK : NFFT3_ERR_CUFFT;
}

// Oversampled transform of ng consecutive grids.  Full: the 3D plan (batched
// for ng = 4).  Pruned, inverse: only the planes l1 with |k1| < N1/2 can be
// nonzero, so 2D FFTs run over those two plane ranges, then 1D FFTs along l1;
// pruned, forward (adjoint): 1D FFTs along l1, then 2D FFTs over the planes
// whose output is kept.
int exec_grid_fft(nfft3_plan p, void *data, int prec, int direction, int ng) {
    if (!p->fft_pruned) return exec_fft(ng == 4 ? p->fft4 : p->fft1, data, prec, direction);
    const int64_t plane = (int64_t)p->n[1] * p->n[2];
    const int64_t nn = plane * p->n[0];
    const size_t esz = prec == 64 ? sizeof(double2) : sizeof(float2);
    for (int q = 0; q < ng; ++q) {
        char *g = (char *)data + esz * nn * q;
        char *lo = g;                                                // l1 in [0, N1/2)
        char *hi = g + esz * plane * (int64_t)(p->n[0] - p->N[0] / 2);  // l1 in [n1 - N1/2, n1)
        int st;
        if (direction == CUFFT_INVERSE) {
            if ((st = exec_fft(p->fft2d, lo, prec, direction)) != NFFT3_OK) return st;
            if ((st = exec_fft(p->fft2d, hi, prec, direction)) != NFFT3_OK) return st;
            if ((st = exec_fft(p->fft1d, g, prec, direction)) != NFFT3_OK) return st;
        } else {
            if ((st = exec_fft(p->fft1d, g, prec, direction)) != NFFT3_OK) return st;
            if ((st = exec_fft(p->fft2d, lo, prec, direction)) != NFFT3_OK) return st;
            if ((st = exec_fft(p->fft2d, hi, prec, direction)) != NFFT3_OK) return st;
        }
    }
    return NFFT3_OK;
}

int set_points_impl(nfft3_plan p, const double *x, int prec, int64_t first_part = 0, cudaEvent_t second = nullptr) {
    if (!p || p->prec != prec) return NFFT3_ERR_ARG;
    if (!x && p->M > 0) return NFFT3_ERR_ARG;
    p->points_ok = 0;
    p->split_ok = 0;
    const int rec = rec_begin(p, kRecSetPoints);
    cudaError_t e;
    const StableSort *stable = p->det ? &p->ss : nullptr;
    if (prec == 64)
        e = launch_points<double>(x, p->pb, p->key, (double *)p->s[0], (double *)p->s[1],
                                  (double *)p->s[2], p->stream, stable, first_part, second);
    else
        e = launch_points<float>(x, p->pb, p->key, (float *)p->s[0], (float *)p->s[1],
                                 (float *)p->s[2], p->stream, stable, first_part, second);
    if (e != cudaSuccess) return NFFT3_ERR_CUDA;
    p->launches += (p->M > 0 ? 4 : 1) + scan_launches(p->pb.nkey + 1);
    if (second && first_part > 0 && first_part < p->M) p->launches += 1;   // the first pass in two parts
    if (stable) p->launches += stable_sort_launches(p->pb);
    if (launch_chunks(p->pb, p->stream) != cudaSuccess) return NFFT3_ERR_CUDA;
    p->launches += 2 + scan_launches(p->pb.ntile + 1);
    const bool split = p->pb.dense_min > 0 && p->M > 0;
    if (split) {
        if (launch_split_lists(p->pb, p->stream) != cudaSuccess) return NFFT3_ERR_CUDA;
        p->launches += split_list_launches(p->pb);
    }
    rec_mark(p, rec, 1);
    rec_end(p, rec, 1);
    int status = 0, nch = 0, nbs[2] = {0, 0};
    if (cudaMemcpyAsync(&status, p->pb.status, sizeof(int), cudaMemcpyDeviceToHost, p->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(&nch, p->pb.chunk_start + p->pb.ntile, sizeof(int), cudaMemcpyDeviceToHost,
                        p->stream) != cudaSuccess)
        return NFFT3_ERR_CUDA;
    if (split && (cudaMemcpyAsync(&nbs[0], p->pb.tile_dense_start + p->pb.ntile, sizeof(int),
                                  cudaMemcpyDeviceToHost, p->stream) != cudaSuccess ||
                  cudaMemcpyAsync(&nbs[1], p->pb.tile_sparse_start + p->pb.ntile, sizeof(int),
                                  cudaMemcpyDeviceToHost, p->stream) != cudaSuccess))
        return NFFT3_ERR_CUDA;
    if (cudaStreamSynchronize(p->stream) != cudaSuccess) return NFFT3_ERR_CUDA;
    if (status & 2) return NFFT3_ERR_CUDA;   // a tile-staged gather timed out on its copy
    if (status & 1) return NFFT3_ERR_POINTS;
    p->nchunks = nch <= p->pb.chunk_cap ? nch : 0;
    p->nbatch = nbs[0];
    p->nsparse = nbs[1];
    p->split_ok = split && nbs[0] <= p->pb.batch_cap && nbs[1] <= p->M;
    p->points_ok = 1;
    return NFFT3_OK;
}

// Padded grid storage for ng grids (allocated on first use, kept by the plan).
int ensure_pgrid(nfft3_plan p, int ng) {
    if (p->pgrid && p->pgrid_count >= ng) return NFFT3_OK;
    const int64_t pn = (int64_t)(p->n[0] + 2 * p->m) * (p->n[1] + 2 * p->m) * (p->n[2] + 2 * p->m);
    const size_t elem = p->prec == 64 ? 16 : 8;   // double-float float4 or float2
    // 64 zero bytes past the last grid: the mixed family's dense gather reads
    // its rows as 16-byte pairs and may read one value past a row's end
    // (with weight zero), past the last row into this slack
    constexpr size_t kSlack = 64;
    void *v = nullptr;
    const int st = dev_alloc(p, &v, elem * pn * ng + kSlack);
    if (st != NFFT3_OK) return st;
    if (cudaMemsetAsync((char *)v + elem * pn * ng, 0, kSlack, p->stream) != cudaSuccess) {
        dev_free(v);
        return NFFT3_ERR_CUDA;
    }
    dev_free(p->pgrid);
    p->pgrid = v;
    p->pgrid_count = ng;
    p->tmap_ok = 0;
    if (p->prec == 32) {
        const Grid3 pg{p->n[0] + 2 * p->m, p->n[1] + 2 * p->m, p->n[2] + 2 * p->m};
        p->tmap_ok = encode_padded_tmap(p->tmap, p->pgrid, pg, p->m) == 0;
    }
    return NFFT3_OK;
}

// Layout shift of the padded grid: the tile-staged kernel (single mixed-family
// grid, tma mode, tensor map and chunk list ready) needs the stencil centre as
// origin (shift m); the column kernels read from the first node (shift 0).
// The choice is recorded so that a stored grid is read the way it was written.
int pad_shift(nfft3_plan p, int ng, bool allow_tile = true) {
    const bool tile = allow_tile && ng == 1 && p->prec == 32 && p->gather_mode == 0 && p->tmap_ok &&
                      p->nchunks > 0;
    p->pgrid_shift = tile ? p->m : 0;
    return p->pgrid_shift;
}

// Gather from the padded grid(s): mixed-family values from TMA-staged tiles
// (tma mode), otherwise the column-parallel kernels.
template <typename R>
cudaError_t gather_padded(nfft3_plan p, int ng, typename Cplx<R>::T *f, typename Cplx<R>::T *grad) {
    constexpr int prec = sizeof(R) == 8 ? 64 : 32;
    const Grid3 g{p->n[0], p->n[1], p->n[2]};
    const Grid3 pg{g.n1 + 2 * p->m, g.n2 + 2 * p->m, g.n3 + 2 * p->m};
    p->launches += 1;
    if (prec == 64)
        return launch_gather_col_df((const float4 *)p->pgrid, pg, p->m, points_view<double>(p), p->wtdf,
                                    p->wt64, p->df_weights_fp64, (double2 *)f, (double2 *)grad, ng, p->stream,
                                    &p->half);
    if (ng == 1 && p->pgrid_shift != 0 && p->tmap_ok && p->nchunks > 0)
        return launch_gather_tma_f32(p->tmap, p->pb.chunks, p->nchunks, p->pb.nt2, p->pb.nt3, g, p->m,
                                     points_view<float>(p), p->wt32, (float2 *)f, p->pb.status,
                                     p->tma_first_wait, p->stream);
    if (p->pgrid_shift != 0) return cudaErrorInvalidValue;  // centre layout, no tile list: not reachable
    if (ng == 1 && p->split_ok) {
        p->launches += (p->nbatch > 0) + (p->nsparse > 0) - 1;
        return launch_gather_split_f32((const float2 *)p->pgrid, pg, p->m, points_view<float>(p), p->wt32,
                                       p->pb.batches, p->nbatch, p->pb.sparse_idx, p->nsparse, (float2 *)f,
                                       p->stream);
    }
    return launch_gather_col_f32((const float2 *)p->pgrid, pg, p->m, points_view<float>(p), p->wt32,
                                 (float2 *)f, (float2 *)grad, ng, p->stream);
}

// Window gather of ng grids (1: value, 4: value + gradient) after the FFT:
// the FP64 family splits the grid into double-float (timed as the split
// stage, mark 3) unless the native FP64 kernel is selected.
template <typename R>
cudaError_t gather_stage(nfft3_plan p, typename Cplx<R>::T *G, int ng, typename Cplx<R>::T *f,
                         typename Cplx<R>::T *grad, int rec) {
    constexpr int prec = sizeof(R) == 8 ? 64 : 32;
    const Grid3 g{p->n[0], p->n[1], p->n[2]};
    const int64_t nn = (int64_t)g.n1 * g.n2 * g.n3;
    cudaError_t e;
    if (p->gather_mode == 0 || p->gather_mode == 3) {
        // padded copy (FP64: split into double-float), then the column gather
        const int st = ensure_pgrid(p, ng);
        if (st != NFFT3_OK) return cudaErrorMemoryAllocation;
        const Grid3 pg{g.n1 + 2 * p->m, g.n2 + 2 * p->m, g.n3 + 2 * p->m};
        if (prec == 64)
            e = launch_pad_grid_df((const double2 *)G, g, (float4 *)p->pgrid, pg, ng, pad_shift(p, ng), p->stream);
        else
            e = launch_pad_grid_f32((const float2 *)G, g, (float2 *)p->pgrid, pg, ng, pad_shift(p, ng), p->stream);
        if (e != cudaSuccess) return e;
        rec_mark(p, rec, 3);
        p->launches += 1;
        return gather_padded<R>(p, ng, f, grad);
    }
    if (prec == 64 && p->gather_mode == 1) {
        e = launch_grid_to_df((double2 *)G, ng * nn, p->stream);
        if (e != cudaSuccess) return e;
        rec_mark(p, rec, 3);
        PointsView<double> v = points_view<double>(p);
        if (ng == 1)
            e = launch_gather_df((const float4 *)G, g, p->m, v, p->wtdf, (double2 *)f, p->stream);
        else
            e = launch_gather_grad_df((const float4 *)G, g, p->m, v, p->wtdf, (double2 *)f,
                                      (double2 *)grad, p->stream);
        p->launches += 2;
        return e;
    }
    rec_mark(p, rec, 3);
    p->launches += 1;
    if (ng == 1) return launch_gather<R>(G, g, p->m, points_view<R>(p), win_table<R>(p), f, p->stream);
    return launch_gather_grad<R>(G, g, p->m, points_view<R>(p), win_table<R>(p), f, grad, p->stream);
}

// Fused forward transform of c into the padded grid(s) (ng = 1 or 4): the
// deconvolution, the three DFT line passes and the padded layout in three
// launches; the column / tile-staged gathers read the result directly.
template <typename R> int fused_transform(nfft3_plan p, const R *c, int ng, bool allow_tile = true) {
    int st = ensure_pgrid(p, ng);
    if (st == NFFT3_OK) st = ensure_fscratch(p, ng);
    if (st != NFFT3_OK) return st;
    const void *tw[3] = {p->tw[0], p->tw[1], p->tw[2]};
    const cudaError_t e = launch_fused_series<R>(
        (const typename Cplx<R>::T *)c, p->N, p->n, (const R *)p->D[0], (const R *)p->D[1],
        (const R *)p->D[2], tw, p->fscratch, p->pgrid, p->m, pad_shift(p, ng, allow_tile), ng, fwd_vexp(p),
        p->stream);
    p->launches += 3;
    return cuda_status(e);
}

// Fused evaluation of ng grids: the transform is timed as the fft stage
// (deconv and split stages are empty), then the gather.
template <typename R> int fused_eval(nfft3_plan p, const R *c, R *f, R *grad, int ng, int rec) {
    using C = typename Cplx<R>::T;
    rec_mark(p, rec, 1);
    const int st = fused_transform<R>(p, c, ng);
    if (st != NFFT3_OK) return st;
    rec_mark(p, rec, 2);
    rec_mark(p, rec, 3);
    const cudaError_t e = gather_padded<R>(p, ng, (C *)f, (C *)grad);
    rec_mark(p, rec, 4);
    return finish(p, cuda_status(e));
}

template <typename R> int eval_impl(nfft3_plan p, const R *c, R *f) {
    using C = typename Cplx<R>::T;
    constexpr int prec = sizeof(R) == 8 ? 64 : 32;
    if (!p || p->prec != prec) return NFFT3_ERR_ARG;
    if (!p->points_ok) return NFFT3_ERR_NO_POINTS;
    if (p->M > 0 && (!c || !f)) return NFFT3_ERR_ARG;
    if (p->M == 0) return NFFT3_OK;
    const Grid3 g{p->n[0], p->n[1], p->n[2]};
    C *G = (C *)p->grid;
    p->stored_ng = 0;
    const int rec = rec_begin(p, kRecEval);
    const int rs = range_scan(p, 0, c, num_coeffs(p));
    if (rs != NFFT3_OK) return rs;
    if (p->fused) return fused_eval<R>(p, c, f, nullptr, 1, rec);
    cudaError_t e = launch_deconv_scatter<R>((const C *)c, p->N[0], p->N[1], p->N[2],
                                             (const R *)p->D[0], (const R *)p->D[1],
                                             (const R *)p->D[2], G, g, 0, fwd_vexp(p), p->stream);
    if (e != cudaSuccess) return NFFT3_ERR_CUDA;
    rec_mark(p, rec, 1);
    int st = exec_grid_fft(p, G, prec, CUFFT_INVERSE, 1);
    if (st != NFFT3_OK) return st;
    p->launches += 1;  // deconv
    rec_mark(p, rec, 2);
    e = gather_stage<R>(p, G, 1, (C *)f, nullptr, rec);
    rec_mark(p, rec, 4);
    return finish(p, cuda_status(e));
}

template <typename R> int ensure_grad_grids(nfft3_plan p) {
    constexpr int prec = sizeof(R) == 8 ? 64 : 32;
    if (p->grid_count == 4 && (p->have_fft4 || p->fft_pruned)) return NFFT3_OK;
    const int64_t nn = (int64_t)p->n[0] * p->n[1] * p->n[2];
    void *g4 = nullptr;
    int st = dev_alloc(p, &g4, 2 * sizeof(R) * nn * 4);
    if (st != NFFT3_OK) return st;
    if (p->fault == kFaultFftPlan) {
        cudaFree(g4);
        return NFFT3_ERR_CUFFT;
    }
    if (!p->fft_pruned) {
        // batched 3D plan; default layout: distance n1 n2 n3 between transforms
        int dims[3] = {p->n[0], p->n[1], p->n[2]};
        cufftHandle h;
        if (cufftPlanMany(&h, 3, dims, nullptr, 1, (int)0, nullptr, 1, 0,
                          prec == 64 ? CUFFT_Z2Z : CUFFT_C2C, 4) != CUFFT_SUCCESS) {
            cudaFree(g4);
            return NFFT3_ERR_CUFFT;
        }
        cufftSetStream(h, p->stream);
        p->fft4 = h;
        p->have_fft4 = 1;
    }
    dev_free(p->grid);
    p->grid = g4;
    p->grid_count = 4;
    return NFFT3_OK;
}

template <typename R> int eval_grad_impl(nfft3_plan p, const R *c, R *f, R *grad) {
    using C = typename Cplx<R>::T;
    constexpr int prec = sizeof(R) == 8 ? 64 : 32;
    if (!p || p->prec != prec) return NFFT3_ERR_ARG;
    if (!p->points_ok) return NFFT3_ERR_NO_POINTS;
    if (p->M > 0 && (!c || !grad)) return NFFT3_ERR_ARG;
    if (p->M == 0) return NFFT3_OK;
    if (p->fused) {
        p->stored_ng = 0;
        const int rec = rec_begin(p, kRecGrad);
        const int rs = range_scan(p, 0, c, num_coeffs(p));
        if (rs != NFFT3_OK) return rs;
        return fused_eval<R>(p, c, f, grad, 4, rec);
    }
    int st = ensure_grad_grids<R>(p);
    if (st != NFFT3_OK) return st;
    const Grid3 g{p->n[0], p->n[1], p->n[2]};
    C *G = (C *)p->grid;
    p->stored_ng = 0;
    const int rec = rec_begin(p, kRecGrad);
    st = range_scan(p, 0, c, num_coeffs(p));
    if (st != NFFT3_OK) return st;
    cudaError_t e = launch_deconv_scatter<R>((const C *)c, p->N[0], p->N[1], p->N[2],
                                             (const R *)p->D[0], (const R *)p->D[1],
                                             (const R *)p->D[2], G, g, 1, fwd_vexp(p), p->stream);
    if (e != cudaSuccess) return NFFT3_ERR_CUDA;
    rec_mark(p, rec, 1);
    st = exec_grid_fft(p, G, prec, CUFFT_INVERSE, 4);
    if (st != NFFT3_OK) return st;
    p->launches += 1;  // deconv
    rec_mark(p, rec, 2);
    e = gather_stage<R>(p, G, 4, (C *)f, (C *)grad, rec);
    rec_mark(p, rec, 4);
    return finish(p, cuda_status(e));
}

template <typename R> int chain_x_impl(nfft3_plan p, const R *G, const R *grad, double *gx) {
    constexpr int prec = sizeof(R) == 8 ? 64 : 32;
    if (!p || p->prec != prec) return NFFT3_ERR_ARG;
    if (p->M == 0) return NFFT3_OK;
    if (!G || !grad || !gx) return NFFT3_ERR_ARG;
    const cudaError_t e = launch_chain_x<R>(G, grad, gx, p->M, p->stream);
    p->launches += 1;
    return finish(p, cuda_status(e));
}

// Deconvolve + FFT + pad the series c into the plan's padded grid(s) and keep
// them: afterwards eval_stored / eval_grad_stored gather at whatever points
// are set, without repeating the FFT (column gather mode only).
template <typename R> int precompute_impl(nfft3_plan p, const R *c, int with_grad) {
    using C = typename Cplx<R>::T;
    constexpr int prec = sizeof(R) == 8 ? 64 : 32;
    if (!p || p->prec != prec || !c || (p->gather_mode != 0 && p->gather_mode != 3)) return NFFT3_ERR_ARG;
    const int ng = with_grad ? 4 : 1;
    p->stored_ng = 0;
    {
        const int rs = range_scan(p, 0, c, num_coeffs(p));
        if (rs != NFFT3_OK) return rs;
    }
    if (p->fused) {
        const int st = fused_transform<R>(p, c, ng);
        if (st != NFFT3_OK) return st;
        p->stored_ng = ng;
        return finish(p, NFFT3_OK);
    }
    int st = ng == 4 ? ensure_grad_grids<R>(p) : NFFT3_OK;
    if (st == NFFT3_OK) st = ensure_pgrid(p, ng);
    if (st != NFFT3_OK) return st;
    p->stored_ng = 0;
    const Grid3 g{p->n[0], p->n[1], p->n[2]};
    const Grid3 pg{g.n1 + 2 * p->m, g.n2 + 2 * p->m, g.n3 + 2 * p->m};
    C *G = (C *)p->grid;
    cudaError_t e = launch_deconv_scatter<R>((const C *)c, p->N[0], p->N[1], p->N[2],
                                             (const R *)p->D[0], (const R *)p->D[1],
                                             (const R *)p->D[2], G, g, ng == 4, fwd_vexp(p), p->stream);
    if (e != cudaSuccess) return NFFT3_ERR_CUDA;
    st = exec_grid_fft(p, G, prec, CUFFT_INVERSE, ng);
    if (st != NFFT3_OK) return st;
    if (prec == 64)
        e = launch_pad_grid_df((const double2 *)G, g, (float4 *)p->pgrid, pg, ng, pad_shift(p, ng), p->stream);
    else
        e = launch_pad_grid_f32((const float2 *)G, g, (float2 *)p->pgrid, pg, ng, pad_shift(p, ng), p->stream);
    if (e != cudaSuccess) return NFFT3_ERR_CUDA;
    p->launches += 2;
    p->stored_ng = ng;
    return finish(p, NFFT3_OK);
}

template <typename R> int eval_stored_impl(nfft3_plan p, R *f, R *grad, int ng) {
    constexpr int prec = sizeof(R) == 8 ? 64 : 32;
    if (!p || p->prec != prec) return NFFT3_ERR_ARG;
    if (p->stored_ng < ng) return NFFT3_ERR_NO_COEFFS;
    if (!p->points_ok) return NFFT3_ERR_NO_POINTS;
    if (p->M == 0) return NFFT3_OK;
    if ((ng == 1 && !f) || (ng == 4 && !grad)) return NFFT3_ERR_ARG;
    const int rec = rec_begin(p, ng == 4 ? kRecGrad : kRecEval);
    rec_mark(p, rec, 1);
    rec_mark(p, rec, 2);
    rec_mark(p, rec, 3);
    const cudaError_t e = gather_padded<R>(p, ng, (typename Cplx<R>::T *)f, (typename Cplx<R>::T *)grad);
    rec_mark(p, rec, 4);
    return finish(p, cuda_status(e));
}

// ---- window-derivative gradient ------------------------------------------------
// One transform of c into the padded grid (origin layout), then the gather
// that differentiates the window (gather_wd.cu).  Padded-grid gather modes
// (default and tma) only.
template <typename R> cudaError_t gather_wd(nfft3_plan p, R *f, R *grad) {
    using C = typename Cplx<R>::T;
    const Grid3 pg{p->n[0] + 2 * p->m, p->n[1] + 2 * p->m, p->n[2] + 2 * p->m};
    p->launches += 1;
    if constexpr (sizeof(R) == 8)
        return launch_gather_wd_df((const float4 *)p->pgrid, pg, p->m, points_view<double>(p), p->wt64, p->n,
                                   (C *)f, (C *)grad, p->stream);
    else
        return launch_gather_wd_f32((const float2 *)p->pgrid, pg, p->m, points_view<float>(p), p->wt32, p->n,
                                    (C *)f, (C *)grad, p->stream);
}

// c -> padded grid (one grid, origin layout), by the fused transform or by
// deconvolution + cuFFT + padding.
template <typename R> int series_to_origin_pgrid(nfft3_plan p, const R *c) {
    using C = typename Cplx<R>::T;
    int st = range_scan(p, 0, c, num_coeffs(p));
    if (st != NFFT3_OK) return st;
    if (p->fused) return fused_transform<R>(p, c, 1, false);
    st = ensure_pgrid(p, 1);
    if (st != NFFT3_OK) return st;
    const Grid3 g{p->n[0], p->n[1], p->n[2]};
    const Grid3 pg{g.n1 + 2 * p->m, g.n2 + 2 * p->m, g.n3 + 2 * p->m};
    C *G = (C *)p->grid;
    cudaError_t e = launch_deconv_scatter<R>((const C *)c, p->N[0], p->N[1], p->N[2], (const R *)p->D[0],
                                             (const R *)p->D[1], (const R *)p->D[2], G, g, 0, fwd_vexp(p),
                                             p->stream);
    if (e != cudaSuccess) return NFFT3_ERR_CUDA;
    st = exec_grid_fft(p, G, sizeof(R) == 8 ? 64 : 32, CUFFT_INVERSE, 1);
    if (st != NFFT3_OK) return st;
    if constexpr (sizeof(R) == 8)
        e = launch_pad_grid_df((const double2 *)G, g, (float4 *)p->pgrid, pg, 1, pad_shift(p, 1, false), p->stream);
    else
        e = launch_pad_grid_f32((const float2 *)G, g, (float2 *)p->pgrid, pg, 1, pad_shift(p, 1, false), p->stream);
    p->launches += 2;
    return cuda_status(e);
}

template <typename R> int eval_grad_window_impl(nfft3_plan p, const R *c, R *f, R *grad) {
    constexpr int prec = sizeof(R) == 8 ? 64 : 32;
    if (!p || p->prec != prec || (p->gather_mode != 0 && p->gather_mode != 3)) return NFFT3_ERR_ARG;
    if (!p->points_ok) return NFFT3_ERR_NO_POINTS;
    if (p->M > 0 && (!c || !grad)) return NFFT3_ERR_ARG;
    if (p->M == 0) return NFFT3_OK;
    p->stored_ng = 0;
    const int rec = rec_begin(p, kRecGrad);
    rec_mark(p, rec, 1);
    const int st = series_to_origin_pgrid<R>(p, c);
    if (st != NFFT3_OK) return st;
    rec_mark(p, rec, 2);
    rec_mark(p, rec, 3);
    const cudaError_t e = gather_wd<R>(p, f, grad);
    rec_mark(p, rec, 4);
    return finish(p, cuda_status(e));
}

template <typename R> int eval_grad_window_stored_impl(nfft3_plan p, R *f, R *grad) {
    constexpr int prec = sizeof(R) == 8 ? 64 : 32;
    if (!p || p->prec != prec) return NFFT3_ERR_ARG;
    if (p->stored_ng < 1) return NFFT3_ERR_NO_COEFFS;
    if (p->pgrid_shift != 0) return NFFT3_ERR_ARG;   // stored in the tile-staged (centre) layout
    if (!p->points_ok) return NFFT3_ERR_NO_POINTS;
    if (p->M == 0) return NFFT3_OK;
    if (!grad) return NFFT3_ERR_ARG;
    const int rec = rec_begin(p, kRecGrad);
    rec_mark(p, rec, 1);
    rec_mark(p, rec, 2);
    rec_mark(p, rec, 3);
    const cudaError_t e = gather_wd<R>(p, f, grad);
    rec_mark(p, rec, 4);
    return finish(p, cuda_status(e));
}

template <typename R> int adjoint_impl(nfft3_plan p, const R *f, R *c_out) {
    using C = typename Cplx<R>::T;
    constexpr int prec = sizeof(R) == 8 ? 64 : 32;
    if (!p || p->prec != prec) return NFFT3_ERR_ARG;
    if (!p->points_ok) return NFFT3_ERR_NO_POINTS;
    if (!c_out || (p->M > 0 && !f)) return NFFT3_ERR_ARG;
    const Grid3 g{p->n[0], p->n[1], p->n[2]};
    const int64_t nn = (int64_t)g.n1 * g.n2 * g.n3;
    C *H = (C *)p->grid;
    p->stored_ng = 0;
    const int rec = rec_begin(p, kRecAdjoint);
    // FP64 family: f's range word, used by the spread (input) and the deconvolution (output)
    const int *avexp = prec == 64 ? p->vexp + 1 : nullptr;
    int st = range_scan(p, 1, f, p->M);
    if (st != NFFT3_OK) return st;
    PointsView<R> pv = points_view<R>(p);
    pv.vexp = avexp;
    cudaError_t e;
    if (p->det) {
        // deterministic: the tile spread flushes exact fixed-point sums
        if (prec != 64 || p->spread_direct) return NFFT3_ERR_ARG;
        e = cudaMemsetAsync(p->Hq, 0, 4 * sizeof(unsigned long long) * nn, p->stream);
        if (e == cudaSuccess && p->nchunks > 0)
            e = launch_spread_tiles<R>((const C *)f, g, p->m, pv, win_table<R>(p), &p->wtdf,
                                       (const WinTableDF *)p->wtdf_dev, p->pb.chunks, p->nchunks, p->pb.nt2,
                                       p->pb.nt3, H, p->Hq, p->stream);
        if (e == cudaSuccess) e = launch_fixed_to_grid(p->Hq, (double2 *)H, nn, p->stream);
        p->launches += 1;
    } else {
        e = cudaMemsetAsync(H, 0, sizeof(C) * nn, p->stream);
        if (e != cudaSuccess) return NFFT3_ERR_CUDA;
        if (!p->spread_direct && p->nchunks > 0)
            e = launch_spread_tiles<R>((const C *)f, g, p->m, pv, win_table<R>(p), prec == 64 ? &p->wtdf : nullptr,
                                       (const WinTableDF *)p->wtdf_dev, p->pb.chunks, p->nchunks, p->pb.nt2,
                                       p->pb.nt3, H, nullptr, p->stream);
        else
            e = launch_spread<R>((const C *)f, g, p->m, pv, win_table<R>(p), H, p->stream);
    }
    if (e != cudaSuccess) return NFFT3_ERR_CUDA;
    rec_mark(p, rec, 1);
    p->launches += p->M > 0 ? 1 : 0;   // the spread
    if (p->fused && !p->adj_cufft) {
        // forward DFT of the band and deconvolution in three line passes
        st = ensure_fscratch(p, 1);
        if (st != NFFT3_OK) return st;
        const void *tw[3] = {p->tw[0], p->tw[1], p->tw[2]};
        e = launch_fused_adjoint<R>(H, p->N, p->n, (const R *)p->D[0], (const R *)p->D[1], (const R *)p->D[2], tw,
                                    p->fscratch, (C *)c_out, avexp, p->stream);
        p->launches += 3;
        rec_mark(p, rec, 2);
        rec_mark(p, rec, 3);
        rec_end(p, rec, 3);
        return finish(p, cuda_status(e));
    }
    st = exec_grid_fft(p, H, prec, CUFFT_FORWARD, 1);
    if (st != NFFT3_OK) return st;
    rec_mark(p, rec, 2);
    e = launch_deconv_gather<R>(H, g, (const R *)p->D[0], (const R *)p->D[1], (const R *)p->D[2],
                                p->N[0], p->N[1], p->N[2], (C *)c_out, avexp, p->stream);
    p->launches += 1;
    rec_mark(p, rec, 3);
    rec_end(p, rec, 3);
    return finish(p, cuda_status(e));
}

// The plan's second and copy streams and their events (created on first use).
int ensure_aux(nfft3_plan p) {
    if (p->aux_stream) return NFFT3_OK;
    bool ok = cudaStreamCreateWithFlags(&p->aux_stream, cudaStreamNonBlocking) == cudaSuccess;
    if (!ok) p->aux_stream = nullptr;
    const bool cs = ok && cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking) == cudaSuccess;
    int nev = 0;
    if (cs)
        while (nev < 5 && cudaEventCreateWithFlags(&p->aux_ev[nev], cudaEventDisableTiming) == cudaSuccess) ++nev;
    if (!cs || nev < 5) {
        for (int i = 0; i < nev; ++i) cudaEventDestroy(p->aux_ev[i]);
        if (cs) cudaStreamDestroy(p->copy_stream);
        if (ok) cudaStreamDestroy(p->aux_stream);
        p->aux_stream = nullptr;
        p->copy_stream = nullptr;
        return NFFT3_ERR_CUDA;
    }
    return NFFT3_OK;
}

// set_points(x) and eval(c) in one call: with the default gather and the
// fused transform, the transform of c runs on the plan's second stream while
// set_points sorts x on the plan's stream (they share no data), and the
// gather waits for both; otherwise the two calls in sequence.
template <typename R> int eval_points_impl(nfft3_plan p, const double *x, const R *c, R *f) {
    constexpr int prec = sizeof(R) == 8 ? 64 : 32;
    if (!p || p->prec != prec) return NFFT3_ERR_ARG;
    if (p->M > 0 && (!x || !c || !f)) return NFFT3_ERR_ARG;
    if (!(p->fused && p->gather_mode == 3 && p->M > 0)) {
        const int st = set_points_impl(p, x, prec);
        return st != NFFT3_OK ? st : eval_impl<R>(p, c, f);
    }
    int st = ensure_aux(p);
    if (st != NFFT3_OK) return st;
    // the second stream starts after the plan's earlier work (a previous
    // gather may still read the padded grid)
    if (cudaEventRecord(p->aux_ev[0], p->stream) != cudaSuccess ||
        cudaStreamWaitEvent(p->aux_stream, p->aux_ev[0], 0) != cudaSuccess)
        return NFFT3_ERR_CUDA;
    cudaStream_t own = p->stream;
    p->stream = p->aux_stream;   // the transform's launches go to the second stream
    st = precompute_impl<R>(p, c, 0);
    p->stream = own;
    if (st != NFFT3_OK || cudaEventRecord(p->aux_ev[4], p->aux_stream) != cudaSuccess) {
        cudaStreamSynchronize(p->aux_stream);
        return st != NFFT3_OK ? st : NFFT3_ERR_CUDA;
    }
    st = set_points_impl(p, x, prec);
    if (st != NFFT3_OK) {
        cudaStreamSynchronize(p->aux_stream);
        return st;
    }
    if (cudaStreamWaitEvent(p->stream, p->aux_ev[4], 0) != cudaSuccess) return NFFT3_ERR_CUDA;
    return eval_stored_impl<R>(p, f, nullptr, 1);
}

template <typename R> int eval_host_impl(nfft3_plan p, const double *x_host, const R *c_host, R *f_host) {
    constexpr int prec = sizeof(R) == 8 ? 64 : 32;
    if (!p || p->prec != prec) return NFFT3_ERR_ARG;
    if (!c_host || (p->M > 0 && (!x_host || !f_host))) return NFFT3_ERR_ARG;
    const int64_t NN = (int64_t)p->N[0] * p->N[1] * p->N[2];
    int st = NFFT3_OK;
    if (!p->x_dev) {
        void *v = nullptr;
        st = dev_alloc(p, &v, sizeof(double) * 3 * (p->M_cap + 1));
        p->x_dev = (double *)v;
        if (st == NFFT3_OK) st = dev_alloc(p, &p->c_dev, 2 * sizeof(R) * NN);
        if (st == NFFT3_OK) st = dev_alloc(p, &p->f_dev, 2 * sizeof(R) * (p->M_cap + 1));
        if (st == NFFT3_OK) st = ensure_aux(p);
        if (st != NFFT3_OK) {
            void *x = p->x_dev;
            dev_free(x);
            p->x_dev = nullptr;
            dev_free(p->c_dev);
            dev_free(p->f_dev);
            return st;
        }
    }
    if (p->fused && p->gather_mode == 3 && p->M > 0) {
        // The copy stream brings c, then x in two parts (each copy gets the
        // whole link); the transform of c runs on the auxiliary stream once
        // c has arrived; set_points' first pass starts on the first part of x
        // and takes the second part when it has arrived; the gather waits for
        // the transform.  Every stream starts after the plan's earlier work.
        const int64_t half = p->M / 2;
        auto drain = [p]() {
            cudaStreamSynchronize(p->copy_stream);
            cudaStreamSynchronize(p->aux_stream);
        };
        if (cudaEventRecord(p->aux_ev[0], p->stream) != cudaSuccess ||
            cudaStreamWaitEvent(p->copy_stream, p->aux_ev[0], 0) != cudaSuccess ||
            cudaMemcpyAsync(p->c_dev, c_host, 2 * sizeof(R) * NN, cudaMemcpyHostToDevice, p->copy_stream) !=
                cudaSuccess ||
            cudaEventRecord(p->aux_ev[1], p->copy_stream) != cudaSuccess ||
            cudaMemcpyAsync(p->x_dev, x_host, sizeof(double) * 3 * half, cudaMemcpyHostToDevice,
                            p->copy_stream) != cudaSuccess ||
            cudaEventRecord(p->aux_ev[2], p->copy_stream) != cudaSuccess ||
            cudaMemcpyAsync(p->x_dev + 3 * half, x_host + 3 * half, sizeof(double) * 3 * (p->M - half),
                            cudaMemcpyHostToDevice, p->copy_stream) != cudaSuccess ||
            cudaEventRecord(p->aux_ev[3], p->copy_stream) != cudaSuccess ||
            cudaStreamWaitEvent(p->aux_stream, p->aux_ev[1], 0) != cudaSuccess ||
            cudaStreamWaitEvent(p->stream, p->aux_ev[2], 0) != cudaSuccess) {
            drain();
            return NFFT3_ERR_CUDA;
        }
        cudaStream_t own = p->stream;
        p->stream = p->aux_stream;   // the transform's launches go to the auxiliary stream
        st = precompute_impl<R>(p, (const R *)p->c_dev, 0);
        p->stream = own;
        if (st != NFFT3_OK || cudaEventRecord(p->aux_ev[4], p->aux_stream) != cudaSuccess) {
            drain();
            return st != NFFT3_OK ? st : NFFT3_ERR_CUDA;
        }
        st = set_points_impl(p, p->x_dev, prec, half, p->aux_ev[3]);
        if (st != NFFT3_OK) {
            drain();
            return st;
        }
        if (cudaStreamWaitEvent(p->stream, p->aux_ev[4], 0) != cudaSuccess) return NFFT3_ERR_CUDA;
        st = eval_stored_impl<R>(p, (R *)p->f_dev, nullptr, 1);
        if (st < 0) return st;
        if (cudaMemcpyAsync(f_host, p->f_dev, 2 * sizeof(R) * p->M, cudaMemcpyDeviceToHost, p->stream) !=
            cudaSuccess)
            return NFFT3_ERR_CUDA;
        return cudaStreamSynchronize(p->stream) == cudaSuccess ? NFFT3_OK : NFFT3_ERR_CUDA;
    }
    // c on the auxiliary stream (after all earlier work of the plan's stream),
    // x and set_points on the plan's stream; eval waits for c
    if (cudaEventRecord(p->aux_ev[0], p->stream) != cudaSuccess ||
        cudaStreamWaitEvent(p->aux_stream, p->aux_ev[0], 0) != cudaSuccess ||
        cudaMemcpyAsync(p->c_dev, c_host, 2 * sizeof(R) * NN, cudaMemcpyHostToDevice, p->aux_stream) !=
            cudaSuccess ||
        cudaEventRecord(p->aux_ev[1], p->aux_stream) != cudaSuccess)
        return NFFT3_ERR_CUDA;
    if (p->M > 0 &&
        cudaMemcpyAsync(p->x_dev, x_host, sizeof(double) * 3 * p->M, cudaMemcpyHostToDevice,
                        p->stream) != cudaSuccess)
        return NFFT3_ERR_CUDA;
    st = set_points_impl(p, p->x_dev, prec);
    if (st != NFFT3_OK) {
        cudaStreamSynchronize(p->aux_stream);
        return st;
    }
    if (cudaStreamWaitEvent(p->stream, p->aux_ev[1], 0) != cudaSuccess) return NFFT3_ERR_CUDA;
    st = eval_impl<R>(p, (const R *)p->c_dev, (R *)p->f_dev);
    if (st < 0) return st;
    if (p->M > 0 &&
        cudaMemcpyAsync(f_host, p->f_dev, 2 * sizeof(R) * p->M, cudaMemcpyDeviceToHost, p->stream) !=
            cudaSuccess)
        return NFFT3_ERR_CUDA;
    return cudaStreamSynchronize(p->stream) == cudaSuccess ? NFFT3_OK : NFFT3_ERR_CUDA;
}

}  // namespace

extern "C" {

int nfft3_choose_m(double eps, double sigma) {
    if (sigma <= 0) sigma = 2.0;
    if (!(sigma > 1.0)) return kMaxM;
    for (int m = 1; m <= kMaxM; ++m)
        if (error_estimate(m, sigma) <= eps) return m;
    return kMaxM;
}

int nfft3d_plan(nfft3_plan *out, int N1, int N2, int N3, int64_t M, int m, double sigma,
                double eps, void *stream) {
    return make_plan(out, 64, N1, N2, N3, M, m, sigma, eps, stream);
}
int nfft3f_plan(nfft3_plan *out, int N1, int N2, int N3, int64_t M, int m, double sigma,
                double eps, void *stream) {
    return make_plan(out, 32, N1, N2, N3, M, m, sigma, eps, stream);
}

int nfft3d_set_points(nfft3_plan p, const double *x) { return finish(p, set_points_impl(p, x, 64)); }
int nfft3f_set_points(nfft3_plan p, const double *x) { return finish(p, set_points_impl(p, x, 32)); }

int nfft3d_eval(nfft3_plan p, const double *c, double *f) { return eval_impl<double>(p, c, f); }
int nfft3f_eval(nfft3_plan p, const float *c, float *f) { return eval_impl<float>(p, c, f); }

int nfft3d_eval_grad(nfft3_plan p, const double *c, double *f, double *grad) {
    return eval_grad_impl<double>(p, c, f, grad);
}
int nfft3f_eval_grad(nfft3_plan p, const float *c, float *f, float *grad) {
    return eval_grad_impl<float>(p, c, f, grad);
}

int nfft3d_chain_x(nfft3_plan p, const double *G, const double *grad, double *gx) {
    return chain_x_impl<double>(p, G, grad, gx);
}
int nfft3f_chain_x(nfft3_plan p, const float *G, const float *grad, double *gx) {
    return chain_x_impl<float>(p, G, grad, gx);
}

int nfft3d_eval_grad_window(nfft3_plan p, const double *c, double *f, double *grad) {
    return eval_grad_window_impl<double>(p, c, f, grad);
}
int nfft3f_eval_grad_window(nfft3_plan p, const float *c, float *f, float *grad) {
    return eval_grad_window_impl<float>(p, c, f, grad);
}
int nfft3d_eval_grad_window_stored(nfft3_plan p, double *f, double *grad) {
    return eval_grad_window_stored_impl<double>(p, f, grad);
}
int nfft3f_eval_grad_window_stored(nfft3_plan p, float *f, float *grad) {
    return eval_grad_window_stored_impl<float>(p, f, grad);
}

int nfft3d_precompute(nfft3_plan p, const double *c, int with_grad) {
    return precompute_impl<double>(p, c, with_grad);
}
int nfft3f_precompute(nfft3_plan p, const float *c, int with_grad) {
    return precompute_impl<float>(p, c, with_grad);
}
int nfft3d_eval_stored(nfft3_plan p, double *f) { return eval_stored_impl<double>(p, f, nullptr, 1); }
int nfft3f_eval_stored(nfft3_plan p, float *f) { return eval_stored_impl<float>(p, f, nullptr, 1); }
int nfft3d_eval_grad_stored(nfft3_plan p, double *f, double *grad) {
    return eval_stored_impl<double>(p, f, grad, 4);
}
int nfft3f_eval_grad_stored(nfft3_plan p, float *f, float *grad) {
    return eval_stored_impl<float>(p, f, grad, 4);
}

int nfft3_set_num_points(nfft3_plan p, int64_t M) {
    if (!p || M < 0) return NFFT3_ERR_ARG;
    if (M > p->M_cap) return NFFT3_ERR_TOO_LARGE;
    p->M = M;
    p->pb.M = M;
    p->points_ok = 0;
    return NFFT3_OK;
}

int nfft3d_adjoint(nfft3_plan p, const double *f, double *c_out) {
    return adjoint_impl<double>(p, f, c_out);
}
int nfft3f_adjoint(nfft3_plan p, const float *f, float *c_out) {
    return adjoint_impl<float>(p, f, c_out);
}

int nfft3d_eval_points(nfft3_plan p, const double *x, const double *c, double *f) {
    return eval_points_impl<double>(p, x, c, f);
}
int nfft3f_eval_points(nfft3_plan p, const double *x, const float *c, float *f) {
    return eval_points_impl<float>(p, x, c, f);
}

int nfft3d_eval_host(nfft3_plan p, const double *x_host, const double *c_host, double *f_host) {
    return eval_host_impl<double>(p, x_host, c_host, f_host);
}
int nfft3f_eval_host(nfft3_plan p, const double *x_host, const float *c_host, float *f_host) {
    return eval_host_impl<float>(p, x_host, c_host, f_host);
}

int nfft3d_destroy(nfft3_plan p) {
    if (p && p->prec != 64) return NFFT3_ERR_ARG;
    release(p);
    return NFFT3_OK;
}
int nfft3f_destroy(nfft3_plan p) {
    if (p && p->prec != 32) return NFFT3_ERR_ARG;
    release(p);
    return NFFT3_OK;
}

int nfft3_plan_info(nfft3_plan p, int *n, int *m, int64_t *M, int *prec) {
    if (!p) return NFFT3_ERR_ARG;
    if (n)
        for (int d = 0; d < 3; ++d) n[d] = p->n[d];
    if (m) *m = p->m;
    if (M) *M = p->M;
    if (prec) *prec = p->prec;
    return NFFT3_OK;
}

int nfft3_window_error(nfft3_plan p, double *max_abs_err) {
    if (!p || !max_abs_err) return NFFT3_ERR_ARG;
    *max_abs_err = p->window_err > p->window_err_df ? p->window_err : p->window_err_df;
    return NFFT3_OK;
}

int nfft3_set_stream(nfft3_plan p, void *stream) {
    if (!p) return NFFT3_ERR_ARG;
    p->stream = (cudaStream_t)stream;
    if (p->fft1 && cufftSetStream(p->fft1, p->stream) != CUFFT_SUCCESS) return NFFT3_ERR_CUFFT;
    if (p->have_fft4 && cufftSetStream(p->fft4, p->stream) != CUFFT_SUCCESS) return NFFT3_ERR_CUFFT;
    return NFFT3_OK;
}

int nfft3_sync(nfft3_plan p) {
    if (!p) return NFFT3_ERR_ARG;
    int status = 0;
    if (cudaMemcpyAsync(&status, p->pb.status, sizeof(int), cudaMemcpyDeviceToHost, p->stream) !=
        cudaSuccess)
        return NFFT3_ERR_CUDA;
    if (cudaStreamSynchronize(p->stream) != cudaSuccess) return NFFT3_ERR_CUDA;
    if (status & 2) return NFFT3_ERR_CUDA;   // a tile-staged gather gave up waiting for its copy
    return cudaGetLastError() == cudaSuccess ? NFFT3_OK : NFFT3_ERR_CUDA;
}

int nfft3_set_deterministic(nfft3_plan p, int on) {
    if (!p) return NFFT3_ERR_ARG;
    p->points_ok = 0;   // the point order changes: set_points must follow
    if (!on) {
        release_deterministic(p);
        return NFFT3_OK;
    }
    if (p->det) return NFFT3_OK;
    if (p->prec != 64) return NFFT3_ERR_ARG;
    const int64_t nn = (int64_t)p->n[0] * p->n[1] * p->n[2];
    const size_t cnt = stable_sort_count_ints(p->M_cap);
    void *v = nullptr;
    int st = dev_alloc(p, &v, sizeof(int) * (p->M_cap + 1));
    p->ss.buf = (int *)v;
    if (st == NFFT3_OK) st = dev_alloc(p, &v, sizeof(int) * cnt), p->ss.counts = (int *)v;
    if (st == NFFT3_OK) st = dev_alloc(p, &v, sizeof(int) * cnt), p->ss.offsets = (int *)v;
    if (st == NFFT3_OK) st = dev_alloc(p, &v, sizeof(int) * scan_tmp_ints((int64_t)cnt)), p->ss.scan_tmp = (int *)v;
    if (st == NFFT3_OK) st = dev_alloc(p, &v, 4 * sizeof(unsigned long long) * nn), p->Hq = (unsigned long long *)v;
    if (st != NFFT3_OK) {
        release_deterministic(p);
        return st;
    }
    p->det = 1;
    return NFFT3_OK;
}

int nfft3_timing_enable(nfft3_plan p, int on) {
    if (!p) return NFFT3_ERR_ARG;
    if (!on && p->nrec) fold_records(p);
    p->timing = on ? 1 : 0;
    return NFFT3_OK;
}

int nfft3_timing_read(nfft3_plan p, double *ms, int64_t *calls, int64_t *launches, int reset) {
    if (!p) return NFFT3_ERR_ARG;
    fold_records(p);
    for (int i = 0; i < NFFT3_NSTAGES; ++i) {
        if (ms) ms[i] = p->stage_ms[i];
        if (calls) calls[i] = p->stage_calls[i];
    }
    if (launches) *launches = p->launches;
    if (reset) {
        for (int i = 0; i < NFFT3_NSTAGES; ++i) p->stage_ms[i] = 0.0, p->stage_calls[i] = 0;
        p->launches = 0;
    }
    return NFFT3_OK;
}

const char *nfft3_error_string(int code) {
    switch (code) {
        case NFFT3_OK: return "ok";
        case NFFT3_WARN_EPS: return "warning: requested eps is below the estimate for this m";
        case NFFT3_ERR_ARG: return "invalid argument";
        case NFFT3_ERR_ALLOC: return "device allocation failed";
        case NFFT3_ERR_CUFFT: return "cuFFT error";
        case NFFT3_ERR_CUDA: return "CUDA error";
        case NFFT3_ERR_NO_POINTS: return "no points set";
        case NFFT3_ERR_POINTS: return "non-finite point coordinate";
        case NFFT3_ERR_TOO_LARGE: return "size exceeds library limits";
        case NFFT3_ERR_NO_COEFFS: return "no precomputed coefficients (call nfft3*_precompute)";
        default: return "unknown status";
    }
}

}  // extern "C"
