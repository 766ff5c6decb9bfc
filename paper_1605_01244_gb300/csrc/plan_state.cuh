// Definition of the plan object shared by the translation units that need
// its fields (plan.cu and noalloc.cu).  Not part of the public ABI.
#pragma once

#include "internal.cuh"

constexpr int kTimingRecords = 64;
constexpr int kTimingMarks = 5;

struct nfft3_plan_s {
    int prec;                 // 64 or 32
    int N[3], n[3], m;
    int64_t M;                // points in use (set_points reads M points)
    int64_t M_cap;            // capacity the point buffers were allocated for
    double b[3];
    cudaStream_t stream;
    int sync_check;           // GBNFFT_SYNC_CHECK set: synchronise after every call
    int fault;                // host-side fault injection (GBNFFT_FAULT)
    int device;
    // window polynomials (both precisions; the family uses one) and their checked error
    gbnfft::WinTable<double> wt64;
    gbnfft::WinTable<float> wt32;
    gbnfft::WinTableDF wtdf;   // FP64 family: double-float copy for the FP32-pipe gather
    void *wtdf_dev;            // FP64 family: wtdf in device memory (read by the adjoint spread)
    double window_err;
    double window_err_df;
    int df_weights_fp64;       // GBNFFT_DF_WEIGHTS: FP64-pipe weights (default) or df ("df")
    gbnfft::HalfTables half;   // FP64 family: half-interval tables of the value gather (mode: GBNFFT_SLOT_WEIGHTS)
    int gather_mode;           // GBNFFT_GATHER: 0 col (default), 1 thread, 2 native (see plan.cu)
    int spread_direct;         // GBNFFT_SPREAD=direct: one thread per point, global atomics only
    int adj_cufft;             // GBNFFT_ADJ_FFT=cufft: adjoint transform by cuFFT + deconvolution kernel
    unsigned tma_first_wait;   // GBNFFT_TMA_FIRST_WAIT (test of the tile-staged gather's bounded wait)
    // tables and grid
    void *D[3];               // deconvolution factors, real type of the family
    void *grid;               // n1 n2 n3 complex (x4 once eval_grad ran)
    int grid_count;           // 1 or 4
    void *pgrid;              // ghost-padded copy for the column gathers, (n+2m)^3 x pgrid_count
    int pgrid_count;
    int pgrid_shift;          // layout shift of its current contents (0 or m)
    int stored_ng;            // grids precomputed by nfft3*_precompute (0: none valid)
    // FP64 family range scaling: device words with the exponent rank of the
    // largest input of the current call; [0] coefficients (eval, eval_grad,
    // precompute; read again by the stored gathers), [1] adjoint values
    int *vexp;
    alignas(64) unsigned char tmap[128];  // CUtensorMap of the padded FP32 grid (tile-staged gather)
    int tmap_ok;
    int nchunks;              // chunks of the tile-staged gather for the current points
    int nbatch, nsparse;      // split gather lists for the current points (mixed family)
    int split_ok;             // the split lists describe the current points
    cufftHandle fft1;
    cufftHandle fft4;
    int have_fft4;
    // pruned transform (default; GBNFFT_FFT=full uses fft1/fft4): batched 2D
    // FFTs over the planes l1 with |k1| < N1/2, then 1D FFTs along l1
    int fft_pruned;
    // fused forward transform (power-of-two n; default for the padded-grid
    // gathers; GBNFFT_FFT=cufft or full selects cuFFT): twiddle tables
    // w_{n_d}^i (double-float float4 or float2) and the two line-pass buffers
    int fused;
    void *tw[3];
    void *fscratch;
    int fscratch_ng;
    cufftHandle fft2d;        // n2 x n3, batch N1/2 planes
    cufftHandle fft1d;        // length n1, stride n2 n3, batch n2 n3
    // points
    int points_ok;
    int4 *key;
    void *s[3];
    gbnfft::PointsBuild pb;
    // host-buffer staging (allocated on first _host call): eval_host copies
    // on copy_stream and, with the fused transform, transforms c on
    // aux_stream while x arrives and set_points runs on the plan's stream
    double *x_dev;
    void *c_dev;
    void *f_dev;
    cudaStream_t aux_stream;
    cudaStream_t copy_stream;   // host-buffer copies of eval_host
    cudaEvent_t aux_ev[5];
    // stage timing (CUDA events on the plan's stream), enabled by nfft3_timing_enable
    int timing;
    int nrec;
    cudaEvent_t ev[kTimingRecords][kTimingMarks];
    int rec_kind[kTimingRecords];
    int ev_ready[kTimingRecords];
    double stage_ms[NFFT3_NSTAGES];
    int64_t stage_calls[NFFT3_NSTAGES];
    int64_t launches;         // kernels this library enqueued (cuFFT's own not counted)
    // deterministic mode (nfft3_set_deterministic): stable point order and
    // exact fixed-point flushes of the adjoint spread
    int det;
    gbnfft::StableSort ss;
    unsigned long long *Hq;   // n1 n2 n3 x 4 int64 limbs
};

// Set-up of the allocation-free entry point on the plan's device (noalloc.cu):
// run by plan creation for FP64 plans; a no-op for plans it cannot serve.
int noalloc_setup(nfft3_plan p);
