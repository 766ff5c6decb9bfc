/*
 * gbnfft -- 3D nonequispaced FFT (type-2 NFFT and its adjoint) for one GB300.
 *
 * The library evaluates the 3D truncated Fourier series of the INFFTM paper
 * (Caliari & Zuccher, arXiv:1605.01244, eq. (fs) and the NFFT transform of
 * Sec. 2.2.1, with the + sign of the physical series)
 *
 *     f_j = sum_{k in I_N} c_k exp(+2 pi i k . x_j),     j = 0..M-1,
 *     I_N = [-N1/2, N1/2) x [-N2/2, N2/2) x [-N3/2, N3/2),
 *
 * at M arbitrary torus points x_j (any real coordinates; the series is
 * 1-periodic, so they are wrapped onto [-1/2, 1/2)^3), its gradient
 * (eq. (Lambda) in torus units) and its adjoint
 *
 *     h_k = sum_j f_j exp(-2 pi i k . x_j).
 *
 * The paper uses the NFFT as a black box with cost O(N log N + M |log eps|^3)
 * (Sec. 1).  This library's approximation: deconvolve by the Fourier
 * transform of a Kaiser-Bessel window and zero-pad into an oversampled grid
 * of n_d >= sigma N_d points, one unnormalised inverse 3D FFT, then a
 * (2m+1)^3-tap window sum per point.
 *
 * Data layout (all device pointers unless a name ends in _host):
 *   c    : N1*N2*N3 complex values, row-major (i3 fastest), entry (i1,i2,i3)
 *          holding k_d = i_d - N_d/2.  Complex = two interleaved reals
 *          (re, im): double for the nfft3d_* family, float for nfft3f_*.
 *   x    : M*3 doubles, row-major (x_j0, x_j1, x_j2), both families.
 *   f    : M complex values (same real type as c).
 *   grad : M*3 complex values, grad[3j+d] = d f_j / d x_{j,d}.
 *
 * Families: nfft3d_* ("FP64") takes and returns FP64 values and meets an
 * FP64 accuracy class (relative l2 error <= 1e-12 at m >= 6, sigma = 2),
 * but its transform, window sums and adjoint spread run in double-float
 * arithmetic: pairs of floats carrying about 48 significant bits, on the
 * FP32 pipe (GB300's FP64 pipe is 64x slower).  The coordinate reduction,
 * the deconvolution tables and the adjoint's FFT and final deconvolution are
 * FP64.  Range: every call scales its input values (c, or f for the adjoint)
 * by the exact power of two that brings the largest magnitude into [1, 2),
 * and scales its results back, so any finite FP64 input is served; input
 * entries below 2^-100 of the largest are dropped (their share of any result
 * is below 2^-100 of its scale).  nfft3f_* ("mixed") keeps the coordinate
 * reduction and the deconvolution tables in FP64 and runs the grid, FFT,
 * window sums and spreading in FP32, with FP32's range.
 *
 * Ownership: the plan owns all device workspaces.  Pointers passed to a call
 * are borrowed for the duration of the call (the work is enqueued on the
 * plan's stream; the caller keeps the buffers alive until that stream has
 * finished the work).  set_points copies what it needs from x.
 *
 * Errors: every call returns an int status: 0 OK, > 0 warning, < 0 error
 * (NFFT3_ERR_*).  No call aborts, throws or prints.  Kernel faults surface
 * as NFFT3_ERR_CUDA from the next call that synchronises (set_points, the
 * _host calls, nfft3_sync).  A plan is used from one host thread and one
 * stream at a time.
 */
#ifndef GBNFFT_H
#define GBNFFT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nfft3_plan_s *nfft3_plan;

enum {
    NFFT3_OK = 0,
    NFFT3_WARN_EPS = 1,        /* the requested eps is below what the plan's m reaches */
    NFFT3_ERR_ARG = -1,        /* bad argument (size, null pointer, precision family) */
    NFFT3_ERR_ALLOC = -2,      /* device allocation failed */
    NFFT3_ERR_CUFFT = -3,      /* cuFFT plan or exec failed */
    NFFT3_ERR_CUDA = -4,       /* CUDA launch or runtime error */
    NFFT3_ERR_NO_POINTS = -5,  /* eval/adjoint before a successful set_points */
    NFFT3_ERR_POINTS = -6,     /* a point coordinate is NaN or infinite */
    NFFT3_ERR_TOO_LARGE = -7,  /* a size exceeds the library's limits */
    NFFT3_ERR_NO_COEFFS = -8   /* *_stored call without a valid *_precompute */
};

/*
 * Create a plan.
 *   N1,N2,N3 : even, >= 2 (paper Sec. 2: N_d even), each <= 4096.
 *   M        : number of points, 0 <= M < 2^31.
 *   m        : window cutoff, 1..8 (2m+1 taps per dimension); if m <= 0 it
 *              is chosen from eps (smallest m whose relative l2 error
 *              estimate 8 exp(-2 pi sqrt(1 - 1/sigma) (m + 1/2)) is <= eps;
 *              the estimate bounds the measured error for flat spectra).
 *              If m > 0, eps is only checked (warning if the estimate
 *              exceeds it); eps <= 0 skips the check.
 *   sigma    : oversampling factor >= 1.25 (<= 0 selects 2); n_d is the
 *              smallest even integer >= sigma N_d with no prime factor > 7.
 *   stream   : cudaStream_t to enqueue all work on (NULL = legacy stream).
 * The plan is created on the device current at the call.
 */
int nfft3d_plan(nfft3_plan *out, int N1, int N2, int N3, int64_t M, int m,
                double sigma, double eps, void *stream);
int nfft3f_plan(nfft3_plan *out, int N1, int N2, int N3, int64_t M, int m,
                double sigma, double eps, void *stream);

/*
 * Set the M points (device pointer x, M*3 doubles).  Each coordinate is
 * wrapped onto [-1/2, 1/2) (the series is periodic; paper Sec. 2.2.1 uses
 * mod(.,1)), reduced with FP64 rounding to its first stencil node and a
 * fractional offset (nfft3_reduce_coords), and the points are bucketed by grid tile.  Synchronises the
 * plan's stream (it reads back a status word).  NaN/Inf coordinates give
 * NFFT3_ERR_POINTS and leave the plan without points.
 */
int nfft3d_set_points(nfft3_plan p, const double *x);
int nfft3f_set_points(nfft3_plan p, const double *x);

/*
 * The per-coordinate reduction of set_points on its own, for inspection:
 * for each of the M doubles x[j] (device) and an oversampled size n with
 * cutoff m (1..8), the first stencil node l0[j] = ceil(u - m - 1/2) wrapped
 * into [0, n), u = n (x_w + 1/2), x_w = x - floor(x + 1/2), and the offset
 * s = l0 - (u - m - 1/2) in [0, 1) as the FP64 family stores it (s) and as
 * the mixed family stores it (s32: the FP64 value's significand truncated to
 * FP32).  Every step rounds like FP64 round-to-nearest arithmetic; for
 * n = 2^L (8 <= n <= 2^30) the steps after x_w + 1/2 run on the integer
 * pipe with the same results, except next to x = -1/2.  Any of l0, s, s32 may be NULL.  *status
 * (device int) is zeroed and gets bit 0 if some x[j] is NaN or infinite
 * (that coordinate is reduced as 0).  Asynchronous on the stream.
 * Coordinate wrap: paper Sec. 2.2.1.
 */
int nfft3_reduce_coords(int n, int m, const double *x, int64_t M, int *l0, double *s, float *s32,
                        int *status, void *stream);

/* f = A c  (type-2 NFFT).  c: N1*N2*N3 complex, f: M complex (overwritten). */
int nfft3d_eval(nfft3_plan p, const double *c, double *f);
int nfft3f_eval(nfft3_plan p, const float *c, float *f);

/*
 * f = A c and grad_d f = A (2 pi i k_d c), d = 1..3 (eq. (Lambda), torus
 * units; physical units divide by b_d - a_d).  f may be NULL.
 * grad: M*3 complex, grad[3j+d].
 */
int nfft3d_eval_grad(nfft3_plan p, const double *c, double *f, double *grad);
int nfft3f_eval_grad(nfft3_plan p, const float *c, float *f, float *grad);

/*
 * Chain rule for the point coordinates, the backward pass of f = A(x) c in x:
 *   gx[3j+d] = Re(conj(G_j) grad[3j+d]) = Re G_j Re grad[3j+d] + Im G_j Im grad[3j+d],
 * with G_j = dL/d(Re f_j) + i dL/d(Im f_j) (M complex, interleaved, the
 * plan's precision) and grad the 3M complex gradient of nfft3*_eval_grad at
 * the same points (torus units, Sec. 2 / eq. (Lambda)).  gx: 3M doubles,
 * written.  All three are device pointers owned by the caller; the kernel
 * runs on the plan's stream (computed in FP64 for both families).
 * NFFT3_ERR_ARG: a NULL pointer with M > 0, or a precision mismatch.
 */
int nfft3d_chain_x(nfft3_plan p, const double *G, const double *grad, double *gx);
int nfft3f_chain_x(nfft3_plan p, const float *G, const float *grad, double *gx);

/*
 * f and grad as nfft3*_eval_grad, by differentiating the window instead of
 * the series: one oversampled transform of c, then
 *   grad_d f_j = sum_l g_l n_d phi'(u_d - l_d) prod_{e != d} phi(u_e - l_e),
 * the derivative of the window sum of eq. (fs)'s NFFT approximation
 * (u = n (x + 1/2), torus units).  One grid and one transform instead of four;
 * the approximation error of the gradient is about ten times that of
 * nfft3*_eval_grad at the same m (one more m gives the same accuracy).
 * Default and tma gather modes only (NFFT3_ERR_ARG otherwise).
 * The _stored variant gathers from the grid of a preceding
 * nfft3*_precompute(c, 0 or 1) (NFFT3_ERR_NO_COEFFS without one;
 * NFFT3_ERR_ARG if that grid was stored in the tile-staged layout).
 */
int nfft3d_eval_grad_window(nfft3_plan p, const double *c, double *f, double *grad);
int nfft3f_eval_grad_window(nfft3_plan p, const float *c, float *f, float *grad);
int nfft3d_eval_grad_window_stored(nfft3_plan p, double *f, double *grad);
int nfft3f_eval_grad_window_stored(nfft3_plan p, float *f, float *grad);

/*
 * nfft3d_eval_grad without allocation.  The paper has no counterpart: this
 * is a service for callers that cannot call cudaMalloc when they evaluate --
 * a process whose device memory is already reserved by another allocator (a
 * framework's caching pool, where cudaMalloc may fail), or a latency-bound
 * loop that cannot take cudaMalloc's implicit device synchronisation.
 * nfft3d_eval_grad allocates its four gradient grids on first use; this
 * variant computes the same f and grad (same layout and meaning) with those
 * grids in a fixed 16 MiB device array compiled into the library.  It calls
 * no cudaMalloc, cudaFree or allocating library routine, and it loads no
 * device code: CUDA loads a library's device code lazily, and loading the
 * code that holds the array is what creates the array on a device, so the
 * set-up happens when an FP64 plan whose grids fit is created
 * (nfft3d_plan looks up the array's device address with
 * cudaGetSymbolAddress, loads the kernels this call launches and runs the
 * plan's FFT once).  From the first such plan on, the device holds the
 * 16 MiB until the process exits.  Create the plan before any stream
 * capture.
 *   Limit: 4 * n1*n2*n3 complex doubles must fit, i.e. n1*n2*n3 <= 262144
 *   (64^3); larger plans get NFFT3_ERR_TOO_LARGE.  FP64 plans only
 *   (NFFT3_ERR_ARG for a mixed plan).
 *   All calls share the array: calls whose work overlaps on the GPU (other
 *   streams or host threads) race and give wrong results.  Each call rewrites
 *   every grid element before reading it, so leftover contents are harmless.
 */
int nfft3d_eval_grad_noalloc(nfft3_plan p, const double *c, double *f, double *grad);

/*
 * Evaluate one series at many point sets: nfft3*_precompute runs the
 * deconvolution, oversampled FFT(s) and padding for c once and keeps the
 * result in the plan (with_grad != 0: also the three gradient grids);
 * nfft3*_eval_stored / nfft3*_eval_grad_stored then gather at the points
 * currently set (f and grad as in eval / eval_grad; grad requires a
 * with_grad precompute).  set_points keeps the stored grids; eval,
 * eval_grad and adjoint overwrite them (a later *_stored call returns
 * NFFT3_ERR_NO_COEFFS).  Default gather mode only.
 */
int nfft3d_precompute(nfft3_plan p, const double *c, int with_grad);
int nfft3f_precompute(nfft3_plan p, const float *c, int with_grad);
int nfft3d_eval_stored(nfft3_plan p, double *f);
int nfft3f_eval_stored(nfft3_plan p, float *f);
int nfft3d_eval_grad_stored(nfft3_plan p, double *f, double *grad);
int nfft3f_eval_grad_stored(nfft3_plan p, float *f, float *grad);

/*
 * Use the first M points of the plan's capacity (0 <= M <= the M given at
 * plan creation): later set_points reads M points and eval writes M values.
 * Clears the points (set_points must follow).
 */
int nfft3_set_num_points(nfft3_plan p, int64_t M);

/*
 * Deterministic mode (on != 0; FP64 plans): set_points orders
 * the points of each tile by original index (a stable radix sort instead of
 * the atomic counting sort), and the adjoint's spread adds its tile boxes to
 * the grid as exact fixed-point sums (two int64 limbs per component,
 * resolution 2^-60 of the range-scaled values) instead of FP64 additions in
 * whatever order the blocks run (atomics, or bulk row reductions), so that
 * adjoint results are bitwise reproducible from run to run.  Allocates
 * 32 bytes per oversampled grid node plus sort buffers; on == 0 releases
 * them.  Either way the points must be set again (NFFT3_ERR_NO_POINTS until
 * then).  NFFT3_ERR_ARG for mixed plans, or the one-thread spread
 * (GBNFFT_SPREAD=direct) at adjoint time.  Eval results are bitwise
 * reproducible in both modes.
 */
int nfft3_set_deterministic(nfft3_plan p, int on);

/* c_out = A^H f  (type-1 adjoint): c_out[k] = sum_j f_j exp(-2 pi i k.x_j). */
int nfft3d_adjoint(nfft3_plan p, const double *f, double *c_out);
int nfft3f_adjoint(nfft3_plan p, const float *f, float *c_out);

/*
 * nfft3*_set_points(x) followed by nfft3*_eval(c, f), in one call, with the
 * same arguments, results and errors as those two calls (device pointers;
 * x is read, c read, f written).  With the default gather and the fused
 * transform (power-of-two oversampled sizes) the transform of c runs on a
 * second stream owned by the plan while set_points sorts x on the plan's
 * stream -- the two share no data -- and the gather waits for both; in
 * other configurations the two calls run in sequence.  Returns after
 * set_points' checks, like nfft3*_set_points; the evaluation completes
 * asynchronously on the plan's stream.
 */
int nfft3d_eval_points(nfft3_plan p, const double *x, const double *c, double *f);
int nfft3f_eval_points(nfft3_plan p, const double *x, const float *c, float *f);

/*
 * Host-buffer variants: copy x_host (M*3 doubles) and c_host (N^3 complex)
 * to plan-owned device buffers, set the points, evaluate, copy f back into
 * f_host (M complex) and synchronise.  Pinned host memory gives full copy
 * bandwidth; pageable memory works but is slower.  With the default gather
 * and the fused transform, c and then x (in two halves) are copied on a copy
 * stream owned by the plan, c is transformed on a second plan-owned stream
 * as soon as it has arrived, and set_points starts on the first half of x
 * on the plan's stream; the gather waits for both.
 */
int nfft3d_eval_host(nfft3_plan p, const double *x_host, const double *c_host, double *f_host);
int nfft3f_eval_host(nfft3_plan p, const double *x_host, const float *c_host, float *f_host);

/* Release the plan and every device buffer it owns.  NULL is accepted. */
int nfft3d_destroy(nfft3_plan p);
int nfft3f_destroy(nfft3_plan p);

/*
 * Plan introspection.  Any output pointer may be NULL.
 *   n[3]: oversampled sizes;  m: cutoff;  M: points;  prec: 64 or 32.
 */
int nfft3_plan_info(nfft3_plan p, int *n, int *m, int64_t *M, int *prec);

/*
 * Largest absolute error of the plan's window weights (each tap's weight is
 * a polynomial fitted at plan creation; weights are normalised to 1 at the
 * window centre), measured on the host in the family's precision.
 */
int nfft3_window_error(nfft3_plan p, double *max_abs_err);

/* Change the stream later calls enqueue on. */
int nfft3_set_stream(nfft3_plan p, void *stream);

/* Wait for the plan's stream and report any asynchronous CUDA error (including
 * a tile-staged gather that gave up waiting for its shared-memory copy). */
int nfft3_sync(nfft3_plan p);

/* Static description of a status code. */
const char *nfft3_error_string(int code);

/*
 * Stage timing.  While enabled, every call records CUDA events on the plan's
 * stream around its stages; nfft3_timing_read waits for them and returns
 * the summed milliseconds and call counts per stage (arrays of
 * NFFT3_NSTAGES, NULL allowed) and the number of kernels this library
 * enqueued since the last reset (cuFFT's internal kernels not counted).
 * Timing adds no synchronisation to the calls themselves.
 */
enum {
    NFFT3_STAGE_SET_POINTS = 0,  /* reduction + counting sort          */
    NFFT3_STAGE_DECONV = 1,      /* deconvolve + zero-pad scatter      */
    NFFT3_STAGE_FFT = 2,         /* oversampled inverse FFT (cuFFT)    */
    NFFT3_STAGE_GATHER = 3,      /* window gather (value or gradient)  */
    NFFT3_STAGE_SPREAD = 4,      /* adjoint: clear + spread            */
    NFFT3_STAGE_FFT_FWD = 5,     /* adjoint: forward FFT (cuFFT)       */
    NFFT3_STAGE_DECONV_ADJ = 6,  /* adjoint: deconvolve + gather of c  */
    NFFT3_STAGE_SPLIT = 7,       /* FP64 family: split the grid into hi/lo floats */
    NFFT3_NSTAGES = 8
};
int nfft3_timing_enable(nfft3_plan p, int on);
int nfft3_timing_read(nfft3_plan p, double *ms, int64_t *calls, int64_t *launches, int reset);

/*
 * One Newton step towards the zero set of psi (vortex cores), for M points
 * (device arrays).  F = (Re psi, Im psi) and J = [Re grad psi; Im grad psi]
 * (2 x 3) come from nfft3*_eval_grad at x (f: M complex, grad: M*3 complex,
 * double2 for prec 64, float2 for prec 32); the minimum-norm step
 * dx = -J^T (J J^T)^{-1} F is added to x (M*3 doubles) for active points.
 * status[j] (int, caller-initialised to 0): 0 active, 1 converged
 * (|psi| < tol at the x it was evaluated at; x not moved), 2 singular
 * J J^T (det <= 1e-30 (|Re grad|^2 + |Im grad|^2)^2), 3 step longer than
 * max_step (torus units).  resid[j] receives |psi| at the evaluated x.
 * The paper finds cores by thresholding rho = |psi|^2 on refined point sets
 * (Sec. 4.3, sftubeeval3); this step refines candidates onto the zero set.
 */
int nfft3_newton_step(int prec, int64_t M, double *x, const void *f, const void *grad,
                      int *status, double *resid, double tol, double max_step, void *stream);

/*
 * keep[i] = 1 when status[i] == 1 and no converged point of lower index lies
 * within radius of x_i (periodic distance on the unit torus); else 0.
 */
int nfft3_dedupe(int64_t M, const double *x, const int *status, double radius, int *keep,
                 void *stream);

/*
 * Dense local-grid core detection.
 * nfft3_lattice_points: x[(i1 R2 + i2) R3 + i3] = lo + i * h (device x, R1 R2 R3 x 3
 * doubles; lo, h: host arrays of 3), the points at which psi is evaluated.
 * nfft3_plaquette_crossings: for psi sampled on that lattice (device, R1 R2 R3
 * complex; double2 for prec 64, float2 for prec 32), finds every lattice face
 * around which the phase of psi winds by +-2 pi (sum of the four phase
 * differences, each wrapped into (-pi, pi]) -- a vortex core crosses that
 * face.  Writes the face centres (out: cap x 3 doubles, torus coordinates)
 * and out_dir = +-(normal direction 1..3) signed by the winding; *count
 * (device unsigned long long, zeroed by the call) receives the total number
 * found, which may exceed cap (then only cap are written).  The paper marks
 * low-density lattice nodes instead (Sec. 5: rho = |psi|^2 <= 0.0012).
 */
int nfft3_lattice_points(double *x, int R1, int R2, int R3, const double *lo, const double *h,
                         void *stream);
int nfft3_plaquette_crossings(int prec, const void *psi, int R1, int R2, int R3, const double *lo,
                              const double *h, double *out, int *out_dir, int64_t cap,
                              unsigned long long *count, void *stream);

/*
 * One- and two-dimensional NFFT (the paper's infft and infft2, Appendix B),
 * FP64, one call:  f_j = sum_k c_k exp(+2 pi i k.x_j), k_d in [-N_d/2, N_d/2),
 * with the 3D path's window (Kaiser-Bessel, half-width m + 1/2 grid cells,
 * sigma = n_d / N_d, n_d the smallest even 7-smooth integer >= sigma N_d):
 * deconvolve + zero-pad, cuFFT inverse transform, window sum.
 *   dim: 1 or 2;  N: host array of dim sizes (even, >= 2);  m in 1..8;
 *   sigma in [1.25, 8] (<= 0: 2);  x: device, M x dim doubles (any finite
 *   values; periodic);  c: device, N1 (x N2) complex doubles, centred order,
 *   row-major;  f: device, M complex doubles (overwritten).
 *   workspace: device memory of nfft_lowdim_workspace_bytes bytes.
 * Synchronises the stream (the non-finite-coordinate check is read back:
 * NFFT3_ERR_POINTS).  Returns NFFT3_ERR_ARG for invalid sizes (0 bytes from
 * the workspace query).
 */
size_t nfft_lowdim_workspace_bytes(int dim, const int *N, int m, double sigma);
int nfft_lowdim_eval(int dim, const int *N, int64_t M, int m, double sigma, const double *x, const double *c,
                     double *f, void *workspace, size_t ws_bytes, void *stream);

/*
 * Evaluation on a rectilinear grid (the paper's igridftn / ndcovlt, Sec. 2.1):
 *   f[(i1 M2 + i2) M3 + i3] = sum_k c_k exp(+2 pi i (k1 y1[i1] + k2 y2[i2] + k3 y3[i3]))
 * for the grid y1 x y2 x y3 (device arrays of M1, M2, M3 torus coordinates),
 * computed exactly (no window approximation) as three dense complex
 * contractions, one dimension at a time (the library's own complex matrix
 * products: FP32 for nfft3f_*, FP64 for nfft3d_* -- or double-float on the
 * FP32 pipe, about 48 significant bits, with GBNFFT_GRID_DF=1).  c as in
 * eval, f: M1 M2 M3 complex (device, overwritten).  workspace: device memory
 * of nfft3_grid_eval_workspace_bytes bytes (the three exponential matrices,
 * two partial contractions and one range word: M1 N1 + M2 N2 + M3 N3 +
 * N1 N2 M3 + N1 M2 M3 + 1 complex).  Asynchronous on the stream.  N1 N2 and
 * M2 M3 must stay below 2^31, N1 N2 and M1, M2 below 65535 * 64 and N1
 * below 65536 (NFFT3_ERR_TOO_LARGE).
 */
size_t nfft3_grid_eval_workspace_bytes(int prec, int N1, int N2, int N3, int M1, int M2, int M3);
int nfft3d_grid_eval(const double *c, int N1, int N2, int N3, const double *y1, int M1, const double *y2, int M2,
                     const double *y3, int M3, double *f, void *workspace, size_t ws_bytes, void *stream);
int nfft3f_grid_eval(const float *c, int N1, int N2, int N3, const double *y1, int M1, const double *y2, int M2,
                     const double *y3, int M3, float *f, void *workspace, size_t ws_bytes, void *stream);

/*
 * One refinement step of the vortex-tube evaluation (Sec. 4.3, sftubeeval3):
 * of the M points x (device, M x 3 doubles) with values psi (device, M
 * complex; double2 for prec 64, float2 for prec 32), keep those with
 * rho = |psi|^2 <= rhobar and write, for the r-th kept point xi (in input
 * order), the 27 points xi + (a h1/3, b h2/3, c h3/3), a, b, c in {-1, 0, 1}
 * (c fastest) to out[27 r .. 27 r + 26] (device, cap x 3 doubles; h: host
 * array of the current step sizes).  *kept (host) receives the number of kept
 * points; the call synchronises the stream to read it.  Returns
 * NFFT3_ERR_TOO_LARGE if 27 * kept > cap (then only the first cap points are
 * written).  workspace: device memory of nfft3_tube_workspace_bytes(M)
 * bytes.  Deterministic (a scan, no atomics).
 */
size_t nfft3_tube_workspace_bytes(int64_t M);
int nfft3_tube_refine(int prec, const double *x, const void *psi, int64_t M, double rhobar, const double *h,
                      double *out, int64_t cap, int64_t *kept, void *workspace, size_t ws_bytes,
                      void *stream);

/*
 * Kernels of the core-proposal CNN (no counterpart in the paper: a learned
 * proposal stage in front of the NFFT + Newton refinement).  All pointers
 * are device pointers; activations and weights are BF16 (bit pattern
 * __nv_bfloat16, passed as void*), accumulations FP32.  Activations are
 * [B][C][D][D][D] row-major, weights [Cout][Cin][k][k][k] with k = 1 or 3 and
 * zero padding k/2 (output size = input size), bias [Cout].
 *   cnn_conv3d_fwd:   y = conv(x, w) + bias, optional ReLU; y_bf16 and/or y_f32.
 *   cnn_conv3d_dgrad: dx = conv^T(dy, w), times the ReLU mask (relu_mask[i] > 0)
 *                     of the layer input when relu_mask != NULL.
 *   cnn_conv3d_wgrad: dw (FP32, same layout as w) and db (FP32, may be NULL);
 *                     takes B (Cout Cin k^3 + Cout) floats of stream-ordered
 *                     scratch (cudaMallocAsync) for the per-batch-entry
 *                     partial sums (NFFT3_ERR_ALLOC if that fails).
 *   k = 1 or 3 with at most 16 channels in and out run the shared-memory tiled
 *   kernels (8 x 8 x 4 voxel tiles); other shapes, or GBNFFT_CNN_NAIVE=1, one
 *   output per thread.  Every sum is in a fixed order (deterministic).
 *   cnn_core_loss:    4-channel head y (FP32: logit, 3 offsets) vs target
 *                     (B D^3 in {0,1}) and off_target (B D^3 x 3): mean BCE,
 *                     positives weighted by pos_weight, + lam * L1 over the
 *                     positive voxels (npos of them);
 *                     writes dy, adds the loss to *loss (caller zeroes it).
 *   cnn_adam:         Adam step `step` (1-based) on FP32 master weights, also
 *                     writing the BF16 copy when w_bf16 != NULL.
 */
int cnn_conv3d_fwd(const void *x, const void *w, const float *bias, int B, int Cin, int Cout, int D,
                   int k, int relu, void *y_bf16, float *y_f32, void *stream);
int cnn_conv3d_dgrad(const float *dy, const void *w, int B, int Cin, int Cout, int D, int k,
                     const void *relu_mask, float *dx, void *stream);
int cnn_conv3d_wgrad(const float *dy, const void *x, int B, int Cin, int Cout, int D, int k, float *dw,
                     float *db, void *stream);
int cnn_core_loss(const float *y, const float *target, const float *off_target, int B, int D, float lam,
                  float pos_weight, float npos, float *dy, float *loss, void *stream);
int cnn_adam(float *w_master, void *w_bf16, const float *g, float *m1, float *m2, int64_t n, float lr,
             float b1, float b2, float eps, int step, void *stream);

/*
 * CUDA-core FMA throughput of the current device in TFLOP/s (2 flops per FMA),
 * measured by a kernel of independent FMA chains on every SM (prec 64 or 32;
 * iters sets the run length).  Used to state the ALU roofline of the window
 * sums; not part of the transform.
 */
int nfft3_fma_peak(int prec, int iters, void *stream, double *tflops);

/*
 * m chosen for (eps, sigma) by the rule documented at nfft3d_plan
 * (returns 1..8, or 8 when eps is below what m = 8 reaches).
 */
int nfft3_choose_m(double eps, double sigma);

/*
 * Gross-Pitaevskii solver: time-splitting pseudospectral (TSSP) integration
 * of the paper's eq. (GPE) (Sec. 3),
 *     psi_t = (i/2) Lap psi + (i/2) (1 - |psi|^2) psi,
 * by the Strang splitting of Sec. 3.1 on a periodic box of sides L1, L2, L3
 * sampled at n1 x n2 x n3 points x = a + L_d i_d / n_d (the solver does not
 * need the origin a).  psi: device, n1*n2*n3 FP64 complex (re, im
 * interleaved), row-major with i3 fastest; it is advanced in place.  A step
 * is a potential half step (exact: psi <- exp(i t (1 - |psi|^2) / 2) psi
 * with t = tau / 2), the kinetic step (exact in Fourier space: psi_hat_k <-
 * exp(-i tau |kappa_k|^2 / 2) psi_hat_k, kappa_d = 2 pi k_d / L_d, cuFFT
 * Z2Z transforms) and a second potential half step; consecutive half steps
 * within one gpe_steps call are merged.  Work is enqueued on the plan's
 * stream.  The plan owns a FP64 complex work grid (for the diagnostics) and
 * a cuFFT plan.
 *   gpe_plan_create: n_d >= 1, L_d > 0; NFFT3_ERR_ALLOC / _CUFFT on failure.
 *   gpe_steps: nsteps >= 0 steps of size tau (the kinetic tables are rebuilt
 *     when tau changes; that call synchronises the stream).
 *   gpe_mass_energy: the discrete mass sum |psi|^2 dV and the energy of the
 *     paper's eq. (energy), (1/2) int |grad psi|^2 + (1/4) int (1 - |psi|^2)^2
 *     (the gradient spectrally), dV = L1 L2 L3 / (n1 n2 n3); synchronises.
 *     Either output pointer may be NULL.
 */
typedef struct gpe_plan_s *gpe_plan;
int gpe_plan_create(gpe_plan *out, int n1, int n2, int n3, double L1, double L2, double L3, void *stream);
int gpe_steps(gpe_plan p, double *psi, double tau, int nsteps);
int gpe_mass_energy(gpe_plan p, const double *psi, double *mass, double *energy);
int gpe_destroy(gpe_plan p);

#ifdef __cplusplus
}
#endif

#endif /* GBNFFT_H */
