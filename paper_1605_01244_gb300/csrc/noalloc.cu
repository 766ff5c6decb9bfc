// nfft3d_eval_grad_noalloc: the FP64 value+gradient evaluation with its four
// oversampled grids taken from a fixed, file-scope device array instead of
// plan-owned memory, so that the call allocates nothing.
//
// Why: nfft3d_eval_grad allocates its four gradient grids with cudaMalloc the
// first time it runs on a plan.  Some callers cannot allow that at call time:
// a process whose device memory is already reserved by another allocator (a
// framework's caching pool) where cudaMalloc may fail, and latency-sensitive
// loops where cudaMalloc's implicit device synchronisation would stall other
// streams.  This entry point serves them for small grids.
//
// Limit: the four grids (4 * n1*n2*n3 complex doubles) must fit in
// kNoAllocBytes = 16 MiB, i.e. n1*n2*n3 <= 262144 (64^3).
//
// Set-up: CUDA loads a library's device code lazily, and loading this file's
// code is what creates the 16 MiB array on a device.  So that the entry point
// itself never triggers a load, creating an FP64 plan whose grids fit does
// the set-up on the plan's device (noalloc_setup below): it looks up the
// array's address (which loads this code and the array), loads the kernels
// the entry point launches, and runs the plan's FFT once.  From then on the
// device holds the array until the process exits.
#include <mutex>

#include "internal.cuh"
#include "plan_state.cuh"

using namespace gbnfft;

namespace {

constexpr size_t kNoAllocBytes = size_t(16) << 20;
constexpr int kMaxDevices = 64;

// Shared by every call on a device: it keeps the last call's grids, and calls
// whose work overlaps on the GPU (two streams, or two host threads) race on it.
static __device__ __align__(256) unsigned char g_noalloc_grids[kNoAllocBytes];

std::mutex g_setup_mutex;
void *g_grids_addr[kMaxDevices];  // device address of g_noalloc_grids, per device

bool fits(const nfft3_plan p) {
    const int64_t nn = (int64_t)p->n[0] * p->n[1] * p->n[2];
    return (uint64_t)nn * 4 * sizeof(double2) <= kNoAllocBytes;
}

// The array's device address on the current device (in host code the symbol
// names a host-side stand-in, not device memory); looked up once per device.
int grids_address(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return NFFT3_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return NFFT3_ERR_TOO_LARGE;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_grids_addr[dev]) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_grids) != cudaSuccess || !ptr) {
            cudaGetLastError();
            return NFFT3_ERR_CUDA;
        }
        g_grids_addr[dev] = ptr;
    }
    *out = g_grids_addr[dev];
    return NFFT3_OK;
}

}  // namespace

// Called by plan creation for FP64 plans, with the plan's device current.
int noalloc_setup(nfft3_plan p) {
    if (p->prec != 64 || !fits(p)) return NFFT3_OK;
    void *base = nullptr;
    int st = grids_address(&base);
    if (st != NFFT3_OK) return st;
    if (preload_grad_kernels<double>(p->m) != cudaSuccess) return NFFT3_ERR_CUDA;
    // cuFFT may also load its kernels on a plan's first execution: run it once
    // on the plan's own (zeroed) grid, which every evaluation overwrites
    const int64_t nn = (int64_t)p->n[0] * p->n[1] * p->n[2];
    if (cudaMemsetAsync(p->grid, 0, sizeof(double2) * nn, p->stream) != cudaSuccess) return NFFT3_ERR_CUDA;
    if (cufftExecZ2Z(p->fft1, (cufftDoubleComplex *)p->grid, (cufftDoubleComplex *)p->grid, CUFFT_INVERSE) !=
        CUFFT_SUCCESS)
        return NFFT3_ERR_CUFFT;
    return cudaStreamSynchronize(p->stream) == cudaSuccess ? NFFT3_OK : NFFT3_ERR_CUDA;
}

extern "C" int nfft3d_eval_grad_noalloc(nfft3_plan p, const double *c, double *f, double *grad) {
    if (!p || p->prec != 64) return NFFT3_ERR_ARG;
    if (!p->points_ok) return NFFT3_ERR_NO_POINTS;
    if (p->M > 0 && (!c || !grad)) return NFFT3_ERR_ARG;
    if (!fits(p)) return NFFT3_ERR_TOO_LARGE;
    if (p->M == 0) return NFFT3_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device) return NFFT3_ERR_ARG;
    void *base = nullptr;
    int st = grids_address(&base);   // set up at plan creation: no CUDA call here
    if (st != NFFT3_OK) return st;
    double2 *G4 = (double2 *)base;
    const int64_t nn = (int64_t)p->n[0] * p->n[1] * p->n[2];
    const Grid3 g{p->n[0], p->n[1], p->n[2]};
    // every grid element (zeros included) is written here, so nothing left
    // over from an earlier call is read
    cudaError_t e = launch_deconv_scatter<double>((const double2 *)c, p->N[0], p->N[1], p->N[2],
                                                  (const double *)p->D[0], (const double *)p->D[1],
                                                  (const double *)p->D[2], G4, g, 1, nullptr, p->stream);
    if (e != cudaSuccess) return NFFT3_ERR_CUDA;
    for (int q = 0; q < 4; ++q) {
        cufftDoubleComplex *gq = (cufftDoubleComplex *)(G4 + q * nn);
        if (cufftExecZ2Z(p->fft1, gq, gq, CUFFT_INVERSE) != CUFFT_SUCCESS) return NFFT3_ERR_CUFFT;
    }
    PointsView<double> v;
    v.key = p->key;
    v.s1 = (const double *)p->s[0];
    v.s2 = (const double *)p->s[1];
    v.s3 = (const double *)p->s[2];
    v.M = p->M;
    v.vexp = nullptr;   // FP64 grids and the FP64-pipe gather: no range scaling needed
    e = launch_gather_grad<double>(G4, g, p->m, v, p->wt64, (double2 *)f, (double2 *)grad,
                                   p->stream);
    if (e != cudaSuccess) return NFFT3_ERR_CUDA;
    // this library's own kernels (deconvolve + scatter, gather); the four
    // cuFFT executions launch cuFFT's kernels, which no call counts
    p->launches += 2;
    if (p->sync_check) {
        if (cudaStreamSynchronize(p->stream) != cudaSuccess) return NFFT3_ERR_CUDA;
        if (cudaGetLastError() != cudaSuccess) return NFFT3_ERR_CUDA;
    }
    return NFFT3_OK;
}
