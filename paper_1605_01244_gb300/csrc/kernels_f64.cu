// Instantiation of kernels.cuh for the FP64 family (double).
#include "kernels.cuh"

namespace gbnfft {
GBNFFT_INSTANTIATE(double)
}  // namespace gbnfft
