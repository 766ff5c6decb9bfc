// Instantiation of kernels.cuh for the mixed family (float).
#include "kernels.cuh"

namespace gbnfft {
GBNFFT_INSTANTIATE(float)
}  // namespace gbnfft
