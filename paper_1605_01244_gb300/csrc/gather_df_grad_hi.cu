// Double-float gather, one thread per point, with the three gradient grids,
// for m = 7, 8 (see gather_df_grad.cu).
#include "gather_df.cuh"

namespace gbnfft {

cudaError_t gather_grad_df_m_gt6(const float4 *G4, Grid3 g, int m, PointsView<double> pts, const WinTableDF &w,
                                 double2 *f, double2 *grad, cudaStream_t st) {
    switch (m) {
        case 7: return df_dispatch<7, 4>(G4, g, pts, w, f, grad, st);
        case 8: return df_dispatch<8, 4>(G4, g, pts, w, f, grad, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace gbnfft
