// Double-float gather, one thread per point, with the three gradient grids,
// for m <= 6 (the kernels are in gather_df.cuh; m = 7, 8 are instantiated in
// gather_df_grad_hi.cu so that the two compile in parallel).
#include "gather_df.cuh"

namespace gbnfft {

cudaError_t gather_grad_df_m_le6(const float4 *G4, Grid3 g, int m, PointsView<double> pts, const WinTableDF &w,
                                 double2 *f, double2 *grad, cudaStream_t st) {
    switch (m) {
        case 1: return df_dispatch<1, 4>(G4, g, pts, w, f, grad, st);
        case 2: return df_dispatch<2, 4>(G4, g, pts, w, f, grad, st);
        case 3: return df_dispatch<3, 4>(G4, g, pts, w, f, grad, st);
        case 4: return df_dispatch<4, 4>(G4, g, pts, w, f, grad, st);
        case 5: return df_dispatch<5, 4>(G4, g, pts, w, f, grad, st);
        case 6: return df_dispatch<6, 4>(G4, g, pts, w, f, grad, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_gather_grad_df(const float4 *G4, Grid3 g, int m, PointsView<double> pts,
                                  const WinTableDF &w, double2 *f, double2 *grad,
                                  cudaStream_t st) {
    if (pts.M == 0) return cudaSuccess;
    return m <= 6 ? gather_grad_df_m_le6(G4, g, m, pts, w, f, grad, st)
                  : gather_grad_df_m_gt6(G4, g, m, pts, w, f, grad, st);
}

}  // namespace gbnfft
