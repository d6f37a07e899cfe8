// hd_nd_rows.cu -- instantiation and launch of k_rows_rcm (row pairs with the operator C_1 of Sec. 5).
#include "hd_nd_kernels.cuh"

namespace hd {

cudaError_t launch_rows_rcm(Eng e, unsigned grid, int T, size_t smem, cudaStream_t st, float2* F, const float2* G,
                            float2* O, RowGeom rg, float scale, const float2* tw, FftPlan pl) {
  auto k = e == Eng::SE    ? k_rows_rcm<kPtsSE, false, true>
           : e == Eng::TC  ? k_rows_rcm<kPts, true, false>
           : e == Eng::TCS ? k_rows_rcm<kPts, true, true>
                           : k_rows_rcm<kPts, false, false>;
  return launch_kernel(k, grid, T, smem, st, F, G, O, rg, scale, tw, pl);
}

}  // namespace hd
