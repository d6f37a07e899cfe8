// hd_nd_adj.cu -- instantiation and launch of k_rows_adj (the adjoint's row pass: C_1 of Sec. 5 on
// (U, G) and (U, F) with the row transforms of U formed once).
#include "hd_nd_kernels.cuh"

namespace hd {

cudaError_t launch_rows_adj(Eng e, unsigned grid, int T, size_t smem, cudaStream_t st, float2* F, float2* G,
                            const float2* U, RowGeom rg, float scale, int outs, const float2* tw, FftPlan pl) {
  auto k = e == Eng::SE ? k_rows_adj<kPtsSE, true> : k_rows_adj<kPts, false>;
  return launch_kernel(k, grid, T, smem, st, F, G, U, rg, scale, outs, tw, pl);
}

}  // namespace hd
