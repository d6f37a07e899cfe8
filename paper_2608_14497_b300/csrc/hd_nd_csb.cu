// hd_nd_csb.cu -- instantiation and launch of k_col_bwd_cs (inverse real residues, Eq. real-accumulation).
#include "hd_nd_kernels.cuh"

namespace hd {

cudaError_t launch_col_bwd_cs(Eng e, unsigned grid, int T, size_t smem, cudaStream_t st, const float2* Y, float* Z,
                              int64_t B, int W, int Lout, int m, int q, float scale, const float2* tw, FftPlan pl_m,
                              FftPlan pl_h, CsMid mid) {
  auto k = (e == Eng::SE && T <= 256) ? k_col_bwd_cs<16, true> : e == Eng::SE ? k_col_bwd_cs<kPtsSE, true> : k_col_bwd_cs<kPts, false>;
  return launch_kernel(k, grid, T, smem, st, Y, Z, B, W, Lout, m, q, scale, tw, pl_m, pl_h, mid);
}

}  // namespace hd
