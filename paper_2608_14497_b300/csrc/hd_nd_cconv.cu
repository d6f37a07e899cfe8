// hd_nd_cconv.cu -- instantiation and launch of k_rows_cconv (complex hybrid row convolutions of hybridCS).
#include "hd_nd_kernels.cuh"

namespace hd {

cudaError_t launch_rows_cconv(Eng e, unsigned grid, int T, size_t smem, cudaStream_t st, float2* F, const float2* G,
                              int Lr, int m, int q, int p, float scale, const float2* tw, FftPlan pl) {
  auto k = (e == Eng::SE && T <= 256) ? k_rows_cconv<16, true> : e == Eng::SE ? k_rows_cconv<kPtsSE, true> : k_rows_cconv<kPts, false>;
  return launch_kernel(k, grid, T, smem, st, F, G, Lr, m, q, p, scale, tw, pl);
}

}  // namespace hd
