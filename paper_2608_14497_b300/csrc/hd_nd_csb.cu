// hd_nd_csb.cu -- instantiation and launch of k_col_bwd_cs (inverse real residues, Eq. real-accumulation).
#include "hd_nd_kernels.cuh"

namespace hd {

cudaError_t launch_col_bwd_cs(Eng e, unsigned grid, int T, size_t smem, cudaStream_t st, const float2* Y, float* Z,
                              int64_t B, int W, int Lout, int m, int q, float scale, const float2* tw, FftPlan pl_m,
                              FftPlan pl_h, CsMid mid) {
  // the residue lengths of the usual 2D/3D sizes with compile-time passes
  if (e == Eng::SE && T <= 256) {
    decltype(&k_col_bwd_cs<16, true>) kk = nullptr;
    switch (m) {
      case 256: kk = k_col_bwd_cs<16, true, 256>; break;
      case 384: kk = k_col_bwd_cs<16, true, 384>; break;
      case 1024: kk = k_col_bwd_cs<16, true, 1024>; break;
      case 2048: kk = k_col_bwd_cs<16, true, 2048>; break;
      case 3072: kk = k_col_bwd_cs<16, true, 3072>; break;
      default: break;
    }
    if (kk) return launch_kernel(kk, grid, T, smem, st, Y, Z, B, W, Lout, m, q, scale, tw, pl_m, pl_h, mid);
  }
  auto k = (e == Eng::SE && T <= 256) ? k_col_bwd_cs<16, true> : e == Eng::SE ? k_col_bwd_cs<kPtsSE, true> : k_col_bwd_cs<kPts, false>;
  return launch_kernel(k, grid, T, smem, st, Y, Z, B, W, Lout, m, q, scale, tw, pl_m, pl_h, mid);
}

}  // namespace hd
