// hd_nd_csf.cu -- instantiation and launch of k_col_fwd_cs (real residues of Sec. 3.1 along the first dimension).
#include "hd_nd_kernels.cuh"

namespace hd {

cudaError_t launch_col_fwd_cs(Eng e, unsigned grid, int T, size_t smem, cudaStream_t st, const float* X, float2* Y,
                              int64_t B, int W, int Lin, int m, int q, int p, const float2* tw, FftPlan pl_m,
                              FftPlan pl_h, CsMid mid) {
  // the residue lengths of the usual 2D/3D sizes with compile-time passes
  if (e == Eng::SE && T <= 256) {
    decltype(&k_col_fwd_cs<16, true>) kk = nullptr;
    switch (m) {
      case 256: kk = k_col_fwd_cs<16, true, 256>; break;
      case 384: kk = k_col_fwd_cs<16, true, 384>; break;
      case 1024: kk = k_col_fwd_cs<16, true, 1024>; break;
      case 2048: kk = k_col_fwd_cs<16, true, 2048>; break;
      case 3072: kk = k_col_fwd_cs<16, true, 3072>; break;
      default: break;
    }
    if (kk) return launch_kernel(kk, grid, T, smem, st, X, Y, B, W, Lin, m, q, p, tw, pl_m, pl_h, mid);
  }
  auto k = (e == Eng::SE && T <= 256) ? k_col_fwd_cs<16, true> : e == Eng::SE ? k_col_fwd_cs<kPtsSE, true> : k_col_fwd_cs<kPts, false>;
  return launch_kernel(k, grid, T, smem, st, X, Y, B, W, Lin, m, q, p, tw, pl_m, pl_h, mid);
}

}  // namespace hd
