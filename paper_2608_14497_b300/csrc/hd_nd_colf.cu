// hd_nd_colf.cu -- instantiation and launch of k_col_fwd (complex hybrid forward transform along a strided dimension).
#include "hd_nd_kernels.cuh"

namespace hd {

cudaError_t launch_col_fwd(Eng e, unsigned grid, int T, size_t smem, cudaStream_t st, const void* X, float2* Y,
                           ColGeom cg, int Lin, int m, int q, int p, int in_mode, int Lreal, const float2* tw,
                           FftPlan pl) {
  // the structured engine at <= 16 points per thread (T <= 256): the 4-CTA-per-SM instance
  // the residue lengths of the usual 2D/3D sizes (L = 256, 384, 1024, 2048,
  // 3000) with compile-time passes
  if (e == Eng::SE && T <= 256) {
    decltype(&k_col_fwd<16, false, true>) kk = nullptr;
    switch (m) {
      case 256: kk = k_col_fwd<16, false, true, 256>; break;
      case 384: kk = k_col_fwd<16, false, true, 384>; break;
      case 1024: kk = k_col_fwd<16, false, true, 1024>; break;
      case 2048: kk = k_col_fwd<16, false, true, 2048>; break;
      case 3072: kk = k_col_fwd<16, false, true, 3072>; break;
      default: break;
    }
    if (kk) return launch_kernel(kk, grid, T, smem, st, X, Y, cg, Lin, m, q, p, in_mode, Lreal, tw, pl);
  }
  auto k = (e == Eng::SE && T <= 256) ? k_col_fwd<16, false, true>
           : e == Eng::SE    ? k_col_fwd<kPtsSE, false, true>
           : e == Eng::TC  ? k_col_fwd<kPts, true, false>
           : e == Eng::TCS ? k_col_fwd<kPts, true, true>
                           : k_col_fwd<kPts, false, false>;
  return launch_kernel(k, grid, T, smem, st, X, Y, cg, Lin, m, q, p, in_mode, Lreal, tw, pl);
}

}  // namespace hd
