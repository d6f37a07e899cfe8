// hd_nd_colb.cu -- instantiation and launch of k_col_bwd (complex hybrid backward transform along a strided dimension).
#include "hd_nd_kernels.cuh"

namespace hd {

cudaError_t launch_col_bwd(Eng e, unsigned grid, int T, size_t smem, cudaStream_t st, const float2* Y, void* Z,
                           ColGeom cg, int Lout, int m, int q, int out_mode, int Lreal, float scale, const float2* tw,
                           FftPlan pl) {
  // the structured engine at <= 16 points per thread (T <= 256): the 4-CTA-per-SM instance
  // the residue lengths of the usual 2D/3D sizes (L = 256, 384, 1024, 2048,
  // 3000) with compile-time passes
  if (e == Eng::SE && T <= 256) {
    decltype(&k_col_bwd<16, false, true>) kk = nullptr;
    switch (m) {
      case 256: kk = k_col_bwd<16, false, true, 256>; break;
      case 384: kk = k_col_bwd<16, false, true, 384>; break;
      case 1024: kk = k_col_bwd<16, false, true, 1024>; break;
      case 2048: kk = k_col_bwd<16, false, true, 2048>; break;
      case 3072: kk = k_col_bwd<16, false, true, 3072>; break;
      default: break;
    }
    if (kk) return launch_kernel(kk, grid, T, smem, st, Y, Z, cg, Lout, m, q, out_mode, Lreal, scale, tw, pl);
  }
  auto k = (e == Eng::SE && T <= 256) ? k_col_bwd<16, false, true>
           : e == Eng::SE    ? k_col_bwd<kPtsSE, false, true>
           : e == Eng::TC  ? k_col_bwd<kPts, true, false>
           : e == Eng::TCS ? k_col_bwd<kPts, true, true>
                           : k_col_bwd<kPts, false, false>;
  return launch_kernel(k, grid, T, smem, st, Y, Z, cg, Lout, m, q, out_mode, Lreal, scale, tw, pl);
}

}  // namespace hd
