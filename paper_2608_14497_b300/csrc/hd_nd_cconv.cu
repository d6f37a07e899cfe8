// hd_nd_cconv.cu -- instantiation and launch of k_rows_cconv (complex hybrid row convolutions of hybridCS).
#include "hd_nd_kernels.cuh"

namespace hd {

cudaError_t launch_rows_cconv(Eng e, unsigned grid, int T, size_t smem, cudaStream_t st, float2* F, const float2* G,
                              int Lr, int m, int q, int p, float scale, const float2* tw, FftPlan pl) {
  // the residue lengths of the usual 2D/3D sizes with compile-time passes
  if (e == Eng::SE) {
    decltype(&k_rows_cconv<16, true>) kk = nullptr;
    const bool small = T <= 256;
    switch (m) {
      case 256: kk = small ? k_rows_cconv<16, true, 256> : k_rows_cconv<kPtsSE, true, 256>; break;
      case 384: kk = small ? k_rows_cconv<16, true, 384> : k_rows_cconv<kPtsSE, true, 384>; break;
      case 1024: kk = small ? k_rows_cconv<16, true, 1024> : k_rows_cconv<kPtsSE, true, 1024>; break;
      case 2048: kk = small ? k_rows_cconv<16, true, 2048> : k_rows_cconv<kPtsSE, true, 2048>; break;
      case 3072: kk = small ? k_rows_cconv<16, true, 3072> : k_rows_cconv<kPtsSE, true, 3072>; break;
      default: break;
    }
    if (kk) return launch_kernel(kk, grid, T, smem, st, F, G, Lr, m, q, p, scale, tw, pl);
  }
  auto k = (e == Eng::SE && T <= 256) ? k_rows_cconv<16, true> : e == Eng::SE ? k_rows_cconv<kPtsSE, true> : k_rows_cconv<kPts, false>;
  return launch_kernel(k, grid, T, smem, st, F, G, Lr, m, q, p, scale, tw, pl);
}

}  // namespace hd
