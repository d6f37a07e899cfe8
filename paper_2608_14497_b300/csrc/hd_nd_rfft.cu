// hd_nd_rfft.cu -- instantiation and launch of k_rows_fft (row DFTs of the explicit baselines).
#include "hd_nd_kernels.cuh"

namespace hd {

cudaError_t launch_rows_fft(Eng e, unsigned grid, int T, size_t smem, cudaStream_t st, RowsIO io, int mode, int n,
                            const float2* tw, int twmul, FftPlan pl) {
  auto k = (e == Eng::SE && T <= 256) ? k_rows_fft<16, true> : e == Eng::SE ? k_rows_fft<kPtsSE, true> : k_rows_fft<kPts, false>;
  return launch_kernel(k, grid, T, smem, st, io, mode, n, tw, twmul, pl);
}

}  // namespace hd
