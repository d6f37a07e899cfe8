// hd_cl_x8b.cu -- explicit-padding baseline instances of the cluster kernel for
// clusters of 8 CTAs and residue lengths m = 256 R3, R3 in {10, 12, 16, 18}.
#include "hd_cl_launch.cuh"

namespace hd {
cudaError_t launch_clx_c8b(int R3, const ClusterLaunch& cl, int nitems, const float* f, const float* g, float* h,
                          cudaStream_t st) {
  switch (R3) {
    case 10: return cl::launch<8, 10, true>(cl, nitems, f, g, h, st);
    case 12: return cl::launch<8, 12, true>(cl, nitems, f, g, h, st);
    case 16: return cl::launch<8, 16, true>(cl, nitems, f, g, h, st);
    case 18: return cl::launch<8, 18, true>(cl, nitems, f, g, h, st);
  }
  return cudaErrorInvalidValue;
}
}  // namespace hd
