// hd_cl_x4.cu -- explicit-padding baseline instances of the cluster kernel for
// clusters of 4 CTAs and residue lengths m = 256 R3, R3 in {5, 6, 8, 9}.
#include "hd_cl_launch.cuh"

namespace hd {
cudaError_t launch_clx_c4(int R3, const ClusterLaunch& cl, int nitems, const float* f, const float* g, float* h,
                          cudaStream_t st) {
  switch (R3) {
    case 5: return cl::launch<4, 5, true>(cl, nitems, f, g, h, st);
    case 6: return cl::launch<4, 6, true>(cl, nitems, f, g, h, st);
    case 8: return cl::launch<4, 8, true>(cl, nitems, f, g, h, st);
    case 9: return cl::launch<4, 9, true>(cl, nitems, f, g, h, st);
  }
  return cudaErrorInvalidValue;
}
}  // namespace hd
