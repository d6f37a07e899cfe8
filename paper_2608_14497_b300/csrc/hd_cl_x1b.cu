// hd_cl_x1b.cu -- explicit-padding baseline instances of the cluster kernel for
// clusters of 1 CTA and residue lengths m = 256 R3, R3 in {8, 9, 10, 12, 16, 18}.
#include "hd_cl_launch.cuh"

namespace hd {
cudaError_t launch_clx_c1b(int R3, const ClusterLaunch& cl, int nitems, const float* f, const float* g, float* h,
                          cudaStream_t st) {
  switch (R3) {
    case 8: return cl::launch<1, 8, true>(cl, nitems, f, g, h, st);
    case 9: return cl::launch<1, 9, true>(cl, nitems, f, g, h, st);
    case 10: return cl::launch<1, 10, true>(cl, nitems, f, g, h, st);
    case 12: return cl::launch<1, 12, true>(cl, nitems, f, g, h, st);
    case 16: return cl::launch<1, 16, true>(cl, nitems, f, g, h, st);
    case 18: return cl::launch<1, 18, true>(cl, nitems, f, g, h, st);
  }
  return cudaErrorInvalidValue;
}
}  // namespace hd
