// hd_cl_x1.cu -- explicit-padding baseline instances of the cluster kernel for
// clusters of 1 CTA and residue lengths m = 256 R3, R3 in {1, 2, 3, 4, 5, 6}.
#include "hd_cl_launch.cuh"

namespace hd {
cudaError_t launch_clx_c1(int R3, const ClusterLaunch& cl, int nitems, const float* f, const float* g, float* h,
                          cudaStream_t st) {
  switch (R3) {
    case 1: return cl::launch<1, 1, true>(cl, nitems, f, g, h, st);
    case 2: return cl::launch<1, 2, true>(cl, nitems, f, g, h, st);
    case 3: return cl::launch<1, 3, true>(cl, nitems, f, g, h, st);
    case 4: return cl::launch<1, 4, true>(cl, nitems, f, g, h, st);
    case 5: return cl::launch<1, 5, true>(cl, nitems, f, g, h, st);
    case 6: return cl::launch<1, 6, true>(cl, nitems, f, g, h, st);
  }
  return cudaErrorInvalidValue;
}
}  // namespace hd
