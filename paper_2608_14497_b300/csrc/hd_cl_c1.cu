// hd_cl_c1.cu -- instances of the cluster hybridRCM kernel for clusters of
// 1 CTA and residue lengths m = 256 R3, R3 in {1, 2, 3, 4, 5, 6}; one file per group
// so the instances compile in parallel.
#include "hd_cl_launch.cuh"

namespace hd {
cudaError_t launch_cl_c1(int R3, const ClusterLaunch& cl, int nitems, const float* f, const float* g, float* h,
                         cudaStream_t st) {
  switch (R3) {
    case 1: return cl::launch<1, 1>(cl, nitems, f, g, h, st);
    case 2: return cl::launch<1, 2>(cl, nitems, f, g, h, st);
    case 3: return cl::launch<1, 3>(cl, nitems, f, g, h, st);
    case 4: return cl::launch<1, 4>(cl, nitems, f, g, h, st);
    case 5: return cl::launch<1, 5>(cl, nitems, f, g, h, st);
    case 6: return cl::launch<1, 6>(cl, nitems, f, g, h, st);
  }
  return cudaErrorInvalidValue;
}
}  // namespace hd
