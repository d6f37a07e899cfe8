// hd_cl_c4b.cu -- instances of the cluster hybridRCM kernel for clusters of
// 4 CTAs and residue lengths m = 256 R3, R3 in {10, 12, 16, 18}; one file per group
// so the instances compile in parallel.
#include "hd_cl_launch.cuh"

namespace hd {
cudaError_t launch_cl_c4b(int R3, const ClusterLaunch& cl, int nitems, const float* f, const float* g, float* h,
                         cudaStream_t st) {
  switch (R3) {
    case 10: return cl::launch<4, 10>(cl, nitems, f, g, h, st);
    case 12: return cl::launch<4, 12>(cl, nitems, f, g, h, st);
    case 16: return cl::launch<4, 16>(cl, nitems, f, g, h, st);
    case 18: return cl::launch<4, 18>(cl, nitems, f, g, h, st);
  }
  return cudaErrorInvalidValue;
}
}  // namespace hd
