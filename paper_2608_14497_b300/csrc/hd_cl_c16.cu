// hd_cl_c16.cu -- instances of the cluster hybridRCM kernel for clusters of
// 16 CTAs and residue lengths m = 256 R3, R3 in {5, 6, 8, 9}; one file per group
// so the instances compile in parallel.
#include "hd_cl_launch.cuh"

namespace hd {
cudaError_t launch_cl_c16(int R3, const ClusterLaunch& cl, int nitems, const float* f, const float* g, float* h,
                         cudaStream_t st) {
  switch (R3) {
    case 5: return cl::launch<16, 5>(cl, nitems, f, g, h, st);
    case 6: return cl::launch<16, 6>(cl, nitems, f, g, h, st);
    case 8: return cl::launch<16, 8>(cl, nitems, f, g, h, st);
    case 9: return cl::launch<16, 9>(cl, nitems, f, g, h, st);
  }
  return cudaErrorInvalidValue;
}
}  // namespace hd
