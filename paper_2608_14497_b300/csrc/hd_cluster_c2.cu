// hd_cluster_c2.cu -- instantiation of the cluster hybridRCM kernel for
// clusters of 2 CTAs (q = 4 residues); one file per cluster size so they
// compile in parallel.
#include "hd_cluster_kernel.cuh"

namespace hd {
cudaError_t launch_cluster_c2(const ClusterLaunch& cl, int nitems, size_t smem, const float* f, const float* g,
                              float* h, cudaStream_t st) {
  return launch_cluster_c<2>(cl, nitems, smem, f, g, h, st);
}
}  // namespace hd
