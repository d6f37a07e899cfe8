// hd_nd.cuh -- multidimensional drivers and explicit-padding baselines.
#pragma once
#include <cuda_runtime.h>

#include "hd_internal.h"

namespace hd {
hd_status explicit_nd(hd_ctx* c, hd_algo algo, int d, const int64_t* L, const float* f, const float* g, float* h,
                      cudaStream_t st);
}  // namespace hd
