// hd_nd.cu -- multidimensional drivers and explicit-padding baselines.
#include "hd_nd.cuh"

namespace hd {
hd_status explicit_nd(hd_ctx*, hd_algo, int, const int64_t*, const float*, const float*, float*, cudaStream_t) {
  return HD_EUNSUPPORTED;
}
}  // namespace hd

extern "C" {
hd_status hd_conv2d(hd_ctx*, hd_algo, hd_prec, const float*, const float*, float*, int64_t, int64_t,
                    const hd_dim_params*, void*) {
  return HD_EUNSUPPORTED;
}
hd_status hd_conv3d(hd_ctx*, hd_algo, hd_prec, const float*, const float*, float*, int64_t, int64_t, int64_t,
                    const hd_dim_params*, void*) {
  return HD_EUNSUPPORTED;
}
hd_status hd_batch_plan_create(hd_ctx*, hd_algo, int32_t, const int64_t*, const int32_t*, hd_batch_plan**) {
  return HD_EUNSUPPORTED;
}
hd_status hd_batch_plan_destroy(hd_batch_plan*) { return HD_OK; }
hd_status hd_conv1d_batched(hd_ctx*, const hd_batch_plan*, const float*, const float*, float*, void*) {
  return HD_EUNSUPPORTED;
}
hd_status hd_conv_adjoint(hd_ctx*, hd_algo, int, const int64_t*, int32_t, const float*, const float*, const float*,
                          float*, float*, void*) {
  return HD_EUNSUPPORTED;
}
}
