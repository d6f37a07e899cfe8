// hd_nd.cuh -- multidimensional drivers and explicit-padding baselines.
#pragma once
#include <cuda_runtime.h>

#include "hd_internal.h"

namespace hd {
// K: output extents per dimension (nullptr: K = L).
hd_status explicit_nd(hd_ctx* c, hd_algo algo, int d, const int64_t* L, const float* f, const float* g, float* h,
                      cudaStream_t st, const int64_t* K = nullptr);
hd_status conv_nd_ext(hd_ctx* c, hd_algo algo, hd_prec prec, const float* f, const float* g, float* h, int d,
                      const int64_t* L, const int64_t* K, const hd_dim_params* prm, cudaStream_t st);
// hybridRCM 2D/3D over `batch` problems of extents L stored back to back.
hd_status conv_nd_batch_rcm(hd_ctx* c, int d, const int64_t* L, int64_t batch, const float* f, const float* g,
                            float* h, cudaStream_t st);
// Gradients of h = conv(f, g) (hybridRCM 2D/3D) for `batch` problems: grad_f =
// rev(conv(rev(u), g)), grad_g = rev(conv(rev(u), f)); either may be NULL.
hd_status adjoint_rcm_nd(hd_ctx* c, int d, const int64_t* L, int64_t batch, const float* u, const float* f,
                         const float* g, float* gf, float* gg, cudaStream_t st);
// Columns per CTA of a column pass over A blocks of B columns (a power of two
// <= 8; host logic, tested without a GPU).
int choose_W(size_t per_col, int pts, int64_t A, int64_t B, size_t max_smem, bool even, int64_t max_pts,
             int num_sms);
}  // namespace hd
