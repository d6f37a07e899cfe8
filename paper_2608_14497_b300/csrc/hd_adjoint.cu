// hd_adjoint.cu -- the adjoint (gradients) of the truncated convolution.
//
// For h = conv(f, g) restricted to the first L outputs per dimension, and an
// output gradient u (same extents), the gradients are the correlations
//   grad_f[j] = sum_k u[k] g[k - j],   grad_g[j] = sum_k u[k] f[k - j].
// Writing rev(x)[i] = x[L - 1 - i] on every axis, grad_f = rev(conv(rev(u), g))
// and grad_g = rev(conv(rev(u), f)): the same truncated convolution with the
// output gradient reversed (the paper has no adjoint; this reading is derived
// from the definition of the adjoint).  Reversal on all axes of a row-major
// array is the reversal of the flat index.  Spectra are recomputed by the
// forward convolution kernels; nothing from the forward call is stored.
#include <cuda_runtime.h>

#include <algorithm>

#include "hd_internal.h"

namespace hd {

__global__ void k_reverse(const float* __restrict__ in, float* __restrict__ out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = in[n - 1 - i];
}

static cudaError_t reverse(const float* in, float* out, int64_t n, cudaStream_t st) {
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 148 * 32);
  k_reverse<<<blocks, 256, 0, st>>>(in, out, n);
  return cudaGetLastError();
}

hd_status ensure_ws2(hd_ctx* c, size_t bytes) {
  if (bytes <= c->ws2_bytes) return HD_OK;
  if (c->ws2) {
    cudaDeviceSynchronize();
    cudaFree(c->ws2);
    c->ws2 = nullptr;
    c->ws2_bytes = 0;
  }
  if (cudaMalloc(&c->ws2, bytes) != cudaSuccess) return HD_ENOMEM;
  c->ws2_bytes = bytes;
  return HD_OK;
}

}  // namespace hd

using namespace hd;

static hd_status conv_any(hd_ctx* c, hd_algo algo, int nd, const int64_t* L, const float* a, const float* b, float* h,
                          void* stream) {
  switch (nd) {
    case 1: return hd_conv1d(c, algo, HD_FP32, a, b, h, L[0], nullptr, stream);
    case 2: return hd_conv2d(c, algo, HD_FP32, a, b, h, L[0], L[1], nullptr, stream);
    case 3: return hd_conv3d(c, algo, HD_FP32, a, b, h, L[0], L[1], L[2], nullptr, stream);
  }
  return HD_EINVAL;
}

extern "C" hd_status hd_conv_adjoint(hd_ctx* c, hd_algo algo, int ndim, const int64_t* Ls, int32_t batch,
                                     const float* grad_h, const float* f, const float* g, float* grad_f,
                                     float* grad_g, void* stream) {
  if (!c || !Ls || !grad_h || batch < 1 || ndim < 1 || ndim > 3) return HD_EINVAL;
  if ((grad_f && !g) || (grad_g && !f)) return HD_EINVAL;
  int64_t n = 1;
  for (int i = 0; i < ndim; ++i) {
    if (Ls[i] < 1) return HD_EINVAL;
    n *= Ls[i];
  }
  cudaSetDevice(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  if (ensure_ws2(c, 2 * sizeof(float) * (size_t)n) != HD_OK) return HD_ENOMEM;
  float* ru = reinterpret_cast<float*>(c->ws2);
  float* tmp = ru + n;
  for (int32_t b = 0; b < batch; ++b) {
    const int64_t o = (int64_t)b * n;
    if (reverse(grad_h + o, ru, n, st) != cudaSuccess) return HD_ECUDA;
    if (grad_f) {
      hd_status s = conv_any(c, algo, ndim, Ls, ru, g + o, tmp, stream);
      if (s != HD_OK) return s;
      if (reverse(tmp, grad_f + o, n, st) != cudaSuccess) return HD_ECUDA;
    }
    if (grad_g) {
      hd_status s = conv_any(c, algo, ndim, Ls, ru, f + o, tmp, stream);
      if (s != HD_OK) return s;
      if (reverse(tmp, grad_g + o, n, st) != cudaSuccess) return HD_ECUDA;
    }
  }
  return HD_OK;
}
