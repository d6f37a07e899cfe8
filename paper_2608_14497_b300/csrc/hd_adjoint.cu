// hd_adjoint.cu -- the adjoint (gradients) of the truncated convolution.
//
// For h = conv(f, g) restricted to the first L outputs per dimension, and an
// output gradient u (same extents), the gradients are the correlations
//   grad_f[j] = sum_k u[k] g[k - j],   grad_g[j] = sum_k u[k] f[k - j].
// Writing rev(x)[i] = x[L - 1 - i] on every axis, grad_f = rev(conv(rev(u), g))
// and grad_g = rev(conv(rev(u), f)): the same truncated convolution with the
// output gradient reversed (the paper has no adjoint; this reading is derived
// from the definition of the adjoint).  Spectra are recomputed; nothing from
// the forward call is stored.
//
// hybridRCM in 2D/3D runs one fused sequence for the whole batch (hd_nd.cu,
// adjoint_rcm_nd): the reversal is folded into the loads of the first outer
// pass and the stores of the last one, and the outer and row transforms of
// rev(u) are formed once for both gradients.  Other cases reverse the whole
// batch in one launch per array and convolve item by item.
#include <cuda_runtime.h>

#include <algorithm>

#include "hd_internal.h"
#include "hd_nd.cuh"

namespace hd {

// Reversal of every item of a batch (items of n floats back to back).
__global__ void k_reverse_items(const float* __restrict__ in, float* __restrict__ out, int64_t n, int64_t total) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t item = i / n, k = i - item * n;
    out[i] = in[item * n + (n - 1 - k)];
  }
}

static cudaError_t reverse_items(const float* in, float* out, int64_t n, int64_t batch, cudaStream_t st) {
  const int64_t total = n * batch;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 148 * 32);
  k_reverse_items<<<blocks, 256, 0, st>>>(in, out, n, total);
  return cudaGetLastError();
}

hd_status ensure_ws2(hd_ctx* c, size_t bytes, cudaStream_t st) {
  if (bytes <= c->ws2_bytes) return HD_OK;
  // stream-ordered: the old area is released after the work already queued
  // on `st`, the new one is usable by what follows; no device synchronisation
  if (c->ws2) cudaFreeAsync(c->ws2, st);
  c->ws2 = nullptr;
  c->ws2_bytes = 0;
  if (cudaMallocAsync(&c->ws2, bytes, st) != cudaSuccess) return HD_ENOMEM;
  c->ws2_bytes = bytes;
  return HD_OK;
}

static bool overlaps(const float* a, const float* b, int64_t n) {
  return a && b && a < b + n && b < a + n;
}

}  // namespace hd

using namespace hd;

extern "C" hd_status hd_conv_adjoint(hd_ctx* c, hd_algo algo, int ndim, const int64_t* Ls, int32_t batch,
                                     const float* grad_h, const float* f, const float* g, float* grad_f,
                                     float* grad_g, void* stream) {
  if (!c || !Ls || !grad_h || batch < 1 || ndim < 1 || ndim > 3) return fail(HD_EINVAL, "adjoint: bad argument");
  if ((grad_f && !g) || (grad_g && !f)) return fail(HD_EINVAL, "adjoint: a requested gradient needs the other input");
  int64_t n = 1;
  for (int i = 0; i < ndim; ++i) {
    if (Ls[i] < 1) return fail(HD_EINVAL, "adjoint: L < 1");
    n *= Ls[i];
  }
  const int64_t tot = n * batch;
  // a gradient may not overlap an input or the other gradient: inputs are
  // read after the first gradient has been written
  if (overlaps(grad_f, grad_h, tot) || overlaps(grad_f, f, tot) || overlaps(grad_f, g, tot) ||
      overlaps(grad_g, grad_h, tot) || overlaps(grad_g, f, tot) || overlaps(grad_g, g, tot) ||
      overlaps(grad_f, grad_g, tot))
    return fail(HD_EINVAL, "adjoint: gradients may not overlap grad_h, f, g or each other");
  if (!grad_f && !grad_g) return HD_OK;
  cudaSetDevice(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  if (algo == HD_HYBRID_RCM && ndim >= 2) return adjoint_rcm_nd(c, ndim, Ls, batch, grad_h, f, g, grad_f, grad_g, st);
  // general case: reverse the batch once, convolve item by item, reverse back
  if (ensure_ws2(c, 2 * sizeof(float) * (size_t)tot, st) != HD_OK) return fail(HD_ENOMEM, "adjoint: workspace");
  float* ru = reinterpret_cast<float*>(c->ws2);
  float* tmp = ru + tot;
  if (reverse_items(grad_h, ru, n, batch, st) != cudaSuccess) return fail(HD_ECUDA, "adjoint: reversal launch");
  for (int pass = 0; pass < 2; ++pass) {
    float* out = pass == 0 ? grad_f : grad_g;
    const float* other = pass == 0 ? g : f;
    if (!out) continue;
    hd_status s = hd_conv_batch(c, algo, HD_FP32, ndim, Ls, batch, ru, other, tmp, stream);
    if (s != HD_OK) return s;
    if (reverse_items(tmp, out, n, batch, st) != cudaSuccess) return fail(HD_ECUDA, "adjoint: reversal launch");
  }
  return HD_OK;
}
