/*
 * hdoracle.c -- FP64 CPU oracle for dealiased real linear convolutions.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library
 * and its Python binding) may link, load or call this file.  Only the tests,
 * the smoke check and the CPU-baseline leg of the benchmark use it.
 *
 * What is computed here is the plain definition of the problem the paper
 * solves (Sec. 2, problem statement before Eq. forwardr): the linear
 * convolution  h_k = sum_j f_j g_{k-j}  of two arrays of length L that a
 * dealiased FFT convolution reproduces exactly (up to rounding) once the data
 * are padded to at least 2L-1 (the paper pads to M = 2L, Sec. 6).
 *
 *   O1  hd_direct_conv   direct FP64 summation, per dimension, 1D/2D/3D.
 *   O1' hd_direct_corr   the adjoint of O1 with respect to f (a correlation).
 *   O2  hd_fft_conv      explicitly zero-padded FFT convolution: pad every
 *                        dimension to a power of two >= 2L-1, radix-2
 *                        complex FFT (own code), pointwise product, inverse,
 *                        crop.  Any padded length >= 2L-1 gives the same
 *                        linear convolution, so no mixed radix is needed.
 *   O1m/O2m hd_direct_conv_multi / hd_fft_conv_multi
 *                        1D convolution of n >= 2 arrays of possibly
 *                        different lengths L_1..L_n (Sec. 4.1, convolutions
 *                        of more than two arrays; Sec. 7, arrays of
 *                        different sizes): h = x^1 * ... * x^n, whose
 *                        support is S = sum L_i - n + 1 samples; the first K
 *                        (1 <= K <= S) are returned.  O1m convolves directly,
 *                        one array after the other, keeping the full
 *                        intermediate result; O2m pads every array to one
 *                        power of two >= S, multiplies the n spectra and
 *                        inverts.
 *
 * Shapes: arrays are row-major with the last dimension contiguous.  The
 * input extents are L[0..d-1]; the output extents K[0..d-1] satisfy
 * 1 <= K[i] <= 2L[i]-1 (K = L returns the first L outputs per dimension).
 *
 * Build: gcc -O2 -fopenmp -fPIC -shared (see oracle/build.py).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define HD_PI 3.14159265358979323846264338327950288

/* Collapse an nD shape to (d0, d1, d2) with missing leading dims = 1. */
static void shape3(int d, const int64_t *in, int64_t out[3]) {
  out[0] = out[1] = out[2] = 1;
  for (int i = 0; i < d; ++i) out[3 - d + i] = in[i];
}

/* ------------------------------------------------------------------------ */
/* O1: direct summation.  h[k] = sum over j with 0 <= j_i < L_i and          */
/* 0 <= k_i - j_i < L_i of f[j] g[k-j], for 0 <= k_i < K_i.                   */
/* ------------------------------------------------------------------------ */
int hd_direct_conv(int d, const int64_t *L_, const int64_t *K_, const double *f,
                   const double *g, double *h) {
  if (d < 1 || d > 3) return 1;
  int64_t L[3], K[3];
  shape3(d, L_, L);
  shape3(d, K_, K);
  for (int i = 0; i < 3; ++i)
    if (L[i] < 1 || K[i] < 1 || K[i] > 2 * L[i] - 1) return 1;
  const int64_t nout = K[0] * K[1] * K[2];
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t o = 0; o < nout; ++o) {
    const int64_t k0 = o / (K[1] * K[2]);
    const int64_t k1 = (o / K[2]) % K[1];
    const int64_t k2 = o % K[2];
    double acc = 0.0;
    const int64_t a0 = k0 - (L[0] - 1) > 0 ? k0 - (L[0] - 1) : 0;
    const int64_t b0 = k0 < L[0] - 1 ? k0 : L[0] - 1;
    const int64_t a1 = k1 - (L[1] - 1) > 0 ? k1 - (L[1] - 1) : 0;
    const int64_t b1 = k1 < L[1] - 1 ? k1 : L[1] - 1;
    const int64_t a2 = k2 - (L[2] - 1) > 0 ? k2 - (L[2] - 1) : 0;
    const int64_t b2 = k2 < L[2] - 1 ? k2 : L[2] - 1;
    for (int64_t j0 = a0; j0 <= b0; ++j0)
      for (int64_t j1 = a1; j1 <= b1; ++j1) {
        const double *fr = f + (j0 * L[1] + j1) * L[2];
        const double *gr = g + ((k0 - j0) * L[1] + (k1 - j1)) * L[2];
        for (int64_t j2 = a2; j2 <= b2; ++j2) acc += fr[j2] * gr[k2 - j2];
      }
    h[o] = acc;
  }
  return 0;
}

/* O1 at chosen output points only: h[k] for the npts multi-indices in
 * pts[npts][d] (each 0 <= k_i < 2L_i - 1), by the same direct sum.  Used to
 * check full-size results where computing every output would take too long. */
int hd_direct_conv_points(int d, const int64_t *L_, int64_t npts, const int64_t *pts, const double *f,
                          const double *g, double *out) {
  if (d < 1 || d > 3) return 1;
  int64_t L[3];
  shape3(d, L_, L);
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t i = 0; i < npts; ++i) {
    int64_t k[3] = {0, 0, 0};
    for (int a = 0; a < d; ++a) k[3 - d + a] = pts[i * d + a];
    double acc = 0.0;
    const int64_t a0 = k[0] - (L[0] - 1) > 0 ? k[0] - (L[0] - 1) : 0, b0 = k[0] < L[0] - 1 ? k[0] : L[0] - 1;
    const int64_t a1 = k[1] - (L[1] - 1) > 0 ? k[1] - (L[1] - 1) : 0, b1 = k[1] < L[1] - 1 ? k[1] : L[1] - 1;
    const int64_t a2 = k[2] - (L[2] - 1) > 0 ? k[2] - (L[2] - 1) : 0, b2 = k[2] < L[2] - 1 ? k[2] : L[2] - 1;
    for (int64_t j0 = a0; j0 <= b0; ++j0)
      for (int64_t j1 = a1; j1 <= b1; ++j1) {
        const double *fr = f + (j0 * L[1] + j1) * L[2];
        const double *gr = g + ((k[0] - j0) * L[1] + (k[1] - j1)) * L[2];
        for (int64_t j2 = a2; j2 <= b2; ++j2) acc += fr[j2] * gr[k[2] - j2];
      }
    out[i] = acc;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* O1': the adjoint of the map f -> h = conv_K(f, g) (K outputs per dim):     */
/* grad_f[j] = sum over k with 0 <= k_i < K_i and 0 <= k_i - j_i < L_i of     */
/* u[k] g[k-j], for 0 <= j_i < L_i.  Written out from the definition of the   */
/* adjoint, <conv(f,g), u> = <f, grad_f>.                                     */
/* ------------------------------------------------------------------------ */
int hd_direct_corr(int d, const int64_t *L_, const int64_t *K_, const double *u,
                   const double *g, double *grad) {
  if (d < 1 || d > 3) return 1;
  int64_t L[3], K[3];
  shape3(d, L_, L);
  shape3(d, K_, K);
  for (int i = 0; i < 3; ++i)
    if (L[i] < 1 || K[i] < 1 || K[i] > 2 * L[i] - 1) return 1;
  const int64_t nin = L[0] * L[1] * L[2];
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t o = 0; o < nin; ++o) {
    const int64_t j0 = o / (L[1] * L[2]);
    const int64_t j1 = (o / L[2]) % L[1];
    const int64_t j2 = o % L[2];
    double acc = 0.0;
    const int64_t e0 = (j0 + L[0] < K[0] ? j0 + L[0] : K[0]);
    const int64_t e1 = (j1 + L[1] < K[1] ? j1 + L[1] : K[1]);
    const int64_t e2 = (j2 + L[2] < K[2] ? j2 + L[2] : K[2]);
    for (int64_t k0 = j0; k0 < e0; ++k0)
      for (int64_t k1 = j1; k1 < e1; ++k1) {
        const double *ur = u + (k0 * K[1] + k1) * K[2];
        const double *gr = g + ((k0 - j0) * L[1] + (k1 - j1)) * L[2];
        for (int64_t k2 = j2; k2 < e2; ++k2) acc += ur[k2] * gr[k2 - j2];
      }
    grad[o] = acc;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* O2: explicitly zero-padded FFT convolution in FP64.                        */
/* ------------------------------------------------------------------------ */

/* In-place iterative radix-2 complex FFT of length n (a power of two) on
 * interleaved (re, im) doubles with element stride `stride` (in complex
 * elements).  sign = +1 computes sum_j x_j e^{+2 pi i jk/n}, sign = -1 the
 * conjugate kernel; no scaling.  Bit reversal, then log2(n) butterfly passes;
 * each twiddle is evaluated directly with cos/sin (no recurrences). */
static void fft_pow2(double *x, int64_t n, int64_t stride, int sign) {
  for (int64_t i = 1, j = 0; i < n; ++i) {
    int64_t bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) {
      double *a = x + 2 * i * stride, *b = x + 2 * j * stride;
      double t0 = a[0], t1 = a[1];
      a[0] = b[0]; a[1] = b[1];
      b[0] = t0; b[1] = t1;
    }
  }
  for (int64_t len = 2; len <= n; len <<= 1) {
    const int64_t half = len >> 1;
    for (int64_t k = 0; k < half; ++k) {
      const double ang = sign * 2.0 * HD_PI * (double)k / (double)len;
      const double wr = cos(ang), wi = sin(ang);
      for (int64_t i = k; i < n; i += len) {
        double *a = x + 2 * i * stride, *b = x + 2 * (i + half) * stride;
        const double br = b[0] * wr - b[1] * wi;
        const double bi = b[0] * wi + b[1] * wr;
        b[0] = a[0] - br; b[1] = a[1] - bi;
        a[0] += br; a[1] += bi;
      }
    }
  }
}

static int64_t next_pow2(int64_t v) {
  int64_t p = 1;
  while (p < v) p <<= 1;
  return p;
}

/* FFT every line of a (P0, P1, P2) complex grid along axis `ax`. */
static void fft_axis(double *x, const int64_t P[3], int ax, int sign) {
  const int64_t n = P[ax];
  if (n == 1) return;
  int64_t stride = 1;
  for (int i = ax + 1; i < 3; ++i) stride *= P[i];
  const int64_t outer = (ax == 0 ? 1 : (ax == 1 ? P[0] : P[0] * P[1]));
  const int64_t inner = stride;
#pragma omp parallel for schedule(static)
  for (int64_t line = 0; line < outer * inner; ++line) {
    const int64_t o = line / inner, i = line % inner;
    fft_pow2(x + 2 * (o * n * inner + i), n, stride, sign);
  }
}

int hd_fft_conv(int d, const int64_t *L_, const int64_t *K_, const double *f,
                const double *g, double *h) {
  if (d < 1 || d > 3) return 1;
  int64_t L[3], K[3], P[3];
  shape3(d, L_, L);
  shape3(d, K_, K);
  for (int i = 0; i < 3; ++i) {
    if (L[i] < 1 || K[i] < 1 || K[i] > 2 * L[i] - 1) return 1;
    P[i] = next_pow2(2 * L[i] - 1);
  }
  const int64_t np = P[0] * P[1] * P[2];
  double *F = (double *)calloc((size_t)(2 * np), sizeof(double));
  double *G = (double *)calloc((size_t)(2 * np), sizeof(double));
  if (!F || !G) {
    free(F);
    free(G);
    return 2;
  }
  /* zero pad: place the L0 x L1 x L2 block at the origin of the P grid */
  for (int64_t a = 0; a < L[0]; ++a)
    for (int64_t b = 0; b < L[1]; ++b)
      for (int64_t c = 0; c < L[2]; ++c) {
        const int64_t src = (a * L[1] + b) * L[2] + c;
        const int64_t dst = (a * P[1] + b) * P[2] + c;
        F[2 * dst] = f[src];
        G[2 * dst] = g[src];
      }
  for (int ax = 0; ax < 3; ++ax) {
    fft_axis(F, P, ax, +1);
    fft_axis(G, P, ax, +1);
  }
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < np; ++i) {
    const double ar = F[2 * i], ai = F[2 * i + 1];
    const double br = G[2 * i], bi = G[2 * i + 1];
    F[2 * i] = ar * br - ai * bi;
    F[2 * i + 1] = ar * bi + ai * br;
  }
  for (int ax = 0; ax < 3; ++ax) fft_axis(F, P, ax, -1);
  const double scale = 1.0 / (double)np;
  for (int64_t a = 0; a < K[0]; ++a)
    for (int64_t b = 0; b < K[1]; ++b)
      for (int64_t c = 0; c < K[2]; ++c)
        h[(a * K[1] + b) * K[2] + c] = F[2 * ((a * P[1] + b) * P[2] + c)] * scale;
  free(F);
  free(G);
  return 0;
}

/* Batched 1D convolutions of uneven lengths on flat arrays: item i occupies
 * [off[i], off[i] + Ls[i]) of f, g and h; K = L outputs per item.  Uses O2
 * per item when use_fft != 0, else O1; items run in parallel. */
int hd_batch_conv1d(int64_t n, const int64_t *off, const int64_t *Ls,
                    const double *f, const double *g, double *h, int use_fft) {
  int bad = 0;
  /* items in parallel; the nested parallel loops inside run single-threaded */
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
  for (int64_t i = 0; i < n; ++i) {
    int64_t L = Ls[i];
    int64_t K = L;
    int rc = use_fft ? hd_fft_conv(1, &L, &K, f + off[i], g + off[i], h + off[i])
                     : hd_direct_conv(1, &L, &K, f + off[i], g + off[i], h + off[i]);
    bad |= rc;
  }
  return bad;
}

/* ------------------------------------------------------------------------ */
/* O1m / O2m: 1D convolution of n arrays of possibly different lengths.     */
/* ------------------------------------------------------------------------ */

static int64_t multi_support(int n, const int64_t *L) {
  int64_t S = 1;
  for (int i = 0; i < n; ++i) S += L[i] - 1;
  return S;
}

int hd_direct_conv_multi(int n, const int64_t *L, const double *const *x, int64_t K, double *h) {
  if (n < 2) return 1;
  for (int i = 0; i < n; ++i)
    if (L[i] < 1 || !x[i]) return 1;
  const int64_t S = multi_support(n, L);
  if (K < 1 || K > S) return 1;
  double *acc = (double *)calloc((size_t)S, sizeof(double));
  double *tmp = (double *)calloc((size_t)S, sizeof(double));
  if (!acc || !tmp) {
    free(acc);
    free(tmp);
    return 2;
  }
  /* acc = x^1; then acc <- acc * x^i (full linear convolution) for i >= 2 */
  int64_t len = L[0];
  memcpy(acc, x[0], sizeof(double) * (size_t)L[0]);
  for (int i = 1; i < n; ++i) {
    const int64_t out = len + L[i] - 1;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < out; ++k) {
      double sum = 0.0;
      const int64_t j0 = k - (L[i] - 1) > 0 ? k - (L[i] - 1) : 0;
      const int64_t j1 = k < len - 1 ? k : len - 1;
      for (int64_t j = j0; j <= j1; ++j) sum += acc[j] * x[i][k - j];
      tmp[k] = sum;
    }
    memcpy(acc, tmp, sizeof(double) * (size_t)out);
    len = out;
  }
  memcpy(h, acc, sizeof(double) * (size_t)K);
  free(acc);
  free(tmp);
  return 0;
}

int hd_fft_conv_multi(int n, const int64_t *L, const double *const *x, int64_t K, double *h) {
  if (n < 2) return 1;
  for (int i = 0; i < n; ++i)
    if (L[i] < 1 || !x[i]) return 1;
  const int64_t S = multi_support(n, L);
  if (K < 1 || K > S) return 1;
  const int64_t P = next_pow2(S);
  double *acc = (double *)calloc((size_t)(2 * P), sizeof(double));
  double *X = (double *)calloc((size_t)(2 * P), sizeof(double));
  if (!acc || !X) {
    free(acc);
    free(X);
    return 2;
  }
  for (int64_t j = 0; j < L[0]; ++j) acc[2 * j] = x[0][j];
  fft_pow2(acc, P, 1, +1);
  for (int i = 1; i < n; ++i) {
    memset(X, 0, sizeof(double) * (size_t)(2 * P));
    for (int64_t j = 0; j < L[i]; ++j) X[2 * j] = x[i][j];
    fft_pow2(X, P, 1, +1);
    for (int64_t k = 0; k < P; ++k) {
      const double ar = acc[2 * k], ai = acc[2 * k + 1];
      const double br = X[2 * k], bi = X[2 * k + 1];
      acc[2 * k] = ar * br - ai * bi;
      acc[2 * k + 1] = ar * bi + ai * br;
    }
  }
  fft_pow2(acc, P, 1, -1);
  for (int64_t k = 0; k < K; ++k) h[k] = acc[2 * k] / (double)P;
  free(acc);
  free(X);
  return 0;
}
