// lnL emulator: a small MLP of lnL(theta) trained on exact evaluations, with
// an ensemble of two heads and a fallback flag (the learned part of the build;
// the paper has no counterpart).
//
// Model: x = (theta - centre) / half_width in [-1, 1]^d (zero-padded to 16
// inputs); lnL(theta) = q(x) + sigma_r f(x), where q is a float64 least-squares
// polynomial in x fitted to the training labels -- products of Legendre
// polynomials of total degree up to the highest that keeps 16 labels per
// coefficient and at most 256 terms (degree 6 for d = 4 from 3360 labels) --
// and f is an MLP with `depth`
// hidden GELU layers of `width` units (gelu(z) = z Phi(z)) and a linear output,
// trained on the normalised residuals (lnL - q) / sigma_r.  The residual is
// small next to lnL itself, so bf16 weights with FP32 accumulation are enough.
//
// Every product runs on tensor cores: in training WMMA bf16 x bf16 -> fp32
// (forward Z = X W^T, data gradient dX = dZ W, weight gradient dW = dZ^T X);
// at inference every layer on tcgen05 with the bias and GELU fused into the
// epilogue (mlp_tc_kernel; the first layer's 16 inputs widened with zeros to
// one 64-column stage).  Master
// weights, gradients and the Adam state are float32; each layer's input
// activations and its weights are rounded to bf16 for the products.
// Prediction averages the two heads; a point is flagged for exact evaluation
// when it lies outside the training box or the heads disagree by more than a
// tolerance.
#include "qmlgb.h"
#include "internal.cuh"
#include "ptx.cuh"

#include <cuda.h>
#include <cuda_bf16.h>
#include <mma.h>

#include <algorithm>
#include <cmath>
#include <type_traits>
#include <string>
#include <functional>
#include <vector>

namespace qmlgb {
void set_last_error(const std::string &msg);
}

using namespace qmlgb;
using namespace nvcuda;

namespace {

constexpr int kIn0 = 16, kOut0 = 16, kMaxDim = 8;
// baseline polynomial: products of Legendre polynomials P_k(x_i) of total
// degree <= deg (well conditioned on the box), at most kMaxFeat terms
constexpr int kMaxFeat = 256, kMaxDeg = 12;
// number of multi-indices of d components with sum <= deg: C(deg + d, d)
inline int nfeat_of(int d, int deg) {
  long long c = 1;
  for (int i = 1; i <= d; ++i) c = c * (deg + i) / i;
  return (int)c;
}
// the feature order: by total degree t = 0..deg; within a degree the first
// exponent from t down to 0, then the second from what is left down to 0,
// and so on, the last taking the rest
void multi_indices(int d, int deg, std::vector<unsigned char> &out) {
  out.clear();
  std::vector<int> m(d);
  for (int t = 0; t <= deg; ++t) {
    // recursive enumeration written as an explicit stack over positions
    std::function<void(int, int)> rec = [&](int pos, int left) {
      if (pos == d - 1) {
        m[pos] = left;
        for (int i = 0; i < d; ++i) out.push_back((unsigned char)m[i]);
        return;
      }
      for (int k = left; k >= 0; --k) {
        m[pos] = k;
        rec(pos + 1, left - k);
      }
    };
    rec(0, t);
  }
}
// degree of the baseline for n training labels: the highest total degree
// with at least 16 labels per coefficient and at most kMaxFeat terms
int baseline_degree(int d, int n) {
  int deg = 1;
  while (deg < kMaxDeg && nfeat_of(d, deg + 1) <= kMaxFeat && 16LL * nfeat_of(d, deg + 1) <= n)
    ++deg;
  return deg;
}
// points in the outer 3 % shell of the box are treated as outside the
// training hull: uniformly drawn samples thin out there and the two heads can
// agree while both extrapolate
constexpr double kHullMargin = 0.97;

// ---------------------------------------------------------- tensor cores --
// C (M x N, fp32 row-major, ldc) = op(A) op(B) [+ C]; A is M x K and B is
// K x N in the given layouts; M, N, K multiples of 16.  4 warps per block,
// 64 x 64 output tile, 2 x 2 fragments per warp.
template <typename ALay, typename BLay>
__global__ void wmma_gemm_kernel(int M, int N, int K, const __nv_bfloat16 *A, int lda,
                                 const __nv_bfloat16 *B, int ldb, float *C, int ldc,
                                 int accumulate) {
  const int warp = threadIdx.x >> 5;
  const int m0 = blockIdx.y * 64 + (warp >> 1) * 32;
  const int n0 = blockIdx.x * 64 + (warp & 1) * 32;
  wmma::fragment<wmma::accumulator, 16, 16, 16, float> acc[2][2];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      if (accumulate && m0 + 16 * i < M && n0 + 16 * j < N)
        wmma::load_matrix_sync(acc[i][j], C + (int64_t)(m0 + 16 * i) * ldc + n0 + 16 * j, ldc,
                               wmma::mem_row_major);
      else
        wmma::fill_fragment(acc[i][j], 0.0f);
    }
  const bool am[2] = {m0 < M, m0 + 16 < M};
  const bool bn[2] = {n0 < N, n0 + 16 < N};
  for (int k = 0; k < K; k += 16) {
    wmma::fragment<wmma::matrix_a, 16, 16, 16, __nv_bfloat16, ALay> a[2];
    wmma::fragment<wmma::matrix_b, 16, 16, 16, __nv_bfloat16, BLay> b[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      if (!am[i]) continue;
      const int r = m0 + 16 * i;
      const __nv_bfloat16 *p = std::is_same<ALay, wmma::row_major>::value
                                   ? A + (int64_t)r * lda + k
                                   : A + r + (int64_t)k * lda;
      wmma::load_matrix_sync(a[i], p, lda);
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      if (!bn[j]) continue;
      const int c = n0 + 16 * j;
      const __nv_bfloat16 *p = std::is_same<BLay, wmma::row_major>::value
                                   ? B + (int64_t)k * ldb + c
                                   : B + (int64_t)c * ldb + k;
      wmma::load_matrix_sync(b[j], p, ldb);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j)
        if (am[i] && bn[j]) wmma::mma_sync(acc[i][j], a[i], b[j], acc[i][j]);
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j)
      if (am[i] && bn[j])
        wmma::store_matrix_sync(C + (int64_t)(m0 + 16 * i) * ldc + n0 + 16 * j, acc[i][j], ldc,
                                wmma::mem_row_major);
}

template <typename ALay, typename BLay>
void wmma_gemm(int M, int N, int K, const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *B,
               int ldb, float *C, int ldc, int accumulate, cudaStream_t st) {
  dim3 grid((N + 63) / 64, (M + 63) / 64);
  wmma_gemm_kernel<ALay, BLay><<<grid, 128, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, accumulate);
  count_launch();
}

// ------------------------------------------------------------ elementwise --
// 2 Phi(z) = 1 + erf(z / sqrt 2), erf from the rational approximation of
// Abramowitz & Stegun 7.1.26 (Hastings): for x >= 0, erf(x) = 1 - (a1 t +
// a2 t^2 + ... + a5 t^5) e^(-x^2) with t = 1 / (1 + p x) and an absolute
// error of at most 1.5e-7; erf(-x) = -erf(x).  So 1 + erf(z / sqrt 2) is
// 2 - Q for z >= 0 and Q for z < 0, Q = poly(t) exp(-z^2 / 2).  Training and
// inference both use it, so the network the inference evaluates is the one
// trained; its error is far below the bf16 rounding of every activation.
__device__ __forceinline__ float two_phi_f(float z) {
  const float x = fabsf(z) * 0.70710678118654752f;
  const float t = __fdividef(1.0f, fmaf(0.3275911f, x, 1.0f));
  const float poly =
      t * fmaf(t, fmaf(t, fmaf(t, fmaf(t, 1.061405429f, -1.453152027f), 1.421413741f), -0.284496736f),
               0.254829592f);
  const float q = poly * __expf(-0.5f * z * z);
  return z >= 0.0f ? 2.0f - q : q;
}
// GELU(z) = z Phi(z) and its derivative Phi(z) + z phi(z)
__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * two_phi_f(z); }
__device__ __forceinline__ float dgelu_f(float z) {
  return 0.5f * two_phi_f(z) + z * __expf(-0.5f * z * z) * 0.3989422804014327f;
}

// Z <- Z + b (row-major B x N); Xn = bf16(gelu(Z)) or bf16(Z)
__global__ void bias_act_kernel(float *Z, int Brows, int N, const float *b, __nv_bfloat16 *Xn,
                                int act) {
  const int64_t total = (int64_t)Brows * N;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int n = (int)(t % N);
    const float z = Z[t] + b[n];
    Z[t] = z;
    if (Xn) Xn[t] = __float2bfloat16_rn(act ? gelu_f(z) : z);
  }
}

// dZ = dX * gelu'(Z), kept in fp32 (bias gradient) and bf16 (products)
__global__ void gelu_bwd_kernel(const float *dX, const float *Z, int64_t total, float *dZf,
                                __nv_bfloat16 *dZh) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const float d = dX[t] * dgelu_f(Z[t]);
    dZf[t] = d;
    dZh[t] = __float2bfloat16_rn(d);
  }
}

// output layer: residual of column 0 over the first nreal rows; gradient of
// the mean squared error; per-block partial loss (fixed-order sum later)
__global__ void loss_grad_kernel(const float *out, const float *t, int Brows, int nreal,
                                 float *dZf, __nv_bfloat16 *dZh, double *partial) {
  __shared__ double red[256];
  double l = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Brows * kOut0;
       i += gridDim.x * blockDim.x) {
    const int b = i / kOut0, c = i % kOut0;
    float g = 0.0f;
    if (c == 0 && b < nreal) {
      const float r = out[i] - t[b];
      g = 2.0f * r / (float)nreal;
      l += (double)r * r;
    }
    dZf[i] = g;
    dZh[i] = __float2bfloat16_rn(g);
  }
  red[threadIdx.x] = l;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void sum_partials_kernel(const double *partial, int np, double scale, double *out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < np; ++i) s += partial[i];
    *out = s * scale;
  }
}

// db[n] = sum_b dZ[b, n] (fixed order over b)
__global__ void colsum_kernel(const float *dZ, int Brows, int N, float *db) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.0f;
  for (int b = 0; b < Brows; ++b) s += dZ[(int64_t)b * N + n];
  db[n] = s;
}

__global__ void adam_kernel(float *p, const float *g, float *m, float *v, int64_t n, float lr,
                            float b1, float b2, float eps, float c1, float c2,
                            __nv_bfloat16 *ph) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    p[i] = pi;
    ph[i] = __float2bfloat16_rn(pi);
  }
}

__global__ void to_bf16_kernel(const float *p, int64_t n, __nv_bfloat16 *ph) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    ph[i] = __float2bfloat16_rn(p[i]);
}

// splitmix64 (Steele, Lea & Flood 2014) of a counter: uniform in [0, 1)
__device__ __forceinline__ double u01(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  x ^= x >> 31;
  return (double)(x >> 11) * (1.0 / 9007199254740992.0);
}

// uniform weights, zero biases: He bound sqrt(6 / fan_in) for the GELU layers
// (keeps the activation scale through depth), Glorot bound sqrt(6 / (fan_in +
// fan_out)) for the linear output layer; padded input columns of layer 0 and
// padded output rows of the last layer stay zero
__global__ void init_layer_kernel(float *W, float *b, int out, int in, int in_real, int out_real,
                                  int is_output, uint64_t seed) {
  const float a = is_output ? sqrtf(6.0f / (float)(in_real + out_real)) : sqrtf(6.0f / (float)in_real);
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < out * in; t += gridDim.x * blockDim.x) {
    const int o = t / in, i = t % in;
    float w = 0.0f;
    if (i < in_real && o < out_real) w = (float)((2.0 * u01(seed * 0x100000000ull + t) - 1.0) * a);
    W[t] = w;
  }
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < out; o += gridDim.x * blockDim.x) b[o] = 0.0f;
}

// normalised inputs of a batch: sample j of the epoch is row
// (off + j stride) mod n; theta is n x d column-major (float64)
__global__ void gather_kernel(const double *theta, int n, int d, const double *centre,
                              const double *half, const float *targ, int Brows, int nreal,
                              int64_t off, int64_t stride, __nv_bfloat16 *X0, float *tb) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < Brows * kIn0; t += gridDim.x * blockDim.x) {
    const int b = t / kIn0, c = t % kIn0;
    float x = 0.0f;
    if (b < nreal && c < d) {
      const int64_t row = (off + (int64_t)b * stride) % n;
      x = (float)((theta[row + (int64_t)c * n] - centre[c]) / half[c]);
    }
    X0[t] = __float2bfloat16_rn(x);
    if (c == 0) {
      if (tb && b < nreal) tb[b] = targ[(off + (int64_t)b * stride) % n];
      else if (tb) tb[b] = 0.0f;
    }
  }
}

// dst (rows x dcols, bf16 row-major) <- src (rows x cols) with zero columns
// cols .. dcols - 1 (the 16 inputs of the first layer widened to one
// 64-column tensor-core stage)
__global__ void pad_cols_kernel(const __nv_bfloat16 *src, int rows, int cols, __nv_bfloat16 *dst,
                                int dcols) {
  const int64_t total = (int64_t)rows * dcols;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / dcols;
    const int c = (int)(t - r * dcols);
    dst[t] = c < cols ? src[r * cols + c] : __float2bfloat16_rn(0.0f);
  }
}

// Legendre values P_0..P_deg of each of the d coordinates (Bonnet's
// recurrence (k + 1) P_{k+1} = (2k + 1) x P_k - k P_{k-1})
__device__ __forceinline__ void legendre_table(const double *x, int d, int deg,
                                               double (*leg)[kMaxDeg + 1]) {
  for (int i = 0; i < d; ++i) {
    leg[i][0] = 1.0;
    if (deg >= 1) leg[i][1] = x[i];
    for (int k = 1; k < deg; ++k)
      leg[i][k + 1] = ((2 * k + 1) * x[i] * leg[i][k] - k * leg[i][k - 1]) / (k + 1);
  }
}
// q(x) = sum_j coef_j prod_i P_{m_ji}(x_i) with the multi-indices m (nf x d)
__device__ __forceinline__ double baseline_value(const double *x, int d, int deg, int nf,
                                                 const unsigned char *midx, const double *coef) {
  double leg[kMaxDim][kMaxDeg + 1];
  legendre_table(x, d, deg, leg);
  double q = 0.0;
  for (int j = 0; j < nf; ++j) {
    double f = 1.0;
    for (int i = 0; i < d; ++i) f *= leg[i][midx[j * d + i]];
    q = fma(coef[j], f, q);
  }
  return q;
}

// The same value for inference, where it runs once per predicted point: the
// constant term in float64 and the other terms in float32 (the float64 pipe
// of this part is narrow).  Each term is a product of Legendre values of
// magnitude <= 1, so the float32 sum is off by at most about 2^-23 sum |coef_j|,
// j >= 1, far below the emulator's tolerance.
__device__ __forceinline__ double baseline_value_fast(const double *x, int d, int deg, int nf,
                                                      const unsigned char *midx,
                                                      const double *coef) {
  float leg[kMaxDim][kMaxDeg + 1];
  for (int i = 0; i < d; ++i) {
    const float xi = (float)x[i];
    leg[i][0] = 1.0f;
    if (deg >= 1) leg[i][1] = xi;
    for (int k = 1; k < deg; ++k)
      leg[i][k + 1] = ((2 * k + 1) * xi * leg[i][k] - k * leg[i][k - 1]) / (float)(k + 1);
  }
  float q = 0.0f;
  for (int j = 1; j < nf; ++j) {
    float f = 1.0f;
    for (int i = 0; i < d; ++i) f *= leg[i][midx[j * d + i]];
    q = fmaf((float)coef[j], f, q);
  }
  return coef[0] + (double)q;
}

// Phi (n x nf, column-major): the features of every training point
__global__ void phi_kernel(const double *theta, int n, int d, int deg, int nf,
                           const unsigned char *midx, const double *centre, const double *half,
                           double *Phi) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
    double x[kMaxDim], leg[kMaxDim][kMaxDeg + 1];
    for (int i = 0; i < d; ++i) x[i] = (theta[s + (int64_t)i * n] - centre[i]) / half[i];
    legendre_table(x, d, deg, leg);
    for (int j = 0; j < nf; ++j) {
      double f = 1.0;
      for (int i = 0; i < d; ++i) f *= leg[i][midx[j * d + i]];
      Phi[s + (int64_t)j * n] = f;
    }
  }
}

// (G + ridge) coef = r by Cholesky, G (nf x nf, column-major, overwritten by
// its factor) and r in global memory; one block, fixed operation order.  The
// ridge, 1e-12 of the mean diagonal, keeps a rank-deficient G solvable.
__global__ void chol_solve_kernel(double *G, const double *r, int nf, double *coef) {
  __shared__ double sd;
  __shared__ double z[kMaxFeat];
  const int tid = threadIdx.x;
  if (tid == 0) {
    double tr = 0.0;
    for (int i = 0; i < nf; ++i) tr += G[i + (int64_t)i * nf];
    sd = 1e-12 * tr / nf;
  }
  __syncthreads();
  for (int i = tid; i < nf; i += blockDim.x) G[i + (int64_t)i * nf] += sd;
  __syncthreads();
  for (int j = 0; j < nf; ++j) {
    if (tid == 0) {
      const double v = G[j + (int64_t)j * nf];
      sd = sqrt(v > 0.0 ? v : 1e-300);
      G[j + (int64_t)j * nf] = sd;
    }
    __syncthreads();
    for (int i = j + 1 + tid; i < nf; i += blockDim.x) G[i + (int64_t)j * nf] /= sd;
    __syncthreads();
    // trailing update of the lower triangle, column by column
    const int m = nf - j - 1;
    for (int t = tid; t < m * m; t += blockDim.x) {
      const int ii = j + 1 + t % m, kk = j + 1 + t / m;
      if (ii >= kk) G[ii + (int64_t)kk * nf] -= G[ii + (int64_t)j * nf] * G[kk + (int64_t)j * nf];
    }
    __syncthreads();
  }
  if (tid == 0) {
    for (int i = 0; i < nf; ++i) {  // L z = r
      double t = r[i];
      for (int k = 0; k < i; ++k) t -= G[i + (int64_t)k * nf] * z[k];
      z[i] = t / G[i + (int64_t)i * nf];
    }
    for (int i = nf - 1; i >= 0; --i) {  // L^T coef = z
      double t = z[i];
      for (int k = i + 1; k < nf; ++k) t -= G[k + (int64_t)i * nf] * coef[k];
      coef[i] = t / G[i + (int64_t)i * nf];
    }
  }
}

// residual r = y - q(x) and its sum of squares partials
__global__ void residual_kernel(const double *theta, const double *y, int n, int d, int deg,
                                int nf, const unsigned char *midx, const double *centre,
                                const double *half, const double *coef, double *res,
                                double *partial) {
  __shared__ double red[256];
  double ss = 0.0;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
    double x[kMaxDim];
    for (int i = 0; i < d; ++i) x[i] = (theta[s + (int64_t)i * n] - centre[i]) / half[i];
    const double r = y[s] - baseline_value(x, d, deg, nf, midx, coef);
    res[s] = r;
    ss += r * r;
  }
  red[threadIdx.x] = ss;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void scale_targets_kernel(const double *res, int n, const double *sumsq, float *targ,
                                     double *sigma) {
  const double sg = sqrt(*sumsq / n) > 0.0 ? sqrt(*sumsq / n) : 1.0;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x)
    targ[s] = (float)(res[s] / sg);
  if (blockIdx.x == 0 && threadIdx.x == 0) *sigma = sg;
}

// prediction: q(x) + sigma (f0 + f1) / 2; flag outside the hull (box minus
// its outer shell) or when the heads differ by more than thr (in lnL units)
__global__ void predict_finish_kernel(const double *theta, int ntot, int off, int cnt, int d,
                                      int deg, int nf, const unsigned char *midx,
                                      const double *centre, const double *half,
                                      const double *coef, const double *sigma, const float *o0,
                                      const float *o1, double thr, double *out, int *flags,
                                      double *dis) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < cnt; j += gridDim.x * blockDim.x) {
    const int s = off + j;
    double x[kMaxDim];
    bool outside = false;
    for (int i = 0; i < d; ++i) {
      x[i] = (theta[s + (int64_t)i * ntot] - centre[i]) / half[i];
      outside |= (fabs(x[i]) > kHullMargin);
    }
    const double q = baseline_value_fast(x, d, deg, nf, midx, coef);
    const double a = o0[(int64_t)j * kOut0], b = o1[(int64_t)j * kOut0];
    out[s] = q + *sigma * 0.5 * (a + b);
    const double dab = *sigma * fabs(a - b);
    if (flags) flags[s] = (outside || dab > thr) ? 1 : 0;
    if (dis) dis[s] = dab;
  }
}

// ------------------------------------------------- tcgen05 inference layer --
// A layer at inference, Y = X W^T + b, on tcgen05 tensor cores (kind::f16:
// bf16 x bf16 -> fp32 in TMEM).  X is the layer's bf16 input (rows x K,
// row-major, rows a multiple of 128), W its bf16 weights (N x K, row-major),
// K a multiple of 64 up to 256.  Persistent: each CTA takes the 128-row tiles
// blockIdx.x, + gridDim.x, ...  Warp 0 (one lane) loads W once (all of K, in
// 128-byte-swizzled stages of 64 columns) and then streams the tiles' X
// through a ring of kTcRing 64-column slots; warp 1 owns the TMEM allocation
// and issues each tile's K / 16 MMAs (M = 128, N) into one of two
// accumulators; warps 2-9 are the epilogue (TMEM lanes 32 (w % 4) .., column
// half (w - 2) / 4), which adds the bias and writes bf16(gelu(Y)) to Xn for a
// hidden layer or fp32 Y to Z for the output layer.  With two accumulators a
// tile's epilogue runs while the next tile's X arrives and is multiplied.
// Every wait is bounded: on expiry the status takes QML_ETIMEOUT, copies and
// MMAs in flight are drained, TMEM is freed, and the rest of the layer is not
// written.
constexpr int kTcMaxStages = 4;  // K <= 256
constexpr int kTcRing = 4;       // X slots of 64 columns
constexpr int kTcThreads = 320;
template <int N>
constexpr size_t tc_smem() {
  return 1024 + (size_t)kTcMaxStages * N * 128 + (size_t)kTcRing * 128 * 128 + 256;
}
template <int N>
__global__ void __launch_bounds__(kTcThreads, 1)
    mlp_tc_kernel(const __grid_constant__ CUtensorMap mX, const __grid_constant__ CUtensorMap mW,
                  int rows, int K, const float *bias, __nv_bfloat16 *Xn, float *Z, DevStatus *st) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  constexpr int kA = 128 * 128, kB = N * 128;  // bytes of one 64-column stage
  constexpr int kCols = N <= 32 ? 32 : (N <= 64 ? 64 : (N <= 128 ? 128 : 256));
  constexpr int kEpiThreads = N > 16 ? 256 : 128;
  constexpr uint32_t kIdescN = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
                               ((uint32_t)(128 >> 4) << 24);
  unsigned char *tB = smem, *tA = smem + kTcMaxStages * kB;
  // bars: wfull, xfull[kTcRing], xempty[kTcRing], accf[2], acce[2], drain
  uint64_t *bars = (uint64_t *)(tA + kTcRing * kA);
  uint32_t *holder = (uint32_t *)(bars + 2 * kTcRing + 6);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nst = K / 64, ntiles = rows / 128;
  const uint32_t wfull = smem_u32(&bars[0]), xfull0 = smem_u32(&bars[1]),
                 xempty0 = smem_u32(&bars[1 + kTcRing]), accf0 = smem_u32(&bars[1 + 2 * kTcRing]),
                 acce0 = smem_u32(&bars[3 + 2 * kTcRing]), drain = smem_u32(&bars[5 + 2 * kTcRing]);
  if (threadIdx.x == 0) {
    mbar_init(wfull, 1);
    for (int q = 0; q < kTcRing; ++q) {
      mbar_init(xfull0 + 8 * q, 1);
      mbar_init(xempty0 + 8 * q, 1);
    }
    for (int q = 0; q < 2; ++q) {
      mbar_init(accf0 + 8 * q, 1);
      mbar_init(acce0 + 8 * q, kEpiThreads);
    }
    mbar_init(drain, 1);
    fence_mbar_init();
  }
  if (warp == 1) tmem_alloc(smem_u32(holder), 2 * kCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *holder;
  const bool go = *((volatile int *)&st->code) == 0;
  if (go && warp == 0 && lane == 0) {
    // ---- producer: W once, then X chunk by chunk through the ring
    int last_phase[kTcRing];
    for (int q = 0; q < kTcRing; ++q) last_phase[q] = -1;
    bool ok = true;
    mbar_expect_tx(wfull, (uint32_t)(nst * kB));
    for (int s2 = 0; s2 < nst; ++s2) tma_load_2d(smem_u32(tB + s2 * kB), &mW, wfull, 64 * s2, 0);
    uint32_t idx = 0;
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x)
      for (int s2 = 0; s2 < nst; ++s2, ++idx) {
        const uint32_t q = idx % kTcRing, ph = (idx / kTcRing) & 1u;
        if (!mbar_wait(xempty0 + 8 * q, ph ^ 1u, st)) { ok = false; break; }
        mbar_expect_tx(xfull0 + 8 * q, (uint32_t)kA);
        tma_load_2d(smem_u32(tA + q * kA), &mX, xfull0 + 8 * q, 64 * s2, 128 * t);
        last_phase[q] = (int)ph;
      }
    // every copy issued into this CTA's shared memory lands before it exits
    mbar_drain_wait(wfull, 0);
    for (int q = 0; q < kTcRing; ++q)
      if (last_phase[q] >= 0) mbar_drain_wait(xfull0 + 8 * q, (uint32_t)last_phase[q]);
  } else if (go && warp == 1 && lane == 0) {
    // ---- MMA issuer
    bool ok = mbar_wait(wfull, 0, st);
    uint32_t idx = 0, it = 0;
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++it) {
      const uint32_t bsel = it & 1u;
      // the epilogue has read this accumulator's previous tile
      if (!mbar_wait(acce0 + 8 * bsel, ((it >> 1) & 1u) ^ 1u, st)) { ok = false; break; }
      tc_fence_after();
      uint32_t on = 0;
      for (int s2 = 0; s2 < nst; ++s2, ++idx) {
        const uint32_t q = idx % kTcRing, ph = (idx / kTcRing) & 1u;
        if (!mbar_wait(xfull0 + 8 * q, ph, st)) { ok = false; break; }
        tc_fence_after();
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          mma_bf16(tbase + bsel * kCols, smem_desc(smem_u32(tA + q * kA) + 32 * kk),
                   smem_desc(smem_u32(tB + s2 * kB) + 32 * kk), kIdescN, on);
          on = 1u;
        }
        mma_commit(xempty0 + 8 * q);  // the slot is free when these MMAs finish
      }
      if (!ok) break;
      mma_commit(accf0 + 8 * bsel);
    }
    mma_commit(drain);  // every MMA issued above has finished when this arrives
    mbar_drain_wait(drain, 0);
  } else if (go && warp >= 2 && (N > 16 || warp < 6)) {
    // ---- epilogue
    const int quad = warp & 3;
    const int half = N > 16 ? (warp - 2) >> 2 : 0;
    constexpr int kW = N > 16 ? N / 2 : N;  // columns per epilogue warp
    uint32_t it = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
      const uint32_t bsel = it & 1u;
      int okw = 1;
      if (lane == 0) okw = mbar_wait(accf0 + 8 * bsel, (it >> 1) & 1u, st) ? 1 : 0;
      okw = __shfl_sync(0xffffffffu, okw, 0);
      __syncwarp();
      if (!okw) break;
      tc_fence_after();
      const int row = 128 * t + quad * 32 + lane;
      const uint32_t lb = tbase + bsel * kCols + ((uint32_t)(quad * 32) << 16) + (uint32_t)(half * kW);
#pragma unroll 1
      for (int cb = 0; cb < kW / 16; ++cb) {
        uint32_t a[16];
        tmem_ld16(lb + 16 * cb, a);
        const int c0 = half * kW + 16 * cb;
        // bias + c0 is 64-byte aligned: every layer's bias starts at a
        // multiple of 16 floats of the parameter block (widths are multiples
        // of 16), and the launch checks the block's alignment
        const float4 *b4 = reinterpret_cast<const float4 *>(bias + c0);
        float y[16];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float4 bv = b4[j];
          y[4 * j] = __uint_as_float(a[4 * j]) + bv.x;
          y[4 * j + 1] = __uint_as_float(a[4 * j + 1]) + bv.y;
          y[4 * j + 2] = __uint_as_float(a[4 * j + 2]) + bv.z;
          y[4 * j + 3] = __uint_as_float(a[4 * j + 3]) + bv.w;
        }
        if (row < rows) {
          if (Xn) {
            __align__(16) __nv_bfloat16 o[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) o[j] = __float2bfloat16_rn(gelu_f(y[j]));
            uint4 *dst = (uint4 *)(Xn + (int64_t)row * N + c0);
            dst[0] = ((const uint4 *)o)[0];
            dst[1] = ((const uint4 *)o)[1];
          } else {
            float4 *dst = (float4 *)(Z + (int64_t)row * N + c0);
#pragma unroll
            for (int j = 0; j < 4; ++j) dst[j] = make_float4(y[4 * j], y[4 * j + 1], y[4 * j + 2], y[4 * j + 3]);
          }
        }
      }
      tc_fence_before();
      mbar_arrive(acce0 + 8 * bsel);  // the accumulator may take the tile after next
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tbase, 2 * kCols);
}

template <int N>
bool launch_mlp_tc(const CUtensorMap &mX, const CUtensorMap &mW, int rows, int K, const float *bias,
                   __nv_bfloat16 *Xn, float *Z, DevStatus *st, cudaStream_t s) {
  if (((uintptr_t)bias & 15) != 0) return false;  // the epilogue reads the bias as float4
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(mlp_tc_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tc_smem<N>()) != cudaSuccess)
      return false;
    attr = true;
  }
  static int nsm = 0;
  if (nsm == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1)
      nsm = 148;
  }
  const int ntiles = rows / 128, grid = ntiles < nsm ? ntiles : nsm;  // persistent
  mlp_tc_kernel<N><<<grid, kTcThreads, tc_smem<N>(), s>>>(mX, mW, rows, K, bias, Xn, Z, st);
  count_launch();
  return true;
}

int grid_of(int64_t total) {
  int64_t b = (total + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

// ======================================================================
struct qml_emu {
  int d = 0, width = 0, depth = 0, nheads = 2;
  uint64_t seed = 0;
  std::vector<std::pair<int, int>> layers;  // (out, in)
  std::vector<int64_t> woff, boff;          // offsets into the flat parameter vector
  int64_t nparam = 0;
  // device
  double *centre = nullptr, *half = nullptr, *coef = nullptr, *sigma = nullptr;
  // baseline: total degree, feature count and multi-indices (nf x d, device)
  int deg = 0, nf = 1;
  unsigned char *midx = nullptr;
  float *p[2] = {nullptr, nullptr}, *m[2] = {nullptr, nullptr}, *v[2] = {nullptr, nullptr};
  __nv_bfloat16 *ph[2] = {nullptr, nullptr};
  float *grad = nullptr;
  int adam_t[2] = {0, 0};
  bool fitted = false;
  // held-out labels, sorted by head disagreement: disagreement and the
  // running maximum of the prediction error up to it
  std::vector<double> val_dis, val_maxerr;
  std::vector<void *> mem;
  // buffers of emu_predict, kept between calls (freed by emu_free)
  void *pcache = nullptr;
  void (*pcache_free)(void *) = nullptr;
};

namespace {

qml_status efail(qml_status s, const std::string &m) {
  set_last_error(m);
  return s;
}

template <class T>
T *emu_alloc(qml_emu *e, size_t count) {
  void *p = nullptr;
  if (cudaMalloc(&p, count * sizeof(T)) != cudaSuccess) return nullptr;
  e->mem.push_back(p);
  return (T *)p;
}

// activations of one batch (Brows a multiple of 16)
struct Acts {
  int B = 0;
  std::vector<__nv_bfloat16 *> X;  // inputs of each layer, B x in_l
  std::vector<float *> Z;          // pre-activations, B x out_l
  float *dZf = nullptr, *dX = nullptr, *tb = nullptr;
  __nv_bfloat16 *dZh = nullptr;
  double *partial = nullptr, *loss = nullptr;
  std::vector<void *> mem;
  ~Acts() {
    for (void *p : mem) cudaFree(p);
  }
  template <class T>
  T *a(size_t count) {
    void *p = nullptr;
    if (cudaMalloc(&p, count * sizeof(T)) != cudaSuccess) return nullptr;
    mem.push_back(p);
    return (T *)p;
  }
  bool make(const qml_emu *e, int Brows) {
    B = Brows;
    int maxw = kIn0;
    for (auto &l : e->layers) maxw = std::max(maxw, std::max(l.first, l.second));
    for (auto &l : e->layers) {
      X.push_back(a<__nv_bfloat16>((size_t)B * l.second));
      Z.push_back(a<float>((size_t)B * l.first));
    }
    dZf = a<float>((size_t)B * maxw);
    dX = a<float>((size_t)B * maxw);
    dZh = a<__nv_bfloat16>((size_t)B * maxw);
    tb = a<float>(B);
    partial = a<double>(256);
    loss = a<double>(1);
    for (auto *p : X) if (!p) return false;
    for (auto *p : Z) if (!p) return false;
    return dZf && dX && dZh && tb && partial && loss;
  }
};

void forward(qml_emu *e, int h, Acts &A, cudaStream_t st) {
  const int nl = (int)e->layers.size();
  for (int l = 0; l < nl; ++l) {
    const int out = e->layers[l].first, in = e->layers[l].second;
    // Z = X W^T: A = X (B x in, row-major), B = W^T (in x out) = W col-major
    wmma_gemm<wmma::row_major, wmma::col_major>(A.B, out, in, A.X[l], in, e->ph[h] + e->woff[l],
                                                in, A.Z[l], out, 0, st);
    __nv_bfloat16 *next = (l + 1 < nl) ? A.X[l + 1] : nullptr;
    bias_act_kernel<<<grid_of((int64_t)A.B * out), 256, 0, st>>>(A.Z[l], A.B, out, e->p[h] + e->boff[l],
                                                                 next, l + 1 < nl ? 1 : 0);
    count_launch();
  }
}

// Inference on tcgen05: every layer (K = width, a multiple of 64 up to 256;
// the first layer's 16 inputs and weights widened with zeros to 64) runs as
// mlp_tc_kernel with bias and activation fused.  Tuning key emu_tc = 0
// selects the WMMA path for every layer, emu_tc0 = 0 for the first one.
bool tc_capable(const qml_emu *e) { return e->width % 64 == 0 && e->width <= 256; }
bool use_tc(const qml_emu *e) { return tune_get("emu_tc", 1) != 0 && tc_capable(e); }

// tensor maps of every layer l >= 1: its input activations (rows x in) and
// head h's weights (out x in)
bool make_tc_maps(const qml_emu *e, int h, const Acts &A, int rows,
                  std::vector<CUtensorMap> &mx, std::vector<CUtensorMap> &mw) {
  const int nl = (int)e->layers.size();
  mx.assign(nl, CUtensorMap{});
  mw.assign(nl, CUtensorMap{});
  for (int l = 1; l < nl; ++l) {
    const int out = e->layers[l].first, in = e->layers[l].second;
    if (!make_map_bf16(&mx[l], A.X[l], in, rows, (int64_t)in * 2, 64, 128)) return false;
    if (!make_map_bf16(&mw[l], e->ph[h] + e->woff[l], in, out, (int64_t)in * 2, 64, out))
      return false;
  }
  return true;
}

bool launch_tc_layer(int out, const CUtensorMap &mx, const CUtensorMap &mw, int rows, int in,
                     const float *b, __nv_bfloat16 *xn, float *z, DevStatus *st, cudaStream_t s) {
  switch (out) {
    case 16: return launch_mlp_tc<16>(mx, mw, rows, in, b, xn, z, st, s);
    case 64: return launch_mlp_tc<64>(mx, mw, rows, in, b, xn, z, st, s);
    case 128: return launch_mlp_tc<128>(mx, mw, rows, in, b, xn, z, st, s);
    case 192: return launch_mlp_tc<192>(mx, mw, rows, in, b, xn, z, st, s);
    case 256: return launch_mlp_tc<256>(mx, mw, rows, in, b, xn, z, st, s);
    default: return false;
  }
}

// m0x / m0w: maps of the first layer's inputs and weights widened to 64
// columns (then the first layer runs on tcgen05 too), or null (WMMA)
bool forward_tc(qml_emu *e, int h, Acts &A, int rows, const std::vector<CUtensorMap> &mx,
                const std::vector<CUtensorMap> &mw, const CUtensorMap *m0x,
                const CUtensorMap *m0w, DevStatus *st, cudaStream_t s) {
  const int nl = (int)e->layers.size();
  {
    const int out = e->layers[0].first, in = e->layers[0].second;
    if (m0x && m0w) {
      if (!launch_tc_layer(out, *m0x, *m0w, rows, 64, e->p[h] + e->boff[0], A.X[1], nullptr, st,
                           s))
        return false;
    } else {
      wmma_gemm<wmma::row_major, wmma::col_major>(A.B, out, in, A.X[0], in,
                                                  e->ph[h] + e->woff[0], in, A.Z[0], out, 0, s);
      bias_act_kernel<<<grid_of((int64_t)A.B * out), 256, 0, s>>>(A.Z[0], A.B, out,
                                                                  e->p[h] + e->boff[0], A.X[1], 1);
      count_launch();
    }
  }
  for (int l = 1; l < nl; ++l) {
    const int out = e->layers[l].first, in = e->layers[l].second;
    __nv_bfloat16 *xn = (l + 1 < nl) ? A.X[l + 1] : nullptr;
    float *z = (l + 1 < nl) ? nullptr : A.Z[l];
    if (!launch_tc_layer(out, mx[l], mw[l], rows, in, e->p[h] + e->boff[l], xn, z, st, s))
      return false;
  }
  return true;
}

// gradient of the mean squared error of head h over the first nreal rows
void backward(qml_emu *e, int h, Acts &A, int nreal, cudaStream_t st) {
  const int nl = (int)e->layers.size();
  loss_grad_kernel<<<64, 256, 0, st>>>(A.Z[nl - 1], A.tb, A.B, nreal, A.dZf, A.dZh, A.partial);
  count_launch();
  sum_partials_kernel<<<1, 32, 0, st>>>(A.partial, 64, 1.0 / nreal, A.loss);
  count_launch();
  for (int l = nl - 1; l >= 0; --l) {
    const int out = e->layers[l].first, in = e->layers[l].second;
    // dW = dZ^T X: A = dZ^T (out x B) = dZ col-major (ld out), B = X (B x in) row-major
    wmma_gemm<wmma::col_major, wmma::row_major>(out, in, A.B, A.dZh, out, A.X[l], in,
                                                e->grad + e->woff[l], in, 0, st);
    colsum_kernel<<<(out + 127) / 128, 128, 0, st>>>(A.dZf, A.B, out, e->grad + e->boff[l]);
    count_launch();
    if (l > 0) {
      // dX = dZ W: A = dZ (B x out) row-major, B = W (out x in) row-major
      wmma_gemm<wmma::row_major, wmma::row_major>(A.B, in, out, A.dZh, out, e->ph[h] + e->woff[l],
                                                  in, A.dX, in, 0, st);
      gelu_bwd_kernel<<<grid_of((int64_t)A.B * in), 256, 0, st>>>(A.dX, A.Z[l - 1],
                                                                  (int64_t)A.B * in, A.dZf, A.dZh);
      count_launch();
    }
  }
}

bool is_dev(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// device copy of a host or device array (owned by `keep` when copied)
const double *dev_in(const double *p, size_t count, std::vector<void *> &keep) {
  if (is_dev(p)) return p;
  void *d = nullptr;
  if (cudaMalloc(&d, count * sizeof(double)) != cudaSuccess) return nullptr;
  keep.push_back(d);
  cudaMemcpy(d, p, count * sizeof(double), cudaMemcpyHostToDevice);
  return (const double *)d;
}

// Predictions (and flags / disagreements when given) at n device points.
// Activations of both heads for emu_predict, their tensor maps and a status
// word, sized for `rows` points per chunk; kept in the emulator between calls
// (the buffers are about a gigabyte at width 256, and allocating and freeing
// them each call would cost more than the inference).
struct PredCache {
  int rows = 0;
  Acts A0, A1;
  bool tc = false;
  std::vector<CUtensorMap> mx0, mw0, mx1, mw1;
  // the first layer widened to 64 input columns: inputs (rows x 64, both
  // heads) and each head's weights (width x 64), refreshed every call
  __nv_bfloat16 *x0p = nullptr, *w0p[2] = {nullptr, nullptr};
  bool tc0 = false;
  CUtensorMap mx0p, mw0p[2];
  DevStatus *dst = nullptr;
  ~PredCache() {
    if (dst) cudaFree(dst);
    if (x0p) cudaFree(x0p);
    for (auto *w : w0p)
      if (w) cudaFree(w);
  }
};

void free_pred_cache(void *p) { delete (PredCache *)p; }

PredCache *pred_cache(qml_emu *e, int rows) {
  PredCache *c = (PredCache *)e->pcache;
  if (c && c->rows >= rows) return c;
  if (c) {
    cudaDeviceSynchronize();
    delete c;
    e->pcache = nullptr;
  }
  c = new PredCache();
  c->rows = rows;
  if (!c->A0.make(e, rows) || !c->A1.make(e, rows) ||
      cudaMalloc(&c->dst, sizeof(DevStatus)) != cudaSuccess) {
    delete c;
    return nullptr;
  }
  // the tensor maps are made whenever the width allows; emu_tc is read per call
  c->tc = tc_capable(e) && make_tc_maps(e, 0, c->A0, rows, c->mx0, c->mw0) &&
          make_tc_maps(e, 1, c->A1, rows, c->mx1, c->mw1);
  if (c->tc) {
    const int w0 = e->layers[0].first;
    c->tc0 = cudaMalloc(&c->x0p, (size_t)rows * 64 * sizeof(__nv_bfloat16)) == cudaSuccess &&
             cudaMalloc(&c->w0p[0], (size_t)w0 * 64 * sizeof(__nv_bfloat16)) == cudaSuccess &&
             cudaMalloc(&c->w0p[1], (size_t)w0 * 64 * sizeof(__nv_bfloat16)) == cudaSuccess &&
             make_map_bf16(&c->mx0p, c->x0p, 64, rows, 128, 64, 128) &&
             make_map_bf16(&c->mw0p[0], c->w0p[0], 64, w0, 128, 64, w0) &&
             make_map_bf16(&c->mw0p[1], c->w0p[1], 64, w0, 128, 64, w0);
  }
  e->pcache = c;
  e->pcache_free = free_pred_cache;
  return c;
}

qml_status run_predict(qml_emu *e, int n, const double *th, double thr, double *od, int *fd,
                       double *dis, cudaStream_t st) {
  // points per pass through the layers (tuning key emu_chunk, a multiple of
  // 128, default 262144): each layer launch then has enough 128-row tiles for
  // its persistent CTAs to pipeline over (2^20 points: 1.55e8 points/s in
  // passes of 65536, 2.07e8 in passes of 262144)
  int chunk = (int)std::min<int64_t>(std::max<int64_t>(tune_get("emu_chunk", 262144), 128), 1 << 22);
  chunk = chunk / 128 * 128;
  // activation rows allocated in whole 128-row tiles (the tcgen05 layers read
  // and write complete tiles; rows past the points are never used)
  const int rows_alloc = (std::min(chunk, (n + 15) / 16 * 16) + 127) / 128 * 128;
  PredCache *pc = pred_cache(e, rows_alloc);
  if (!pc) return QML_ENOMEM;
  Acts &A0 = pc->A0, &A1 = pc->A1;
  bool tc = pc->tc && use_tc(e);
  const std::vector<CUtensorMap> &mx0 = pc->mx0, &mw0 = pc->mw0, &mx1 = pc->mx1, &mw1 = pc->mw1;
  DevStatus *dst = pc->dst;
  if (cudaMemsetAsync(dst, 0, sizeof(DevStatus), st) != cudaSuccess) return QML_ENOMEM;
  const bool tc0 = tc && pc->tc0 && tune_get("emu_tc0", 1) != 0;
  if (tc0) {
    const int w0 = e->layers[0].first;
    for (int h = 0; h < 2; ++h) {
      pad_cols_kernel<<<grid_of((int64_t)w0 * 64), 256, 0, st>>>(e->ph[h] + e->woff[0], w0, kIn0,
                                                                 pc->w0p[h], 64);
      count_launch();
    }
  }
  for (int off = 0; off < n; off += chunk) {
    const int cnt = std::min(chunk, n - off);
    const int Bc = (cnt + 15) / 16 * 16;
    A0.B = A1.B = Bc;
    gather_kernel<<<grid_of((int64_t)Bc * kIn0), 256, 0, st>>>(th + off, n, e->d, e->centre, e->half,
                                                               nullptr, Bc, cnt, 0, 1, A0.X[0], nullptr);
    count_launch();
    cudaMemcpyAsync(A1.X[0], A0.X[0], (size_t)Bc * kIn0 * sizeof(__nv_bfloat16),
                    cudaMemcpyDeviceToDevice, st);
    const int rows_tc = (Bc + 127) / 128 * 128;
    if (tc0) {
      pad_cols_kernel<<<grid_of((int64_t)Bc * 64), 256, 0, st>>>(A0.X[0], Bc, kIn0, pc->x0p, 64);
      count_launch();
    }
    if (!tc ||
        !forward_tc(e, 0, A0, rows_tc, mx0, mw0, tc0 ? &pc->mx0p : nullptr,
                    tc0 ? &pc->mw0p[0] : nullptr, dst, st) ||
        !forward_tc(e, 1, A1, rows_tc, mx1, mw1, tc0 ? &pc->mx0p : nullptr,
                    tc0 ? &pc->mw0p[1] : nullptr, dst, st)) {
      if (tc) {  // a launch was refused: finish on the WMMA path
        tc = false;
        cudaGetLastError();
      }
      forward(e, 0, A0, st);
      forward(e, 1, A1, st);
    }
    const int nl = (int)e->layers.size();
    predict_finish_kernel<<<grid_of(cnt), 256, 0, st>>>(th, n, off, cnt, e->d, e->deg, e->nf,
                                                        e->midx, e->centre, e->half, e->coef,
                                                        e->sigma, A0.Z[nl - 1],
                                                        A1.Z[nl - 1], thr, od, fd, dis);
    count_launch();
  }
  {
    DevStatus hs{};
    cudaMemcpyAsync(&hs, dst, sizeof(hs), cudaMemcpyDeviceToHost, st);
    const cudaError_t err = cudaStreamSynchronize(st);
    if (err != cudaSuccess)
      return efail(QML_ECUDA, std::string("emulator inference: ") + cudaGetErrorString(err));
    if (hs.code != 0)
      return efail(QML_ETIMEOUT, "emulator inference: a tensor-core wait ran out of time");
  }
  return QML_OK;
}

// Disagreement threshold for accuracy target tol: at most tol / 2, and below
// the smallest held-out disagreement whose running maximum error exceeds
// 0.8 tol (so every held-out point that would be accepted is within 0.8 tol).
double flag_threshold(const qml_emu *e, double tol) {
  double thr = 0.5 * tol;
  for (size_t i = 0; i < e->val_dis.size(); ++i)
    if (e->val_maxerr[i] > 0.8 * tol) {
      thr = std::min(thr, std::nextafter(e->val_dis[i], 0.0));
      break;
    }
  return thr;
}

// seeded permutation of 0..n-1 (splitmix64 stream, Fisher-Yates)
std::vector<int> permutation(int n, uint64_t seed) {
  std::vector<int> p(n);
  for (int i = 0; i < n; ++i) p[i] = i;
  uint64_t z = seed * 0xD1B54A32D192ED03ull + 0x8CB92BA72F3D8DD7ull;
  for (int i = n - 1; i > 0; --i) {
    z += 0x9E3779B97F4A7C15ull;
    uint64_t x = z;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    x ^= x >> 31;
    const int j = (int)(x % (uint64_t)(i + 1));
    std::swap(p[i], p[j]);
  }
  return p;
}

}  // namespace

extern "C" {

int64_t emu_param_count(const qml_emu *emu) { return emu ? emu->nparam : 0; }

qml_status emu_create(int32_t ndim, const double *lo, const double *hi, int32_t width,
                      int32_t depth, uint64_t seed, qml_emu **out) {
  if (!out || !lo || !hi || ndim < 1 || ndim > kMaxDim || width < 16 || width % 16 || depth < 1 ||
      depth > 16)
    return efail(QML_EINVAL, "emu_create: need 1 <= ndim <= 8, width a multiple of 16, depth >= 1");
  qml_emu *e = new qml_emu();
  e->d = ndim;
  e->width = width;
  e->depth = depth;
  e->seed = seed;
  int in = kIn0;
  for (int l = 0; l < depth; ++l) {
    e->layers.push_back({width, in});
    in = width;
  }
  e->layers.push_back({kOut0, in});
  for (auto &l : e->layers) {
    e->woff.push_back(e->nparam);
    e->nparam += (int64_t)l.first * l.second;
    e->boff.push_back(e->nparam);
    e->nparam += l.first;
  }
  std::vector<double> c(ndim), hw(ndim);
  for (int i = 0; i < ndim; ++i) {
    if (!(hi[i] > lo[i])) {
      delete e;
      return efail(QML_EINVAL, "emu_create: need hi > lo in every dimension");
    }
    c[i] = 0.5 * (hi[i] + lo[i]);
    hw[i] = 0.5 * (hi[i] - lo[i]);
  }
  e->centre = emu_alloc<double>(e, ndim);
  e->half = emu_alloc<double>(e, ndim);
  e->coef = emu_alloc<double>(e, kMaxFeat);
  e->midx = emu_alloc<unsigned char>(e, kMaxFeat * kMaxDim);
  e->sigma = emu_alloc<double>(e, 1);
  e->grad = emu_alloc<float>(e, e->nparam);
  for (int h = 0; h < 2; ++h) {
    e->p[h] = emu_alloc<float>(e, e->nparam);
    e->m[h] = emu_alloc<float>(e, e->nparam);
    e->v[h] = emu_alloc<float>(e, e->nparam);
    e->ph[h] = emu_alloc<__nv_bfloat16>(e, e->nparam);
  }
  if (!e->centre || !e->half || !e->coef || !e->midx || !e->sigma || !e->grad || !e->p[1] ||
      !e->ph[1]) {
    emu_free(e);
    return efail(QML_ENOMEM, "emu_create: device allocation failed");
  }
  cudaMemcpy(e->centre, c.data(), ndim * sizeof(double), cudaMemcpyHostToDevice);
  cudaMemcpy(e->half, hw.data(), ndim * sizeof(double), cudaMemcpyHostToDevice);
  cudaMemset(e->coef, 0, kMaxFeat * sizeof(double));
  cudaMemset(e->midx, 0, kMaxFeat * kMaxDim);  // untrained: one constant feature, q = 0
  const double one = 1.0;
  cudaMemcpy(e->sigma, &one, sizeof(double), cudaMemcpyHostToDevice);
  for (int h = 0; h < 2; ++h) {
    for (size_t l = 0; l < e->layers.size(); ++l) {
      const int o = e->layers[l].first, i = e->layers[l].second;
      const int in_real = (l == 0) ? ndim : i;
      const int out_real = (l + 1 == e->layers.size()) ? 1 : o;
      init_layer_kernel<<<64, 256>>>(e->p[h] + e->woff[l], e->p[h] + e->boff[l], o, i, in_real,
                                     out_real, l + 1 == e->layers.size() ? 1 : 0,
                                     seed * 16 + 2 * h + 1 + 64 * l);
      count_launch();
    }
    to_bf16_kernel<<<grid_of(e->nparam), 256>>>(e->p[h], e->nparam, e->ph[h]);
    count_launch();
    cudaMemset(e->m[h], 0, e->nparam * sizeof(float));
    cudaMemset(e->v[h], 0, e->nparam * sizeof(float));
  }
  if (cudaDeviceSynchronize() != cudaSuccess) {
    emu_free(e);
    return efail(QML_ECUDA, "emu_create: initialisation failed");
  }
  *out = e;
  return QML_OK;
}

void emu_free(qml_emu *emu) {
  if (!emu) return;
  cudaDeviceSynchronize();
  if (emu->pcache && emu->pcache_free) emu->pcache_free(emu->pcache);
  for (void *p : emu->mem) cudaFree(p);
  delete emu;
}

qml_status emu_train(qml_emu *e, int32_t n, const double *theta, const double *lnl,
                     int32_t epochs, int32_t batch, double lr, double *final_loss, void *stream) {
  if (!e || n < 16 || !theta || !lnl || epochs < 1 || batch < 16 || batch % 16 || lr <= 0.0)
    return efail(QML_EINVAL, "emu_train: need n >= 16, batch a positive multiple of 16, lr > 0");
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<void *> keep;
  // a seeded eighth of the labels (n >= 512) is held out of training and
  // calibrates the fallback threshold afterwards
  const int n_all = n;
  const int n_val = n_all >= 512 ? n_all / 8 : 0;
  n = n_all - n_val;
  std::vector<double> th_h((size_t)n_all * e->d), y_h(n_all);
  cudaStreamSynchronize(st);
  if (cudaMemcpy(th_h.data(), theta, th_h.size() * sizeof(double), cudaMemcpyDefault) != cudaSuccess ||
      cudaMemcpy(y_h.data(), lnl, y_h.size() * sizeof(double), cudaMemcpyDefault) != cudaSuccess)
    return efail(QML_ECUDA, "emu_train: reading theta / lnl failed");
  {
    const std::vector<int> perm = permutation(n_all, e->seed ^ 0x5EEDull);
    std::vector<double> tp(th_h.size()), yp(n_all);
    for (int s2 = 0; s2 < n_all; ++s2) {
      yp[s2] = y_h[perm[s2]];
      for (int i = 0; i < e->d; ++i) {
        // training rows first (0..n-1), held-out rows after; each block
        // column-major with its own row count
        const int64_t dst = s2 < n ? s2 + (int64_t)i * n
                                   : (int64_t)n * e->d + (s2 - n) + (int64_t)i * n_val;
        tp[dst] = th_h[perm[s2] + (size_t)i * n_all];
      }
    }
    th_h.swap(tp);
    y_h.swap(yp);
  }
  const double *th = dev_in(th_h.data(), (size_t)n_all * e->d, keep);
  const double *y = dev_in(y_h.data(), n_all, keep);
  double *res = nullptr, *part = nullptr, *sumsq = nullptr, *phi = nullptr, *gram = nullptr;
  float *targ = nullptr;
  // the baseline's degree and feature order for this many training labels
  e->deg = baseline_degree(e->d, n);
  e->nf = nfeat_of(e->d, e->deg);
  const int nf = e->nf;
  {
    std::vector<unsigned char> mi;
    multi_indices(e->d, e->deg, mi);
    cudaMemcpy(e->midx, mi.data(), mi.size(), cudaMemcpyHostToDevice);
  }
  cudaMalloc(&res, n * sizeof(double));
  cudaMalloc(&part, 256 * sizeof(double));
  cudaMalloc(&sumsq, sizeof(double));
  cudaMalloc(&targ, n * sizeof(float));
  cudaMalloc(&phi, (size_t)n * nf * sizeof(double));
  cudaMalloc(&gram, (size_t)nf * (nf + 1) * sizeof(double));
  keep.push_back(res);
  keep.push_back(part);
  keep.push_back(sumsq);
  keep.push_back(targ);
  keep.push_back(phi);
  keep.push_back(gram);
  auto cleanup = [&]() {
    cudaStreamSynchronize(st);
    for (void *p : keep) cudaFree(p);
  };
  if (!th || !y || !res || !part || !sumsq || !targ || !phi || !gram) {
    cleanup();
    return efail(QML_ENOMEM, "emu_train: allocation failed");
  }
  // polynomial baseline (float64 least squares: Phi^T Phi c = Phi^T y by
  // Cholesky) and normalised residual targets
  phi_kernel<<<grid_of(n), 256, 0, st>>>(th, n, e->d, e->deg, nf, e->midx, e->centre, e->half,
                                         phi);
  count_launch();
  launch_dgemm_fixed(1, 0, nf, nf, n, 1.0, phi, n, phi, n, 0.0, gram, nf, 0, nullptr, st);
  launch_dgemm_fixed(1, 0, nf, 1, n, 1.0, phi, n, y, n, 0.0, gram + (size_t)nf * nf, nf, 0,
                     nullptr, st);
  chol_solve_kernel<<<1, 256, 0, st>>>(gram, gram + (size_t)nf * nf, nf, e->coef);
  count_launch();
  residual_kernel<<<64, 256, 0, st>>>(th, y, n, e->d, e->deg, nf, e->midx, e->centre, e->half,
                                      e->coef, res, part);
  count_launch();
  sum_partials_kernel<<<1, 32, 0, st>>>(part, 64, 1.0, sumsq);
  count_launch();
  scale_targets_kernel<<<grid_of(n), 256, 0, st>>>(res, n, sumsq, targ, e->sigma);
  count_launch();
  Acts A;
  if (!A.make(e, batch)) {
    cleanup();
    return efail(QML_ENOMEM, "emu_train: activation allocation failed");
  }
  const int steps_per_epoch = (n + batch - 1) / batch;
  const int64_t total_steps = (int64_t)steps_per_epoch * epochs;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int h = 0; h < 2; ++h) {
    int64_t step = 0;
    for (int ep = 0; ep < epochs; ++ep) {
      // epoch order: off + j stride (mod n) with stride coprime to n
      uint64_t hsh = (e->seed + 1000003ull * (ep + 1) + 7919ull * (h + 1)) * 0x9E3779B97F4A7C15ull;
      int64_t stride = (int64_t)(hsh % (uint64_t)n) | 1;
      auto gcd = [](int64_t a, int64_t b) { while (b) { int64_t t = a % b; a = b; b = t; } return a; };
      while (gcd(stride, n) != 1) stride += 2;
      const int64_t off = (int64_t)((hsh >> 20) % (uint64_t)n);
      for (int sb = 0; sb < steps_per_epoch; ++sb, ++step) {
        const int nreal = std::min(batch, n - sb * batch);
        gather_kernel<<<grid_of((int64_t)batch * kIn0), 256, 0, st>>>(
            th, n, e->d, e->centre, e->half, targ, batch, nreal, off + (int64_t)sb * batch * stride,
            stride, A.X[0], A.tb);
        count_launch();
        forward(e, h, A, st);
        backward(e, h, A, nreal, st);
        // learning rate: constant for the first 80 % of the steps (the network
        // needs them to leave its initial plateau), then a cosine decay to 2 %
        const double frac = (double)step / (double)std::max<int64_t>(1, total_steps - 1);
        const double dec = frac < 0.8 ? 1.0
                                       : 0.02 + 0.98 * 0.5 * (1.0 + cos(3.141592653589793 * (frac - 0.8) / 0.2));
        const float lrs = (float)(lr * dec);
        e->adam_t[h] += 1;
        const float c1 = 1.0f / (1.0f - powf(b1, (float)e->adam_t[h]));
        const float c2 = 1.0f / (1.0f - powf(b2, (float)e->adam_t[h]));
        adam_kernel<<<grid_of(e->nparam), 256, 0, st>>>(e->p[h], e->grad, e->m[h], e->v[h],
                                                        e->nparam, lrs, b1, b2, eps, c1, c2,
                                                        e->ph[h]);
        count_launch();
      }
    }
    if (final_loss) {
      // loss of the trained head over (up to) the first 4096 samples
      const int ne = std::min(n, 4096);
      Acts E;
      const int Be = (ne + 15) / 16 * 16;
      if (E.make(e, Be)) {
        gather_kernel<<<grid_of((int64_t)Be * kIn0), 256, 0, st>>>(th, n, e->d, e->centre, e->half,
                                                                   targ, Be, ne, 0, 1, E.X[0], E.tb);
        count_launch();
        forward(e, h, E, st);
        backward(e, h, E, ne, st);
        cudaMemcpyAsync(&final_loss[h], E.loss, sizeof(double), cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
      }
    }
  }
  e->fitted = true;
  e->val_dis.clear();
  e->val_maxerr.clear();
  if (n_val > 0) {
    // flags with an infinite threshold mark the held-out points outside the
    // hull: those are always evaluated exactly and do not calibrate
    double *vd = nullptr, *vo = nullptr;
    int *vf = nullptr;
    cudaMalloc(&vd, n_val * sizeof(double));
    cudaMalloc(&vo, n_val * sizeof(double));
    cudaMalloc(&vf, n_val * sizeof(int));
    keep.push_back(vd);
    keep.push_back(vo);
    keep.push_back(vf);
    const qml_status ps = (!vd || !vo || !vf)
                              ? QML_ENOMEM
                              : run_predict(e, n_val, th + (int64_t)n * e->d, INFINITY, vo, vf,
                                            vd, st);
    if (ps != QML_OK) {
      cleanup();
      e->fitted = false;
      return ps == QML_ENOMEM ? efail(QML_ENOMEM, "emu_train: held-out evaluation failed") : ps;
    }
    std::vector<double> dh(n_val), oh(n_val);
    std::vector<int> fh(n_val);
    cudaMemcpyAsync(dh.data(), vd, n_val * sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(oh.data(), vo, n_val * sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(fh.data(), vf, n_val * sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    std::vector<int> ord;
    for (int i = 0; i < n_val; ++i)
      if (!fh[i]) ord.push_back(i);
    std::sort(ord.begin(), ord.end(), [&](int a, int b) { return dh[a] < dh[b]; });
    double mx = 0.0;
    for (int i : ord) {
      mx = std::max(mx, std::fabs(oh[i] - y_h[n + i]));
      e->val_dis.push_back(dh[i]);
      e->val_maxerr.push_back(mx);
    }
  }
  cudaError_t err = cudaStreamSynchronize(st);
  cleanup();
  if (err != cudaSuccess) return efail(QML_ECUDA, std::string("emu_train: ") + cudaGetErrorString(err));
  return QML_OK;
}

qml_status emu_predict(qml_emu *e, int32_t n, const double *theta, double tol, double *out,
                       int32_t *flags, void *stream) {
  if (!e || n < 1 || !theta || !out) return efail(QML_EINVAL, "emu_predict: bad arguments");
  if (!e->fitted) return efail(QML_EINVAL, "emu_predict: emulator not trained");
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<void *> keep;
  const double *th = dev_in(theta, (size_t)n * e->d, keep);
  double *od = out;
  int *fd = flags;
  const bool out_host = !is_dev(out), flags_host = flags && !is_dev(flags);
  if (out_host) {
    cudaMalloc(&od, n * sizeof(double));
    keep.push_back(od);
  }
  if (flags_host) {
    cudaMalloc(&fd, n * sizeof(int));
    keep.push_back(fd);
  }
  const qml_status ps = (!th || !od || (flags && !fd))
                            ? QML_ENOMEM
                            : run_predict(e, n, th, flag_threshold(e, tol), od, fd, nullptr, st);
  if (ps != QML_OK) {
    for (void *p : keep) cudaFree(p);
    return ps == QML_ENOMEM ? efail(QML_ENOMEM, "emu_predict: allocation failed") : ps;
  }
  if (out_host) cudaMemcpyAsync(out, od, n * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (flags_host) cudaMemcpyAsync(flags, fd, n * sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaError_t err = cudaStreamSynchronize(st);
  for (void *p : keep) cudaFree(p);
  if (err != cudaSuccess) return efail(QML_ECUDA, std::string("emu_predict: ") + cudaGetErrorString(err));
  return QML_OK;
}

qml_status emu_threshold(const qml_emu *e, double tol, double *thr, int32_t *nheld) {
  if (!e || !thr || !(tol > 0.0)) return efail(QML_EINVAL, "emu_threshold: bad arguments");
  if (!e->fitted) return efail(QML_EINVAL, "emu_threshold: emulator not trained");
  *thr = flag_threshold(e, tol);
  if (nheld) *nheld = (int32_t)e->val_dis.size();
  return QML_OK;
}

qml_status emu_params(qml_emu *e, int32_t head, float *out) {
  if (!e || head < 0 || head > 1 || !out) return efail(QML_EINVAL, "emu_params: bad arguments");
  cudaDeviceSynchronize();
  if (cudaMemcpy(out, e->p[head], e->nparam * sizeof(float), cudaMemcpyDefault) != cudaSuccess)
    return efail(QML_ECUDA, "emu_params: copy failed");
  return QML_OK;
}

qml_status emu_baseline(const qml_emu *e, double *coef, int32_t *nfeat_out, double *sigma) {
  if (!e || !coef || !nfeat_out || !sigma) return efail(QML_EINVAL, "emu_baseline: bad arguments");
  const int nf = e->nf;
  cudaDeviceSynchronize();
  if (cudaMemcpy(coef, e->coef, nf * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(sigma, e->sigma, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
    return efail(QML_ECUDA, "emu_baseline: copy failed");
  *nfeat_out = nf;
  return QML_OK;
}

qml_status emu_loss_grad(qml_emu *e, int32_t head, int32_t n, const double *x, const double *t,
                         double *loss, float *grad) {
  if (!e || head < 0 || head > 1 || n < 1 || !x || !t || !loss || !grad)
    return efail(QML_EINVAL, "emu_loss_grad: bad arguments");
  // x: n x 16 normalised inputs (row-major, host), t: n targets (host)
  const int Bp = (n + 15) / 16 * 16;
  Acts A;
  if (!A.make(e, Bp)) return efail(QML_ENOMEM, "emu_loss_grad: allocation failed");
  std::vector<__nv_bfloat16> xh((size_t)Bp * kIn0, __float2bfloat16_rn(0.0f));
  std::vector<float> th(Bp, 0.0f);
  for (int b = 0; b < n; ++b) {
    for (int c = 0; c < kIn0; ++c) xh[(size_t)b * kIn0 + c] = __float2bfloat16_rn((float)x[(size_t)b * kIn0 + c]);
    th[b] = (float)t[b];
  }
  cudaMemcpy(A.X[0], xh.data(), xh.size() * sizeof(__nv_bfloat16), cudaMemcpyHostToDevice);
  cudaMemcpy(A.tb, th.data(), Bp * sizeof(float), cudaMemcpyHostToDevice);
  forward(e, head, A, 0);
  backward(e, head, A, n, 0);
  cudaMemcpy(loss, A.loss, sizeof(double), cudaMemcpyDeviceToHost);
  if (cudaMemcpy(grad, e->grad, e->nparam * sizeof(float), cudaMemcpyDefault) != cudaSuccess)
    return efail(QML_ECUDA, "emu_loss_grad: copy failed");
  return QML_OK;
}

}  // extern "C"
