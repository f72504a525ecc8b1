// Dense float64 building blocks on CUDA cores: tiled GEMM, diagonal-block
// Cholesky with its triangular inverse, and small elementwise helpers.
//
// GB300's float64 rate is a few fused multiply-adds per clock per SM, so a
// 64x64 register-tiled kernel with shared-memory staging is bound by the
// float64 pipe, not by memory: each 64x64x16 step issues 65k FMAs against
// 16 KB of shared traffic.  Thread (tx, ty) of a 16x16 block owns rows
// tx + 16 i and columns ty + 16 j (i, j < 4), so a warp's stores cover 16
// consecutive rows of 2 columns and its shared reads broadcast.
#include "internal.cuh"

#include <math.h>

namespace qmlgb {

namespace {

constexpr int BM = 64, BN = 64, BK = 16;

template <bool TA, bool TB>
__global__ void __launch_bounds__(256) dgemm_kernel(int64_t M, int64_t N, int64_t K, double alpha,
                                                    const double *A, int64_t lda, const double *B,
                                                    int64_t ldb, double beta, double *C,
                                                    int64_t ldc, int lower,
                                                    const DevStatus *status) {
  if (status && *((volatile const int *)&status->code) != 0) return;
  const int64_t m0 = (int64_t)blockIdx.x * BM;
  const int64_t n0 = (int64_t)blockIdx.y * BN;
  if (lower && m0 + BM - 1 < n0) return;  // tile strictly above the diagonal
  __shared__ double As[2][BK][BM + 1];
  __shared__ double Bs[2][BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  double ra[4], rb[4];
  auto load_a = [&](int64_t k0) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int mm, kk;
      if (!TA) { mm = tid & 63; kk = (tid >> 6) + 4 * r; }
      else { kk = tid & 15; mm = (tid >> 4) + 16 * r; }
      int64_t gm = m0 + mm, gk = k0 + kk;
      double v = 0.0;
      if (gm < M && gk < K) v = TA ? A[gk + gm * lda] : A[gm + gk * lda];
      ra[r] = v;
    }
  };
  auto store_a = [&](int buf) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int mm, kk;
      if (!TA) { mm = tid & 63; kk = (tid >> 6) + 4 * r; }
      else { kk = tid & 15; mm = (tid >> 4) + 16 * r; }
      As[buf][kk][mm] = ra[r];
    }
  };
  auto load_b = [&](int64_t k0) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int nn, kk;
      if (!TB) { kk = tid & 15; nn = (tid >> 4) + 16 * r; }
      else { nn = tid & 63; kk = (tid >> 6) + 4 * r; }
      int64_t gn = n0 + nn, gk = k0 + kk;
      double v = 0.0;
      if (gn < N && gk < K) v = TB ? B[gn + gk * ldb] : B[gk + gn * ldb];
      rb[r] = v;
    }
  };
  auto store_b = [&](int buf) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int nn, kk;
      if (!TB) { kk = tid & 15; nn = (tid >> 4) + 16 * r; }
      else { nn = tid & 63; kk = (tid >> 6) + 4 * r; }
      Bs[buf][kk][nn] = rb[r];
    }
  };

  const int64_t nk = (K + BK - 1) / BK;
  if (nk > 0) {
    load_a(0);
    load_b(0);
    store_a(0);
    store_b(0);
  }
  __syncthreads();
  for (int64_t t = 0; t < nk; ++t) {
    const int buf = (int)(t & 1);
    if (t + 1 < nk) {
      load_a((t + 1) * BK);
      load_b((t + 1) * BK);
    }
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[buf][kk][tx + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[buf][kk][ty + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    if (t + 1 < nk) {
      store_a(buf ^ 1);
      store_b(buf ^ 1);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t gm = m0 + tx + 16 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t gn = n0 + ty + 16 * j;
      if (gn >= N) continue;
      if (lower && gm < gn) continue;
      double *cp = C + gm + gn * ldc;
      double v = alpha * acc[i][j];
      if (beta != 0.0) v = fma(beta, *cp, v);
      *cp = v;
    }
  }
}

// ------------------------------------------------ diagonal-block Cholesky --
// The factor L lives in the lower triangle of the shared tile a; its inverse
// is written into the strict upper triangle (inv[i][j] at a[j][i], i > j)
// and its diagonal into invd, so one 64 x 65 tile (33 KB) holds both.
// Column-parallel forward substitution: 256 threads = 64 columns x 4 partial
// sums; every lane reaches the shuffles (inactive columns contribute zero).
__device__ __forceinline__ double inv_at(double (*a)[kNB + 1], const double *invd, int k, int c) {
  return k == c ? invd[c] : a[c][k];
}

// (float64 division is expensive on this part: one reciprocal per diagonal
// entry, reused by every product)
__device__ void invert_lower_shared(double (*a)[kNB + 1], double *invd, int jb) {
  const int tid = threadIdx.x;
  const int col = tid >> 2, part = tid & 3;
  if (col < jb && part == 0) invd[col] = 1.0 / a[col][col];
  __syncthreads();
  for (int i = 1; i < jb; ++i) {
    double s = 0.0;
    if (col < i)
      for (int k = col + part; k < i; k += 4) s = fma(a[i][k], inv_at(a, invd, k, col), s);
    s += __shfl_down_sync(0xffffffffu, s, 2, 4);
    s += __shfl_down_sync(0xffffffffu, s, 1, 4);
    if (col < i && part == 0) a[col][i] = -s * invd[i];
    __syncthreads();
  }
}

// One CTA factors a jb x jb (jb <= 64) diagonal block in shared memory:
// right-looking unblocked Cholesky with a pivot check, then the inverse of
// the lower factor.  With factor == 0 the block already holds L and only the
// inverse is formed (blockIdx.x selects the block: j0 = blockIdx.x * kNB).
__global__ void __launch_bounds__(256) potrf_diag_kernel(double *A, int64_t lda, int64_t n,
                                                         int64_t j0, double *Linv,
                                                         double *logdet_part,
                                                         DevStatus *status, int factor) {
  __shared__ double a[kNB][kNB + 1];
  __shared__ double invd[kNB];
  __shared__ double rpiv;
  __shared__ int bad;
  const int tid = threadIdx.x;
  if (status && *((volatile int *)&status->code) != 0) return;
  if (!factor) {
    j0 = (int64_t)blockIdx.x * kNB;
    A += j0 + j0 * lda;
    Linv += (int64_t)blockIdx.x * kNB * kNB;
  }
  const int jb = (int)((n - j0) < kNB ? (n - j0) : kNB);
  if (tid == 0) bad = 0;
  for (int t = tid; t < kNB * kNB; t += blockDim.x) {
    int i = t % kNB, j = t / kNB;
    a[i][j] = (i < jb && j < jb && i >= j) ? A[i + j * lda] : 0.0;
  }
  __syncthreads();
  if (factor) {
    for (int c = 0; c < jb; ++c) {
      if (tid == 0) {
        double piv = a[c][c];
        if (!(piv > 0.0) || !isfinite(piv)) {
          bad = 1;
          status->info = (int)(j0 + c + 1);
          atomicExch(&status->code, 2 /* QML_ENOTSPD */);
        } else {
          const double d = sqrt(piv);
          a[c][c] = d;
          rpiv = 1.0 / d;
        }
      }
      __syncthreads();
      if (bad) return;
      const double r = rpiv;
      for (int i = c + 1 + tid; i < jb; i += blockDim.x) a[i][c] *= r;
      __syncthreads();
      // trailing rank-1 update: row i = c+1+(tid % 64), columns strided by 4
      {
        const int i = c + 1 + (tid & 63);
        if (i < jb) {
          const double aic = a[i][c];
          for (int j = c + 1 + (tid >> 6); j <= i; j += 4) a[i][j] = fma(-aic, a[j][c], a[i][j]);
        }
      }
      __syncthreads();
    }
    for (int t = tid; t < jb * jb; t += blockDim.x) {
      int i = t % jb, j = t / jb;
      if (i >= j) A[i + j * lda] = a[i][j];
    }
    // logs in parallel, summed in a fixed order
    if (tid < jb) invd[tid] = log(a[tid][tid]);
    __syncthreads();
    if (tid == 0) {
      double s = 0.0;
      for (int c = 0; c < jb; ++c) s += invd[c];
      *logdet_part = 2.0 * s;
    }
    __syncthreads();
  }
  invert_lower_shared(a, invd, jb);
  for (int t = tid; t < kNB * kNB; t += blockDim.x) {
    int i = t % kNB, j = t / kNB;
    double v = 0.0;
    if (i < jb && j < jb && i >= j) v = (i == j) ? invd[i] : a[j][i];
    Linv[i + j * kNB] = v;
  }
}

__global__ void sum_logdet_kernel(const double *parts, int nparts, double *out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < nparts; ++i) s += parts[i];
    *out = s;
  }
}

__global__ void copy_lower_kernel(const double *src, int64_t lds, double *dst, int64_t ldd,
                                  int64_t n) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * n;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = t % n, j = t / n;
    if (i >= j) dst[i + j * ldd] = src[i + j * lds];
  }
}

__global__ void symmetrize_kernel(double *A, int64_t lda, int64_t n) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * n;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = t % n, j = t / n;
    if (i < j) A[i + j * lda] = A[j + i * lda];
  }
}

__global__ void copy_matrix_kernel(const double *src, int64_t lds, double *dst, int64_t ldd,
                                   int64_t rows, int64_t cols) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < rows * cols;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = t % rows, j = t / rows;
    dst[i + j * ldd] = src[i + j * lds];
  }
}

__global__ void add_matrix_kernel(const double *src, int64_t lds, double *dst, int64_t ldd,
                                  int64_t rows, int64_t cols) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < rows * cols;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = t % rows, j = t / rows;
    dst[i + j * ldd] += src[i + j * lds];
  }
}

// squared norm of each column, fixed-order tree reduction (deterministic)
__global__ void colnorm2_kernel(const double *X, int64_t ldx, int64_t rows, double *out) {
  const int64_t j = blockIdx.x;
  __shared__ double red[256];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < rows; i += blockDim.x) {
    double v = X[i + j * ldx];
    s = fma(v, v, s);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[j] = red[0];
}

__global__ void loglike_finish_kernel(const double *chi2, const double *logdet, int nmaps,
                                      double *lnL) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < nmaps) lnL[j] = -0.5 * (chi2[j] + *logdet);
}

__global__ void set_identity_kernel(double *X, int64_t ld, int64_t n) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ld * ld;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = t % ld, j = t / ld;
    X[t] = (i == j && i < n) ? 1.0 : 0.0;
  }
}

int grid_for(int64_t total) {
  int64_t b = (total + 255) / 256;
  if (b > 152 * 32) b = 152 * 32;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

void launch_dgemm(int ta, int tb, int64_t M, int64_t N, int64_t K, double alpha,
                  const double *A, int64_t lda, const double *B, int64_t ldb, double beta,
                  double *C, int64_t ldc, int lower, const DevStatus *status, cudaStream_t st) {
  if (M <= 0 || N <= 0) return;
  dim3 grid((unsigned)((M + BM - 1) / BM), (unsigned)((N + BN - 1) / BN));
  if (!ta && !tb)
    { dgemm_kernel<false, false><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, lower, status); count_launch(); }
  else if (!ta && tb)
    { dgemm_kernel<false, true><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, lower, status); count_launch(); }
  else if (ta && !tb)
    { dgemm_kernel<true, false><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, lower, status); count_launch(); }
  else
    { dgemm_kernel<true, true><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, lower, status); count_launch(); }
}

void launch_potrf_diag(double *A, int64_t lda, int64_t n, int64_t j0, double *Linv,
                       double *logdet_part, DevStatus *status, cudaStream_t st) {
  { potrf_diag_kernel<<<1, 256, 0, st>>>(A, lda, n, j0, Linv, logdet_part, status, 1); count_launch(); }
}

void launch_trtri_blocks(const double *L, int64_t lda, int64_t n, double *Linv,
                         DevStatus *status, cudaStream_t st) {
  const int nb = (int)((n + kNB - 1) / kNB);
  { potrf_diag_kernel<<<nb, 256, 0, st>>>(const_cast<double *>(L), lda, n, 0, Linv, nullptr,
                                        status, 0); count_launch(); }
}

void launch_sum_logdet(const double *parts, int nparts, double *out, cudaStream_t st) {
  { sum_logdet_kernel<<<1, 32, 0, st>>>(parts, nparts, out); count_launch(); }
}

void launch_copy_lower(const double *src, int64_t lds, double *dst, int64_t ldd, int64_t n,
                       cudaStream_t st) {
  { copy_lower_kernel<<<grid_for(n * n), 256, 0, st>>>(src, lds, dst, ldd, n); count_launch(); }
}

void launch_symmetrize_lower(double *A, int64_t lda, int64_t n, cudaStream_t st) {
  { symmetrize_kernel<<<grid_for(n * n), 256, 0, st>>>(A, lda, n); count_launch(); }
}

void launch_copy_matrix(const double *src, int64_t lds, double *dst, int64_t ldd, int64_t rows,
                        int64_t cols, cudaStream_t st) {
  { copy_matrix_kernel<<<grid_for(rows * cols), 256, 0, st>>>(src, lds, dst, ldd, rows, cols); count_launch(); }
}

void launch_add_matrix(const double *src, int64_t lds, double *dst, int64_t ldd, int64_t rows,
                       int64_t cols, cudaStream_t st) {
  { add_matrix_kernel<<<grid_for(rows * cols), 256, 0, st>>>(src, lds, dst, ldd, rows, cols); count_launch(); }
}

void launch_colnorm2(const double *X, int64_t ldx, int64_t rows, int64_t cols, double *out,
                     cudaStream_t st) {
  if (cols > 0) { colnorm2_kernel<<<(unsigned)cols, 256, 0, st>>>(X, ldx, rows, out); count_launch(); }
}

void launch_loglike_finish(const double *chi2, const double *logdet, int nmaps, double *lnL,
                           cudaStream_t st) {
  { loglike_finish_kernel<<<(nmaps + 127) / 128, 128, 0, st>>>(chi2, logdet, nmaps, lnL); count_launch(); }
}

void launch_set_identity(double *X, int64_t ld, int64_t n, cudaStream_t st) {
  { set_identity_kernel<<<grid_for(ld * ld), 256, 0, st>>>(X, ld, n); count_launch(); }
}

}  // namespace qmlgb
