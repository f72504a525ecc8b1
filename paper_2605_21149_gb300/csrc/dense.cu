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
#include "dfloat.cuh"
#include "ptx.cuh"

#include <math.h>

#include <string>

namespace qmlgb {

namespace {

constexpr int BK = 16;

// strided batch of products: blockIdx.z selects A + z sA, B + z sB, C + z sC
struct DgBatch {
  int count;
  int64_t sA, sB, sC;
};

// RM x RN outputs per thread: a (16 RM) x (16 RN) tile per CTA.  Small
// products take small tiles so that the grid still covers the SMs: with a
// float64 pipe this narrow the per-SM rate, not the operand traffic, sets
// the time, so spreading the work over more SMs is what pays.
template <bool TA, bool TB, int RM, int RN>
__global__ void __launch_bounds__(256) dgemm_kernel(int64_t M, int64_t N, int64_t K, double alpha,
                                                    const double *A, int64_t lda, const double *B,
                                                    int64_t ldb, double beta, double *C,
                                                    int64_t ldc, int lower,
                                                    const DevStatus *status, DgBatch bt) {
  constexpr int BM = 16 * RM, BN = 16 * RN;
  A += (int64_t)blockIdx.z * bt.sA;
  B += (int64_t)blockIdx.z * bt.sB;
  C += (int64_t)blockIdx.z * bt.sC;
  if (status && *((volatile const int *)&status->code) != 0) return;
  const int64_t m0 = (int64_t)blockIdx.x * BM;
  const int64_t n0 = (int64_t)blockIdx.y * BN;
  if (lower && m0 + BM - 1 < n0) return;  // tile strictly above the diagonal
  __shared__ double As[2][BK][BM + 1];
  __shared__ double Bs[2][BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  double acc[RM][RN];
#pragma unroll
  for (int i = 0; i < RM; ++i)
#pragma unroll
    for (int j = 0; j < RN; ++j) acc[i][j] = 0.0;

  // tile element r of this thread: (mm, kk) of the BK x BM slab of op(A)
  auto a_at = [&](int r, int &mm, int &kk) {
    if (!TA) { mm = tid % BM; kk = tid / BM + (256 / BM) * r; }
    else { kk = tid & 15; mm = (tid >> 4) + 16 * r; }
  };
  auto b_at = [&](int r, int &nn, int &kk) {
    if (!TB) { kk = tid & 15; nn = (tid >> 4) + 16 * r; }
    else { nn = tid % BN; kk = tid / BN + (256 / BN) * r; }
  };
  double ra[RM], rb[RN];
  auto load_a = [&](int64_t k0) {
#pragma unroll
    for (int r = 0; r < RM; ++r) {
      int mm, kk;
      a_at(r, mm, kk);
      int64_t gm = m0 + mm, gk = k0 + kk;
      double v = 0.0;
      if (gm < M && gk < K) v = TA ? A[gk + gm * lda] : A[gm + gk * lda];
      ra[r] = v;
    }
  };
  auto store_a = [&](int buf) {
#pragma unroll
    for (int r = 0; r < RM; ++r) {
      int mm, kk;
      a_at(r, mm, kk);
      As[buf][kk][mm] = ra[r];
    }
  };
  auto load_b = [&](int64_t k0) {
#pragma unroll
    for (int r = 0; r < RN; ++r) {
      int nn, kk;
      b_at(r, nn, kk);
      int64_t gn = n0 + nn, gk = k0 + kk;
      double v = 0.0;
      if (gn < N && gk < K) v = TB ? B[gn + gk * ldb] : B[gk + gn * ldb];
      rb[r] = v;
    }
  };
  auto store_b = [&](int buf) {
#pragma unroll
    for (int r = 0; r < RN; ++r) {
      int nn, kk;
      b_at(r, nn, kk);
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
      double a[RM], b[RN];
#pragma unroll
      for (int i = 0; i < RM; ++i) a[i] = As[buf][kk][tx + 16 * i];
#pragma unroll
      for (int j = 0; j < RN; ++j) b[j] = Bs[buf][kk][ty + 16 * j];
#pragma unroll
      for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < RN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    if (t + 1 < nk) {
      store_a(buf ^ 1);
      store_b(buf ^ 1);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < RM; ++i) {
    const int64_t gm = m0 + tx + 16 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < RN; ++j) {
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
// One CTA (256 threads, 8 warps) factors a jb x jb (jb <= 64) diagonal block
// in shared memory and inverts the lower factor.  On this part a float64
// operation that depends on the previous one waits tens of clocks and one
// SM retires under two float64 lanes per clock, so the kernel is built
// around short dependency chains: panels of kPW = 8 columns factored by one
// warp in registers (pivots and column entries travel by shuffle), rank-8
// trailing updates and the blocked inverse with independent partial sums.
//
// Dynamic shared memory: the tile a (factor L in its lower triangle), the
// dense inverse x (zeros above the diagonal), 1 / L_cc, a scratch block;
// row stride kLDA = 65 doubles keeps column reads free of bank conflicts.
constexpr int kLDA = kNB + 1;
constexpr int kPW = 8;
constexpr size_t kDiagSmem =
    (size_t)(2 * kNB * kLDA + kNB + (kNB / kPW - 1) * kPW * kPW) * sizeof(double) + 16;

// Inverse X = L^-1 into x (invd holds 1 / L_cc; x zeroed by the caller):
//  1. warp I inverts the 8 x 8 diagonal block I by forward substitution
//     (lane c < 8 owns column c);
//  2. block rows I = 1 .. 7 in turn: T_IJ = sum_{J <= K < I} L_IK X_KJ for all
//     J < I (four interleaved partial sums), then X_IJ = -D_I T_IJ (X_IJ needs
//     only block rows above I, so one step per block row).
__device__ void invert_lower_blocked(double (*a)[kLDA], double (*x)[kLDA], const double *invd,
                                     int jb, double *tmp /* >= 7 * 64 doubles */) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nbk = (jb + kPW - 1) / kPW;
  if (warp < nbk && lane < kPW) {
    const int b0 = warp * kPW, col = b0 + lane;
    const int bend = (b0 + kPW < jb) ? b0 + kPW : jb;
    if (col < bend) {
      x[col][col] = invd[col];
      for (int r = col + 1; r < bend; ++r) {
        double s0 = 0.0, s1 = 0.0;
        int k = col;
        for (; k + 1 < r; k += 2) {
          s0 = fma(a[r][k], x[k][col], s0);
          s1 = fma(a[r][k + 1], x[k + 1][col], s1);
        }
        if (k < r) s0 = fma(a[r][k], x[k][col], s0);
        x[r][col] = -(s0 + s1) * invd[r];
      }
    }
  }
  __syncthreads();
  for (int I = 1; I < nbk; ++I) {
    const int rI = I * kPW, rend = (rI + kPW < jb) ? rI + kPW : jb;
    for (int t = tid; t < I * kPW * kPW; t += blockDim.x) {
      const int J = t / (kPW * kPW), r = (t / kPW) % kPW, c = t % kPW;
      const int row = rI + r, xc = J * kPW + c;
      double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
      if (row < rend)
        for (int k = J * kPW; k < rI; k += 4) {  // rI - J kPW is a multiple of 4
          s0 = fma(a[row][k], x[k][xc], s0);
          s1 = fma(a[row][k + 1], x[k + 1][xc], s1);
          s2 = fma(a[row][k + 2], x[k + 2][xc], s2);
          s3 = fma(a[row][k + 3], x[k + 3][xc], s3);
        }
      tmp[t] = (s0 + s1) + (s2 + s3);
    }
    __syncthreads();
    for (int t = tid; t < I * kPW * kPW; t += blockDim.x) {
      const int J = t / (kPW * kPW), r = (t / kPW) % kPW, c = t % kPW;
      const int row = rI + r;
      if (row < rend) {
        double s0 = 0.0, s1 = 0.0;
        int q = 0;
        for (; q + 1 <= r; q += 2) {
          s0 = fma(x[row][rI + q], tmp[J * kPW * kPW + q * kPW + c], s0);
          s1 = fma(x[row][rI + q + 1], tmp[J * kPW * kPW + (q + 1) * kPW + c], s1);
        }
        if (q <= r) s0 = fma(x[row][rI + q], tmp[J * kPW * kPW + q * kPW + c], s0);
        x[row][J * kPW + c] = -(s0 + s1);
      }
    }
    __syncthreads();
  }
}

// mode 1: factor and invert; mode 2: factor only, and Linv receives the
// scaled coefficients of the row solve x L^T = b (trsm_rows_kernel) instead of
// an inverse, Linv[c kNB + j] = L_jc / L_jj (j > c), 1 / L_cc (j = c), 0
// otherwise; mode 0: the block already holds L and only the inverse is formed
// (blockIdx.x selects the block: j0 = blockIdx.x * kNB);
// mode 3: as mode 0, but the factor comes from the float-float slot that
// potrf_diag_df_kernel left at Linv (packed L~ and the row exponents k_i,
// L_ij = L~_ij 2^k_i): it is written into A (lower triangle), 2 sum ln L_ii
// goes to logdet_part[blockIdx.x], and the inverse replaces the slot.
__global__ void __launch_bounds__(256, 1) potrf_diag_kernel(double *A, int64_t lda, int64_t n,
                                                         int64_t j0, double *Linv,
                                                         double *logdet_part,
                                                         DevStatus *status, int mode) {
  const int factor = mode == 1 || mode == 2;
  extern __shared__ __align__(16) double dsm[];
  double(*a)[kLDA] = (double(*)[kLDA])dsm;
  double(*x)[kLDA] = (double(*)[kLDA])(dsm + kNB * kLDA);
  double *invd = dsm + 2 * kNB * kLDA;
  double *tmp = invd + kNB;
  int *bad = (int *)(tmp + (kNB / kPW - 1) * kPW * kPW);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (status && *((volatile int *)&status->code) != 0) return;
  if (!factor) {
    j0 = (int64_t)blockIdx.x * kNB;
    A += j0 + j0 * lda;
    Linv += (int64_t)blockIdx.x * kNB * kNB;
  }
  const int jb = (int)((n - j0) < kNB ? (n - j0) : kNB);
  if (mode == 3) {
    const float2 *slot = (const float2 *)Linv;
    const int *kx = (const int *)(slot + packed_off(kNB, kNB));
    for (int t = tid; t < kNB * kNB; t += blockDim.x) {
      const int i = t % kNB, j = t / kNB;
      double v = 0.0;
      if (i >= j && i < jb && j < jb) {
        const float2 f = slot[packed_off(j, kNB) + (i - j)];
        v = df_to_double({f.x, f.y}, kx[i]);
        A[i + j * lda] = v;
      }
      a[i][j] = v;
      x[i][j] = 0.0;
    }
    __syncthreads();
    // log det part: one log per thread of warps 0 and 1, fixed-order sums
    if (warp < 2) {
      double sl = tid < jb ? log(a[tid][tid]) : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sl += __shfl_xor_sync(0xffffffffu, sl, o);
      if (lane == 0) tmp[warp] = sl;
    }
    __syncthreads();
    if (tid == 0) logdet_part[blockIdx.x] = 2.0 * (tmp[0] + tmp[1]);
    if (tid < jb) invd[tid] = 1.0 / a[tid][tid];
    __syncthreads();
    invert_lower_blocked(a, x, invd, jb, tmp);
    for (int t = tid; t < kNB * kNB; t += blockDim.x) {
      int i = t % kNB, j = t / kNB;
      Linv[i + j * kNB] = (i < jb && j < jb) ? x[i][j] : 0.0;
    }
    return;
  }
  // the tile's loads in two batches of 8 per thread, each batch in flight together
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int t = tid + 256 * (8 * h + u), i = t % kNB, j = t / kNB;
      v[u] = (i < jb && j < jb && i >= j) ? A[i + j * lda] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int t = tid + 256 * (8 * h + u), i = t % kNB, j = t / kNB;
      a[i][j] = v[u];
      x[i][j] = 0.0;
    }
  }
  if (tid == 0) *bad = 0;
  __syncthreads();
  if (factor) {
    // Warps 0-2 each factor the panel's 8 x 8 pivot block in lanes 0-7 (the
    // same operations on the same values, so identical results) and carry 24
    // rows of their own below it in lanes 8-31: one row per lane, and the
    // panel's float64 instructions spread over three SM sub-partitions (a
    // float64 warp instruction holds its sub-partition for ~76 clocks).
    // Lane-dependent conditions are selects, so each step is one basic block.
    for (int c0 = 0; c0 < jb; c0 += kPW) {
      const int cend = (c0 + kPW < jb) ? c0 + kPW : jb;
      if (warp == 0 || (warp < 3 && c0 + kPW + 24 * warp < jb)) {
        const int row = lane < kPW ? c0 + lane : c0 + kPW + 24 * warp + (lane - kPW);
        const bool live = row < jb;
        double v[kPW];
#pragma unroll
        for (int q = 0; q < kPW; ++q) v[q] = (c0 + q < cend && live) ? a[row][c0 + q] : 0.0;
        int fail_col = -1;
#pragma unroll
        for (int q = 0; q < kPW; ++q) {
          const int c = c0 + q;
          if (c < cend && fail_col < 0) {
            const double d = __shfl_sync(0xffffffffu, v[q], q);  // a_cc: lane q holds row c
            const double r = rsqrt(d);
            if (!(r > 0.0) || !isfinite(r)) {  // a_cc <= 0, infinite or NaN
              fail_col = c;
            } else {
              // row c: L_cc = a_cc r; rows below: l_ic = a_ic r
              const double sc = (row == c ? d : v[q]) * r;
              v[q] = row >= c ? sc : v[q];
              if (warp == 0 && lane == 0) invd[c] = r;
              double lj[kPW];
#pragma unroll
              for (int qj = q + 1; qj < kPW; ++qj) lj[qj] = __shfl_sync(0xffffffffu, v[q], qj);
#pragma unroll
              for (int qj = q + 1; qj < kPW; ++qj) {
                const double nv = fma(-v[q], lj[qj], v[qj]);
                v[qj] = row >= c0 + qj ? nv : v[qj];
              }
            }
          }
        }
        if (fail_col >= 0) {
          if (warp == 0 && lane == 0) {
            *bad = 1;
            // the first error of the call is the one reported
            if (atomicCAS(&status->code, 0, 2 /* QML_ENOTSPD */) == 0)
              status->info = (int)(j0 + fail_col + 1);
          }
        } else if (live && (warp == 0 || lane >= kPW)) {
#pragma unroll
          for (int q = 0; q < kPW; ++q)
            if (c0 + q < cend && row >= c0 + q) a[row][c0 + q] = v[q];
        }
      }
      __syncthreads();
      if (*bad) return;
      // rank-(cend - c0) update of the trailing triangle cend <= j <= i < jb,
      // two elements per pass, each with two partial sums (a full panel takes
      // the branch-free form)
      const int m = jb - cend;
      const int T = m * (m + 1) / 2;
      const bool full = cend - c0 == kPW;
      for (int t = tid; t < T; t += 2 * blockDim.x) {
        int ii[2], jj[2];
        bool on[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int tu = t + u * (int)blockDim.x;
          on[u] = tu < T;
          int r = (int)((sqrtf(8.0f * tu + 1.0f) - 1.0f) * 0.5f);
          while ((r + 1) * (r + 2) / 2 <= tu) ++r;
          while (r * (r + 1) / 2 > tu) --r;
          ii[u] = cend + r;
          jj[u] = cend + (tu - r * (r + 1) / 2);
          if (!on[u]) ii[u] = jj[u] = cend;  // harmless in-range indices
        }
        double v[2], w[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          v[u] = a[ii[u]][jj[u]];
          w[u] = 0.0;
        }
        if (full) {
#pragma unroll
          for (int q = 0; q < kPW; q += 2) {
#pragma unroll
            for (int u = 0; u < 2; ++u) {
              v[u] = fma(-a[ii[u]][c0 + q], a[jj[u]][c0 + q], v[u]);
              w[u] = fma(-a[ii[u]][c0 + q + 1], a[jj[u]][c0 + q + 1], w[u]);
            }
          }
        } else {
          for (int q = 0; q < cend - c0; ++q) {
#pragma unroll
            for (int u = 0; u < 2; ++u) v[u] = fma(-a[ii[u]][c0 + q], a[jj[u]][c0 + q], v[u]);
          }
        }
#pragma unroll
        for (int u = 0; u < 2; ++u)
          if (on[u]) a[ii[u]][jj[u]] = v[u] + w[u];
      }
      __syncthreads();
    }
    for (int t = tid; t < jb * jb; t += blockDim.x) {
      int i = t % jb, j = t / jb;
      if (i >= j) A[i + j * lda] = a[i][j];
    }
    // log det part: logs in parallel, a fixed-order shuffle tree over them
    if (warp == 0) {
      double s = (lane < jb ? log(a[lane][lane]) : 0.0) +
                 (lane + 32 < jb ? log(a[lane + 32][lane + 32]) : 0.0);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) *logdet_part = 2.0 * s;
    }
    if (mode == 2) {
      for (int t = tid; t < kNB * kNB; t += blockDim.x) {
        const int j = t % kNB, c = t / kNB;
        double v = 0.0;
        if (j < jb && c < jb) v = j > c ? a[j][c] * invd[j] : (j == c ? invd[c] : 0.0);
        Linv[t] = v;
      }
      return;
    }
  } else {
    if (tid < jb) invd[tid] = 1.0 / a[tid][tid];
    __syncthreads();
  }
  invert_lower_blocked(a, x, invd, jb, tmp);
  for (int t = tid; t < kNB * kNB; t += blockDim.x) {
    int i = t % kNB, j = t / kNB;
    Linv[i + j * kNB] = (i < jb && j < jb) ? x[i][j] : 0.0;
  }
}

// X = B L^-T for the m x ib rows B (ld ldb) and a lower-triangular ib x ib
// block L, i.e. each row solves x L^T = b by forward substitution,
//   x_c = b_c / L_cc - sum_{k<c} (L_ck / L_cc) x_k,
// from the scaled coefficients S (kNB x kNB, S[k kNB + c] = L_ck / L_cc for
// c > k, S[c kNB + c] = 1 / L_cc: mode 2 of potrf_diag_kernel).  One warp per
// CTA, two rows per warp, 16 lanes per row: lane g keeps columns g, g + 16,
// g + 32, g + 48 in registers, x_c reaches the row's other lanes by shuffle and
// every later column takes one fma per step (the current column by a select).
// S comes into shared memory by one bulk copy (bounded wait).  X goes to B (in
// place) and to T (ld ldt).
constexpr int kTrsmRows = 2;
__global__ void __launch_bounds__(32) trsm_rows_kernel(const double *S, int ib, double *B,
                                                       int64_t ldb, int64_t m, double *T,
                                                       int64_t ldt, DevStatus *status) {
  __shared__ __align__(128) double s[kNB * kNB];
  __shared__ __align__(8) uint64_t bar;
  if (*((volatile int *)&status->code) != 0) return;
  const int lane = threadIdx.x, g = lane & 15;
  const int64_t row = (int64_t)blockIdx.x * kTrsmRows + (lane >> 4);
  const bool on = row < m;
  const uint32_t b = smem_u32(&bar);
  if (lane == 0) {
    mbar_init(b, 1);
    fence_mbar_init();
    mbar_expect_tx(b, (uint32_t)sizeof(s));
    bulk_load(smem_u32(s), S, (uint32_t)sizeof(s), b);
  }
  double v[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int col = g + 16 * q;
    v[q] = (on && col < ib) ? B[row + (int64_t)col * ldb] : 0.0;
  }
  __syncwarp();
  if (!mbar_wait(b, 0, status)) {
    mbar_drain_wait(b, 0);
    return;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) v[q] *= s[(g + 16 * q) * (kNB + 1)];
#pragma unroll
  for (int qc = 0; qc < 4; ++qc) {
#pragma unroll
    for (int g0 = 0; g0 < 16; ++g0) {
      const int c = 16 * qc + g0;
      const double xc = __shfl_sync(0xffffffffu, v[qc], g0, 16);
      const double nv = fma(-s[c * kNB + g + 16 * qc], xc, v[qc]);
      v[qc] = g > g0 ? nv : v[qc];
#pragma unroll
      for (int q = qc + 1; q < 4; ++q) v[q] = fma(-s[c * kNB + g + 16 * q], xc, v[q]);
    }
  }
  if (on) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int col = g + 16 * q;
      if (col < ib) {
        B[row + (int64_t)col * ldb] = v[q];
        T[row + (int64_t)col * ldt] = v[q];
      }
    }
  }
}

// Float-float factor of one diagonal block of the split-precision Cholesky
// (rows and columns j0 .. j0 + jb - 1 of A, lower triangle; A is only read).
// The block is scaled symmetrically by powers of two, a~_ij = a_ij
// 2^-(k_i + k_j) with k_i = floor(e_i / 2) for the binary exponent e_i of a_ii
// (so a~_ii lies in [1, 4) and every float-float entry stays far from the
// float range limits), then factored right-looking as in potrf_diag_kernel:
// eight-column panels in warps 0-2 (each with the pivot block in lanes 0-7,
// column entries by shuffle), rank-8 updates of the trailing triangle by all
// threads.  Two outputs of
// kSlot float2 each (packed lower triangle, then the 64 exponents as int):
//   Lslot: L~, with L_ij = L~_ij 2^k_i (mode 3 of potrf_diag_kernel turns it
//          into float64 L, the log det part and the inverse);
//   Sout:  the coefficients of the row solve x L^T = b (trsm_rows_df_kernel),
//          S(j, c) = L~_jc / L~_jj for j > c and S(c, c) = 1 / L~_cc.
// A pivot that is not positive and finite sets QML_ENOTSPD with its column.
constexpr int kSlot = packed_off(kNB, kNB) + kNB / 2;
__global__ void __launch_bounds__(256, 1) potrf_diag_df_kernel(const double *A, int64_t lda,
                                                                int64_t n, int64_t j0,
                                                                float2 *Lslot, float2 *Sout,
                                                                DevStatus *status) {
  __shared__ dfl a[kNB][kNB + 1];
  __shared__ dfl rd[kNB];
  __shared__ int kx[kNB];
  __shared__ int bad;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (*((volatile int *)&status->code) != 0) return;
  const int jb = (int)((n - j0) < kNB ? (n - j0) : kNB);
  constexpr int kPer = kNB * kNB / 256;
  double raw[kPer];  // all loads of the tile in flight together
#pragma unroll
  for (int u = 0; u < kPer; ++u) {
    const int t = tid + 256 * u, i = t % kNB, j = t / kNB;
    raw[u] = (i < jb && j < jb && i >= j) ? A[i + j * lda] : 0.0;
  }
#pragma unroll
  for (int u = 0; u < kPer; ++u) {
    const int t = tid + 256 * u, i = t % kNB, j = t / kNB;
    if (i == j) {
      const int E = (int)(((unsigned)__double2hiint(raw[u]) >> 20) & 0x7FFu);
      kx[i] = (E == 0 || E == 0x7FF) ? 0 : ((E - 1023) >> 1);
    }
  }
  if (tid == 0) bad = 0;
  __syncthreads();
#pragma unroll
  for (int u = 0; u < kPer; ++u) {
    const int t = tid + 256 * u, i = t % kNB, j = t / kNB;
    a[i][j] = df_from_double(raw[u], kx[i] + kx[j]);
  }
  __syncthreads();
  // Lane-dependent conditions below are selects, not branches, so that the
  // independent float-float chains of a step stay in one basic block and
  // interleave (each step is a dependent chain of 4-cycle float32 operations).
  for (int c0 = 0; c0 < jb; c0 += kPW) {
    const int cend = (c0 + kPW < jb) ? c0 + kPW : jb;
    // Warps 0-2 each factor the panel's 8 x 8 pivot block in lanes 0-7 (the
    // same operations on the same values, so identical results) and carry 24
    // rows of their own below it in lanes 8-31: no exchange between warps,
    // one row per lane.  dg is every lane's copy of the pivot block's diagonal,
    // updated by the same operations as its owner's entry, so a pivot needs
    // no shuffle.
    if (warp == 0 || (warp < 3 && c0 + kPW + 24 * warp < jb)) {
      const int row = lane < kPW ? c0 + lane : c0 + kPW + 24 * warp + (lane - kPW);
      const bool live = row < jb;
      dfl v[kPW], dg[kPW];
#pragma unroll
      for (int q = 0; q < kPW; ++q) {
        v[q] = (c0 + q < cend && live) ? a[row][c0 + q] : dfl{0.0f, 0.0f};
        dg[q] = c0 + q < cend ? a[c0 + q][c0 + q] : dfl{0.0f, 0.0f};
      }
      int fail_col = -1;
#pragma unroll
      for (int q = 0; q < kPW; ++q) {
        const int c = c0 + q;
        if (c < cend && fail_col < 0) {
          const dfl d = dg[q];
          if (!(d.h > 0.0f) || !isfinite(d.h)) {  // a_cc <= 0, infinite or NaN
            fail_col = c;
          } else {
            const dfl r = df_rsqrt(d);
            const dfl s0 = df_mul(v[q], r), lcc = df_mul(d, r);
            v[q] = row > c ? s0 : (row == c ? lcc : v[q]);
            if (warp == 0 && lane == 0) rd[c] = r;
            dfl lj[kPW];
#pragma unroll
            for (int qj = q + 1; qj < kPW; ++qj)  // l(c0 + qj, c): lane qj of every warp
              lj[qj] = {__shfl_sync(0xffffffffu, v[q].h, qj), __shfl_sync(0xffffffffu, v[q].l, qj)};
#pragma unroll
            for (int qj = q + 1; qj < kPW; ++qj) {
              const dfl n = df_fms(v[qj], v[q], lj[qj]);
              v[qj] = row >= c0 + qj ? n : v[qj];
              dg[qj] = df_fms(dg[qj], lj[qj], lj[qj]);
            }
          }
        }
      }
      if (fail_col >= 0) {
        if (warp == 0 && lane == 0) {
          bad = 1;
          // the first error of the call is the one reported
          if (atomicCAS(&status->code, 0, 2 /* QML_ENOTSPD */) == 0)
            status->info = (int)(j0 + fail_col + 1);
        }
      } else if (live && (warp == 0 || lane >= kPW)) {
#pragma unroll
        for (int q = 0; q < kPW; ++q)
          if (c0 + q < cend && row >= c0 + q) a[row][c0 + q] = v[q];
      }
    }
    __syncthreads();
    if (bad) return;
    // rank-(cend - c0) update of the trailing triangle cend <= j <= i < jb,
    // two elements per pass, each with two partial sums (a full panel takes
    // the branch-free form)
    const int m = jb - cend;
    const int T = m * (m + 1) / 2;
    const bool full = cend - c0 == kPW;
    for (int t = tid; t < T; t += 2 * blockDim.x) {
      int ii[2], jj[2];
      bool on[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int tu = t + u * (int)blockDim.x;
        on[u] = tu < T;
        int r = (int)((sqrtf(8.0f * tu + 1.0f) - 1.0f) * 0.5f);
        while ((r + 1) * (r + 2) / 2 <= tu) ++r;
        while (r * (r + 1) / 2 > tu) --r;
        ii[u] = cend + r;
        jj[u] = cend + (tu - r * (r + 1) / 2);
        if (!on[u]) ii[u] = jj[u] = cend;  // harmless in-range indices
      }
      dfl v[2], w[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        v[u] = a[ii[u]][jj[u]];
        w[u] = dfl{0.0f, 0.0f};
      }
      if (full) {
#pragma unroll
        for (int q = 0; q < kPW; q += 2) {
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            v[u] = df_fms(v[u], a[ii[u]][c0 + q], a[jj[u]][c0 + q]);
            w[u] = df_fms(w[u], a[ii[u]][c0 + q + 1], a[jj[u]][c0 + q + 1]);
          }
        }
      } else {
        for (int q = 0; q < cend - c0; ++q) {
#pragma unroll
          for (int u = 0; u < 2; ++u) v[u] = df_fms(v[u], a[ii[u]][c0 + q], a[jj[u]][c0 + q]);
        }
      }
#pragma unroll
      for (int u = 0; u < 2; ++u)
        if (on[u]) a[ii[u]][jj[u]] = df_add(v[u], w[u]);
    }
    __syncthreads();
  }
#pragma unroll 4
  for (int t = tid; t < kNB * kNB; t += blockDim.x) {
    const int j = t % kNB, c = t / kNB;
    const bool in = j < jb;
    const dfl l = in ? a[j][c] : dfl{0.0f, 0.0f};
    const dfl sm = df_mul(l, rd[j]);
    const dfl sc = !in ? dfl{0.0f, 0.0f} : (j == c ? rd[c] : sm);
    if (j >= c) {
      const int p = packed_off(c, kNB) + (j - c);
      Lslot[p] = make_float2(l.h, l.l);
      Sout[p] = make_float2(sc.h, sc.l);
    }
  }
  if (tid < kNB) {
    ((int *)(Lslot + packed_off(kNB, kNB)))[tid] = kx[tid];
    ((int *)(Sout + packed_off(kNB, kNB)))[tid] = kx[tid];
  }
}

// X = B L^-T for the m x ib rows B (ld ldb) and the diagonal block factored
// by potrf_diag_df_kernel: each row solves sum_k L~_ck x_k = b_c 2^-k_c by
// forward substitution in float-float,
//   x_c = b_c 2^-k_c / L~_cc - sum_{k<c} (L~_ck / L~_cc) x_k,
// from its coefficients S (kSlot float2, brought into shared memory by one
// bulk copy with a bounded wait).  One warp per CTA, two rows per warp, 16
// lanes per row: lane g keeps columns g, g + 16, g + 32, g + 48, x_c reaches
// the row's other lanes by shuffle and every later column takes one
// float-float multiply-subtract per step.  X (float64) goes to B (in place)
// and to T (ld ldt).
__global__ void __launch_bounds__(32) trsm_rows_df_kernel(const float2 *S, int ib, double *B,
                                                          int64_t ldb, int64_t m, double *T,
                                                          int64_t ldt, DevStatus *status) {
  __shared__ __align__(128) float2 s[kSlot];
  __shared__ __align__(8) uint64_t bar;
  if (*((volatile int *)&status->code) != 0) return;
  const int lane = threadIdx.x, g = lane & 15;
  const int64_t row = (int64_t)blockIdx.x * kTrsmRows + (lane >> 4);
  const bool on = row < m;
  const uint32_t b = smem_u32(&bar);
  if (lane == 0) {
    mbar_init(b, 1);
    fence_mbar_init();
    mbar_expect_tx(b, (uint32_t)sizeof(s));
    bulk_load(smem_u32(s), S, (uint32_t)sizeof(s), b);
  }
  double raw[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int col = g + 16 * q;
    raw[q] = (on && col < ib) ? B[row + (int64_t)col * ldb] : 0.0;
  }
  __syncwarp();
  if (!mbar_wait(b, 0, status)) {
    mbar_drain_wait(b, 0);
    return;
  }
  const int *kx = (const int *)(s + packed_off(kNB, kNB));
  dfl v[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int col = g + 16 * q;
    const float2 r = s[packed_off(col, kNB)];
    v[q] = df_mul(df_from_double(raw[q], kx[col]), dfl{r.x, r.y});
  }
#pragma unroll
  for (int qc = 0; qc < 4; ++qc) {
#pragma unroll
    for (int g0 = 0; g0 < 16; ++g0) {
      const int c = 16 * qc + g0;
      const dfl xc = {__shfl_sync(0xffffffffu, v[qc].h, g0, 16),
                      __shfl_sync(0xffffffffu, v[qc].l, g0, 16)};
      // column qc of this lane is later than c only where g > g0 (a select);
      // columns q > qc always are
      {
        const float2 sc = s[packed_off(c, kNB) + (g + 16 * qc - c)];  // in range for g <= g0 too
        const dfl nv = df_fms(v[qc], dfl{sc.x, sc.y}, xc);
        v[qc] = g > g0 ? nv : v[qc];
      }
#pragma unroll
      for (int q = qc + 1; q < 4; ++q) {
        const float2 sc = s[packed_off(c, kNB) + (g + 16 * q - c)];
        v[q] = df_fms(v[q], dfl{sc.x, sc.y}, xc);
      }
    }
  }
  if (on) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int col = g + 16 * q;
      if (col < ib) {
        const double xv = df_to_double(v[q], 0);
        B[row + (int64_t)col * ldb] = xv;
        T[row + (int64_t)col * ldt] = xv;
      }
    }
  }
}

void set_diag_smem() {
  static bool done = false;
  if (!done) {
    cudaFuncSetAttribute(potrf_diag_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kDiagSmem);
    done = true;
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

int grid_for(int64_t total) {
  int64_t b = (total + 255) / 256;
  if (b > 152 * 32) b = 152 * 32;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

namespace {

// number of CTAs that do work for a bm x bn tiling
int64_t dgemm_ctas(int64_t M, int64_t N, int bm, int bn, int lower) {
  const int64_t gx = (M + bm - 1) / bm, gy = (N + bn - 1) / bn;
  if (!lower) return gx * gy;
  int64_t n = 0;
  for (int64_t y = 0; y < gy; ++y) {
    const int64_t first = (y * bn) / bm;  // first x with x*bm + bm - 1 >= y*bn
    n += gx - (first > gx ? gx : first);
  }
  return n;
}

template <bool TA, bool TB, int RM, int RN>
void dgemm_go(int64_t M, int64_t N, int64_t K, double alpha, const double *A, int64_t lda,
              const double *B, int64_t ldb, double beta, double *C, int64_t ldc, int lower,
              const DevStatus *status, cudaStream_t st, DgBatch bt) {
  dim3 grid((unsigned)((M + 16 * RM - 1) / (16 * RM)), (unsigned)((N + 16 * RN - 1) / (16 * RN)),
            (unsigned)bt.count);
  dgemm_kernel<TA, TB, RM, RN><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc,
                                                     lower, status, bt);
  count_launch();
}

template <bool TA, bool TB>
void dgemm_tile(int rm, int rn, int64_t M, int64_t N, int64_t K, double alpha, const double *A,
                int64_t lda, const double *B, int64_t ldb, double beta, double *C, int64_t ldc,
                int lower, const DevStatus *status, cudaStream_t st, DgBatch bt) {
#define QMLGB_DG(R1, R2)                                                                          \
  if (rm == R1 && rn == R2) {                                                                     \
    dgemm_go<TA, TB, R1, R2>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, lower, status, st, bt); \
    return;                                                                                       \
  }
  QMLGB_DG(4, 4) QMLGB_DG(2, 2) QMLGB_DG(1, 1) QMLGB_DG(1, 4) QMLGB_DG(2, 4) QMLGB_DG(4, 1)
  QMLGB_DG(4, 2)
#undef QMLGB_DG
  // any other pair: the full tile, which is safe for every aliasing
  dgemm_go<TA, TB, 4, 4>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, lower, status, st, bt);
}

void dgemm_dispatch(int ta, int tb, int rm, int rn, int64_t M, int64_t N, int64_t K,
                    double alpha, const double *A, int64_t lda, const double *B, int64_t ldb,
                    double beta, double *C, int64_t ldc, int lower, const DevStatus *status,
                    cudaStream_t st, DgBatch bt = DgBatch{1, 0, 0, 0}) {
  if (!ta && !tb) dgemm_tile<false, false>(rm, rn, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, lower, status, st, bt);
  else if (!ta && tb) dgemm_tile<false, true>(rm, rn, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, lower, status, st, bt);
  else if (ta && !tb) dgemm_tile<true, false>(rm, rn, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, lower, status, st, bt);
  else dgemm_tile<true, true>(rm, rn, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, lower, status, st, bt);
}

const int kCand[7][2] = {{4, 4}, {2, 4}, {4, 2}, {2, 2}, {1, 4}, {4, 1}, {1, 1}};

// Autotuner: time every candidate tile on this shape (output into a scratch
// matrix, beta = 0, so the caller's C is untouched) and keep the fastest.
// Every tile computes each output as the same in-order fused sum over k, so
// the choice changes the time, never the result.  Returns false (no entry)
// when the measurement could not be made.
bool dgemm_autotune(int ta, int tb, int64_t M, int64_t N, int64_t K, const double *A,
                    int64_t lda, const double *B, int64_t ldb, int lower,
                    const DevStatus *status, cudaStream_t st, int &rm, int &rn) {
  double *scratch = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  bool ok = cudaMalloc(&scratch, (size_t)M * N * sizeof(double)) == cudaSuccess &&
            cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
  float best = 0.0f;
  int found = -1;
  for (int i = 0; ok && i < 7; ++i) {
    const int r1 = kCand[i][0], r2 = kCand[i][1];
    dgemm_dispatch(ta, tb, r1, r2, M, N, K, 1.0, A, lda, B, ldb, 0.0, scratch, M, lower, status, st);
    cudaEventRecord(e0, st);
    for (int r = 0; r < 3; ++r)
      dgemm_dispatch(ta, tb, r1, r2, M, N, K, 1.0, A, lda, B, ldb, 0.0, scratch, M, lower, status,
                     st);
    cudaEventRecord(e1, st);
    float ms = 0.0f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      ok = false;
      break;
    }
    if (found < 0 || ms < best) {
      best = ms;
      found = i;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (scratch) cudaFree(scratch);
  if (!ok || found < 0) {
    cudaGetLastError();
    return false;
  }
  rm = kCand[found][0];
  rn = kCand[found][1];
  return true;
}

}  // namespace

// Tile choice: a measured entry of the tuning table for this shape (tuned
// on first use when allowed), else the largest tile whose grid still gives
// every SM two CTAs, else the smallest.  In-place products keep what makes
// them safe: C == A (C's rows read only by their own CTA) needs the whole of
// N in one tile, C == B the whole of M; callers only alias with N (resp. M)
// <= 64, and those shapes are never timed.
namespace {
void launch_dgemm_impl(int ta, int tb, int64_t M, int64_t N, int64_t K, double alpha,
                       const double *A, int64_t lda, const double *B, int64_t ldb, double beta,
                       double *C, int64_t ldc, int lower, const DevStatus *status,
                       cudaStream_t st, bool may_tune) {
  if (M <= 0 || N <= 0) return;
  const bool aliasA = (C == A), aliasB = (C == B);
  const std::string key = "dgemm:" + std::to_string(ta) + "," + std::to_string(tb) + "," +
                          std::to_string(lower) + "," + std::to_string(M) + "," +
                          std::to_string(N) + "," + std::to_string(K) + "," +
                          std::to_string((aliasA ? 1 : 0) + (aliasB ? 2 : 0));
  int64_t tv;
  bool known = false;
  if (tune_find(key, tv))
    for (int i = 0; i < 7; ++i)
      known |= (tv == 10 * kCand[i][0] + kCand[i][1]);
  if (known && !(aliasA && tv % 10 != 4) && !(aliasB && tv / 10 != 4)) {
    dgemm_dispatch(ta, tb, (int)(tv / 10), (int)(tv % 10), M, N, K, alpha, A, lda, B, ldb, beta,
                   C, ldc, lower, status, st);
    return;
  }
  if (may_tune && !aliasA && !aliasB && M * N <= (1 << 24) && K <= 4096 &&
      tune_get("dgemm_autotune", 1)) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone) {
      int rm = 4, rn = 4;
      if (dgemm_autotune(ta, tb, M, N, K, A, lda, B, ldb, lower, status, st, rm, rn)) {
        tune_put(key, 10 * rm + rn);
        dgemm_dispatch(ta, tb, rm, rn, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, lower, status,
                       st);
        return;
      }
    }
    cudaGetLastError();
  }
  const int64_t want = 2 * 152;
  int rm = 4, rn = 4;
  int64_t best = -1;
  for (int i = 0; i < 7; ++i) {
    const int r1 = kCand[i][0], r2 = kCand[i][1];
    if (aliasA && r2 != 4) continue;
    if (aliasB && r1 != 4) continue;
    const int64_t n = dgemm_ctas(M, N, 16 * r1, 16 * r2, lower);
    if (n >= want) {  // candidates run from the largest tile down
      rm = r1;
      rn = r2;
      best = n;
      break;
    }
    if (n > best) {
      best = n;
      rm = r1;
      rn = r2;
    }
  }
  dgemm_dispatch(ta, tb, rm, rn, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, lower, status, st);
}
}  // namespace

void launch_dgemm(int ta, int tb, int64_t M, int64_t N, int64_t K, double alpha,
                  const double *A, int64_t lda, const double *B, int64_t ldb, double beta,
                  double *C, int64_t ldc, int lower, const DevStatus *status, cudaStream_t st) {
  launch_dgemm_impl(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, lower, status, st, true);
}

void launch_dgemm_fixed(int ta, int tb, int64_t M, int64_t N, int64_t K, double alpha,
                        const double *A, int64_t lda, const double *B, int64_t ldb, double beta,
                        double *C, int64_t ldc, int lower, const DevStatus *status,
                        cudaStream_t st) {
  launch_dgemm_impl(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, lower, status, st, false);
}

// count products C_z <- alpha op(A_z) op(B_z) + beta C_z, X_z = X + z sX; the
// tile is the largest whose grid (over all products) gives every SM two CTAs
void launch_dgemm_batched(int ta, int tb, int64_t M, int64_t N, int64_t K, double alpha,
                          const double *A, int64_t lda, int64_t sA, const double *B,
                          int64_t ldb, int64_t sB, double beta, double *C, int64_t ldc,
                          int64_t sC, int count, const DevStatus *status, cudaStream_t st) {
  if (M <= 0 || N <= 0 || count <= 0) return;
  int rm = 1, rn = 1;
  for (int i = 0; i < 7; ++i) {
    if (dgemm_ctas(M, N, 16 * kCand[i][0], 16 * kCand[i][1], 0) * count >= 2 * 152) {
      rm = kCand[i][0];
      rn = kCand[i][1];
      break;
    }
  }
  dgemm_dispatch(ta, tb, rm, rn, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, 0, status, st,
                 DgBatch{count, sA, sB, sC});
}

void launch_potrf_diag(double *A, int64_t lda, int64_t n, int64_t j0, double *Linv,
                       double *logdet_part, DevStatus *status, cudaStream_t st) {
  set_diag_smem();
  { potrf_diag_kernel<<<1, 256, kDiagSmem, st>>>(A, lda, n, j0, Linv, logdet_part, status, 1); count_launch(); }
}

void launch_potrf_diag_factor(double *A, int64_t lda, int64_t n, int64_t j0, double *S,
                              double *logdet_part, DevStatus *status, cudaStream_t st) {
  set_diag_smem();
  { potrf_diag_kernel<<<1, 256, kDiagSmem, st>>>(A, lda, n, j0, S, logdet_part, status, 2); count_launch(); }
}

void launch_trsm_rows(const double *S, int64_t ib, double *B, int64_t ldb, int64_t m, double *T,
                      int64_t ldt, DevStatus *status, cudaStream_t st) {
  if (m <= 0 || ib <= 0) return;
  const unsigned grid = (unsigned)((m + kTrsmRows - 1) / kTrsmRows);
  { trsm_rows_kernel<<<grid, 32, 0, st>>>(S, (int)ib, B, ldb, m, T, ldt, status); count_launch(); }
}

void launch_potrf_diag_df(const double *A, int64_t lda, int64_t n, int64_t j0, double *Lslot,
                          double *S, DevStatus *status, cudaStream_t st) {
  { potrf_diag_df_kernel<<<1, 256, 0, st>>>(A, lda, n, j0, (float2 *)Lslot, (float2 *)S, status); count_launch(); }
}

void launch_trsm_rows_df(const double *S, int64_t ib, double *B, int64_t ldb, int64_t m,
                         double *T, int64_t ldt, DevStatus *status, cudaStream_t st) {
  if (m <= 0 || ib <= 0) return;
  const unsigned grid = (unsigned)((m + kTrsmRows - 1) / kTrsmRows);
  { trsm_rows_df_kernel<<<grid, 32, 0, st>>>((const float2 *)S, (int)ib, B, ldb, m, T, ldt, status); count_launch(); }
}

void launch_trtri_blocks_df(double *L, int64_t lda, int64_t n, double *Linv,
                            double *logdet_parts, DevStatus *status, cudaStream_t st) {
  const int nb = (int)((n + kNB - 1) / kNB);
  set_diag_smem();
  { potrf_diag_kernel<<<nb, 256, kDiagSmem, st>>>(L, lda, n, 0, Linv, logdet_parts, status, 3); count_launch(); }
}

void launch_trtri_blocks(const double *L, int64_t lda, int64_t n, double *Linv,
                         DevStatus *status, cudaStream_t st) {
  const int nb = (int)((n + kNB - 1) / kNB);
  set_diag_smem();
  { potrf_diag_kernel<<<nb, 256, kDiagSmem, st>>>(const_cast<double *>(L), lda, n, 0, Linv, nullptr,
                                        status, 0); count_launch(); }
}

void launch_sum_logdet(const double *parts, int nparts, double *out, cudaStream_t st) {
  { sum_logdet_kernel<<<1, 32, 0, st>>>(parts, nparts, out); count_launch(); }
}

namespace {
// A <- (A + A^T) / 2 (both triangles), one thread per strictly lower entry
__global__ void symmetrize_avg_kernel(double *A, int64_t lda, int64_t n) {
  const int64_t total = n * (n - 1) / 2;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    // t -> (i, j), i > j, row by row of the strict lower triangle
    int64_t i = (int64_t)((sqrt(8.0 * (double)t + 1.0) + 1.0) * 0.5);
    while (i * (i - 1) / 2 > t) --i;
    while ((i + 1) * i / 2 <= t) ++i;
    const int64_t j = t - i * (i - 1) / 2;
    const double v = 0.5 * (A[i + j * lda] + A[j + i * lda]);
    A[i + j * lda] = v;
    A[j + i * lda] = v;
  }
}
}  // namespace

void launch_symmetrize_avg(double *A, int64_t lda, int64_t n, cudaStream_t st) {
  if (n < 2) return;
  { symmetrize_avg_kernel<<<grid_for(n * (n - 1) / 2), 256, 0, st>>>(A, lda, n); count_launch(); }
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

// Native binning (Sect. 2.4): bin B of the binned index covers the per-l
// rows bstart[B] .. bstart[B] + bcount[B] - 1.
// dst (nab x ncols, ld nab) <- per-bin sums of the rows of src (na x ncols, ld na)
__global__ void bin_rows_kernel(const double *src, int na, int ncols, const int *bstart,
                                const int *bcount, int nab, double *dst) {
  const int64_t total = (int64_t)nab * ncols;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int B = (int)(t % nab);
    const int64_t j = t / nab;
    double s = 0.0;
    for (int u = 0; u < bcount[B]; ++u) s += src[bstart[B] + u + j * na];
    dst[B + j * nab] = s;
  }
}

// Fb (nab x nab) <- per-(bin, bin') block sums of the symmetric F (na x na);
// (B, B') and (B', B) add the same entries in the same order, so Fb is exactly
// symmetric
__global__ void bin_fisher_kernel(const double *F, int na, const int *bstart, const int *bcount,
                                  int nab, double *Fb) {
  const int64_t total = (int64_t)nab * nab;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int B = (int)(t % nab), B2 = (int)(t / nab);
    const int lo = B < B2 ? B : B2, hi = B < B2 ? B2 : B;
    double s = 0.0;
    for (int u = 0; u < bcount[hi]; ++u)
      for (int v = 0; v < bcount[lo]; ++v)
        s += F[(bstart[lo] + v) + (int64_t)(bstart[hi] + u) * na];
    Fb[t] = s;
  }
}

void launch_bin_rows(const double *src, int na, int ncols, const int *bstart, const int *bcount,
                     int nab, double *dst, cudaStream_t st) {
  if (nab <= 0 || ncols <= 0) return;
  { bin_rows_kernel<<<grid_for((int64_t)nab * ncols), 256, 0, st>>>(src, na, ncols, bstart, bcount, nab, dst); count_launch(); }
}

void launch_bin_fisher(const double *F, int na, const int *bstart, const int *bcount, int nab,
                       double *Fb, cudaStream_t st) {
  if (nab <= 0) return;
  { bin_fisher_kernel<<<grid_for((int64_t)nab * nab), 256, 0, st>>>(F, na, bstart, bcount, nab, Fb); count_launch(); }
}

// X (ld x ld, first n rows / columns used) <- block diagonal of the kNB x kNB
// inverses Dinv (consecutive blocks of kNB * kNB), zeros elsewhere
__global__ void place_diag_kernel(const double *Dinv, int64_t n, double *X, int64_t ld) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ld * ld;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t % ld, c = t / ld;
    double v = 0.0;
    if (r < n && c < n && r / kNB == c / kNB)
      v = Dinv[(r / kNB) * kNB * kNB + (r % kNB) + (c % kNB) * kNB];
    X[t] = v;
  }
}

void launch_place_diag_inverses(const double *Dinv, int64_t n, double *X, int64_t ld,
                                cudaStream_t st) {
  { place_diag_kernel<<<grid_for(ld * ld), 256, 0, st>>>(Dinv, n, X, ld); count_launch(); }
}

}  // namespace qmlgb
