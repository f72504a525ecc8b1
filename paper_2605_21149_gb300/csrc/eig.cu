// Symmetric eigendecomposition of the Fisher matrix for the decorrelated
// normalisation (paper Sect. 2.5, Eq. decorrelated: F = U Xi U^T,
// F^-1/2 = U Xi^-1/2 U^T with eigenvalues below 1e-12 x max set to zero) and
// the inverse used by the deconvolved normalisation (Eq. deconvolved).
//
// Parallel cyclic Jacobi (round-robin pair ordering): in each of the n-1
// rounds of a sweep the n indices form n/2 disjoint pairs; every pair gets the
// Jacobi rotation that zeroes its off-diagonal entry, and because the pairs
// are disjoint the update A <- J^T A J splits into independent 2x2 blocks
// R_a^T A[pair a, pair b] R_b.  One cooperative kernel runs all rounds: each
// round computes the n/2 rotations once, then applies them; grid barriers
// separate the phases (A is double-buffered).  float64 on CUDA cores is a
// few FMAs per clock per SM on GB300, so the work of a round is spread over
// every SM rather than one CTA.  Only blocks a <= b are computed and mirrored,
// which keeps A exactly symmetric.  Barrier waits are bounded: after
// kSpinLimit polls a block records QML_ETIMEOUT and every block returns.
#include "internal.cuh"

#include <math.h>

namespace qmlgb {

namespace {

// Grid barrier without a contended counter: block b publishes the epoch it
// has reached in its own 128-byte line (release store after a fence, so the
// block's writes come first), then every block reads all the lines (acquire
// loads spread over its threads) until each shows this epoch.  A single
// counter would serialise one atomic per block at one L2 slice.  The wait is
// bounded: after kSpinLimit / 8 polls the block records QML_ETIMEOUT, and a
// block that sees an error status leaves; both return false.
constexpr int kFlagStride = 32;  // unsigned words per flag line
constexpr int kJacobiThreads = 512;
// the barrier flags live in the reduction area, after the per-block partial
// sums (2 doubles per block): 4096 doubles hold 256 flag lines
constexpr int kFlagOffset = 4096;
constexpr int kMaxJacobiBlocks = 256;
// largest matrix the schedule tables hold (na = nspec * nl <= 6 * 94 at
// l <= 95, padded to even)
constexpr int kMaxJacobiN = 2048;

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned *p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ bool grid_barrier(DevStatus *st, unsigned *flags, unsigned &epoch, unsigned nblocks) {
  ++epoch;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    st_release(flags + (size_t)blockIdx.x * kFlagStride, epoch);
  }
  for (long long spins = 0;; ++spins) {
    bool here = true;
    for (unsigned b = threadIdx.x; b < nblocks; b += blockDim.x)
      here &= ((int)(ld_acquire(flags + (size_t)b * kFlagStride) - epoch) >= 0);
    if (__syncthreads_and(here)) return true;
    if ((spins & 63) == 63) {
      int bad = 0;
      if (threadIdx.x == 0) {
        bad = *((volatile int *)&st->code) != 0;
        if (!bad && spins > kSpinLimit / 8) {
          atomicExch(&st->code, 5 /* QML_ETIMEOUT */);
          bad = 1;
        }
      }
      if (__syncthreads_or(bad)) return false;
    }
  }
}

// round-robin (circle) schedule: slot a of round r holds player(a, r); slots
// a and n-1-a (a < n/2) form a pair, player 0 never moves
__device__ __forceinline__ int player(int x, int r, int n) {
  return x == 0 ? 0 : ((x - 1 + r) % (n - 1)) + 1;
}
__device__ __forceinline__ int slot_of(int y, int r, int n) {
  return y == 0 ? 0 : (((y - 1 - r) % (n - 1)) + (n - 1)) % (n - 1) + 1;
}

// Rotation (c, s) that (nearly) zeroes a_pq.  float64 operations that depend
// on one another cost tens of clocks each on this part, so the angle comes
// from float32 arithmetic and only the last step is float64: with d = a_qq -
// a_pp, the rotation angle phi has tan phi = sgn(d) 2 a_pq / (|d| +
// sqrt(d^2 + 4 a_pq^2)) (Golub & Van Loan, Sect. 8.5); tau = tan(phi / 2)
// = t / (1 + sqrt(1 + t^2)) in float32 (d and 2 a_pq first scaled by a power
// of two so neither overflows nor underflows), then in float64
//   c = (1 - tau^2) / (1 + tau^2),  s = 2 tau / (1 + tau^2),
// so that c^2 + s^2 = 1 to float64 rounding for any tau.  The angle is
// accurate to float32 only; the update applies J^T B J exactly (diagonal
// blocks included, the residual a_pq kept), so every step is an orthogonal
// similarity and the sweeps still drive the off-diagonal norm to zero.
__device__ __forceinline__ void rotation(double app, double aqq, double apq, double *out) {
  double c = 1.0, sn = 0.0;
  const double d = aqq - app, tw = 2.0 * apq;
  if (tw != 0.0 && isfinite(d) && isfinite(tw)) {
    // 2^-e with e the larger binary exponent of |d| and |tw|
    const long long bd = __double_as_longlong(d), bt = __double_as_longlong(tw);
    const int ed = (int)((bd >> 52) & 0x7FF), et = (int)((bt >> 52) & 0x7FF);
    const int e = ed > et ? ed : et;  // biased; |x| < 2^(e - 1022)
    double tv;
    if (e >= 1 && e <= 2045) {
      // 2^(1023 - e): the larger of |d|, |tw| lands in [1, 2)
      const double scale = __longlong_as_double((long long)(2 * 1023 - e) << 52);
      const float ds = (float)(d * scale), ts = (float)(tw * scale);
      const float r = sqrtf(ds * ds + ts * ts);
      const float t = (ds >= 0.0f ? ts : -ts) / (fabsf(ds) + r);  // |t| <= 1
      tv = (double)(t / (1.0f + sqrtf(1.0f + t * t)));
    } else {  // subnormal or near-overflow entries: the same steps in float64
      const double m = fmax(fabs(d), fabs(tw));
      const double ds = d / m, ts = tw / m;
      const double t = (ds >= 0.0 ? ts : -ts) / (fabs(ds) + sqrt(ds * ds + ts * ts));
      tv = t / (1.0 + sqrt(1.0 + t * t));
    }
    if (!isfinite(tv)) tv = 0.0;
    const double t2 = tv * tv;
    const double w = 1.0 / (1.0 + t2);
    c = (1.0 - t2) * w;
    sn = (2.0 * tv) * w;
  }
  out[0] = c;
  out[1] = sn;
}

// J^T B J for the symmetric 2 x 2 block B = [[x00, x01], [x01, x11]] of one
// pair: the two diagonal entries
__device__ __forceinline__ void rotated_diag(double x00, double x01, double x11, double c,
                                             double s, double &d0, double &d1) {
  const double cc = c * c, ss = s * s, cs2 = 2.0 * c * s;
  d0 = fma(cc, x00, fma(-cs2, x01, ss * x11));
  d1 = fma(ss, x00, fma(cs2, x01, cc * x11));
}

// One cooperative kernel runs every sweep.  Round r applies the rotations in
// rot_cur (one per pair); the thread that updates the 2 x 2 block holding a
// pair of round r+1 also forms that pair's rotation into rot_next from the
// updated entries (the off-diagonal one it has just computed, the diagonal
// ones recomputed from round r's rotations), so each round needs one grid
// barrier.
__global__ void __launch_bounds__(kJacobiThreads) jacobi_kernel(double *A0, double *A1, double *V, int n,
                                                     int max_sweeps, double *red, double *rot,
                                                     DevStatus *st) {
  const unsigned nblocks = gridDim.x;
  const int64_t gtid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t gsize = (int64_t)gridDim.x * blockDim.x;
  const int h = n / 2;
  const int64_t nblk = (int64_t)h * (h + 1) / 2;
  const int64_t nvt = (int64_t)n * h;
  double *Aold = A0, *Anew = A1;
  double *rcur = rot, *rnext = rot + 4 * (int64_t)h;
  const int64_t tbase =
      ((int64_t)blockIdx.x + (int64_t)nblocks * (threadIdx.x >> 5)) * 32 + (threadIdx.x & 31);
  double prev_off = 0.0;
  __shared__ double sred[2][kJacobiThreads / 32];
  // the round-robin schedule in shared memory, three rounds deep (buffer
  // r mod 3): slot -> player and player -> slot.  Round r reads its own and
  // round r+1's tables; the tables of round r+2 are written while the block
  // waits at round r's barrier, into the buffer round r-1 used.
  __shared__ short s_pt[3][kMaxJacobiN], s_sl[3][kMaxJacobiN];
  auto fill_tables = [&](int r) {
    short *pt = s_pt[r % 3], *sl = s_sl[r % 3];
    for (int x = threadIdx.x; x < n; x += blockDim.x) {
      pt[x] = (short)player(x, r, n);
      sl[x] = (short)slot_of(x, r, n);
    }
  };
  unsigned *flags = (unsigned *)(red + kFlagOffset);
  unsigned epoch = 0;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    // convergence test on the current matrix
    double off = 0.0, dia = 0.0;
    for (int64_t e = gtid; e < (int64_t)n * n; e += gsize) {
      int64_t i = e % n, j = e / n;
      double v = Aold[e];
      if (i == j) dia += v * v; else off += v * v;
    }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_down_sync(0xffffffffu, off, o);
      dia += __shfl_down_sync(0xffffffffu, dia, o);
    }
    if ((threadIdx.x & 31) == 0) {
      sred[0][threadIdx.x >> 5] = off;
      sred[1][threadIdx.x >> 5] = dia;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double so = 0.0, sd = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        so += sred[0][w];
        sd += sred[1][w];
      }
      red[2 * blockIdx.x] = so;
      red[2 * blockIdx.x + 1] = sd;
    }
    if (!grid_barrier(st, flags, epoch, nblocks)) return;
    double to = 0.0, td = 0.0;
    for (unsigned b = 0; b < nblocks; ++b) {
      to += ((volatile double *)red)[2 * b];
      td += ((volatile double *)red)[2 * b + 1];
    }
    // converged, or stalled at the float64 rounding floor (quadratic
    // convergence ends there; every block takes the same decision)
    if (to <= 1e-32 * td) break;
    if (sweep > 0 && to > 0.25 * prev_off && to <= 1e-20 * td) break;
    prev_off = to;
    fill_tables(0);
    fill_tables(1);
    // rotations of round 0, one per block
    if (threadIdx.x == 0)
      for (int a = blockIdx.x; a < h; a += nblocks) {
        const int pa = player(a, 0, n), qa = player(n - 1 - a, 0, n);
        rotation(Aold[pa + (int64_t)pa * n], Aold[qa + (int64_t)qa * n],
                 Aold[pa + (int64_t)qa * n], rcur + 4 * a);
      }
    if (!grid_barrier(st, flags, epoch, nblocks)) return;

    for (int r = 0; r < n - 1; ++r) {
      const bool more = (r + 1 < n - 1);
      const short *s_p0 = s_pt[r % 3], *s_p1 = s_pt[(r + 1) % 3], *s_s1 = s_sl[(r + 1) % 3];
      // tasks dealt out warp by warp across the blocks (warp w of block b takes
      // tasks 32 (b + nblocks w) ..), so every SM gets the same share of the
      // float64-heavy 2 x 2 blocks and of the eigenvector rows, and a warp's
      // eigenvector rows stay contiguous
      for (int64_t task = tbase; task < nblk + nvt; task += gsize) {
        if (task < nblk) {
          // upper-triangular block index (bb <= a)
          int a = (int)((sqrtf(8.0f * (float)task + 1.0f) - 1.0f) * 0.5f);
          while ((int64_t)(a + 1) * (a + 2) / 2 <= task) ++a;
          while ((int64_t)a * (a + 1) / 2 > task) --a;
          const int bb = (int)(task - (int64_t)a * (a + 1) / 2);
          const int pa = s_p0[bb], qa = s_p0[n - 1 - bb];
          const int pb = s_p0[a], qb = s_p0[n - 1 - a];
          const double ca = rcur[4 * bb], sa = rcur[4 * bb + 1];
          if (a == bb) {
            // J^T B J on the pair's own block; the residual off-diagonal kept
            const double x00 = Aold[pa + (int64_t)pa * n], x01 = Aold[pa + (int64_t)qa * n];
            const double x11 = Aold[qa + (int64_t)qa * n];
            double d0, d1;
            rotated_diag(x00, x01, x11, ca, sa, d0, d1);
            const double y00 = ca * x00 - sa * x01, y01 = sa * x00 + ca * x01;
            const double y10 = ca * x01 - sa * x11, y11 = sa * x01 + ca * x11;
            const double z01 = 0.5 * ((ca * y01 - sa * y11) + (sa * y00 + ca * y10));
            Anew[pa + (int64_t)pa * n] = d0;
            Anew[qa + (int64_t)qa * n] = d1;
            Anew[pa + (int64_t)qa * n] = z01;
            Anew[qa + (int64_t)pa * n] = z01;
          } else {
            const double cb = rcur[4 * a], sb = rcur[4 * a + 1];
            const double x00 = Aold[pa + (int64_t)pb * n], x01 = Aold[pa + (int64_t)qb * n];
            const double x10 = Aold[qa + (int64_t)pb * n], x11 = Aold[qa + (int64_t)qb * n];
            // diagonal blocks of both old pairs, read with the entries above
            // (needed only when a rotation of round r+1 is formed here)
            const double g00 = Aold[pa + (int64_t)pa * n], g01 = Aold[pa + (int64_t)qa * n];
            const double g11 = Aold[qa + (int64_t)qa * n], h00 = Aold[pb + (int64_t)pb * n];
            const double h01 = Aold[pb + (int64_t)qb * n], h11 = Aold[qb + (int64_t)qb * n];
            // pairs of round r+1 among the four entries: at most two (the
            // pairs of a round are disjoint), found with integer tests only
            int m0 = -1, m1 = -1, a20 = 0, a21 = 0;
            if (more) {
              const int xs[4] = {pa, pa, qa, qa}, ys[4] = {pb, qb, pb, qb};
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                const int sx = s_s1[xs[e]];
                const int a2 = sx < h ? sx : n - 1 - sx;  // pair index in round r+1
                if (s_p1[n - 1 - a2] == (sx < h ? ys[e] : -1) ||
                    (sx >= h && s_p1[a2] == ys[e])) {
                  if (m0 < 0) { m0 = e; a20 = a2; } else { m1 = e; a21 = a2; }
                }
              }
            }
            // X J_b, J = [[c, s], [-s, c]]
            const double y00 = cb * x00 - sb * x01, y01 = sb * x00 + cb * x01;
            const double y10 = cb * x10 - sb * x11, y11 = sb * x10 + cb * x11;
            // J_a^T (X J_b)
            const double z[4] = {ca * y00 - sa * y10, ca * y01 - sa * y11,
                                 sa * y00 + ca * y10, sa * y01 + ca * y11};
            Anew[pa + (int64_t)pb * n] = z[0];
            Anew[pa + (int64_t)qb * n] = z[1];
            Anew[qa + (int64_t)pb * n] = z[2];
            Anew[qa + (int64_t)qb * n] = z[3];
            Anew[pb + (int64_t)pa * n] = z[0];
            Anew[qb + (int64_t)pa * n] = z[1];
            Anew[pb + (int64_t)qa * n] = z[2];
            Anew[qb + (int64_t)qa * n] = z[3];
            if (m0 >= 0) {
              // diagonal entries after round r of both old pairs
              double dp[2], dq[2];  // [0]: player pa / pb, [1]: qa / qb
              rotated_diag(g00, g01, g11, ca, sa, dp[0], dp[1]);
              rotated_diag(h00, h01, h11, cb, sb, dq[0], dq[1]);
              // entry e = 2 i + j is (x, y) = ({pa, qa}[i], {pb, qb}[j]); the
              // rotation wants (a_p2p2, a_q2q2) with p2 = player(a2, r + 1)
              auto diag_pair = [&](int e, int a2, double &dpp, double &dqq) {
                const int x = (e >> 1) ? qa : pa;
                const double dx = dp[e >> 1], dy = dq[e & 1];
                const bool x_is_p = (s_p1[a2] == x);
                dpp = x_is_p ? dx : dy;
                dqq = x_is_p ? dy : dx;
              };
              auto zsel = [&](int e) {
                return e == 0 ? z[0] : (e == 1 ? z[1] : (e == 2 ? z[2] : z[3]));
              };
              double u0, v0;
              diag_pair(m0, a20, u0, v0);
              if (m1 >= 0) {
                double u1, v1;
                diag_pair(m1, a21, u1, v1);
                rotation(u0, v0, zsel(m0), rnext + 4 * a20);
                rotation(u1, v1, zsel(m1), rnext + 4 * a21);
              } else {
                rotation(u0, v0, zsel(m0), rnext + 4 * a20);
              }
            }
          }
        } else {
          const int vt = (int)(task - nblk);
          const int a = vt / n, row = vt - a * n;
          const int pa = s_p0[a], qa = s_p0[n - 1 - a];
          const double ca = rcur[4 * a], sa = rcur[4 * a + 1];
          const double vp = V[row + (int64_t)pa * n], vq = V[row + (int64_t)qa * n];
          V[row + (int64_t)pa * n] = ca * vp - sa * vq;
          V[row + (int64_t)qa * n] = sa * vp + ca * vq;
        }
      }
      fill_tables(r + 2);  // made visible by the barrier's __syncthreads
      if (!grid_barrier(st, flags, epoch, nblocks)) return;
      double *tmp = Aold;
      Aold = Anew;
      Anew = tmp;
      tmp = rcur;
      rcur = rnext;
      rnext = tmp;
    }
  }
  // leave the final matrix in A0
  if (Aold != A0) {
    for (int64_t e = gtid; e < (int64_t)n * n; e += gsize) A0[e] = Aold[e];
  }
}

__global__ void eig_setup_kernel(const double *F, int na, int n, double *A, double *V) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(e % n), j = (int)(e / n);
    double v;
    if (i < na && j < na) v = 0.5 * (F[i + (int64_t)j * na] + F[j + (int64_t)i * na]);
    else v = (i == j) ? 1.0 : 0.0;  // decoupled padding index
    A[e] = v;
    V[e] = (i == j) ? 1.0 : 0.0;
  }
}

// eigenvalue range (true indices only) and per-column factors 1 / x and,
// above the cut, x^-1/2 (one division or square root per eigenvalue)
__global__ void eig_factor_kernel(const double *A, int na, int n, double cut, double *fac,
                                  double *minmax, DevStatus *st) {
  __shared__ double smx[256], smn[256];
  double mx = -1e308, mn = 1e308;
  for (int i = threadIdx.x; i < na; i += blockDim.x) {
    const double x = A[i + (int64_t)i * n];
    mx = fmax(mx, x);
    mn = fmin(mn, x);
  }
  smx[threadIdx.x] = mx;
  smn[threadIdx.x] = mn;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      smx[threadIdx.x] = fmax(smx[threadIdx.x], smx[threadIdx.x + o]);
      smn[threadIdx.x] = fmin(smn[threadIdx.x], smn[threadIdx.x + o]);
    }
    __syncthreads();
  }
  const double xmax = smx[0], xmin = smn[0];
  if (threadIdx.x == 0) {
    minmax[0] = xmin;
    minmax[1] = xmax;
    if (!(xmin > 0.0)) {
      // the first error of the call is the one reported
      if (atomicCAS(&st->code, 0, 2 /* QML_ENOTSPD */) == 0) st->info = -1;
    }
  }
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    const double x = (c < na) ? A[c + (int64_t)c * n] : 1.0;
    fac[c] = (x != 0.0) ? 1.0 / x : 0.0;
    fac[n + c] = (c < na && x >= cut * xmax && x > 0.0) ? rsqrt(x) : 0.0;
  }
}

// the two scaled copies of V: S1 = V Xi^-1, S2 = V Xi_cut^-1/2
__global__ void eig_scale_kernel(const double *V, int n, const double *fac, double *S1,
                                 double *S2) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e / n);
    S1[e] = V[e] * fac[c];
    S2[e] = V[e] * fac[n + c];
  }
}

}  // namespace

size_t fisher_eig_work_doubles(int na) {
  size_t n = (size_t)(na + (na & 1));
  return 5 * n * n + 2 * 4096 + 4 * n;
}

cudaError_t run_fisher_eig(const double *F, int na, double *work, double *Finv, double *Fm12,
                           double *eig_minmax, DevStatus *status, cudaStream_t st) {
  const int n = na + (na & 1);
  if (n > kMaxJacobiN) return cudaErrorInvalidValue;  // callers check this first
  const size_t nn = (size_t)n * n;
  double *A0 = work, *A1 = work + nn, *V = work + 2 * nn, *S1 = work + 3 * nn,
         *S2 = work + 4 * nn, *red = work + 5 * nn, *rot = red + 2 * 4096;
  eig_setup_kernel<<<64, 256, 0, st>>>(F, na, n, A0, V);
  count_launch();
  int dev = 0;
  cudaGetDevice(&dev);
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, jacobi_kernel, kJacobiThreads, 0);
  int nblocks = nsm * (occ > 0 ? 1 : 0);
  if (nblocks > kMaxJacobiBlocks) nblocks = kMaxJacobiBlocks;
  if (nblocks < 1) return cudaErrorLaunchFailure;
  // barrier flags start at zero
  cudaMemsetAsync(red + kFlagOffset, 0, (size_t)kMaxJacobiBlocks * kFlagStride * sizeof(unsigned), st);
  int max_sweeps = 30;
  int nn_arg = n;
  void *args[] = {(void *)&A0, (void *)&A1, (void *)&V, (void *)&nn_arg, (void *)&max_sweeps,
                  (void *)&red, (void *)&rot, (void *)&status};
  cudaError_t e = cudaLaunchCooperativeKernel((const void *)jacobi_kernel, dim3(nblocks),
                                              dim3(kJacobiThreads), args, 0, st);
  if (e != cudaSuccess) return e;
  count_launch();
  // red is free again: per-column factors
  eig_factor_kernel<<<1, 256, 0, st>>>(A0, na, n, 1e-12, red, eig_minmax, status);
  count_launch();
  eig_scale_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(V, n, red, S1, S2);
  count_launch();
  // F^-1 = V Xi^-1 V^T, F^-1/2 = V Xi_cut^-1/2 V^T (rows / columns < na)
  launch_dgemm(0, 1, na, na, n, 1.0, S1, n, V, n, 0.0, Finv, na, 0, nullptr, st);
  launch_dgemm(0, 1, na, na, n, 1.0, S2, n, V, n, 0.0, Fm12, na, 0, nullptr, st);
  return cudaGetLastError();
}

}  // namespace qmlgb
