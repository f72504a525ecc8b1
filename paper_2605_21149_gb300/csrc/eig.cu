// Symmetric eigendecomposition of the Fisher matrix for the decorrelated
// normalisation (paper Sect. 2.5, Eq. decorrelated: F = U Xi U^T,
// F^-1/2 = U Xi^-1/2 U^T with eigenvalues below 1e-12 x max set to zero) and
// the inverse used by the deconvolved normalisation (Eq. deconvolved).
//
// Two forms.  The default is the two-sided form that follows, which by
// default (tuning key eig_mixed) first runs float32 sweeps on one
// thread-block cluster and starts its float64 sweeps from the rotated matrix
// (the float32 pre-rotation phase, further below).  The other
// (tuning key eig_onesided = 1) is a one-sided Jacobi on the Cholesky factor
// of F (ojacobi_kernel below) with one grid barrier a sweep; on this part it
// is the slower one (TQU Nside 16: qml_fisher 52.3 against 45.8 ms), since
// each of its rounds pays for block reductions and a rotation in dependent
// float64 operations, which cost more than the grid barrier it saves.
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
#include "jacobi_sched.cuh"
#include "ptx.cuh"

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
// a and n-1-a (a < n/2) form a pair, player 0 never moves (jacobi_sched.cuh)
__device__ __forceinline__ int player(int x, int r, int n) { return jac_player(x, r, n); }
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
    // converged: off(A) <= eps ||A||_F with eps = 2^-52 (the cyclic-Jacobi
    // tolerance of Golub & Van Loan, Sect. 8.5, in squares: 2^-104), which
    // is where the float64 rounding floor of the off-diagonal sum lies; or
    // stalled at that floor (every block takes the same decision)
    if (to <= 0x1p-104 * (td + to)) break;
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

// ---------------------------------------------------- one-sided Jacobi --
// F = L L^T = G^T G with G = L^T (Cholesky of the padded F, computed first).
// One-sided (Hestenes) Jacobi rotates pairs of columns of G until they are
// orthogonal: G V = W, so V^T F V = W^T W is diagonal, F = V diag(|w_j|^2) V^T
// (eigenvalues |w_j|^2, eigenvectors the columns of V).  The rotation of a
// pair is the two-sided Jacobi rotation of its 2 x 2 Gram matrix
// [[|g_p|^2, g_p.g_q], [g_p.g_q, |g_q|^2]] (the same `rotation` as above).
//
// Parallel form: CTA a holds the columns in slots a and n-1-a (G and V, in
// shared memory), rotates them, then the columns move one slot along the
// round-robin ring (slot 0 fixed, x -> x+1, n-1 -> 1), so after n-1 rounds
// every pair has met once and every column is back in its own slot.  A
// column moves to a neighbouring CTA through a mailbox in global memory
// (two buffers by round parity) and a flag the sender raises with a release
// store; the receiver waits for its own flags only.  Sending and receiving
// are mutual between neighbours, so a sender cannot overwrite a buffer
// before its reader has taken it.  One grid barrier a sweep decides
// convergence: max over the sweep's pairs of (g_p.g_q)^2 / (|g_p|^2 |g_q|^2)
// at most tol2.  Every wait is bounded (QML_ETIMEOUT).
constexpr int kOjThreads = 256;
constexpr int kOjFlagStride = 32;

__device__ __forceinline__ int oj_owner(int y, int h) { return y < h ? y : 2 * h - 1 - y; }

// wait until flag >= want (acquire); false on timeout or another failure
__device__ bool oj_wait_flag(const unsigned *flag, unsigned want, DevStatus *st) {
  for (long long spins = 0;; ++spins) {
    if ((int)(ld_acquire(flag) - want) >= 0) return true;
    if ((spins & 63) == 63) {
      if (*((volatile int *)&st->code) != 0) return false;
      if (spins > kSpinLimit) {
        atomicCAS(&st->code, 0, 5 /* QML_ETIMEOUT */);
        return false;
      }
    }
  }
}

// Deterministic block sum of three per-thread partials (warp shuffles, then
// the warps' partials in a fixed order by every thread).
__device__ __forceinline__ void oj_sum3(double &x, double &y, double &z, double (*sh)[kOjThreads / 32]) {
  for (int o = 16; o > 0; o >>= 1) {
    x += __shfl_down_sync(0xffffffffu, x, o);
    y += __shfl_down_sync(0xffffffffu, y, o);
    z += __shfl_down_sync(0xffffffffu, z, o);
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    sh[0][w] = x;
    sh[1][w] = y;
    sh[2][w] = z;
  }
  __syncthreads();
  x = y = z = 0.0;
  for (int q = 0; q < kOjThreads / 32; ++q) {
    x += sh[0][q];
    y += sh[1][q];
    z += sh[2][q];
  }
  __syncthreads();
}

// L: the Cholesky factor (n x n lower, ld n; only i >= j read).  mbox: 8 h n
// doubles (two parities of 2 h entries of 2 n); pflags: 2 h kOjFlagStride words (zero on entry); red / gflags: the
// grid barrier's partials and flags (flags zero on entry).  Output: V (n x n),
// and the eigenvalues on the diagonal of D (D[j + j n]).
__global__ void __launch_bounds__(kOjThreads) ojacobi_kernel(const double *L, int n, int max_sweeps,
                                                          double tol2, double *mbox,
                                                          unsigned *pflags, double *red,
                                                          unsigned *gflags, double *V, double *D,
                                                          DevStatus *st) {
  extern __shared__ double ojs[];
  double *g0 = ojs, *g1 = ojs + n, *v0 = ojs + 2 * n, *v1 = ojs + 3 * n;
  __shared__ double sred[3][kOjThreads / 32];
  __shared__ double srot[2];
  const int h = n / 2, a = blockIdx.x, tid = threadIdx.x;
  const int slot[2] = {a, n - 1 - a};
  const size_t col = 2 * (size_t)n;  // one mailbox entry: a G column, then a V column
  // initial columns: g_x = row x of L, v_x = e_x
  for (int pos = 0; pos < 2; ++pos) {
    double *g = pos ? g1 : g0, *v = pos ? v1 : v0;
    const int x = slot[pos];
    for (int i = tid; i < n; i += kOjThreads) {
      g[i] = i <= x ? L[x + (size_t)i * n] : 0.0;
      v[i] = i == x ? 1.0 : 0.0;
    }
  }
  __syncthreads();
  unsigned R = 0, epoch = 0;  // rounds so far (all sweeps); grid-barrier epoch
  double worst = 0.0, wprev = 0.0;
  if (*((volatile int *)&st->code) != 0) return;  // e.g. F not positive definite
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    for (int r = 0; r < n - 1; ++r) {
      double al = 0.0, be = 0.0, ga = 0.0;
      for (int i = tid; i < n; i += kOjThreads) {
        const double x = g0[i], y = g1[i];
        al = fma(x, x, al);
        be = fma(y, y, be);
        ga = fma(x, y, ga);
      }
      oj_sum3(al, be, ga, sred);
      if (tid == 0) {
        rotation(al, be, ga, srot);
        const double ab = al * be;
        if (ab > 0.0) worst = fmax(worst, (ga * ga) / ab);
      }
      __syncthreads();
      const double c = srot[0], s = srot[1];
      // [g0 g1] <- [g0 g1] J, J = [[c, s], [-s, c]]; the same for V
      for (int i = tid; i < n; i += kOjThreads) {
        const double x = g0[i], y = g1[i];
        g0[i] = c * x - s * y;
        g1[i] = s * x + c * y;
        const double p = v0[i], q = v1[i];
        v0[i] = c * p - s * q;
        v1[i] = s * p + c * q;
      }
      __syncthreads();
      // send: the column in slot x goes to slot x + 1 (n - 1 -> 1; slot 0 stays)
      const size_t par = (size_t)(R & 1u) * 2 * h * col;  // 2h entries a parity
      for (int pos = 0; pos < 2; ++pos) {
        const int x = slot[pos];
        if (x == 0) continue;
        const int y = (x == n - 1) ? 1 : x + 1;
        const int b = oj_owner(y, h), q = y < h ? 0 : 1;
        double *dst = mbox + par + ((size_t)b * 2 + q) * col;
        const double *g = pos ? g1 : g0, *v = pos ? v1 : v0;
        for (int i = tid; i < n; i += kOjThreads) {
          dst[i] = g[i];
          dst[n + i] = v[i];
        }
      }
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        for (int pos = 0; pos < 2; ++pos) {
          const int x = slot[pos];
          if (x == 0) continue;
          const int y = (x == n - 1) ? 1 : x + 1;
          st_release(pflags + ((size_t)oj_owner(y, h) * 2 + (y < h ? 0 : 1)) * kOjFlagStride, R + 1);
        }
      }
      // receive into both positions (slot 0 keeps its column)
      int ok = 1;
      if (tid == 0)
        for (int pos = 0; pos < 2; ++pos)
          if (slot[pos] != 0 && !oj_wait_flag(pflags + ((size_t)a * 2 + pos) * kOjFlagStride, R + 1, st))
            ok = 0;
      if (!__syncthreads_and(ok)) return;
      for (int pos = 0; pos < 2; ++pos) {
        if (slot[pos] == 0) continue;
        const double *src = mbox + par + ((size_t)a * 2 + pos) * col;
        double *g = pos ? g1 : g0, *v = pos ? v1 : v0;
        for (int i = tid; i < n; i += kOjThreads) {
          g[i] = src[i];
          v[i] = src[n + i];
        }
      }
      __syncthreads();
      ++R;
    }
    // every column is home again: one grid barrier decides convergence
    if (tid == 0) red[a] = worst;
    if (!grid_barrier(st, gflags, epoch, gridDim.x)) return;
    double w = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) w = fmax(w, ((volatile double *)red)[b]);
    // the partials are read before anyone writes the next sweep's
    if (!grid_barrier(st, gflags, epoch, gridDim.x)) return;
    worst = 0.0;
    // converged, or stalled at the rounding floor of the dot products
    if (w <= tol2 || (sweep > 0 && w > 0.25 * wprev && w <= 1e-20)) break;
    wprev = w;
  }
  // eigenvalues |w_x|^2 on D's diagonal, eigenvectors into V
  for (int pos = 0; pos < 2; ++pos) {
    const double *g = pos ? g1 : g0, *v = pos ? v1 : v0;
    const int x = slot[pos];
    double nn = 0.0, d1 = 0.0, d2 = 0.0;
    for (int i = tid; i < n; i += kOjThreads) nn = fma(g[i], g[i], nn);
    oj_sum3(nn, d1, d2, sred);
    if (tid == 0) D[x + (size_t)x * n] = nn;
    for (int i = tid; i < n; i += kOjThreads) V[i + (size_t)x * n] = v[i];
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

// ------------------------------------------- float32 pre-rotation phase --
// The same cyclic Jacobi, first in float32 on one thread-block cluster
// (float32 arithmetic is 64 times the float64 rate on this part, and a
// cluster barrier is far cheaper than a grid barrier).  Only its rotations
// are kept: each is stored as its half-angle tau, from which an orthogonal
// basis V0 is rebuilt in float64 exactly as the float64 rounds build theirs
// (c = (1 - tau^2) / (1 + tau^2), s = 2 tau / (1 + tau^2)), so V0 is
// orthogonal to float64 rounding whatever float32 did.  The float64 sweeps
// then start from V0^T F V0, which is diagonal to float32 accuracy and needs
// two sweeps where F itself needs about seven; the eigenpairs are still
// those of the float64 sweeps and their stopping rule.
//
// Layout: CTA c of the cluster owns pairs [c h / CN, (c + 1) h / CN); a pair
// a holds the columns in slots a (side P) and n - 1 - a (side Q), float32,
// rows indexed by player, double-buffered by round parity.  A round: every
// CTA forms all h rotations from their three entries (a_pp, a_qq, a_qp, in
// a table of its own), then applies J^T B J to each 2 x 2 block of its own
// column pairs and writes the result where the column sits in the next round
// (slot x -> x - 1 for x >= 2, slot 1 -> n - 1, slot 0 fixed: pair a's P
// column goes to P(a - 1), except P(1) -> Q(0) and P(0) -> P(0); its Q column
// to Q(a + 1), except Q(h - 1) -> P(h - 1)).  The thread that writes one of
// the next round's three entries of a pair also stores it into every CTA's
// table, so that no CTA waits on a remote load after the cluster barrier
// that ends the round.  Between that barrier's arrive and its wait a CTA
// stores its half-angles to global memory and builds the player table of a
// later round, so neither delays the barrier.  Every CTA takes the same sweep
// decision from the same sums, so all of them pass the same barriers.
constexpr int kJ32Threads = 512;
constexpr int kJ32MaxSweeps = 8;
// largest padded order of the float32 phase (its columns fit in shared
// memory at 16 CTAs per cluster)
constexpr int kJ32MaxN = 640;

__host__ __device__ constexpr size_t j32_smem_bytes(int n, int cn) {
  return 16 * (size_t)((n / 2 + cn - 1) / cn) * n  // columns
         + 32                                        // partial sums, decision
         + 8 * (size_t)(n / 2)                       // rotations (c, s)
         + 24 * (size_t)(n / 2)                      // rotation inputs, two rounds
         + 8 * (size_t)n                             // players of four rounds
         + (size_t)(n / 2) + 16;                     // owner of each pair
}

// half-angle of the Jacobi rotation zeroing a_pq (the steps of the float64
// `rotation` above, in float32 with the fast reciprocal and square root: the
// float64 sweeps do not depend on this angle's accuracy)
__device__ __forceinline__ float rotation_tau32(float app, float aqq, float apq) {
  const float d = aqq - app, tw = 2.0f * apq;
  const float m = fmaxf(fabsf(d), fabsf(tw));
  if (!(m > 0.0f) || !isfinite(m)) return 0.0f;
  const float inv = __fdividef(1.0f, m);
  const float ds = d * inv, ts = tw * inv;
  const float r2 = ds * ds + ts * ts;  // in [1, 2]
  const float t = __fdividef(ds >= 0.0f ? ts : -ts, fabsf(ds) + r2 * rsqrtf(r2));
  const float u = 1.0f + t * t;  // in [1, 2]
  const float tau = __fdividef(t, 1.0f + u * rsqrtf(u));
  return isfinite(tau) ? tau : 0.0f;
}

template <int CN>
__global__ void __launch_bounds__(kJ32Threads) jacobi32_kernel(const double *A, int n, int max_sweeps,
                                                                float *taus, int *rounds_out) {
  extern __shared__ __align__(16) unsigned char j32_smem[];
  const int h = n / 2;
  const int rank = (int)cluster_ctarank();
  const int lo = j32_lo(rank, h, CN), np = j32_lo(rank + 1, h, CN) - lo;
  const int maxp = (h + CN - 1) / CN;
  float *cols = (float *)j32_smem;
  double *part = (double *)(j32_smem + 16 * (size_t)maxp * n);
  int *s_go = (int *)(part + 2);
  float2 *rot = (float2 *)(part + 4);
  float *inp = (float *)(rot + h);  // [2][h][3]: a_pp, a_qq, a_qp of each pair
  short *tab = (short *)(inp + 6 * h);  // [4][n]: round g's players in table g mod 4
  unsigned char *own = (unsigned char *)(tab + 4 * n);
  __shared__ double sred[2][kJ32Threads / 32];
  auto col = [&](int par, int la, int side) { return cols + ((size_t)(par * maxp + la) * 2 + side) * n; };
  for (int a = threadIdx.x; a < h; a += blockDim.x) own[a] = (unsigned char)j32_owner(a, h, CN);
  // scale by 2^-e, e the binary exponent of the largest diagonal entry
  double mx = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) mx = fmax(mx, fabs(A[i + (size_t)i * n]));
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) sred[0][threadIdx.x >> 5] = mx;
  __syncthreads();
  mx = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, sred[0][w]);
  int ex = 0;
  if (mx > 0.0 && isfinite(mx)) frexp(mx, &ex);
  const double sc = ldexp(1.0, -ex);
  for (int e = threadIdx.x; e < np * 2 * n; e += blockDim.x) {
    const int i = e % n, cs = e / n, la = cs >> 1, side = cs & 1;
    const int j = side ? n - 1 - (lo + la) : lo + la;
    col(0, la, side)[i] = (float)(A[i + (size_t)j * n] * sc);
  }
  for (int x = threadIdx.x; x < n; x += blockDim.x)
    for (int k = 0; k < 3; ++k) tab[k * n + x] = (short)player(x, k, n);
  // the first round's rotation inputs (pair a: players a and n - 1 - a)
  for (int a = threadIdx.x; a < h; a += blockDim.x) {
    const int q = n - 1 - a;
    inp[3 * a] = (float)(A[a + (size_t)a * n] * sc);
    inp[3 * a + 1] = (float)(A[q + (size_t)q * n] * sc);
    inp[3 * a + 2] = (float)(A[q + (size_t)a * n] * sc);
  }
  cluster_sync_all();  // every CTA of the cluster has started and loaded its columns
  const uint32_t part_u32 = smem_u32(part), inp_u32 = smem_u32(inp);
  // this thread's first 2 x 2 block (local pair la, row pair b) and its stride
  const int la0 = (int)threadIdx.x / h, b0 = (int)threadIdx.x - la0 * h;
  const int dla = (int)blockDim.x / h, db = (int)blockDim.x - dla * h;
  int par = 0, g = 0;
  double prev = 0.0;
  for (int sweep = 0;; ++sweep) {
    // off-diagonal and diagonal sums of squares of this CTA's columns (at a
    // sweep's start slot x holds player x)
    double off = 0.0, dia = 0.0;
    for (int e = threadIdx.x; e < np * 2 * n; e += blockDim.x) {
      const int i = e % n, cs = e / n, la = cs >> 1, side = cs & 1;
      const int j = side ? n - 1 - (lo + la) : lo + la;
      const double v = (double)col(par, la, side)[i];
      if (i == j) dia += v * v; else off += v * v;
    }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_down_sync(0xffffffffu, off, o);
      dia += __shfl_down_sync(0xffffffffu, dia, o);
    }
    __syncthreads();  // sred is free again
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
      part[0] = so;
      part[1] = sd;
    }
    cluster_sync_all();
    if (threadIdx.x == 0) {
      // the same sums in the same order in every CTA: the same decision
      double to = 0.0, td = 0.0;
      for (int c = 0; c < CN; ++c) {
        to += dsm_ld_f64(dsm_map(part_u32, (uint32_t)c));
        td += dsm_ld_f64(dsm_map(part_u32 + 8, (uint32_t)c));
      }
      int go = 1;
      if (sweep >= max_sweeps) go = 0;
      else if (to <= 0x1p-46 * (td + to)) go = 0;  // float32 rounding level
      else if (sweep > 0 && to > 0.25 * prev) go = 0;  // stalled
      prev = to;
      *s_go = go;
    }
    __syncthreads();
    if (!*s_go) break;
    for (int r = 0; r < n - 1; ++r, ++g) {
      const short *pl = tab + (g & 3) * n, *pl2 = tab + ((g + 1) & 3) * n;
      // one pair per thread (h <= kJ32MaxN / 2 < kJ32Threads)
      float my_tau = 0.0f;
      if ((int)threadIdx.x < h) {
        const float *in = inp + 3 * ((size_t)par * h + threadIdx.x);
        my_tau = rotation_tau32(in[0], in[1], in[2]);
        const float t2 = my_tau * my_tau, w = __fdividef(1.0f, 1.0f + t2);
        rot[threadIdx.x] = make_float2((1.0f - t2) * w, 2.0f * my_tau * w);
      }
      __syncthreads();
      const uint32_t nin = inp_u32 + 12u * (uint32_t)((par ^ 1) * h);  // next round's table
      auto bcast = [&](int pair, int slot, float v) {
#pragma unroll
        for (int c = 0; c < CN; ++c) dsm_st_f32(dsm_map(nin + 4u * (uint32_t)(3 * pair + slot), (uint32_t)c), v);
      };
      for (int la = la0, b = b0; la < np;) {
        const int a = lo + la;
        const float2 ra = rot[a], rb = rot[b];
        const int pb = pl[b], qb = pl[n - 1 - b];
        const float *P = col(par, la, 0), *Q = P + n;
        const float x00 = P[pb], x01 = Q[pb], x10 = P[qb], x11 = Q[qb];
        // X J_a (the pair's columns), then J_b^T (rows pb, qb)
        const float y00 = ra.x * x00 - ra.y * x01, y01 = ra.y * x00 + ra.x * x01;
        const float y10 = ra.x * x10 - ra.y * x11, y11 = ra.y * x10 + ra.x * x11;
        const float z00 = rb.x * y00 - rb.y * y10, z10 = rb.y * y00 + rb.x * y10;
        const float z01 = rb.x * y01 - rb.y * y11, z11 = rb.y * y01 + rb.x * y11;
        int dpa, dps, dqa, dqs;
        j32_dest_P(a, dpa, dps);
        j32_dest_Q(a, h, dqa, dqs);
        const int cp = own[dpa], cq = own[dqa];
        float *DP = col(par ^ 1, dpa - j32_lo(cp, h, CN), dps);
        float *DQ = col(par ^ 1, dqa - j32_lo(cq, h, CN), dqs);
        if (cp == rank) {
          DP[pb] = z00;
          DP[qb] = z10;
        } else {
          const uint32_t d = dsm_map(smem_u32(DP), (uint32_t)cp);
          dsm_st_f32(d + 4u * pb, z00);
          dsm_st_f32(d + 4u * qb, z10);
        }
        if (cq == rank) {
          DQ[pb] = z01;
          DQ[qb] = z11;
        } else {
          const uint32_t d = dsm_map(smem_u32(DQ), (uint32_t)cq);
          dsm_st_f32(d + 4u * pb, z01);
          dsm_st_f32(d + 4u * qb, z11);
        }
        // the next round's rotation inputs among these entries, into every
        // CTA's table
        int tp[4], ts[4], te[4];
        const int m = j32_next_inputs(a, b, h, pb, qb, dps == 0 ? (int)pl2[n - 1 - dpa] : -1,
                                      dqs == 0 ? (int)pl2[h] : -1, tp, ts, te);
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (i < m) bcast(tp[i], ts[i], te[i] == 0 ? z00 : (te[i] == 1 ? z10 : (te[i] == 2 ? z01 : z11)));
        la += dla;
        b += db;
        if (b >= h) {
          b -= h;
          ++la;
        }
      }
      cluster_arrive_release();
      if (rank == 0 && (int)threadIdx.x < h) taus[(size_t)g * h + threadIdx.x] = my_tau;
      // the table of round g + 3 (last read in round g - 1; first read after
      // the next round's barrier, which every thread reaches after this)
      for (int x = threadIdx.x; x < n; x += blockDim.x) tab[((g + 3) & 3) * n + x] = (short)player(x, g + 3, n);
      __syncwarp();
      cluster_wait_acquire();
      par ^= 1;
    }
  }
  if (rank == 0 && threadIdx.x == 0) *rounds_out = g;
  cluster_sync_all();  // no CTA leaves while another may read its shared memory
}

// (c, s) in float64 of every stored rotation, from its half-angle
__global__ void rot_cs_kernel(const float *taus, const int *rounds, int h, double2 *cs) {
  const int64_t total = (int64_t)(*rounds) * h;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    double t = (double)taus[e];
    if (!isfinite(t)) t = 0.0;
    const double t2 = t * t;
    const double w = 1.0 / (1.0 + t2);
    cs[e] = make_double2((1.0 - t2) * w, (2.0 * t) * w);
  }
}

// V0 = J_1 J_2 ... J_R, one CTA per row (rows are independent: v <- v J_g);
// thread a applies pair a's rotation each round, the (c, s) of the next
// rounds loaded ahead
__global__ void vbuild_kernel(const double2 *cs, const int *rounds, int n, double *V) {
  extern __shared__ double vrow[];
  const int row = blockIdx.x, h = n / 2, a = threadIdx.x;
  for (int i = threadIdx.x; i < n; i += blockDim.x) vrow[i] = (i == row) ? 1.0 : 0.0;
  __syncthreads();
  const int R = *rounds;
  const bool act = a < h;
  auto fetch = [&](int g) {
    return (act && g < R) ? cs[(size_t)g * h + a] : make_double2(1.0, 0.0);
  };
  double2 c0 = fetch(0), c1 = fetch(1), c2 = fetch(2), c3 = fetch(3);
  int p = act ? player(a, 0, n) : 0, q = act ? player(n - 1 - a, 0, n) : 0;
  for (int g = 0; g < R; ++g) {
    const double2 cur = c0;
    c0 = c1;
    c1 = c2;
    c2 = c3;
    c3 = fetch(g + 4);
    if (act) {
      const double vp = vrow[p], vq = vrow[q];
      vrow[p] = cur.x * vp - cur.y * vq;
      vrow[q] = cur.y * vp + cur.x * vq;
      // players of pair a in the next round (slot a > 0 and slot n - 1 - a
      // advance by one along 1 .. n - 1; slot 0 holds player 0)
      p = p == 0 ? 0 : (p == n - 1 ? 1 : p + 1);
      q = q == n - 1 ? 1 : q + 1;
    }
    __syncthreads();
  }
  for (int j = threadIdx.x; j < n; j += blockDim.x) V[row + (size_t)j * n] = vrow[j];
}

// A <- (A + A^T) / 2 in place
__global__ void symmetrize_kernel(double *A, int n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % n), j = (int)(e / n);
    if (i < j) {
      const double v = 0.5 * (A[e] + A[j + (int64_t)i * n]);
      A[e] = v;
      A[j + (int64_t)i * n] = v;
    }
  }
}

}  // namespace

namespace {
// doubles of the work area before the float32 phase's buffers (even, so
// that the (c, s) pairs after them are 16-byte aligned)
size_t eig_base_doubles(size_t n) {
  const size_t h = n / 2, nb = (n + kNB - 1) / kNB;
  // two-sided: A0, A1, V, S1, S2, the barrier area, rotations; one-sided adds
  // the 64-block inverses and log parts of the Cholesky, pair flags, grid
  // flags and the mailboxes
  const size_t b = 5 * n * n + 2 * 4096 + 4 * n + nb * kNB * kNB + nb + 8 + 32 * h + 16 * h + 8 * h * n;
  return b + (b & 1);
}
// stored rotations of the float32 phase
size_t j32_rotations(size_t n) { return (size_t)kJ32MaxSweeps * (n - 1) * (n / 2); }
}  // namespace

size_t fisher_eig_work_doubles(int na) {
  const size_t n = (size_t)(na + (na & 1));
  size_t total = eig_base_doubles(n);
  // float32 phase: half-angles (float), (c, s) pairs, the round count
  if (n <= (size_t)kJ32MaxN) {
    const size_t cnt = j32_rotations(n);
    total += (cnt + 1) / 2 + ((cnt + 1) / 2 & 1) + 2 * cnt + 2;
  }
  return total;
}

namespace {
// the float32 phase on one cluster of CN CTAs; false (nothing launched, no
// error left behind) when this part cannot run it
template <int CN>
bool launch_j32(const double *A0, int n, float *taus, int *rounds, cudaStream_t st) {
  const size_t smem = j32_smem_bytes(n, CN);
  if (smem > 227 * 1024) return false;
  if (cudaFuncSetAttribute(jacobi32_kernel<CN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess ||
      (CN > 8 && cudaFuncSetAttribute(jacobi32_kernel<CN>,
                                      cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)) {
    cudaGetLastError();
    return false;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CN);
  cfg.blockDim = dim3(kJ32Threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CN;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int ncl = 0;
  if (cudaOccupancyMaxActiveClusters(&ncl, jacobi32_kernel<CN>, &cfg) != cudaSuccess || ncl < 1) {
    cudaGetLastError();
    return false;
  }
  if (cudaLaunchKernelEx(&cfg, jacobi32_kernel<CN>, A0, n, kJ32MaxSweeps, taus, rounds) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  count_launch();
  return true;
}

// F = L L^T in place in A (n x n, ld n, lower) by 64-wide blocks: factor and
// invert each diagonal block, solve the rows below with the inverse, update
// the rest (the float64 kernels of the Cholesky path).  A non-positive pivot
// sets QML_ENOTSPD.
void small_potrf(double *A, int n, double *Linv, double *ldp, DevStatus *status, cudaStream_t st) {
  for (int j = 0; j < n; j += kNB) {
    const int jb = (n - j) < kNB ? (n - j) : kNB;
    double *Lb = Linv + (size_t)(j / kNB) * kNB * kNB;
    launch_potrf_diag(A + j + (size_t)j * n, n, n, j, Lb, ldp + j / kNB, status, st);
    if (j + jb < n) {
      const int m2 = n - j - jb;
      double *A21 = A + (j + jb) + (size_t)j * n;
      double *A22 = A + (j + jb) + (size_t)(j + jb) * n;
      launch_dgemm(0, 1, m2, jb, jb, 1.0, A21, n, Lb, kNB, 0.0, A21, n, 0, status, st);
      launch_dgemm(0, 1, m2, m2, jb, -1.0, A21, n, A21, n, 1.0, A22, n, 1, status, st);
    }
  }
}
}  // namespace

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
  int max_sweeps = 30;
  int nn_arg = n;
  cudaError_t e = cudaSuccess;
  // one-sided form (opt-in, tuning key eig_onesided) when the n / 2 column
  // pairs fit on the GPU at once, which the pairwise waits require
  const int h = n / 2;
  const size_t oj_smem = 4 * (size_t)n * sizeof(double);
  bool one = tune_get("eig_onesided", 0) != 0;
  if (one) {
    if (oj_smem > 48 * 1024 &&
        cudaFuncSetAttribute(ojacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)oj_smem) != cudaSuccess)
      one = false;
    int occ1 = 0;
    if (one && (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ1, ojacobi_kernel, kOjThreads,
                                                              oj_smem) != cudaSuccess ||
                (long long)occ1 * nsm < h))
      one = false;
  }
  if (one) {
    const size_t nb = (size_t)(n + kNB - 1) / kNB;
    double *Linv = rot + 4 * (size_t)n;
    double *ldp = Linv + nb * kNB * kNB;
    unsigned *pflags = (unsigned *)(ldp + nb + 8);
    unsigned *gflags = pflags + 64 * (size_t)h;
    double *mbox = (double *)(gflags + 32 * (size_t)h);
    small_potrf(A0, n, Linv, ldp, status, st);
    cudaMemsetAsync(pflags, 0, 96 * (size_t)h * sizeof(unsigned), st);  // pair and grid flags
    double tol2 = (double)n * 0x1p-104;  // |cos| <= sqrt(n) eps between every pair
    void *args[] = {(void *)&A0, (void *)&nn_arg, (void *)&max_sweeps, (void *)&tol2,
                    (void *)&mbox, (void *)&pflags, (void *)&red, (void *)&gflags, (void *)&V,
                    (void *)&A0, (void *)&status};
    e = cudaLaunchCooperativeKernel((const void *)ojacobi_kernel, dim3(h), dim3(kOjThreads), args,
                                    oj_smem, st);
    if (e != cudaSuccess) return e;
    count_launch();
  } else {
    // float32 pre-rotation (tuning key eig_mixed, default on): the float64
    // sweeps below then start from A0 = V0^T A0 V0 with V = V0
    if (tune_get("eig_mixed", 1) != 0 && n <= kJ32MaxN && h >= 32) {
      const size_t cnt = j32_rotations((size_t)n);
      double *mix = work + eig_base_doubles((size_t)n);
      float *taus = (float *)mix;
      const size_t tw = (cnt + 1) / 2 + ((cnt + 1) / 2 & 1);
      double2 *cs = (double2 *)(mix + tw);
      int *rounds = (int *)(mix + tw + 2 * cnt);
      const int want = (int)tune_get("eig_cluster", 16);
      const bool ran = (want >= 16 && launch_j32<16>(A0, n, taus, rounds, st)) ||
                       launch_j32<8>(A0, n, taus, rounds, st);
      if (ran) {
        rot_cs_kernel<<<4 * (unsigned)nsm, 256, 0, st>>>(taus, rounds, h, cs);
        count_launch();
        vbuild_kernel<<<(unsigned)n, (unsigned)((h + 31) / 32 * 32), (size_t)n * sizeof(double), st>>>(
            cs, rounds, n, V);
        count_launch();
        launch_dgemm(0, 0, n, n, n, 1.0, A0, n, V, n, 0.0, A1, n, 0, nullptr, st);
        launch_dgemm(1, 0, n, n, n, 1.0, V, n, A1, n, 0.0, A0, n, 0, nullptr, st);
        symmetrize_kernel<<<64, 256, 0, st>>>(A0, n);
        count_launch();
      }
    }
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, jacobi_kernel, kJacobiThreads, 0);
    int nblocks = nsm * (occ > 0 ? 1 : 0);
    if (nblocks > kMaxJacobiBlocks) nblocks = kMaxJacobiBlocks;
    if (nblocks < 1) return cudaErrorLaunchFailure;
    // barrier flags start at zero
    cudaMemsetAsync(red + kFlagOffset, 0, (size_t)kMaxJacobiBlocks * kFlagStride * sizeof(unsigned),
                    st);
    void *args[] = {(void *)&A0, (void *)&A1, (void *)&V, (void *)&nn_arg, (void *)&max_sweeps,
                    (void *)&red, (void *)&rot, (void *)&status};
    e = cudaLaunchCooperativeKernel((const void *)jacobi_kernel, dim3(nblocks),
                                    dim3(kJacobiThreads), args, 0, st);
    if (e != cudaSuccess) return e;
    count_launch();
  }
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
