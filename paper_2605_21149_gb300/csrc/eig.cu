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

__device__ bool grid_barrier(DevStatus *st, unsigned nblocks) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned *gen = &st->bar_gen;
    const unsigned g = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(&st->bar_count, 1u) + 1u;
    if (arrived == nblocks) {
      st->bar_count = 0;
      __threadfence();
      atomicAdd(&st->bar_gen, 1u);
    } else {
      long long spins = 0;
      while (*gen == g) {
        if (++spins > kSpinLimit) {
          atomicExch(&st->code, 5 /* QML_ETIMEOUT */);
          break;
        }
        if (*((volatile int *)&st->code) != 0) break;
        __nanosleep(64);
      }
    }
    __threadfence();
    s_ok = (*((volatile int *)&st->code) == 0);
  }
  __syncthreads();
  return s_ok != 0;
}

__device__ __forceinline__ int player(int x, int r, int n) {
  return x == 0 ? 0 : ((x - 1 + r) % (n - 1)) + 1;
}

__device__ __forceinline__ void rotation(double app, double aqq, double apq, double &c, double &s,
                                         double &t) {
  if (apq == 0.0) {
    c = 1.0;
    s = 0.0;
    t = 0.0;
    return;
  }
  const double theta = (aqq - app) / (2.0 * apq);
  if (fabs(theta) > 1e150) {
    t = 0.5 / theta;
  } else {
    t = 1.0 / (fabs(theta) + sqrt(theta * theta + 1.0));
    if (theta < 0.0) t = -t;
  }
  c = 1.0 / sqrt(t * t + 1.0);
  s = t * c;
}

__global__ void __launch_bounds__(256) jacobi_kernel(double *A0, double *A1, double *V, int n,
                                                     int max_sweeps, double *red, double *rot,
                                                     DevStatus *st) {
  const unsigned nblocks = gridDim.x;
  const int64_t gtid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t gsize = (int64_t)gridDim.x * blockDim.x;
  const int h = n / 2;
  const int64_t nblk = (int64_t)h * (h + 1) / 2;
  const int64_t nvt = (int64_t)n * h;
  double *Aold = A0, *Anew = A1;
  double prev_off = 0.0;
  __shared__ double sred[2][8];
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
    if (!grid_barrier(st, nblocks)) return;
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
    if (!grid_barrier(st, nblocks)) return;

    for (int r = 0; r < n - 1; ++r) {
      // phase 1: one rotation per pair, computed once (float64 division and
      // square root are expensive on this part)
      for (int64_t a = gtid; a < h; a += gsize) {
        const int pa = player((int)a, r, n), qa = player(n - 1 - (int)a, r, n);
        double c, sn, t;
        const double apq = Aold[pa + (int64_t)qa * n];
        rotation(Aold[pa + (int64_t)pa * n], Aold[qa + (int64_t)qa * n], apq, c, sn, t);
        rot[4 * a] = c;
        rot[4 * a + 1] = sn;
        rot[4 * a + 2] = t * apq;
      }
      if (!grid_barrier(st, nblocks)) return;
      // phase 2: apply every 2x2 block update and the eigenvector rotation
      for (int64_t task = gtid; task < nblk + nvt; task += gsize) {
        if (task < nblk) {
          // upper-triangular block index (bb <= a)
          int a = (int)((sqrt(8.0 * task + 1.0) - 1.0) * 0.5);
          while ((int64_t)(a + 1) * (a + 2) / 2 <= task) ++a;
          while ((int64_t)a * (a + 1) / 2 > task) --a;
          const int bb = (int)(task - (int64_t)a * (a + 1) / 2);
          const int pa = player(bb, r, n), qa = player(n - 1 - bb, r, n);
          const int pb = player(a, r, n), qb = player(n - 1 - a, r, n);
          const double ca = rot[4 * bb], sa = rot[4 * bb + 1];
          if (a == bb) {
            const double tapq = rot[4 * bb + 2];
            Anew[pa + (int64_t)pa * n] = Aold[pa + (int64_t)pa * n] - tapq;
            Anew[qa + (int64_t)qa * n] = Aold[qa + (int64_t)qa * n] + tapq;
            Anew[pa + (int64_t)qa * n] = 0.0;
            Anew[qa + (int64_t)pa * n] = 0.0;
          } else {
            const double cb = rot[4 * a], sb = rot[4 * a + 1];
            const double x00 = Aold[pa + (int64_t)pb * n], x01 = Aold[pa + (int64_t)qb * n];
            const double x10 = Aold[qa + (int64_t)pb * n], x11 = Aold[qa + (int64_t)qb * n];
            // X J_b, J = [[c, s], [-s, c]]
            const double y00 = cb * x00 - sb * x01, y01 = sb * x00 + cb * x01;
            const double y10 = cb * x10 - sb * x11, y11 = sb * x10 + cb * x11;
            // J_a^T (X J_b)
            const double z00 = ca * y00 - sa * y10, z01 = ca * y01 - sa * y11;
            const double z10 = sa * y00 + ca * y10, z11 = sa * y01 + ca * y11;
            Anew[pa + (int64_t)pb * n] = z00;
            Anew[pa + (int64_t)qb * n] = z01;
            Anew[qa + (int64_t)pb * n] = z10;
            Anew[qa + (int64_t)qb * n] = z11;
            Anew[pb + (int64_t)pa * n] = z00;
            Anew[qb + (int64_t)pa * n] = z01;
            Anew[pb + (int64_t)qa * n] = z10;
            Anew[qb + (int64_t)qa * n] = z11;
          }
        } else {
          const int64_t vt = task - nblk;
          const int row = (int)(vt % n), a = (int)(vt / n);
          const int pa = player(a, r, n), qa = player(n - 1 - a, r, n);
          const double ca = rot[4 * a], sa = rot[4 * a + 1];
          const double vp = V[row + (int64_t)pa * n], vq = V[row + (int64_t)qa * n];
          V[row + (int64_t)pa * n] = ca * vp - sa * vq;
          V[row + (int64_t)qa * n] = sa * vp + ca * vq;
        }
      }
      if (!grid_barrier(st, nblocks)) return;
      double *tmp = Aold;
      Aold = Anew;
      Anew = tmp;
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

// eigenvalue range (true indices only) and the two scaled copies of V
__global__ void eig_scale_kernel(const double *A, const double *V, int na, int n, double cut,
                                 double *S1, double *S2, double *minmax, DevStatus *st) {
  __shared__ double smax;
  if (threadIdx.x == 0) {
    double mx = -1e308, mn = 1e308;
    for (int i = 0; i < na; ++i) {
      double x = A[i + (int64_t)i * n];
      mx = fmax(mx, x);
      mn = fmin(mn, x);
    }
    smax = mx;
    minmax[0] = mn;
    minmax[1] = mx;
    if (!(mn > 0.0)) {
      st->info = -1;
      atomicExch(&st->code, 2 /* QML_ENOTSPD */);
    }
  }
  __syncthreads();
  for (int64_t e = threadIdx.x; e < (int64_t)n * n; e += blockDim.x) {
    int c = (int)(e / n);
    double x = (c < na) ? A[c + (int64_t)c * n] : 1.0;
    double inv = (x != 0.0) ? 1.0 / x : 0.0;
    double irt = (c < na && x >= cut * smax && x > 0.0) ? 1.0 / sqrt(x) : 0.0;
    S1[e] = V[e] * inv;
    S2[e] = V[e] * irt;
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
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, jacobi_kernel, 256, 0);
  int nblocks = nsm * (occ > 0 ? 1 : 0);
  if (nblocks > 4096) nblocks = 4096;
  if (nblocks < 1) return cudaErrorLaunchFailure;
  // barrier words start at zero
  cudaMemsetAsync(&status->bar_count, 0, 2 * sizeof(unsigned), st);
  int max_sweeps = 30;
  int nn_arg = n;
  void *args[] = {(void *)&A0, (void *)&A1, (void *)&V, (void *)&nn_arg, (void *)&max_sweeps,
                  (void *)&red, (void *)&rot, (void *)&status};
  cudaError_t e = cudaLaunchCooperativeKernel((const void *)jacobi_kernel, dim3(nblocks),
                                              dim3(256), args, 0, st);
  if (e != cudaSuccess) return e;
  count_launch();
  eig_scale_kernel<<<1, 1024, 0, st>>>(A0, V, na, n, 1e-12, S1, S2, eig_minmax, status);
  count_launch();
  // F^-1 = V Xi^-1 V^T, F^-1/2 = V Xi_cut^-1/2 V^T (rows / columns < na)
  launch_dgemm(0, 1, na, na, n, 1.0, S1, n, V, n, 0.0, Finv, na, 0, nullptr, st);
  launch_dgemm(0, 1, na, na, n, 1.0, S2, n, V, n, 0.0, Fm12, na, 0, nullptr, st);
  return cudaGetLastError();
}

}  // namespace qmlgb
