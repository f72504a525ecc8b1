// Cross-QML of two data sets on one pixel set (Sect. 2.2, Eq. q_cross):
// each set i is filtered by its own C_i = S + N_i, W_i = Y^T C_i^-1 Y and
// w_i = Y^T C_i^-1 d_i (transfer folded into Y), and
//   q_x,a  = 1/2 d1^T C1^-1 P_a C2^-1 d2 = 1/2 sum_{(u,v) in a} sum_i w1[u i] w2[v i],
//   Wx_ab  = 1/2 tr[C1^-1 P_a C2^-1 P_b]
//          = 1/2 sum_{i in l, j in l'} sum_{(u,v) in a, (u',v') in b} W1[v i, u' j] W2[u i, v' j],
// with no noise bias for independent noise, and C_x = Wx^-1 q_x.  Wx is not
// symmetric, so the block sums keep all nc^4 products of the two component
// blocks (no pairing of equal products as in the Fisher matrix) and the
// solve is a general LU with partial pivoting.
#include "internal.cuh"

namespace qmlgb {

namespace {

// Per (l >= l') block: parts[tt][X NP + Y] = sum_{i in l, j in l'} B1[X] B2[Y],
// B_k[c NC + c'] = W_k[c i, c' j].  One CTA per block, largest first; warp
// shuffles then a fixed-order sum over warps (bitwise reproducible).
template <int NC>
__global__ void __launch_bounds__(128) cross_blocksum_kernel(const double *W1, const double *W2,
                                                             int64_t ldw, int k0, int lmin,
                                                             int nl, double *parts) {
  constexpr int NP = NC * NC;
  constexpr int NQ = NP * NP;
  const int nblk = nl * (nl + 1) / 2;
  const int tt = nblk - 1 - (int)blockIdx.x;
  int L = (int)((sqrt(8.0 * tt + 1.0) - 1.0) * 0.5);
  while ((L + 1) * (L + 2) / 2 <= tt) ++L;
  while (L * (L + 1) / 2 > tt) --L;
  const int Lp = tt - L * (L + 1) / 2;
  const int l = lmin + L, lp = lmin + Lp;
  const int ni = 2 * l + 1, nj = 2 * lp + 1;
  const int64_t offi = (int64_t)l * l - (int64_t)lmin * lmin;
  const int64_t offj = (int64_t)lp * lp - (int64_t)lmin * lmin;
  double acc[NQ];
#pragma unroll
  for (int u = 0; u < NQ; ++u) acc[u] = 0.0;
  const int total = ni * nj;
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    const int i = e % ni, j = e / ni;
    double B1[NP], B2[NP];
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
      for (int cp = 0; cp < NC; ++cp) {
        const int64_t at = ((int64_t)c * k0 + offi + i) + ((int64_t)cp * k0 + offj + j) * ldw;
        B1[c * NC + cp] = W1[at];
        B2[c * NC + cp] = W2[at];
      }
#pragma unroll
    for (int X = 0; X < NP; ++X)
#pragma unroll
      for (int Y = 0; Y < NP; ++Y) acc[X * NP + Y] = fma(B1[X], B2[Y], acc[X * NP + Y]);
  }
  __shared__ double red[4][NQ];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int u = 0; u < NQ; ++u) {
    double v = acc[u];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][u] = v;
  }
  __syncthreads();
  const int nw = blockDim.x >> 5;
  for (int u = threadIdx.x; u < NQ; u += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += red[w][u];
    parts[(int64_t)tt * NQ + u] = s;
  }
}

__device__ __forceinline__ int npairs_x(const int *uv) { return uv[2] < 0 ? 1 : 2; }

// Wx (na x na) from the block sums.  For l >= l' the entry takes the stored
// block's products B1[v][u'] B2[u][v']; for l < l' the stored (l', l) block
// holds the transposed component blocks (W1, W2 symmetric), so the same sum
// is B1[u'][v] B2[v'][u] there.
__global__ void cross_assemble_kernel(const double *parts, int nc, int nl, int nspec,
                                      const int *spec_uv, double *Wx) {
  const int na = nspec * nl;
  const int NP = nc * nc, NQ = NP * NP;
  const int64_t total = (int64_t)na * na;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int ra = (int)(e % na), rb = (int)(e / na);
    const int A = ra / nl, L = ra % nl, Bs = rb / nl, Lp = rb % nl;
    const bool swap = L < Lp;
    const int tt = swap ? Lp * (Lp + 1) / 2 + L : L * (L + 1) / 2 + Lp;
    const double *P = parts + (int64_t)tt * NQ;
    const int *ua = spec_uv + 4 * A, *ub = spec_uv + 4 * Bs;
    double s = 0.0;
    for (int pa = 0; pa < npairs_x(ua); ++pa) {
      const int u = ua[2 * pa], v = ua[2 * pa + 1];
      for (int pb = 0; pb < npairs_x(ub); ++pb) {
        const int up = ub[2 * pb], vp = ub[2 * pb + 1];
        const int X = swap ? up * nc + v : v * nc + up;
        const int Y = swap ? vp * nc + u : u * nc + vp;
        s += P[X * NP + Y];
      }
    }
    Wx[ra + (int64_t)rb * na] = 0.5 * s;
  }
}

// q_x for every (l, sim): one CTA per (l, sim), threads over the 2l+1 modes;
// P[u][v] = sum_i w1[u i] w2[v i], then q_a = 1/2 sum_{(u,v) in a} P[u][v].
__global__ void quad_cross_kernel(const double *w1, const double *w2, int64_t ldw, int nc,
                                  int k0, int lmin, int nl, int nspec, const int *spec_uv,
                                  double *q) {
  const int L = blockIdx.x, sim = blockIdx.y;
  const int l = lmin + L;
  const int ni = 2 * l + 1;
  const int64_t off = (int64_t)l * l - (int64_t)lmin * lmin;
  const double *a1 = w1 + (int64_t)sim * ldw, *a2 = w2 + (int64_t)sim * ldw;
  double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int i = threadIdx.x; i < ni; i += blockDim.x) {
    double x[3], y[3];
    for (int c = 0; c < nc; ++c) {
      x[c] = a1[(int64_t)c * k0 + off + i];
      y[c] = a2[(int64_t)c * k0 + off + i];
    }
    for (int u = 0; u < nc; ++u)
      for (int v = 0; v < nc; ++v) acc[u * 3 + v] += x[u] * y[v];
  }
  __shared__ double red[8][9];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int u = 0; u < 9; ++u) {
    double v = acc[u];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][u] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = blockDim.x >> 5;
    double s[9];
    for (int u = 0; u < 9; ++u) {
      s[u] = 0.0;
      for (int w = 0; w < nw; ++w) s[u] += red[w][u];
    }
    const int na = nspec * nl;
    for (int A = 0; A < nspec; ++A) {
      const int *uv = spec_uv + 4 * A;
      double val = 0.0;
      for (int p = 0; p < npairs_x(uv); ++p) val += s[uv[2 * p] * 3 + uv[2 * p + 1]];
      q[(int64_t)A * nl + L + (int64_t)sim * na] = 0.5 * val;
    }
  }
}

// A X = B for a general n x n A (column-major, overwritten by its LU factors)
// and B n x nrhs (overwritten by X): one CTA, LU with partial pivoting (the
// largest |A[i, k]| of column k, ties to the smallest row), rows of B swapped
// with those of A, then forward and back substitution, one thread per right-
// hand side.  A zero pivot sets the status to QML_ENOTSPD with info -2.
__global__ void __launch_bounds__(1024) lu_solve_kernel(double *A, int n, double *B, int nrhs,
                                                        DevStatus *status) {
  __shared__ double sv[32];
  __shared__ int si[32];
  __shared__ int piv_s;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
  for (int k = 0; k < n; ++k) {
    // pivot: largest magnitude in column k below the diagonal
    double best = -1.0;
    int bi = n;
    for (int i = k + tid; i < n; i += nt) {
      const double v = fabs(A[i + (int64_t)k * n]);
      if (v > best || (v == best && i < bi)) { best = v; bi = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_down_sync(0xffffffffu, best, o);
      const int oi = __shfl_down_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if (lane == 0) { sv[warp] = best; si[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
      double b = -1.0;
      int p = n;
      for (int w = 0; w < (nt >> 5); ++w)
        if (sv[w] > b || (sv[w] == b && si[w] < p)) { b = sv[w]; p = si[w]; }
      if (!(b > 0.0)) {
        if (atomicCAS(&status->code, 0, 2 /* QML_ENOTSPD */) == 0) status->info = -2;
        p = -1;
      }
      piv_s = p;
    }
    __syncthreads();
    const int p = piv_s;
    if (p < 0) return;
    if (p != k) {
      for (int j = tid; j < n; j += nt) {
        const double t = A[k + (int64_t)j * n];
        A[k + (int64_t)j * n] = A[p + (int64_t)j * n];
        A[p + (int64_t)j * n] = t;
      }
      for (int j = tid; j < nrhs; j += nt) {
        const double t = B[k + (int64_t)j * n];
        B[k + (int64_t)j * n] = B[p + (int64_t)j * n];
        B[p + (int64_t)j * n] = t;
      }
    }
    __syncthreads();
    const double inv = 1.0 / A[k + (int64_t)k * n];
    for (int i = k + 1 + tid; i < n; i += nt) A[i + (int64_t)k * n] *= inv;
    __syncthreads();
    const int m = n - k - 1;
    for (int64_t e = tid; e < (int64_t)m * m; e += nt) {
      const int i = k + 1 + (int)(e % m), j = k + 1 + (int)(e / m);
      A[i + (int64_t)j * n] = fma(-A[i + (int64_t)k * n], A[k + (int64_t)j * n],
                                  A[i + (int64_t)j * n]);
    }
    __syncthreads();
  }
  for (int c = tid; c < nrhs; c += nt) {
    double *b = B + (int64_t)c * n;
    for (int i = 1; i < n; ++i) {  // L y = b (unit diagonal)
      double s = b[i];
      for (int j = 0; j < i; ++j) s = fma(-A[i + (int64_t)j * n], b[j], s);
      b[i] = s;
    }
    for (int i = n - 1; i >= 0; --i) {  // U x = y
      double s = b[i];
      for (int j = i + 1; j < n; ++j) s = fma(-A[i + (int64_t)j * n], b[j], s);
      b[i] = s / A[i + (int64_t)i * n];
    }
  }
}

}  // namespace

void launch_cross_blocksum(const double *W1, const double *W2, int64_t ldw, int nc, int k0,
                           int lmin, int lmax, double *parts, cudaStream_t st) {
  const int nl = lmax - lmin + 1;
  const int nblk = nl * (nl + 1) / 2;
  if (nc == 1)
    { cross_blocksum_kernel<1><<<nblk, 128, 0, st>>>(W1, W2, ldw, k0, lmin, nl, parts); count_launch(); }
  else if (nc == 2)
    { cross_blocksum_kernel<2><<<nblk, 128, 0, st>>>(W1, W2, ldw, k0, lmin, nl, parts); count_launch(); }
  else
    { cross_blocksum_kernel<3><<<nblk, 128, 0, st>>>(W1, W2, ldw, k0, lmin, nl, parts); count_launch(); }
}

void launch_cross_assemble(const double *parts, int nc, int nl, int nspec, const int *spec_uv,
                           double *Wx, cudaStream_t st) {
  const int64_t na = (int64_t)nspec * nl;
  const int blocks = (int)((na * na + 255) / 256);
  { cross_assemble_kernel<<<blocks, 256, 0, st>>>(parts, nc, nl, nspec, spec_uv, Wx); count_launch(); }
}

void launch_quad_cross(const double *w1, const double *w2, int64_t ldw, int nsims, int nc, int k0,
                       int lmin, int lmax, int nspec, const int *spec_uv, double *q,
                       cudaStream_t st) {
  const int nl = lmax - lmin + 1;
  dim3 grid(nl, nsims);
  { quad_cross_kernel<<<grid, 128, 0, st>>>(w1, w2, ldw, nc, k0, lmin, nl, nspec, spec_uv, q); count_launch(); }
}

void launch_lu_solve(double *A, int n, double *B, int nrhs, DevStatus *status, cudaStream_t st) {
  { lu_solve_kernel<<<1, 1024, 0, st>>>(A, n, B, nrhs, status); count_launch(); }
}

}  // namespace qmlgb
