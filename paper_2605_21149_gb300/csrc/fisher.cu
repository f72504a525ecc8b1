// Fisher block sums (paper App. C.1, Eq. sparse_trace) and the quadratic
// estimates (Eq. q_harmonic).
//
// With W = Y^T C^-1 Y (transfer folded into Y) and the selector E_a of one
// spectrum entry a = (XY, l) (ones at modes (X,l,i),(Y,l,i) and symmetric),
//   F_ab = 1/2 sum_{i in l, j in l'} sum_{(u,v) in a, (u',v') in b}
//          W[v i, u' j] W[u i, v' j].
// For one pair of modes (i, j) the nc x nc component block B_ij of W enters
// only through the products B[v][u'] B[u][v']; the kernel accumulates every
// distinct product (nc^2 (nc^2+1)/2 of them: 1, 10 or 45) over the (l, l')
// block once, and the spectra are assembled from those sums afterwards, so
// the float64 work per (i, j) does not grow with the number of spectra.
// One CTA per (l >= l') block, the largest blocks first; W is read once with
// coalesced loads along i.  Reductions: warp shuffles, then a fixed-order sum
// over warps (results are bitwise reproducible).
//
// The noise bias uses the exact identity
//   1/2 tr[C^-1 P_a] = sum_b F_ab C^fid_b + b_a
// (expectation of Eq. q_ell with <q> = F C, exact when C = sum_b C_b P_b + N,
// which holds because the signal band equals the estimation window and F is
// built over every spectrum of the fields present): b = t/2 - F_full c_fid with
// t_a = tr[E_a W] from the diagonal (l = l') blocks.
#include "internal.cuh"

namespace qmlgb {

namespace {

template <int NC>
__global__ void __launch_bounds__(128) fisher_blocksum_kernel(const double *W, int64_t ldw, int k0,
                                                              int lmin, int nl, double *parts,
                                                              double *diag) {
  constexpr int NP = NC * NC;
  constexpr int NU = NP * (NP + 1) / 2;
  const int nblk = nl * (nl + 1) / 2;
  const int tt = nblk - 1 - (int)blockIdx.x;  // largest (l, l') first
  int L = (int)((sqrt(8.0 * tt + 1.0) - 1.0) * 0.5);
  while ((L + 1) * (L + 2) / 2 <= tt) ++L;
  while (L * (L + 1) / 2 > tt) --L;
  const int Lp = tt - L * (L + 1) / 2;
  const int l = lmin + L, lp = lmin + Lp;
  const int ni = 2 * l + 1, nj = 2 * lp + 1;
  const int64_t offi = (int64_t)l * l - (int64_t)lmin * lmin;
  const int64_t offj = (int64_t)lp * lp - (int64_t)lmin * lmin;

  double acc[NU];
#pragma unroll
  for (int u = 0; u < NU; ++u) acc[u] = 0.0;
  double dacc[NP];
#pragma unroll
  for (int u = 0; u < NP; ++u) dacc[u] = 0.0;

  const int total = ni * nj;
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    const int i = e % ni, j = e / ni;
    double B[NP];
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
      for (int cp = 0; cp < NC; ++cp)
        B[c * NC + cp] = W[((int64_t)c * k0 + offi + i) + ((int64_t)cp * k0 + offj + j) * ldw];
    int idx = 0;
#pragma unroll
    for (int X = 0; X < NP; ++X)
#pragma unroll
      for (int Y = X; Y < NP; ++Y) {
        acc[idx] = fma(B[X], B[Y], acc[idx]);
        ++idx;
      }
    if (L == Lp && i == j) {
#pragma unroll
      for (int X = 0; X < NP; ++X) dacc[X] += B[X];
    }
  }
  // block reduction: shuffles inside the warp, then warps in fixed order
  __shared__ double red[4][NU + NP];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int u = 0; u < NU; ++u) {
    double v = acc[u];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][u] = v;
  }
#pragma unroll
  for (int u = 0; u < NP; ++u) {
    double v = dacc[u];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][NU + u] = v;
  }
  __syncthreads();
  const int nw = blockDim.x >> 5;
  for (int u = threadIdx.x; u < NU + NP; u += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += red[w][u];
    if (u < NU)
      parts[(int64_t)tt * NU + u] = s;
    else if (L == Lp)
      diag[(int64_t)L * NP + (u - NU)] = s;
  }
}

// spec_uv: for each spectrum 4 ints (u0, v0, u1, v1) of local component
// positions; (u1, v1) = (-1, -1) for an auto spectrum (single pair).
__device__ __forceinline__ int npairs(const int *uv) { return uv[2] < 0 ? 1 : 2; }

__global__ void fisher_assemble_kernel(const double *parts, const double *diag, int nc, int nl,
                                       int nspec, const int *spec_uv, double *F, double *t) {
  const int na = nspec * nl;
  const int NP = nc * nc;
  const int NU = NP * (NP + 1) / 2;
  const int64_t total = (int64_t)na * na;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int ra = (int)(e % na), rb = (int)(e / na);
    int A = ra / nl, L = ra % nl, Bs = rb / nl, Lp = rb % nl;
    // use the stored (L >= Lp) block; swapping the roles of (a, l) and (b, l')
    // is the symmetry F_ab = F_ba
    if (L < Lp) {
      int tA = A; A = Bs; Bs = tA;
      int tL = L; L = Lp; Lp = tL;
    }
    const int tt = L * (L + 1) / 2 + Lp;
    const double *P = parts + (int64_t)tt * NU;
    const int *ua = spec_uv + 4 * A, *ub = spec_uv + 4 * Bs;
    double s = 0.0;
    for (int pa = 0; pa < npairs(ua); ++pa) {
      int u = ua[2 * pa], v = ua[2 * pa + 1];
      for (int pb = 0; pb < npairs(ub); ++pb) {
        int up = ub[2 * pb], vp = ub[2 * pb + 1];
        int X = v * nc + up, Y = u * nc + vp;
        if (X > Y) { int tmp = X; X = Y; Y = tmp; }
        // index of (X, Y), X <= Y, in the row-major upper triangle of NP x NP
        int idx = X * NP - X * (X - 1) / 2 + (Y - X);
        s += P[idx];
      }
    }
    F[ra + (int64_t)rb * na] = 0.5 * s;
    if (rb == 0) {
      // t_a = tr[E_a W] for a = ra
      int A2 = ra / nl, L2 = ra % nl;
      const int *u2 = spec_uv + 4 * A2;
      double tsum = 0.0;
      for (int pa = 0; pa < npairs(u2); ++pa) {
        int u = u2[2 * pa], v = u2[2 * pa + 1];
        tsum += diag[(int64_t)L2 * NP + v * nc + u];
      }
      t[ra] = tsum;
    }
  }
}

__global__ void fisher_select_kernel(const double *F_full, const double *t_full,
                                     const double *cl_fid, int ldcl, int lmin, int lmax,
                                     int nspec_full,
                                     const int *full_spec_ids, int nspec, const int *sel,
                                     double *F, double *b) {
  const int nl = lmax - lmin + 1;
  const int naf = nspec_full * nl;
  const int na = nspec * nl;
  const int64_t total = (int64_t)na * na;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total + na;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (e < total) {
      int a = (int)(e % na), bb = (int)(e / na);
      int fa = sel[a / nl] * nl + a % nl, fb = sel[bb / nl] * nl + bb % nl;
      F[e] = F_full[fa + (int64_t)fb * naf];
    } else {
      int a = (int)(e - total);
      int fa = sel[a / nl] * nl + a % nl;
      // b_a = t_a / 2 - sum_b F_ab C_b  (fixed order over b)
      double s = 0.0;
      for (int fb = 0; fb < naf; ++fb) {
        int sid = full_spec_ids[fb / nl];
        int l = lmin + fb % nl;
        s = fma(F_full[fa + (int64_t)fb * naf], cl_fid[sid * ldcl + l], s);
      }
      b[a] = 0.5 * t_full[fa] - s;
    }
  }
}

// y for every (l, sim): one CTA, threads over the 2l+1 modes
__global__ void quad_y_kernel(const double *w, int64_t ldw, int nc, int k0, int lmin, int nl,
                              int nspec, const int *spec_uv, double *y) {
  const int L = blockIdx.x, sim = blockIdx.y;
  const int l = lmin + L;
  const int ni = 2 * l + 1;
  const int64_t off = (int64_t)l * l - (int64_t)lmin * lmin;
  const double *ws = w + (int64_t)sim * ldw;
  double acc[6] = {0, 0, 0, 0, 0, 0};  // (u, v) u <= v, row-major upper triangle
  for (int i = threadIdx.x; i < ni; i += blockDim.x) {
    double v[3];
    for (int c = 0; c < nc; ++c) v[c] = ws[(int64_t)c * k0 + off + i];
    int idx = 0;
    for (int a = 0; a < nc; ++a)
      for (int b = a; b < nc; ++b) acc[idx++] += v[a] * v[b];
  }
  __shared__ double red[8][6];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int u = 0; u < 6; ++u) {
    double v = acc[u];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][u] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = blockDim.x >> 5;
    double s[6];
    for (int u = 0; u < 6; ++u) {
      s[u] = 0.0;
      for (int q = 0; q < nw; ++q) s[u] += red[q][u];
    }
    const int na = nspec * nl;
    for (int A = 0; A < nspec; ++A) {
      const int *uv = spec_uv + 4 * A;
      int a = uv[0], b = uv[1];
      if (a > b) { int t = a; a = b; b = t; }
      int idx = a * nc - a * (a - 1) / 2 + (b - a);
      // auto: 1/2 sum w_X^2 ; cross: 1/2 (w_X w_Y + w_Y w_X) = sum w_X w_Y
      double val = (npairs(uv) == 1) ? 0.5 * s[idx] : s[idx];
      y[(int64_t)A * nl + L + (int64_t)sim * na] = val;
    }
  }
}

__global__ void sub_bias_kernel(const double *y, const double *b, int na, int nsims, double *q) {
  int64_t total = (int64_t)na * nsims;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x)
    q[e] = y[e] - b[e % na];
}

}  // namespace

void launch_fisher_blocksum(const double *W, int64_t ldw, int nc, int k0, int lmin, int lmax,
                            double *parts, double *diag, cudaStream_t st) {
  const int nl = lmax - lmin + 1;
  const int nblk = nl * (nl + 1) / 2;
  if (nc == 1)
    { fisher_blocksum_kernel<1><<<nblk, 128, 0, st>>>(W, ldw, k0, lmin, nl, parts, diag); count_launch(); }
  else if (nc == 2)
    { fisher_blocksum_kernel<2><<<nblk, 128, 0, st>>>(W, ldw, k0, lmin, nl, parts, diag); count_launch(); }
  else
    { fisher_blocksum_kernel<3><<<nblk, 128, 0, st>>>(W, ldw, k0, lmin, nl, parts, diag); count_launch(); }
}

void launch_fisher_assemble(const double *parts, const double *diag, int nc, int nl,
                            int nspec_full, const int *spec_uv, double *F_full, double *t_full,
                            cudaStream_t st) {
  int64_t na = (int64_t)nspec_full * nl;
  int blocks = (int)((na * na + 255) / 256);
  { fisher_assemble_kernel<<<blocks, 256, 0, st>>>(parts, diag, nc, nl, nspec_full, spec_uv,
                                                 F_full, t_full); count_launch(); }
}

void launch_fisher_select(const double *F_full, const double *t_full, const double *cl_fid,
                          int lmin, int lmax, int nspec_full, const int *full_spec_ids,
                          int nspec, const int *sel, double *F, double *b, cudaStream_t st,
                          int ldcl) {
  int64_t na = (int64_t)nspec * (lmax - lmin + 1);
  int blocks = (int)((na * na + na + 255) / 256);
  if (ldcl <= 0) ldcl = lmax + 1;
  { fisher_select_kernel<<<blocks, 256, 0, st>>>(F_full, t_full, cl_fid, ldcl, lmin, lmax,
                                               nspec_full, full_spec_ids, nspec, sel, F, b); count_launch(); }
}

void launch_quad_y(const double *w, int64_t ldw, int nsims, int nc, int k0, int lmin, int lmax,
                   int nspec, const int *spec_uv, double *y, cudaStream_t st) {
  const int nl = lmax - lmin + 1;
  dim3 grid(nl, nsims);
  { quad_y_kernel<<<grid, 128, 0, st>>>(w, ldw, nc, k0, lmin, nl, nspec, spec_uv, y); count_launch(); }
}

void launch_sub_bias(const double *y, const double *b, int na, int nsims, double *q,
                     cudaStream_t st) {
  int64_t total = (int64_t)na * nsims;
  int blocks = (int)((total + 255) / 256);
  if (blocks < 1) blocks = 1;
  { sub_bias_kernel<<<blocks, 256, 0, st>>>(y, b, na, nsims, q); count_launch(); }
}

}  // namespace qmlgb
