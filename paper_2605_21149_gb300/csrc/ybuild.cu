// Y builder: real spin-0 / spin-2 harmonics at pixel centres, transfer folded in.
//
// Math (paper Sect. 2.3.1 Eq. real_ylm; App. A.2 Eqs. spin_y_def, EB_from_spin;
// App. A.3 Eq. wigner_recurrence):
//   sY_lm = sqrt((2l+1)/4pi) d^l_{m,-s}(theta) e^{i m phi}
//   E_lm = -(2Y + -2Y)/2 = F1 e^{imphi},  B_lm = i(2Y - -2Y)/2 = i F2 e^{imphi}
//   F1 = -sqrt((2l+1)/4pi)(d^l_{m,2} + d^l_{m,-2})/2
//   F2 =  sqrt((2l+1)/4pi)(d^l_{m,-2} - d^l_{m,2})/2
// Real columns (m > 0 carries sqrt2, m = 0 does not):
//   T cos/sin : lam cos / lam sin                       (lam = sqrt((2l+1)/4pi) d^l_{m0})
//   E cos     : Q  F1 cos, U -F2 sin      E sin: Q F1 sin, U F2 cos
//   B cos     : Q  F2 sin, U  F1 cos      B sin: Q -F2 cos, U F1 sin
// d^l_{m,s} for fixed (m, s) follows the three-term recurrence in l
//   l sqrt(((l+1)^2-m^2)((l+1)^2-s^2)) d^{l+1}
//     = (2l+1)(l(l+1) cos(theta) - m s) d^l - (l+1) sqrt((l^2-m^2)(l^2-s^2)) d^{l-1},
// started at l0 = max(|m|, |s|) from the half-angle closed form (factorials
// through lgamma so that nothing overflows at large l).
//
// One thread owns one pixel (one row of Y for T, the Q and U rows for P) and
// writes its row across all columns; consecutive threads write consecutive
// rows, so every store of a warp is one coalesced 256-byte segment of a column.
#include "internal.cuh"

#include <math.h>

namespace qmlgb {

namespace {

constexpr double kInv4Pi = 0.07957747154594767;  // 1/(4 pi)
constexpr double kSqrt2 = 1.4142135623730951;

// d^{l0}_{m,s} at l0 = max(m, |s|), m >= 0, s in {-2, 0, 2}.
__device__ double wigner_start(int m, int s, double lc, double ls, double c, double sn) {
  int as = s < 0 ? -s : s;
  if (m >= as) {
    // d^m_{m,s} = (-1)^(m-s) sqrt((2m)! / ((m+s)!(m-s)!)) c^(m+s) sn^(m-s)
    double lg = 0.5 * (lgamma(2.0 * m + 1.0) - lgamma(m + s + 1.0) - lgamma(m - s + 1.0));
    double e = lg;
    if (m + s > 0) e += (m + s) * lc;
    if (m - s > 0) e += (m - s) * ls;
    double v = exp(e);
    return ((m - s) & 1) ? -v : v;
  }
  // m in {0, 1} < |s| = 2, l0 = 2
  // d^2_{m,2}  = sqrt(24/((2+m)!(2-m)!)) c^(2+m) sn^(2-m)
  // d^2_{m,-2} = (-1)^m sqrt(24/((2-m)!(2+m)!)) c^(2-m) sn^(2+m)
  const double f = (m == 0) ? 2.449489742783178 /* sqrt(24/4) */ : 2.0 /* sqrt(24/6) */;
  if (s > 0) {
    double v = f;
    for (int i = 0; i < 2 + m; ++i) v *= c;
    for (int i = 0; i < 2 - m; ++i) v *= sn;
    return v;
  }
  double v = (m & 1) ? -f : f;
  for (int i = 0; i < 2 - m; ++i) v *= c;
  for (int i = 0; i < 2 + m; ++i) v *= sn;
  return v;
}

// Recurrence coefficients, one entry per (m, l) (index m (lmax+1) + l):
//   d^{l+1} = (alpha x - beta) d^l - gamma d^{l-1}
//   alpha = (2l+1) l (l+1) / den,  beta = (2l+1) m s / den,
//   gamma = (l+1) sqrt((l^2-m^2)(l^2-s^2)) / den,
//   den = l sqrt(((l+1)^2-m^2)((l+1)^2-s^2))
// Spin 0 (s = 0) uses c0 = (alpha, gamma); spin 2 uses c2 = (alpha, beta(s=2),
// gamma), and s = -2 flips the sign of beta.  At l = 0 (m = s = 0 only)
// d^1 = x: alpha = 1, beta = gamma = 0.
struct RecCoef {
  double a0, g0, a2, b2, g2;
};

__global__ void rec_coef_kernel(int lmax, RecCoef *tab) {
  const int L = lmax + 1;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < L * L; t += gridDim.x * blockDim.x) {
    const int m = t / L, l = t % L;
    RecCoef c = {0, 0, 0, 0, 0};
    const double lp = l + 1.0, m2 = (double)m * m;
    if (l == 0) {
      c.a0 = 1.0;
    } else if (l >= m) {
      double den0 = (double)l * sqrt((lp * lp - m2) * lp * lp);
      c.a0 = (2.0 * l + 1.0) * (double)l * lp / den0;
      c.g0 = lp * sqrt(((double)l * l - m2) * (double)l * l) / den0;
      if (l >= 2) {
        double den2 = (double)l * sqrt((lp * lp - m2) * (lp * lp - 4.0));
        c.a2 = (2.0 * l + 1.0) * (double)l * lp / den2;
        c.b2 = (2.0 * l + 1.0) * 2.0 * m / den2;
        c.g2 = lp * sqrt(((double)l * l - m2) * ((double)l * l - 4.0)) / den2;
      }
    }
    tab[t] = c;
  }
}

// one thread per (pixel, m): the l recurrence of d^l_{m,0}; writes the m
// columns of its pixel's row for every l >= max(lmin, m)
__global__ void ybuild_T_kernel(YArgs a, const RecCoef *tab, double *Y, int64_t ldy) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int L = a.lmax + 1;
  if (t >= (int64_t)a.npix_T * L) return;
  const int p = (int)(t % a.npix_T), m = (int)(t / a.npix_T);
  const double th = a.theta_T[p], ph = a.phi_T[p];
  const double x = cos(th);
  const double c = cos(0.5 * th), sn = sin(0.5 * th);
  const double lc = log(c), ls = log(sn);
  const int lmin = a.lmin, lmax = a.lmax;
  double *row = Y + p;
  double sm, cm;
  sincos((double)m * ph, &sm, &cm);
  const RecCoef *tc = tab + (int64_t)m * L;
  double dm1 = 0.0, d0 = wigner_start(m, 0, lc, ls, c, sn);
  for (int l = m; l <= lmax; ++l) {
    if (l >= lmin) {
      const double lam = sqrt((2.0 * l + 1.0) * kInv4Pi) * d0 * a.transfer_T[l];
      const int64_t col = (int64_t)l * l - (int64_t)lmin * lmin;
      if (m == 0) {
        row[col * ldy] = lam;
      } else {
        row[(col + 2 * m - 1) * ldy] = kSqrt2 * lam * cm;
        row[(col + 2 * m) * ldy] = kSqrt2 * lam * sm;
      }
    }
    if (l < lmax) {
      const RecCoef cc = tc[l];
      const double dn = cc.a0 * x * d0 - cc.g0 * dm1;
      dm1 = d0;
      d0 = dn;
    }
  }
}

__global__ void ybuild_P_kernel(YArgs a, const RecCoef *tab, double *Y, int64_t ldy,
                                int64_t colE, int64_t colB, int64_t rowQ, int64_t rowU) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int L = a.lmax + 1;
  if (t >= (int64_t)a.npix_P * L) return;
  const int p = (int)(t % a.npix_P), m = (int)(t / a.npix_P);
  const double th = a.theta_P[p], ph = a.phi_P[p];
  const double x = cos(th);
  const double c = cos(0.5 * th), sn = sin(0.5 * th);
  const double lc = log(c), ls = log(sn);
  const int lmin = a.lmin, lmax = a.lmax;
  double *rq = Y + rowQ + p;
  double *ru = Y + rowU + p;
  double sm, cm;
  sincos((double)m * ph, &sm, &cm);
  const RecCoef *tc = tab + (int64_t)m * L;
  const int l0 = m > 2 ? m : 2;
  double pm1 = 0.0, p0 = wigner_start(m, 2, lc, ls, c, sn);    // d^l_{m,2}
  double qm1 = 0.0, q0 = wigner_start(m, -2, lc, ls, c, sn);   // d^l_{m,-2}
  for (int l = l0; l <= lmax; ++l) {
    if (l >= lmin) {
      const double nrm = sqrt((2.0 * l + 1.0) * kInv4Pi) * a.transfer_P[l];
      const double F1 = -0.5 * nrm * (p0 + q0);
      const double F2 = 0.5 * nrm * (q0 - p0);
      const int64_t col = (int64_t)l * l - (int64_t)lmin * lmin;
      if (m == 0) {
        rq[(colE + col) * ldy] = F1;
        ru[(colE + col) * ldy] = 0.0;
        rq[(colB + col) * ldy] = 0.0;
        ru[(colB + col) * ldy] = F1;
      } else {
        const double f1c = kSqrt2 * F1 * cm, f1s = kSqrt2 * F1 * sm;
        const double f2c = kSqrt2 * F2 * cm, f2s = kSqrt2 * F2 * sm;
        const int64_t ic = col + 2 * m - 1, is = col + 2 * m;
        rq[(colE + ic) * ldy] = f1c;
        ru[(colE + ic) * ldy] = -f2s;
        rq[(colE + is) * ldy] = f1s;
        ru[(colE + is) * ldy] = f2c;
        rq[(colB + ic) * ldy] = f2s;
        ru[(colB + ic) * ldy] = f1c;
        rq[(colB + is) * ldy] = -f2c;
        ru[(colB + is) * ldy] = f1s;
      }
    }
    if (l < lmax) {
      const RecCoef cc = tc[l];
      const double ax = cc.a2 * x;
      const double pn = (ax - cc.b2) * p0 - cc.g2 * pm1;
      const double qn = (ax + cc.b2) * q0 - cc.g2 * qm1;
      pm1 = p0;
      p0 = pn;
      qm1 = q0;
      q0 = qn;
    }
  }
}

// zero the cross blocks (T rows x E/B columns and Q/U rows x T columns)
__global__ void zero_block_kernel(double *Y, int64_t ldy, int64_t r0, int64_t nr, int64_t c0,
                                  int64_t nc) {
  int64_t total = nr * nc;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = t % nr, cidx = t / nr;
    Y[(r0 + r) + (c0 + cidx) * ldy] = 0.0;
  }
}

}  // namespace

void launch_ybuild(const YArgs &a, double *Y, int64_t ldy, cudaStream_t st) {
  const int k0 = (a.lmax + 1) * (a.lmax + 1) - a.lmin * a.lmin;
  const int nT = a.has_T ? a.npix_T : 0;
  const int nP = a.has_P ? a.npix_P : 0;
  const int L = a.lmax + 1;
  // recurrence coefficient table ((lmax+1)^2 entries) in the caller's workspace
  RecCoef *tab = (RecCoef *)a.coef;
  { rec_coef_kernel<<<(L * L + 255) / 256, 256, 0, st>>>(a.lmax, tab); count_launch(); }
  const int threads = 128;
  if (nT > 0) {
    const int64_t tot = (int64_t)nT * L;
    { ybuild_T_kernel<<<(unsigned)((tot + threads - 1) / threads), threads, 0, st>>>(a, tab, Y, ldy); count_launch(); }
  }
  if (nP > 0) {
    int64_t colE = a.has_T ? k0 : 0;
    const int64_t tot = (int64_t)nP * L;
    { ybuild_P_kernel<<<(unsigned)((tot + threads - 1) / threads), threads, 0, st>>>(
        a, tab, Y, ldy, colE, colE + k0, nT, (int64_t)nT + nP); count_launch(); }
  }
  if (nT > 0 && nP > 0) {
    // T rows x (E, B) columns and (Q, U) rows x T columns are structurally zero
    { zero_block_kernel<<<1024, 256, 0, st>>>(Y, ldy, 0, nT, k0, 2 * (int64_t)k0); count_launch(); }
    { zero_block_kernel<<<1024, 256, 0, st>>>(Y, ldy, nT, 2 * (int64_t)nP, 0, k0); count_launch(); }
  }
}

// ------------------------------------------------------- Lambda factors --
namespace {

// Per l: the nc x nc block of spectra (fields comps[]) and its lower
// Cholesky factor; a pivot that is not positive (a spectrum set to zero)
// gives a zero column, i.e. a factor of the positive semi-definite block.
__global__ void lambda_factor_kernel(const double *cl, int ldcl, int lmin, int lmax, int nc,
                                     int c0, int c1, int c2, double *lamL) {
  int il = blockIdx.x * blockDim.x + threadIdx.x;
  int l = lmin + il;
  if (l > lmax) return;
  const int L = ldcl;  // row stride of the [6][.] spectrum array
  const int comps[3] = {c0, c1, c2};
  // spectrum index of the (x, y) component pair
  auto sidx = [](int x, int y) {
    if (x > y) { int t = x; x = y; y = t; }
    if (x == y) return x;                  // TT=0 EE=1 BB=2
    if (x == 0 && y == 1) return 3;        // TE
    if (x == 0 && y == 2) return 4;        // TB
    return 5;                              // EB
  };
  double A[3][3];
  for (int i = 0; i < nc; ++i)
    for (int j = 0; j < nc; ++j) A[i][j] = cl[sidx(comps[i], comps[j]) * L + l];
  double Lf[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  double scale = 0.0;
  for (int i = 0; i < nc; ++i) scale = fmax(scale, fabs(A[i][i]));
  for (int j = 0; j < nc; ++j) {
    double d = A[j][j];
    for (int k = 0; k < j; ++k) d -= Lf[j][k] * Lf[j][k];
    if (d > 1e-14 * scale && d > 0.0) {
      double r = sqrt(d);
      Lf[j][j] = r;
      for (int i = j + 1; i < nc; ++i) {
        double v = A[i][j];
        for (int k = 0; k < j; ++k) v -= Lf[i][k] * Lf[j][k];
        Lf[i][j] = v / r;
      }
    }
  }
  for (int i = 0; i < nc; ++i)
    for (int j = 0; j < nc; ++j) lamL[(size_t)il * nc * nc + i * nc + j] = Lf[i][j];
}

// Per l: Li = L_l^-1 of the nc x nc lower factor (lower triangular, row-major
// like lamL).  A pivot <= 0 (a fiducial block that is not positive definite)
// sets the status word to QML_EINVAL with info = l + 1 and leaves zeros.
__global__ void lambda_inverse_kernel(const double *lamL, int nl, int nc, int lmin,
                                      double *lamLi, DevStatus *status) {
  const int il = blockIdx.x * blockDim.x + threadIdx.x;
  if (il >= nl) return;
  const double *Lf = lamL + (size_t)il * nc * nc;
  double X[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  bool ok = true;
  for (int j = 0; j < nc; ++j) ok = ok && Lf[j * nc + j] > 0.0;
  if (ok) {
    // forward substitution column by column: L X = I
    for (int c = 0; c < nc; ++c)
      for (int i = c; i < nc; ++i) {
        double v = (i == c) ? 1.0 : 0.0;
        for (int k = c; k < i; ++k) v -= Lf[i * nc + k] * X[k][c];
        X[i][c] = v / Lf[i * nc + i];
      }
  } else if (status) {
    if (atomicCAS(&status->code, 0, 1 /* QML_EINVAL */) == 0) status->info = lmin + il + 1;
  }
  for (int i = 0; i < nc; ++i)
    for (int j = 0; j < nc; ++j) lamLi[(size_t)il * nc * nc + i * nc + j] = X[i][j];
}

// G[p, (X, l, i)] = sum_X' Y[p, (X', l, i)] L_l[X', X], in place: one thread
// owns one (row, mode) and all components of it.
__global__ void mix_lambda_kernel(double *Y, int64_t ldy, int n, int nc, int k0, int lmin,
                                  int lmax, const double *lamL) {
  int64_t total = (int64_t)n * k0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    int p = (int)(t % n);
    int i = (int)(t / n);
    // l of mode i: i = l^2 - lmin^2 + r, 0 <= r <= 2l
    int l = (int)floor(sqrt((double)(i + lmin * lmin)));
    if (l * l > i + lmin * lmin) --l;
    if ((l + 1) * (l + 1) <= i + lmin * lmin) ++l;
    const double *Lf = lamL + (size_t)(l - lmin) * nc * nc;
    double v[3], g[3];
    for (int c = 0; c < nc; ++c) v[c] = Y[p + ((int64_t)c * k0 + i) * ldy];
    for (int x = 0; x < nc; ++x) {
      double s = 0.0;
      for (int xp = 0; xp < nc; ++xp) s += v[xp] * Lf[xp * nc + x];
      g[x] = s;
    }
    for (int c = 0; c < nc; ++c) Y[p + ((int64_t)c * k0 + i) * ldy] = g[c];
  }
}

}  // namespace

size_t ybuild_coef_bytes(int lmax) { return (size_t)(lmax + 1) * (lmax + 1) * sizeof(RecCoef); }

void launch_lambda_factor(const double *cl, int lmin, int lmax, int nc, const int *comps,
                          double *lamL, cudaStream_t st, int ldcl) {
  int nl = lmax - lmin + 1;
  if (ldcl <= 0) ldcl = lmax + 1;
  { lambda_factor_kernel<<<(nl + 63) / 64, 64, 0, st>>>(cl, ldcl, lmin, lmax, nc, comps[0],
                                                      nc > 1 ? comps[1] : 0,
                                                      nc > 2 ? comps[2] : 0, lamL); count_launch(); }
}

void launch_lambda_inverse(const double *lamL, int nl, int nc, int lmin, double *lamLi,
                           DevStatus *status, cudaStream_t st) {
  { lambda_inverse_kernel<<<(nl + 63) / 64, 64, 0, st>>>(lamL, nl, nc, lmin, lamLi, status); count_launch(); }
}

void launch_mix_lambda(double *Y, int64_t ldy, int n, int nc, int k0, int lmin, int lmax,
                       const double *lamL, cudaStream_t st) {
  int64_t total = (int64_t)n * k0;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  { mix_lambda_kernel<<<blocks, 256, 0, st>>>(Y, ldy, n, nc, k0, lmin, lmax, lamL); count_launch(); }
}

}  // namespace qmlgb
