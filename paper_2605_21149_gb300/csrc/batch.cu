// Kernels of the batched likelihood scan (harmonic form, paper Sect. 2.3.2
// Eqs. smw, logdet; App. B Eq. quad_form_smw; App. C.3 stable congruent form).
//
// With G = Y L_Lambda (L_Lambda the lower factor of the per-(l,m) spectrum
// block) and M = Y^T N^-1 Y:
//   |C| = |N| |I + L_Lambda^T M L_Lambda|,
//   d^T C^-1 d = d^T N^-1 d - z^T Kt^-1 z,  z = L_Lambda^T Y^T N^-1 d,
// Kt = I + L_Lambda^T M L_Lambda has eigenvalues >= 1, so its Cholesky is
// well conditioned for any spectra (also singular Lambda).
#include "internal.cuh"

namespace qmlgb {

namespace {

__device__ __forceinline__ int l_of_mode(int i, int lmin) {
  int l = (int)floor(sqrt((double)(i + lmin * lmin)));
  if (l * l > i + lmin * lmin) --l;
  if ((l + 1) * (l + 1) <= i + lmin * lmin) ++l;
  return l;
}

// Kt (lower triangle) from M (k x k, full) and the per-l factors lamL
// (row-major nc x nc, lower): one thread per mode pair (i, j), all nc x nc
// component entries of that pair.
__global__ void form_ktilde_kernel(const double *M, int64_t ldm, int nc, int k0, int lmin,
                                   const double *lamL, double *K, int64_t ldk) {
  const int64_t total = (int64_t)k0 * k0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % k0), j = (int)(t / k0);
    const double *Li = lamL + (size_t)(l_of_mode(i, lmin) - lmin) * nc * nc;
    const double *Lj = lamL + (size_t)(l_of_mode(j, lmin) - lmin) * nc * nc;
    double B[3][3], T[3][3];
    for (int a = 0; a < nc; ++a)
      for (int b = 0; b < nc; ++b) B[a][b] = M[((int64_t)a * k0 + i) + ((int64_t)b * k0 + j) * ldm];
    // T = B L_j  (T[a][y] = sum_b B[a][b] L_j[b][y])
    for (int a = 0; a < nc; ++a)
      for (int y = 0; y < nc; ++y) {
        double sacc = 0.0;
        for (int b = y; b < nc; ++b) sacc = fma(B[a][b], Lj[b * nc + y], sacc);
        T[a][y] = sacc;
      }
    for (int x = 0; x < nc; ++x)
      for (int y = 0; y < nc; ++y) {
        const int64_t r = (int64_t)x * k0 + i, c = (int64_t)y * k0 + j;
        if (r < c) continue;
        double sacc = (r == c) ? 1.0 : 0.0;
        for (int a = x; a < nc; ++a) sacc = fma(Li[a * nc + x], T[a][y], sacc);
        K[r + c * ldk] = sacc;
      }
  }
}

// z = L_Lambda^T v for nmaps columns (k x nmaps, ld k)
__global__ void lambda_t_apply_kernel(const double *v, int64_t ldv, int nc, int k0, int lmin,
                                      const double *lamL, int nmaps, double *z, int64_t ldz) {
  const int64_t total = (int64_t)k0 * nmaps;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % k0), s = (int)(t / k0);
    const double *Li = lamL + (size_t)(l_of_mode(i, lmin) - lmin) * nc * nc;
    double in[3];
    for (int a = 0; a < nc; ++a) in[a] = v[(int64_t)a * k0 + i + (int64_t)s * ldv];
    for (int x = 0; x < nc; ++x) {
      double sacc = 0.0;
      for (int a = x; a < nc; ++a) sacc = fma(Li[a * nc + x], in[a], sacc);
      z[(int64_t)x * k0 + i + (int64_t)s * ldz] = sacc;
    }
  }
}

// lnL, chi2, logdet of one item from ||L_Kt^-1 z||^2, d^T N^-1 d, ln|N|, ln|Kt|
__global__ void batch_finish_kernel(const double *rr, const double *dnd, const double *lnN,
                                    const double *lnK, int nmaps, double *lnL, double *chi2,
                                    double *logdet) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  const double ld = *lnN + *lnK;
  if (s < nmaps) {
    const double c2 = dnd[s] - rr[s];
    if (chi2) chi2[s] = c2;
    if (lnL) lnL[s] = -0.5 * (c2 + ld);
  }
  if (s == 0 && logdet) *logdet = ld;
}

}  // namespace

void launch_form_ktilde(const double *M, int64_t ldm, int nc, int k0, int lmin,
                        const double *lamL, double *K, int64_t ldk, cudaStream_t st) {
  int64_t total = (int64_t)k0 * k0;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 152 * 32) blocks = 152 * 32;
  { form_ktilde_kernel<<<blocks, 256, 0, st>>>(M, ldm, nc, k0, lmin, lamL, K, ldk); count_launch(); }
}

void launch_lambda_t_apply(const double *v, int64_t ldv, int nc, int k0, int lmin,
                           const double *lamL, int nmaps, double *z, int64_t ldz,
                           cudaStream_t st) {
  int64_t total = (int64_t)k0 * nmaps;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 152 * 32) blocks = 152 * 32;
  if (blocks < 1) blocks = 1;
  { lambda_t_apply_kernel<<<blocks, 256, 0, st>>>(v, ldv, nc, k0, lmin, lamL, nmaps, z, ldz); count_launch(); }
}

void launch_batch_finish(const double *rr, const double *dnd, const double *lnN,
                         const double *lnK, int nmaps, double *lnL, double *chi2, double *logdet,
                         cudaStream_t st) {
  { batch_finish_kernel<<<(nmaps + 127) / 128, 128, 0, st>>>(rr, dnd, lnN, lnK, nmaps, lnL, chi2, logdet); count_launch(); }
}

}  // namespace qmlgb
