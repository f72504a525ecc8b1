// Internal declarations shared by the kernel translation units of libqmlgb.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

namespace qmlgb {

// Device status word written by kernels (first int: qml_status code,
// second: detail such as the failing Cholesky column + 1).
struct DevStatus {
  int code;
  int info;
  unsigned bar_count;   // grid barrier arrival counter
  unsigned bar_gen;     // grid barrier generation
};

// Count of kernel launches made by this library (reported by qml_launch_count).
void count_launch(int n = 1);

// Tuning table (tune.cu): named integer settings and measured tile shapes.
int64_t tune_get(const std::string &key, int64_t dflt);
bool tune_find(const std::string &key, int64_t &value);
void tune_put(const std::string &key, int64_t value);

// Iteration budget of every device-side spin wait (~1 s with 64 ns sleeps).
constexpr long long kSpinLimit = 1LL << 24;

// ---------------------------------------------------------------- ybuild --
struct YArgs {
  int has_T, has_P;
  int npix_T, npix_P;
  const double *theta_T, *phi_T, *theta_P, *phi_P;
  int lmin, lmax;
  const double *transfer_T, *transfer_P;
  void *coef;  // workspace of ybuild_coef_bytes(lmax) bytes (recurrence coefficients)
};
size_t ybuild_coef_bytes(int lmax);
void launch_ybuild(const YArgs &a, double *Y, int64_t ldy, cudaStream_t st);

// Mix the columns of Y inside every (l, m) by the lower Cholesky factor of the
// 3x3 spectrum block: G = Y L_Lambda, so that G G^T = Y Lambda Y^T.
// lamL holds per l the nc x nc lower factor (row-major, nc*nc doubles).
// cl is [6][ldcl] (ldcl <= 0: lmax + 1).
void launch_lambda_factor(const double *cl, int lmin, int lmax, int nc, const int *comps,
                          double *lamL, cudaStream_t st, int ldcl = 0);
// Per l the inverse of the nc x nc lower factor (same layout); a block that is
// not positive definite sets status QML_EINVAL (info = l + 1).
void launch_lambda_inverse(const double *lamL, int nl, int nc, int lmin, double *lamLi,
                           DevStatus *status, cudaStream_t st);
void launch_mix_lambda(double *Y, int64_t ldy, int n, int nc, int k0, int lmin, int lmax,
                       const double *lamL, cudaStream_t st);

// ----------------------------------------------------------------- dense --
// C <- alpha op(A) op(B) + beta C (float64 CUDA-core tiles); see qml_gemm.
void launch_dgemm(int ta, int tb, int64_t M, int64_t N, int64_t K, double alpha,
                  const double *A, int64_t lda, const double *B, int64_t ldb, double beta,
                  double *C, int64_t ldc, int lower, const DevStatus *status, cudaStream_t st);
// launch_dgemm without the autotuner: a measured tuning-table entry for the
// shape when one exists, else the heuristic tile.  Never allocates, creates
// events or synchronises (for callers that may not).
void launch_dgemm_fixed(int ta, int tb, int64_t M, int64_t N, int64_t K, double alpha,
                        const double *A, int64_t lda, const double *B, int64_t ldb, double beta,
                        double *C, int64_t ldc, int lower, const DevStatus *status,
                        cudaStream_t st);
// strided batch: product z uses A + z sA, B + z sB, C + z sC (no aliasing)
void launch_dgemm_batched(int ta, int tb, int64_t M, int64_t N, int64_t K, double alpha,
                          const double *A, int64_t lda, int64_t sA, const double *B,
                          int64_t ldb, int64_t sB, double beta, double *C, int64_t ldc,
                          int64_t sC, int count, const DevStatus *status, cudaStream_t st);

constexpr int kNB = 64;  // Cholesky / TRSM block size

// Factor the diagonal block of the n x n matrix A (lda) that starts at row and
// column j0 (size min(kNB, n - j0); A points at the matrix origin plus
// j0 + j0 lda), lower in place; write its inverse into Linv (ld kNB) and
// 2 sum ln L_ii into *logdet_part.
void launch_potrf_diag(double *A, int64_t lda, int64_t n, int64_t j0, double *Linv,
                       double *logdet_part, DevStatus *status, cudaStream_t st);
// Factor only (mode 2 of the diagonal kernel): S (kNB x kNB) receives the
// scaled coefficients of the row solve, S[k kNB + c] = L_ck / L_cc (c > k),
// S[c kNB + c] = 1 / L_cc, and *logdet_part 2 sum ln L_ii.  S must be
// 16-byte aligned.
void launch_potrf_diag_factor(double *A, int64_t lda, int64_t n, int64_t j0, double *S,
                              double *logdet_part, DevStatus *status, cudaStream_t st);
// B <- B L^-T (m rows, ib <= kNB columns, ld ldb) by float64 forward
// substitution from the coefficients S of launch_potrf_diag_factor; the
// result also goes to T (ld ldt).
void launch_trsm_rows(const double *S, int64_t ib, double *B, int64_t ldb, int64_t m, double *T,
                      int64_t ldt, DevStatus *status, cudaStream_t st);
// Split-precision diagonal blocks in float-float (opt-in, tuning key
// split_diag_df).  launch_potrf_diag_df
// factors the diagonal block at row / column j0 (A at the matrix origin plus
// j0 + j0 lda, n the matrix size; A is only read) and writes two slots of
// kDfSlotDoubles doubles: Lslot (the scaled float-float factor, packed, with
// its row exponents) and S (the coefficients of its row solve).
constexpr int kDfSlotDoubles = kNB * (kNB + 1) / 2 + kNB / 2;
void launch_potrf_diag_df(const double *A, int64_t lda, int64_t n, int64_t j0, double *Lslot,
                          double *S, DevStatus *status, cudaStream_t st);
// B <- B L^-T (m rows, ib <= kNB columns, ld ldb) from the coefficients S of
// launch_potrf_diag_df; the result also goes to T (ld ldt).  S must be
// 16-byte aligned.
void launch_trsm_rows_df(const double *S, int64_t ib, double *B, int64_t ldb, int64_t m,
                         double *T, int64_t ldt, DevStatus *status, cudaStream_t st);
// For every kNB block b of an n x n region L (ld lda) whose float-float
// factor slot is at Linv + b kNB^2: float64 L into the region's lower
// triangle, 2 sum ln L_ii into logdet_parts[b], and the block's inverse into
// Linv + b kNB^2 (ld kNB), replacing the slot.
void launch_trtri_blocks_df(double *L, int64_t lda, int64_t n, double *Linv,
                            double *logdet_parts, DevStatus *status, cudaStream_t st);
// Inverses of every kNB diagonal block of an existing lower factor L
// (block b at Linv + b kNB^2, ld kNB), one CTA per block.
void launch_trtri_blocks(const double *L, int64_t lda, int64_t n, double *Linv,
                         DevStatus *status, cudaStream_t st);
// X <- block diagonal of the kNB x kNB inverses Dinv (first n rows), zeros
// elsewhere in its ld x ld
void launch_place_diag_inverses(const double *Dinv, int64_t n, double *X, int64_t ld,
                                cudaStream_t st);

void launch_sum_logdet(const double *parts, int nparts, double *out, cudaStream_t st);
// Native binning: dst (nab x ncols, ld nab) <- per-bin row sums of src (na x
// ncols, ld na), bin B = rows bstart[B] .. + bcount[B] - 1 (device arrays);
// Fb (nab x nab) <- per-(bin, bin') block sums of the symmetric F (na x na).
void launch_bin_rows(const double *src, int na, int ncols, const int *bstart, const int *bcount,
                     int nab, double *dst, cudaStream_t st);
void launch_bin_fisher(const double *F, int na, const int *bstart, const int *bcount, int nab,
                       double *Fb, cudaStream_t st);
void launch_copy_lower(const double *src, int64_t lds, double *dst, int64_t ldd, int64_t n,
                       cudaStream_t st);
void launch_symmetrize_lower(double *A, int64_t lda, int64_t n, cudaStream_t st);
// A <- (A + A^T) / 2
void launch_symmetrize_avg(double *A, int64_t lda, int64_t n, cudaStream_t st);
void launch_copy_matrix(const double *src, int64_t lds, double *dst, int64_t ldd, int64_t rows,
                        int64_t cols, cudaStream_t st);
void launch_add_matrix(const double *src, int64_t lds, double *dst, int64_t ldd, int64_t rows,
                       int64_t cols, cudaStream_t st);
void launch_colnorm2(const double *X, int64_t ldx, int64_t rows, int64_t cols, double *out,
                     cudaStream_t st);
void launch_loglike_finish(const double *chi2, const double *logdet, int nmaps, double *lnL,
                           cudaStream_t st);

// ---------------------------------------------------------------- fisher --
// Block sums of W (k x k symmetric, full) over all (l >= l') pairs.
// parts: per (l,l') pair nc^4 sums of W[v i,u' j] W[u i,v' j]; diag: per l
// nc^2 sums of W[v i, u i].
void launch_fisher_blocksum(const double *W, int64_t ldw, int nc, int k0, int lmin, int lmax,
                            double *parts, double *diag, cudaStream_t st);
// Assemble F_full (na_full x na_full), t_full (na_full) from the parts.
// spec_full: canonical spectra for the fields present (component indices).
void launch_fisher_assemble(const double *parts, const double *diag, int nc, int nl,
                            int nspec_full, const int *spec_uv /* 4 ints per spectrum */,
                            double *F_full, double *t_full, cudaStream_t st);
// b = t/2 - F_full c_fid restricted; F = F_full restricted.
// cl_fid is [6][ldcl] (ldcl <= 0: lmax + 1).
void launch_fisher_select(const double *F_full, const double *t_full, const double *cl_fid,
                          int lmin, int lmax, int nspec_full, const int *full_spec_ids,
                          int nspec, const int *sel /* positions into full */, double *F,
                          double *b, cudaStream_t st, int ldcl = 0);
// y_a = 1/2 w^T E_a w for every column of w (k x nsims).
void launch_quad_y(const double *w, int64_t ldw, int nsims, int nc, int k0, int lmin, int lmax,
                   int nspec, const int *spec_uv, double *y, cudaStream_t st);
// q = y - b (columns), nsims columns of na.
void launch_sub_bias(const double *y, const double *b, int na, int nsims, double *q,
                     cudaStream_t st);

// ----------------------------------------------------------------- cross --
// Cross-QML (cross.cu): per (l >= l') block the nc^4 sums of W1 x W2
// component products; the mixing matrix Wx from them; q_x = 1/2 w1^T E_a w2;
// a general dense solve A X = B (one CTA, LU with partial pivoting).
void launch_cross_blocksum(const double *W1, const double *W2, int64_t ldw, int nc, int k0,
                           int lmin, int lmax, double *parts, cudaStream_t st);
void launch_cross_assemble(const double *parts, int nc, int nl, int nspec, const int *spec_uv,
                           double *Wx, cudaStream_t st);
void launch_quad_cross(const double *w1, const double *w2, int64_t ldw, int nsims, int nc, int k0,
                       int lmin, int lmax, int nspec, const int *spec_uv, double *q,
                       cudaStream_t st);
void launch_lu_solve(double *A, int n, double *B, int nrhs, DevStatus *status, cudaStream_t st);

// ------------------------------------------------------------------- eig --
// Symmetric eigendecomposition of F (na x na) by parallel cyclic Jacobi
// (cooperative grid, bounded barriers).  Outputs Finv = F^-1 and
// Fm12 = F^-1/2 (eigenvalues < cut * max dropped), both na x na, and
// eig_minmax[2].
cudaError_t run_fisher_eig(const double *F, int na, double *work, double *Finv, double *Fm12,
                           double *eig_minmax, DevStatus *status, cudaStream_t st);
size_t fisher_eig_work_doubles(int na);

// ---------------------------------------------------------------- batch --
// Kt = I + L_Lambda^T M L_Lambda (lower triangle), z = L_Lambda^T v, and the
// per-item lnL / chi2 / logdet (batched likelihood scan, harmonic form).
void launch_form_ktilde(const double *M, int64_t ldm, int nc, int k0, int lmin,
                        const double *lamL, double *K, int64_t ldk, cudaStream_t st);
void launch_lambda_t_apply(const double *v, int64_t ldv, int nc, int k0, int lmin,
                           const double *lamL, int nmaps, double *z, int64_t ldz,
                           cudaStream_t st);
void launch_batch_finish(const double *rr, const double *dnd, const double *lnN,
                         const double *lnK, int nmaps, double *lnL, double *chi2, double *logdet,
                         cudaStream_t st);

// ---------------------------------------------------------------- ozaki --
// Split-precision float64 GEMM (bf16 digits on tcgen05, exact FP32 chunks,
// float64 recombination); same operand conventions as launch_dgemm.  `work`
// must hold ozaki_workspace_bytes(...) bytes.  nslices = 0 picks the default.
void ozaki_choose(int64_t K, int nslices, int &S, int &beta);
size_t ozaki_workspace_bytes(int64_t M, int64_t N, int64_t K, int nslices, bool shared_operand);
// reserve_sms: SMs the persistent kernel leaves free for other work.
cudaError_t ozaki_gemm(int ta, int tb, int64_t M, int64_t N, int64_t K, double alpha,
                       const double *A, int64_t lda, const double *B, int64_t ldb, double beta_c,
                       double *C, int64_t ldc, int lower, int nslices, void *work,
                       DevStatus *status, cudaStream_t st, int reserve_sms = 0);

}  // namespace qmlgb
