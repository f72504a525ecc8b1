/*
 * qmlgb.h -- C ABI of the GB300 (sm_103a) QML / pixel-likelihood library.
 *
 * The method (Sect. 2 of the paper): data d = s + n with total covariance
 * C = S + N (Eqs. data_model, total_cov), N a general dense SPD matrix;
 * S = Y Lambda Y^T through the real harmonic matrix Y (Eqs. addition_theorem,
 * S_factored, real_ylm; App. A for spin 2, Eqs. V_spin2 .. Lambda_TEB).
 * Outputs: the Fisher matrix F (Eq. fisher, evaluated as Eq. sparse_trace on
 * W = Y^T C^-1 Y, Eq. projected_inv), quadratic estimates y and the noise bias
 * b (Eqs. q_ell, noise_bias, q_harmonic), Cl in the deconvolved, decorrelated
 * and convolved normalisations (Eqs. deconvolved, decorrelated, convolved),
 * and the Gaussian pixel log-likelihood (Eq. pixel_likelihood).
 *
 * ---------------------------------------------------------------- layout --
 * All matrices are column-major float64 with the leading dimension equal to
 * the row count unless an argument says otherwise.
 *   pixels (rows of Y, rows/cols of N and C):  T pixels, then Q pixels, then
 *       U pixels of the kept (unmasked) set, n = npix_T + 2 npix_P.
 *   modes (columns of Y):  component-major over the fields present (T, then
 *       E, then B), then l = lmin..lmax, then inside l: index 0 for m = 0,
 *       2m-1 for cos(m phi), 2m for sin(m phi).  k0 = (lmax+1)^2 - lmin^2 per
 *       component, k = ncomp * k0.  The transfer function T_l = B_l p_l of
 *       each field is folded into its columns, so Lambda holds plain Cl.
 *   spectra: index 0..5 = TT, EE, BB, TE, TB, EB.  cl arrays are [6][lmax+1].
 *   Fisher / estimate index a = (spectrum position in spec[]) * nl + (l - lmin),
 *       nl = lmax - lmin + 1, na = nspec * nl.
 *   several maps / simulations are columns: maps is n x nsims, outputs are
 *       na x nsims.
 *
 * ------------------------------------------------------ pointers, memory --
 * Every array argument may point to device memory or to host memory (pinned
 * or pageable); the library tells them apart with cudaPointerGetAttributes.
 * Host inputs are copied to device workspace on `stream`, host outputs are
 * copied back before the call returns.  Inputs are read-only and never kept;
 * the caller owns every buffer it passes.  The library allocates its
 * workspace with cudaMallocAsync on `stream` and frees it before returning,
 * except what a qml_plan keeps until qml_plan_free.
 * `stream` is a cudaStream_t passed as void*; NULL means the legacy default
 * stream.  Every call synchronises `stream` before it returns, so the status
 * covers device-side failures (not SPD, wait timeouts).
 *
 * --------------------------------------------------------------- errors --
 * Calls return a qml_status; on anything but QML_OK the outputs are
 * undefined and qml_last_error() (thread-local) holds a message.
 * No call aborts the process.
 */
#ifndef QMLGB_H
#define QMLGB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  QML_OK = 0,
  QML_EINVAL = 1,     /* bad argument (sizes, pointers, spectra, lmin) */
  QML_ENOTSPD = 2,    /* a Cholesky pivot was <= 0: matrix not positive definite */
  QML_ENOMEM = 3,     /* device workspace allocation failed */
  QML_ECUDA = 4,      /* a CUDA runtime call failed */
  QML_ETIMEOUT = 5    /* a device-side wait exceeded its iteration budget */
} qml_status;

typedef enum {
  QML_FP64 = 0,        /* every contraction in native float64 */
  QML_SPLIT_BF16 = 1   /* large contractions as exact bf16-slice products on
                          tcgen05 tensor cores (Ozaki-style splitting),
                          recombined in float64; panels, logdets stay float64 */
} qml_precision;

/* Description of one analysis (Sect. 2.1; App. A.1.3 for several fields).
 * theta_*, phi_*: colatitude / longitude (radians) of the kept pixel centres
 * of the T field and of the Q/U field (any geometry).  transfer_*: T_l for
 * l = 0..lmax.  cl_fid: fiducial spectra [6][lmax+1] defining C = S + N.
 * N: n x n SPD noise covariance (only its lower triangle is read). */
typedef struct {
  int32_t has_T, has_P;
  int32_t npix_T, npix_P;
  const double *theta_T, *phi_T;
  const double *theta_P, *phi_P;
  int32_t lmin, lmax;            /* signal band = estimation window, lmin >= 2 */
  const double *transfer_T, *transfer_P;
  int32_t nspec;                 /* number of estimated spectra, 1..6 */
  int32_t spec[6];               /* their indices (TT=0 .. EB=5), no repeats */
  const double *cl_fid;
  const double *N;
  int32_t precision;             /* qml_precision */
  int32_t nslices;               /* bf16 slices per operand for QML_SPLIT_BF16
                                    (0 = library default) */
  /* Native multipole binning (Sect. 2.4), read by qml_fisher only: 0 = one
   * bin per multipole; else nbins bins per spectrum with HOST edges
   * bin_edges[0] = lmin < bin_edges[1] < ... < bin_edges[nbins] = lmax + 1,
   * bin b = [bin_edges[b], bin_edges[b+1]).  The bin derivative
   * P_b = sum_{l in b} P_l replaces P_l: F, the noise bias and y become
   * nspec x nbins entries (spectrum-major) and the three normalisations act
   * on the binned F. */
  int32_t nbins;
  const int32_t *bin_edges;
  /* Multipole switching (Sect. 2.3.4, Eqs. C_switched and N_eff), read by
   * qml_fisher only: the signal band [lmin_sig, lmax_sig] contains the
   * inference window [lmin, lmax]; 0 means equal to the window.  The fiducial
   * signal outside the window is held fixed (in C, or in N_eff for the
   * harmonic basis) and only the window is estimated.  transfer_* and cl_fid
   * then hold lmax_sig + 1 entries per field and spectrum (cl_fid is
   * [6][lmax_sig + 1]).  2 <= lmin_sig <= lmin, lmax <= lmax_sig <= 2048. */
  int32_t lmin_sig, lmax_sig;
  /* Computation basis of qml_fisher (Sect. 2.3, Sect. 3 "Computation
   * basis"): QML_BASIS_PIXEL, QML_BASIS_HARMONIC or QML_BASIS_AUTO. */
  int32_t basis;
} qml_problem;

typedef enum {
  QML_BASIS_PIXEL = 0,     /* C = Y Lambda Y^T + N factored by Cholesky; W = X^T X */
  QML_BASIS_HARMONIC = 1,  /* SMW: M = Y^T N^-1 Y, the inner matrix Kt = I + L^T M L
                              (Lambda = L L^T per (l, m)) factored in float64, and
                              W = L^-T Kt^-1 L^T M, the subtraction-free form of
                              M - M K^-1 M (App. C.3); needs the fiducial Lambda
                              positive definite at every window multipole */
  QML_BASIS_AUTO = 2       /* the cheaper of the two by this library's cost model:
                              harmonic when 3 n^2 > 7 k^2 (n pixels, k window modes) */
} qml_basis;

typedef struct qml_plan qml_plan;   /* opaque; owned by the library */

/* Library version (major*10000 + minor*100 + patch). */
int32_t qml_version(void);

/* Number of CUDA kernels this library has launched in this process so far
 * (all threads, all devices); lets a caller count the launches of a region. */
int64_t qml_launch_count(void);

/* Thread-local message of the last failing call on this thread. */
const char *qml_last_error(void);

/* Y (n x k, leading dimension ldy >= n): the real spin-0 / spin-2 harmonic
 * matrix at the pixel centres with the transfer folded into its columns
 * (Eqs. real_ylm, spin_y_def, EB_from_spin; Wigner d^l_{m,s} by the
 * three-term recurrence in l of App. A.3 started from the half-angle closed
 * form at l = max(|m|,|s|)). */
qml_status qml_ybuild(const qml_problem *prob, double *Y, int64_t ldy, void *stream);

/* Synthetic maps d = Y a + noise (Eq. data_model with s = Y a): alm is
 * k x nsims real harmonic coefficients (same mode layout), noise is n x nsims.
 * Output maps n x nsims.  Used to draw simulations from seeded inputs. */
qml_status qml_synthesize(const qml_problem *prob, const double *alm, const double *noise,
                          int32_t nsims, double *maps, void *stream);

/* Fisher matrix F (na x na) of the spectra in prob->spec (Eq. fisher via
 * Eqs. projected_inv, fisher_harmonic, sparse_trace) on the pixel basis:
 * C = Y Lambda_fid Y^T + N, C = L L^T, X = L^-1 Y, W = X^T X, block sums.
 * If plan is not NULL, *plan receives a plan holding L, X, F, the noise bias
 * and the normalisation matrices for qml_estimate (the analogue of handing a
 * Fisher object to the spectra stage).  na = nspec (lmax - lmin + 1) must
 * not exceed 2048 (QML_EINVAL).  prob->basis selects the pixel or the
 * harmonic (SMW) evaluation (Sect. 2.3.2); both give the same F, noise bias
 * and estimates.  With a signal band wider than the window (lmin_sig,
 * lmax_sig) the out-of-window fiducial signal is part of C (pixel basis) or
 * of N_eff (harmonic basis) and F covers the window.  With prob->nbins > 0 (Sect. 2.4) F is the
 * binned Fisher matrix, na_b x na_b with na_b = nspec nbins, and the plan's
 * noise bias and normalisations are binned too.  The plan's F^-1 and F^-1/2
 * come from a Jacobi eigendecomposition of F on the device (tuning keys
 * eig_onesided, eig_mixed, eig_cluster).  Errors: QML_ENOTSPD if C is not
 * positive definite (info = the failing column) or F has an eigenvalue <= 0
 * (info = -1); QML_EINVAL for bad bin edges, a bad signal band, or (harmonic
 * basis) a fiducial block that is not positive definite. */
qml_status qml_fisher(const qml_problem *prob, double *F, qml_plan **plan, void *stream);

/* Quadratic estimates for nsims maps (n x nsims) against a plan from
 * qml_fisher: y (na x nsims, Eq. q_harmonic without the bias), b (na, noise
 * bias, Eq. noise_bias), cl_deconv = F^-1 (y - b) (Eq. deconvolved),
 * cl_decorr = F^-1/2 (y - b) with eigenvalues below 1e-12 x max dropped
 * (Eq. decorrelated), q_conv = y - b whose window matrix is F itself
 * (Eq. convolved).  Any output pointer may be NULL to skip it.  nsims = 0
 * (maps may then be NULL) only writes b.  For a binned plan every na above
 * is na_b = nspec nbins: y and b summed over each bin's multipoles. */
qml_status qml_estimate(qml_plan *plan, const double *maps, int32_t nsims,
                        double *y, double *b, double *cl_deconv, double *cl_decorr,
                        double *q_conv, void *stream);

/* Release a plan (NULL is accepted). */
void qml_plan_free(qml_plan *plan);

/* Cross-QML of two data sets observed through the same pixels (Sect. 2.2,
 * Eq. q_cross): plan1 and plan2 come from qml_fisher on problems that differ
 * only in their noise N_i (same pixels, fields, window and spectra; per-l,
 * no bins; either basis or precision).  Each data set is filtered by its own
 * C_i = S + N_i: W_i = Y^T C_i^-1 Y, w_i = Y^T C_i^-1 d_i, and
 *   Wx (na x na)     = 1/2 tr[C1^-1 P_a C2^-1 P_b]  (mode-mixing matrix,
 *                      not symmetric in general),
 *   q  (na x nsims)  = 1/2 d1^T C1^-1 P_a C2^-1 d2,
 *   cl (na x nsims)  = Wx^-1 q  (LU with partial pivoting).
 * With independent noise there is no noise bias.  maps1, maps2 are n x nsims;
 * nsims = 0 computes only Wx (maps, q, cl may then be NULL); q and cl may be
 * NULL.  Errors: QML_EINVAL for plans that do not match, QML_ENOTSPD when Wx
 * is singular. */
qml_status qml_cross(qml_plan *plan1, qml_plan *plan2, const double *maps1, const double *maps2,
                     int32_t nsims, double *Wx, double *q, double *cl, void *stream);

/* The basis a plan was computed in (QML_BASIS_PIXEL or QML_BASIS_HARMONIC;
 * -1 for NULL), e.g. to see what QML_BASIS_AUTO chose. */
int32_t qml_plan_basis(const qml_plan *plan);

/* Gaussian pixel log-likelihood of nmaps maps (n x nmaps) at spectra cl_theta
 * ([6][lmax+1]): lnL = -1/2 (d^T C^-1 d + ln|C|), constant dropped
 * (Eq. pixel_likelihood), C = Y Lambda(theta) Y^T + N factored by Cholesky,
 * ln|C| = 2 sum ln L_ii.  Outputs lnL, chi2 (length nmaps) and logdet (1);
 * any may be NULL.  prob->cl_fid and prob->spec are ignored. */
qml_status pix_loglike(const qml_problem *prob, const double *cl_theta, const double *maps,
                       int32_t nmaps, double *lnL, double *chi2, double *logdet, void *stream);

/* One mask of a batched likelihood scan: its problem (geometry, transfer,
 * noise N, precision; cl_fid and spec are ignored) and the nmaps maps
 * (n x nmaps) observed through it. */
typedef struct {
  qml_problem prob;
  const double *maps;
  int32_t nmaps;
} lnl_mask;

/* Batched pixel log-likelihood over a parameter scan with mixed masks
 * (Sect. 2.6, Eq. pixel_likelihood, evaluated through the SMW identity and the
 * determinant lemma, Eqs. smw, logdet and quad_form_smw, in the congruent form
 * Kt = I + L^T M L with M = Y^T N^-1 Y and Lambda(theta) = L L^T per (l, m),
 * App. C.3): ln|C| = ln|N| + ln|Kt|, d^T C^-1 d = d^T N^-1 d - |Lk^-1 L^T Y^T
 * N^-1 d|^2.  masks: HOST array of nmask descriptors (same fields and
 * multipole band).  With QML_SPLIT_BF16 masks the per-mask products are split
 * precision and each item's Kt is factored in float64 (tuning key
 * batch_split_kt = 1: split trailing updates for Kt as well).
 * Item i uses mask item_mask[i] (host or device, nitems) and
 * spectra item_cl + i*6*(lmax+1).  Outputs (row-major per item, leading
 * dimension ld_out >= the largest nmaps): lnL[i*ld_out + j], chi2[...] and
 * logdet[i]; any may be NULL.  The per-mask part (Cholesky of N, M, Y^T N^-1 d)
 * runs once; items are spread round-robin over internal worker streams
 * (tuning key batch_streams, default 4).  Errors: QML_EINVAL,
 * QML_ENOTSPD (N not positive definite), QML_ETIMEOUT. */
qml_status pix_loglike_batch(const lnl_mask *masks, int32_t nmask, int32_t nitems,
                             const int32_t *item_mask, const double *item_cl, int32_t ld_out,
                             double *lnL, double *chi2, double *logdet, void *stream);

/* ---- lnL emulator (the learned part; the paper has none) ---------------- *
 * An MLP surrogate of lnL(theta) over a box of d <= 8 parameters, trained on
 * exact evaluations (e.g. from pix_loglike_batch): lnL = q(x) + sigma f(x),
 * x = theta mapped to [-1, 1]^d, q a float64 least-squares polynomial (cubic
 * for d <= 5, quadratic above), f an MLP
 * with `depth` hidden GELU layers of `width` units (bf16 weights, FP32
 * accumulation on tensor cores), two independently initialised heads.  All
 * training (forward, backward, Adam) runs in this library's kernels. */
typedef struct qml_emu qml_emu;

/* New emulator over the box [lo, hi] (host arrays of ndim); seed fixes the
 * weight initialisation (counter-based generator). */
qml_status emu_create(int32_t ndim, const double *lo, const double *hi, int32_t width,
                      int32_t depth, uint64_t seed, qml_emu **emu);
/* Train on n samples: theta n x ndim (column-major), lnl n; host or device.
 * epochs passes of minibatches of `batch` (a multiple of 16) with Adam at
 * learning rate lr (constant, then a cosine decay over the last 20 % of the
 * steps).  When n >= 512 a seeded eighth of the samples is held out of
 * training; after training the two heads' disagreement and prediction error
 * on them calibrate the fallback threshold of emu_predict.  final_loss (host,
 * 2 doubles, may be NULL) receives each head's mean squared error on the
 * normalised targets of the training samples. */
qml_status emu_train(qml_emu *emu, int32_t n, const double *theta, const double *lnl,
                     int32_t epochs, int32_t batch, double lr, double *final_loss, void *stream);
/* Predict lnL at n points (theta n x ndim column-major; out n; flags n, may be
 * NULL; host or device).  flags[i] = 1 when point i lies outside the training
 * hull (the box without its outer 3 % shell in normalised coordinates) or the
 * two heads differ by more than a threshold derived from the accuracy target
 * tol (|delta lnL|): tol / 2, lowered below the smallest held-out disagreement
 * at which a held-out point (or one of lower disagreement) missed by more
 * than 0.8 tol.  The caller evaluates flagged points exactly
 * (pix_loglike_batch).  The emulator keeps its inference buffers between
 * calls (both heads' activations for up to 65536 points, about a gigabyte at
 * width 256; released by emu_free), so calls on one emulator must not overlap;
 * each call returns after its work has finished.  QML_ETIMEOUT when a
 * tensor-core wait ran out of time. */
qml_status emu_predict(qml_emu *emu, int32_t n, const double *theta, double tol, double *out,
                       int32_t *flags, void *stream);
/* The head-disagreement threshold emu_predict applies for accuracy target
 * tol (host outputs; nheld, may be NULL, receives the number of held-out
 * points inside the hull that calibrated it). */
qml_status emu_threshold(const qml_emu *emu, double tol, double *thr, int32_t *nheld);
/* Number of parameters of one head and their float32 values (host or device;
 * layout: per layer W (out x in, row-major) then b, inputs padded to 16). */
int64_t emu_param_count(const qml_emu *emu);
qml_status emu_params(qml_emu *emu, int32_t head, float *out);
/* The float64 baseline polynomial and residual scale of a trained emulator
 * (host outputs): lnL = q(x) + sigma (f_0(x) + f_1(x)) / 2 with q(x) =
 * sum_k coef[k] phi_k(x), phi_k(x) = prod_i P_{m_ki}(x_i) (Legendre
 * polynomials of the normalised coordinates) over the multi-indices m of
 * total degree <= D: by total degree t = 0..D, within a degree m_k0 from t
 * down to 0, then m_k1 from what is left down to 0, and so on, the last
 * component taking the rest.  D is the highest degree with at most 256 terms
 * and at least 16 training labels (after the held-out eighth) per term; *nfeat
 * receives the term count C(D + d, d), coef must hold 256 doubles.  Exposes
 * the model so that its inference can be checked term by term. */
qml_status emu_baseline(const qml_emu *emu, double *coef, int32_t *nfeat, double *sigma);
/* Mean squared error of head `head` on n given normalised inputs (host, n x 16
 * row-major) and targets (host, n), and its gradient (float32, host or
 * device) -- exposes the training kernels for testing. */
qml_status emu_loss_grad(qml_emu *emu, int32_t head, int32_t n, const double *x, const double *t,
                         double *loss, float *grad);
void emu_free(qml_emu *emu);

/* ---- dense building blocks (exposed for testing the kernels one by one) -- */

/* In-place lower Cholesky A = L L^T of an n x n SPD matrix (lower triangle
 * read and overwritten; the strict upper triangle is left untouched).
 * *logdet (host or device, may be NULL) receives ln|A| = 2 sum ln L_ii.
 * precision QML_FP64: float64 throughout; QML_SPLIT_BF16: 512-wide panels
 * whose diagonal blocks (and ln|A|) are factored in float64, panel solves and
 * trailing updates as split-precision products (the scheme of qml_fisher);
 * with the tuning entry split_diag_df = 1 (qml_tune_set) the 64-wide blocks
 * inside each diagonal block and their row solves run in float-float
 * (about 2^-46 per operation) instead.
 * Errors: QML_ENOTSPD with the failing column in the message. */
qml_status qml_potrf(int64_t n, double *A, int64_t lda, double *logdet, int32_t precision,
                     void *stream);

/* B <- L^-1 B for lower-triangular L (n x n, from qml_potrf) and B n x nrhs.
 * QML_SPLIT_BF16: the inverses of the 512-wide diagonal blocks are formed in
 * float64, every product with them and with the off-diagonal blocks is split. */
qml_status qml_trsm(int64_t n, int64_t nrhs, const double *L, int64_t lda, double *B,
                    int64_t ldb, int32_t precision, void *stream);

/* C <- alpha op(A) op(B) + beta C, op(X) = X or X^T (trans flags 0/1),
 * op(A) m x kk, op(B) kk x nn, C m x nn.  lower != 0 writes only the lower
 * triangle (i >= j) of a square C.  C must not overlap A or B.  m = 0 or
 * nn = 0 is a no-op; with kk = 0, C <- beta C and A, B may be NULL. */
qml_status qml_gemm(int32_t transA, int32_t transB, int64_t m, int64_t nn, int64_t kk,
                    double alpha, const double *A, int64_t lda, const double *B, int64_t ldb,
                    double beta, double *C, int64_t ldc, int32_t lower, int32_t precision,
                    void *stream);

/* ---- tuning table ----------------------------------------------------
 * One process-wide table of named integer settings; the paper has no
 * counterpart (it concerns how this library schedules its kernels, not what
 * they compute).  Keys:
 *   dgemm_autotune  1 (default) / 0: time every float64 GEMM tile candidate
 *                   the first time a small or medium product shape is met
 *                   (C at most 2^24 entries, K at most 4096, C not aliasing A
 *                   or B, the stream not capturing) and keep the fastest.  The
 *                   first call with a new shape synchronises its stream.
 *                   Every tile gives bit-identical results.
 *   dgemm:<ta>,<tb>,<lower>,<M>,<N>,<K>,<alias>  a measured tile (10 RM + RN,
 *                   tile 16 RM x 16 RN); unknown values are ignored
 *   batch_streams   worker streams of pix_loglike_batch (default 4, 1..16)
 *   batch_graphs    1 (default) / 0: pix_loglike_batch replays each worker's
 *                   per-item kernel sequence as a captured CUDA graph
 *   ozaki_stages    3 (default) / 2: depth of the split kernel's TMA ring
 *                   (stages of 64 KB; always 2 for more than 8 digits)
 *   ozaki_pairs     1 (default) / 0: the split kernel runs in clusters of two
 *                   CTAs on pairs of tile rows that share their B digit tiles
 *                   (loaded once from L2, multicast to both) / one CTA per
 *                   tile; the results are bit-identical
 *   emu_tc          1 (default) / 0: emulator inference runs its layers on
 *                   tcgen05 (width a multiple of 64, at most 256) / every
 *                   layer through the WMMA product
 *   emu_chunk       262144 (default): points per pass of emu_predict through
 *                   the network (a multiple of 128)
 *   emu_tc0         1 (default) / 0: with emu_tc, the first layer (16
 *                   inputs, widened with zeros to 64) on tcgen05 too / WMMA
 *   ozaki_band      6 (default): row pairs per band of the split kernel's
 *                   work order (column by column inside a band; 1 = row pair
 *                   after row pair); the results are the same for any value
 *   ozaki_prefetch_c 1 (default) / 0: with beta != 0 the split kernel
 *                   fetches each output tile's C into L2 when the tile
 *                   starts / reads it from memory when the tile is written
 *   eig_onesided    0 (default) / 1: the eigendecomposition of F for the
 *                   decorrelated and deconvolved normalisations by two-sided
 *                   parallel Jacobi on F (a grid barrier a rotation round) /
 *                   by one-sided Jacobi on its Cholesky factor (column pairs
 *                   moving between neighbouring CTAs, one grid barrier a
 *                   sweep; slower on this part); both within the parity
 *                   tolerances
 *   eig_mixed       1 (default) / 0: the two-sided form first runs float32
 *                   Jacobi sweeps on one thread-block cluster, rebuilds
 *                   their rotations in float64 as an orthogonal V0 and starts
 *                   the float64 sweeps from V0^T F V0 (same stopping rule,
 *                   two float64 sweeps instead of about seven at TQU Nside
 *                   16) / float64 sweeps only.  Used for padded orders
 *                   64 .. 640; other orders take the float64 sweeps only
 *   eig_cluster     16 (default) / 8: CTAs in the float32 phase's cluster
 *                   (16 falls back to 8 where the part cannot launch it)
 *   split_lookahead 1 (default) / 0: the split-precision Cholesky runs the
 *                   next panel's float64 diagonal chain on a second,
 *                   high-priority stream beside the trailing update and the
 *                   forward substitution (not while the stream is being
 *                   captured) / everything in order on the caller's stream;
 *                   the results are bit-identical
 *   split_lookahead_sms  8 (default): SMs the split kernel leaves free for
 *                   that chain while they overlap
 *   split_diag_df   0 (default) / 1: the split-precision Cholesky factors
 *                   its 64-wide diagonal blocks and their row solves in
 *                   float64 / in float-float (about 2^-46 per operation)
 *   batch_split_kt  0 (default) / 1: with QML_SPLIT_BF16 masks,
 *                   pix_loglike_batch factors each item's inner matrix Kt in
 *                   native float64 / with split-precision trailing updates
 *                   and panel products (float64 diagonal blocks and ln|Kt|)
 *   test_wait_timeout  0 (default) / 1: for testing the failure path only:
 *                   the split-precision product issues no copies and its
 *                   waits give up after 1 ms, so the call returns
 *                   QML_ETIMEOUT (no fault; the context stays usable)
 * qml_tune_set / qml_tune_get: one entry (key without white space; get
 * returns QML_EINVAL when absent).  qml_tune_table writes the table as text,
 * one "key value" line per entry, into buf (capacity cap bytes, NUL
 * included) and returns the size it needs (nothing is written when cap is
 * smaller).  qml_tune_load merges such text into the table (lines starting
 * with '#' are comments); a malformed line leaves the table unchanged. */
qml_status qml_tune_set(const char *key, int64_t value);
qml_status qml_tune_get(const char *key, int64_t *value);
int64_t qml_tune_table(char *buf, int64_t cap);
qml_status qml_tune_load(const char *text);

/* qml_potrf without any device allocation.  The paper has no counterpart:
 * this exists for callers that cannot allocate device memory (code running
 * inside a host runtime that owns all GPU memory and hands its callees
 * pre-allocated buffers, or hot loops that cannot afford the device
 * synchronisation of cudaMalloc / cudaFree).  Same kernels and result as
 * qml_potrf with precision QML_FP64, except that it never runs the float64
 * GEMM tile autotuner (which allocates): each product uses the tuning table's
 * tile for its shape when present, else the heuristic tile, which changes the
 * time only.  A (n x n, lda) and logdet (may be NULL) must be DEVICE
 * pointers.  Its scratch is a static device array sized for n <= 4096
 * (2.1 MB held on every GPU that loads the library until exit); larger n
 * returns QML_EINVAL.  All calls share that array, so calls that overlap on
 * the GPU race and must be serialised by the caller.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress).  Like
 * the other calls it reads its status back and synchronises `stream` before
 * returning. */
qml_status qml_potrf_noalloc(int64_t n, double *A, int64_t lda, double *logdet, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* QMLGB_H */
