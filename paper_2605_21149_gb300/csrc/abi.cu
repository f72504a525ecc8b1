// extern "C" entry points of libqmlgb (declared in include/qmlgb.h): argument
// validation, host/device pointer staging, workspace, and the enqueue order
// of the kernels for each call.  Everything numeric happens in the kernels of
// ybuild.cu, dense.cu, fisher.cu and eig.cu.
#include "qmlgb.h"
#include "internal.cuh"

#include <cuda_runtime.h>

#include <atomic>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <string>
#include <vector>

using namespace qmlgb;

namespace {
std::atomic<long long> g_launches{0};
}  // namespace

void qmlgb::count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

namespace {
thread_local std::string g_err;
}  // namespace

namespace qmlgb {
void set_last_error(const std::string &msg) { g_err = msg; }
}  // namespace qmlgb

namespace {

qml_status fail(qml_status s, const std::string &msg) {
  g_err = msg;
  return s;
}

void set_pool_threshold() {
  static bool done = false;
  if (done) return;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;  // keep freed blocks cached in the pool
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  done = true;
}

bool is_device_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// One ABI call: stream, workspace, staging of host buffers, device status.
struct Call {
  cudaStream_t st;
  std::vector<void *> bufs;
  struct Back {
    void *host;
    const void *dev;
    size_t bytes;
  };
  std::vector<Back> backs;
  DevStatus *status = nullptr;
  qml_status err = QML_OK;

  explicit Call(void *s) : st((cudaStream_t)s) { set_pool_threshold(); }
  ~Call() {
    for (void *p : bufs) cudaFreeAsync(p, st);
  }

  bool cuda_ok(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return true;
    if (err == QML_OK) {
      err = (e == cudaErrorMemoryAllocation) ? QML_ENOMEM : QML_ECUDA;
      g_err = std::string(what) + ": " + cudaGetErrorString(e);
    }
    return false;
  }

  template <class T>
  T *alloc(size_t count, const char *what = "workspace") {
    if (err != QML_OK) return nullptr;
    if (count == 0) count = 1;
    void *p = nullptr;
    if (!cuda_ok(cudaMallocAsync(&p, count * sizeof(T), st), what)) return nullptr;
    bufs.push_back(p);
    return (T *)p;
  }

  // device view of an input array (copied in when it lives on the host)
  template <class T>
  const T *in(const T *p, size_t count, const char *what) {
    if (err != QML_OK || !p) return p;
    if (is_device_ptr(p)) return p;
    T *d = alloc<T>(count, what);
    if (!d) return nullptr;
    cuda_ok(cudaMemcpyAsync(d, p, count * sizeof(T), cudaMemcpyHostToDevice, st), what);
    return d;
  }

  // device view of an output array (copied back at finish when on the host)
  template <class T>
  T *out(T *p, size_t count, const char *what) {
    if (err != QML_OK || !p) return p;
    if (is_device_ptr(p)) return p;
    T *d = alloc<T>(count, what);
    if (!d) return nullptr;
    backs.push_back({(void *)p, d, count * sizeof(T)});
    return d;
  }

  bool make_status() {
    status = alloc<DevStatus>(1, "status");
    if (!status) return false;
    return cuda_ok(cudaMemsetAsync(status, 0, sizeof(DevStatus), st), "status");
  }

  // copy host outputs back, wait, and translate the device status
  qml_status finish() {
    if (err != QML_OK) {
      cudaStreamSynchronize(st);
      return err;
    }
    cuda_ok(cudaGetLastError(), "kernel launch");
    for (auto &b : backs)
      cuda_ok(cudaMemcpyAsync(b.host, b.dev, b.bytes, cudaMemcpyDeviceToHost, st), "copy out");
    DevStatus hs{};
    if (status) cuda_ok(cudaMemcpyAsync(&hs, status, sizeof(hs), cudaMemcpyDeviceToHost, st), "status");
    cuda_ok(cudaStreamSynchronize(st), "synchronize");
    if (err != QML_OK) return err;
    if (hs.code == QML_ENOTSPD) {
      char buf[160];
      if (hs.info > 0)
        snprintf(buf, sizeof buf, "matrix not positive definite (Cholesky pivot at column %d)",
                 hs.info - 1);
      else if (hs.info == -2)
        snprintf(buf, sizeof buf, "cross-spectrum mixing matrix is singular");
      else
        snprintf(buf, sizeof buf, "Fisher matrix not positive definite");
      return fail(QML_ENOTSPD, buf);
    }
    if (hs.code == QML_ETIMEOUT) return fail(QML_ETIMEOUT, "device wait exceeded its budget");
    if (hs.code == QML_EINVAL)
      return fail(QML_EINVAL, "harmonic basis: the fiducial spectrum block at l = " +
                                  std::to_string(hs.info - 1) + " is not positive definite");
    if (hs.code != 0) return fail(QML_ECUDA, "device status " + std::to_string(hs.code));
    return QML_OK;
  }
};

// ------------------------------------------------------------- problems --
const int kSpecX[6] = {0, 1, 2, 0, 0, 1};
const int kSpecY[6] = {0, 1, 2, 1, 2, 2};

struct Dims {
  int nT = 0, nP = 0, n = 0;
  int nc = 0, comps[3] = {0, 0, 0}, pos[3] = {-1, -1, -1};
  int lmin = 0, lmax = 0, nl = 0, k0 = 0, k = 0;
  int nspec_full = 0, full_ids[6];
  int lsig0 = 0, lsig1 = 0;  // signal band (= the window unless switching)
};

// modes of one field over the multipoles l0 .. l1
inline int band_k0(int l0, int l1) { return (l1 + 1) * (l1 + 1) - l0 * l0; }

qml_status check_problem(const qml_problem *p, Dims &d, bool need_spec, bool need_N) {
  if (!p) return fail(QML_EINVAL, "problem is NULL");
  if (!p->has_T && !p->has_P) return fail(QML_EINVAL, "no field (has_T and has_P both 0)");
  if (p->lmin < 2) return fail(QML_EINVAL, "lmin must be >= 2");
  if (p->lmax < p->lmin || p->lmax > 2048) return fail(QML_EINVAL, "need lmin <= lmax <= 2048");
  if (p->has_T && (p->npix_T <= 0 || !p->theta_T || !p->phi_T || !p->transfer_T))
    return fail(QML_EINVAL, "T field needs npix_T > 0, theta_T, phi_T, transfer_T");
  if (p->has_P && (p->npix_P <= 0 || !p->theta_P || !p->phi_P || !p->transfer_P))
    return fail(QML_EINVAL, "P field needs npix_P > 0, theta_P, phi_P, transfer_P");
  if (p->precision != QML_FP64 && p->precision != QML_SPLIT_BF16)
    return fail(QML_EINVAL, "precision must be QML_FP64 or QML_SPLIT_BF16");
  if (p->nslices < 0 || p->nslices > 10) return fail(QML_EINVAL, "nslices must be 0..10");
  if (p->basis < QML_BASIS_PIXEL || p->basis > QML_BASIS_AUTO)
    return fail(QML_EINVAL, "basis must be QML_BASIS_PIXEL, QML_BASIS_HARMONIC or QML_BASIS_AUTO");
  d.lsig0 = p->lmin_sig > 0 ? p->lmin_sig : p->lmin;
  d.lsig1 = p->lmax_sig > 0 ? p->lmax_sig : p->lmax;
  if (p->lmin_sig < 0 || p->lmax_sig < 0 || d.lsig0 < 2 || d.lsig0 > p->lmin ||
      d.lsig1 < p->lmax || d.lsig1 > 2048)
    return fail(QML_EINVAL,
                "signal band must contain the window: 2 <= lmin_sig <= lmin <= lmax <= lmax_sig "
                "<= 2048");
  d.nT = p->has_T ? p->npix_T : 0;
  d.nP = p->has_P ? p->npix_P : 0;
  d.n = d.nT + 2 * d.nP;
  d.nc = 0;
  if (p->has_T) { d.pos[0] = d.nc; d.comps[d.nc++] = 0; }
  if (p->has_P) {
    d.pos[1] = d.nc; d.comps[d.nc++] = 1;
    d.pos[2] = d.nc; d.comps[d.nc++] = 2;
  }
  d.lmin = p->lmin;
  d.lmax = p->lmax;
  d.nl = d.lmax - d.lmin + 1;
  d.k0 = (d.lmax + 1) * (d.lmax + 1) - d.lmin * d.lmin;
  d.k = d.nc * d.k0;
  d.nspec_full = 0;
  for (int s = 0; s < 6; ++s)
    if (d.pos[kSpecX[s]] >= 0 && d.pos[kSpecY[s]] >= 0) d.full_ids[d.nspec_full++] = s;
  if (need_spec) {
    if (p->nspec < 1 || p->nspec > 6) return fail(QML_EINVAL, "nspec must be 1..6");
    bool seen[6] = {false, false, false, false, false, false};
    for (int i = 0; i < p->nspec; ++i) {
      int s = p->spec[i];
      if (s < 0 || s > 5) return fail(QML_EINVAL, "spectrum index outside 0..5");
      if (seen[s]) return fail(QML_EINVAL, "spectrum listed twice");
      seen[s] = true;
      if (d.pos[kSpecX[s]] < 0 || d.pos[kSpecY[s]] < 0)
        return fail(QML_EINVAL, "spectrum needs a field that is absent");
    }
    if (!p->cl_fid) return fail(QML_EINVAL, "cl_fid is NULL");
  }
  if (need_N && !p->N) return fail(QML_EINVAL, "N is NULL");
  return QML_OK;
}

void spec_uv(const Dims &d, int s, int *uv) {
  int x = d.pos[kSpecX[s]], y = d.pos[kSpecY[s]];
  uv[0] = x;
  uv[1] = y;
  if (x == y) {
    uv[2] = -1;
    uv[3] = -1;
  } else {
    uv[2] = y;
    uv[3] = x;
  }
}

struct Staged {
  YArgs y;
  const double *cl = nullptr, *N = nullptr;
};

// transfer arrays cover the signal band (lsig1 + 1 entries); cl holds
// 6 x cl_ld entries (cl_ld = 0: lmax + 1)
bool stage_problem(Call &c, const qml_problem *p, const Dims &d, Staged &s, const double *cl,
                   bool need_N, size_t cl_ld = 0) {
  const size_t L = (size_t)d.lsig1 + 1;
  if (cl_ld == 0) cl_ld = (size_t)d.lmax + 1;
  s.y.has_T = p->has_T;
  s.y.has_P = p->has_P;
  s.y.npix_T = d.nT;
  s.y.npix_P = d.nP;
  s.y.lmin = d.lmin;
  s.y.lmax = d.lmax;
  s.y.theta_T = p->has_T ? c.in(p->theta_T, d.nT, "theta_T") : nullptr;
  s.y.phi_T = p->has_T ? c.in(p->phi_T, d.nT, "phi_T") : nullptr;
  s.y.transfer_T = p->has_T ? c.in(p->transfer_T, L, "transfer_T") : nullptr;
  s.y.theta_P = p->has_P ? c.in(p->theta_P, d.nP, "theta_P") : nullptr;
  s.y.phi_P = p->has_P ? c.in(p->phi_P, d.nP, "phi_P") : nullptr;
  s.y.transfer_P = p->has_P ? c.in(p->transfer_P, L, "transfer_P") : nullptr;
  s.y.coef = c.alloc<unsigned char>(ybuild_coef_bytes(d.lsig1), "recurrence coefficients");
  if (cl) s.cl = c.in(cl, 6 * cl_ld, "cl");
  if (need_N) s.N = c.in(p->N, (size_t)d.n * d.n, "N");
  return c.err == QML_OK;
}

template <class T>
T *upload(Call &c, const T *host, size_t count, const char *what) {
  T *d = c.alloc<T>(count, what);
  if (d) c.cuda_ok(cudaMemcpyAsync(d, host, count * sizeof(T), cudaMemcpyHostToDevice, c.st), what);
  return d;
}

// ------------------------------------------------------ blocked drivers --
// Right-looking blocked Cholesky (block kNB): factor + invert the diagonal
// block, panel A21 <- A21 L11^-T as a product with the inverse, trailing
// A22 <- A22 - A21 A21^T on the lower triangle.
void potrf_blocked(Call &c, double *A, int64_t n, int64_t lda, double *Linv, double *ldparts,
                   double *logdet) {
  for (int64_t j = 0; j < n; j += kNB) {
    const int64_t jb = (n - j) < kNB ? (n - j) : kNB;
    double *Lb = Linv + (j / kNB) * kNB * kNB;
    launch_potrf_diag(A + j + j * lda, lda, n, j, Lb, ldparts + j / kNB, c.status, c.st);
    if (j + jb < n) {
      const int64_t m2 = n - j - jb;
      double *A21 = A + (j + jb) + j * lda;
      double *A22 = A + (j + jb) + (j + jb) * lda;
      launch_dgemm(0, 1, m2, jb, jb, 1.0, A21, lda, Lb, kNB, 0.0, A21, lda, 0, c.status, c.st);
      launch_dgemm(0, 1, m2, m2, jb, -1.0, A21, lda, A21, lda, 1.0, A22, lda, 1, c.status, c.st);
    }
  }
  if (logdet) launch_sum_logdet(ldparts, (int)((n + kNB - 1) / kNB), logdet, c.st);
}

// Blocked forward substitution B <- L^-1 B using the diagonal-block inverses.
void trsm_blocked(Call &c, const double *L, int64_t n, int64_t lda, const double *Linv,
                  double *B, int64_t nrhs, int64_t ldb) {
  for (int64_t j = 0; j < n; j += kNB) {
    const int64_t jb = (n - j) < kNB ? (n - j) : kNB;
    const double *Lb = Linv + (j / kNB) * kNB * kNB;
    launch_dgemm(0, 0, jb, nrhs, jb, 1.0, Lb, kNB, B + j, ldb, 0.0, B + j, ldb, 0, c.status, c.st);
    if (j + jb < n)
      launch_dgemm(0, 0, n - j - jb, nrhs, jb, -1.0, L + (j + jb) + j * lda, lda, B + j, ldb, 1.0,
                   B + j + jb, ldb, 0, c.status, c.st);
  }
}

// B <- L^-T B (backward substitution with the diagonal-block inverses):
// from the last block up, B_j <- Linv_j^T B_j, then B_0..j-1 -= L_j,0..j-1^T B_j.
void trsm_blocked_t(Call &c, const double *L, int64_t n, int64_t lda, const double *Linv,
                    double *B, int64_t nrhs, int64_t ldb) {
  const int64_t nb = (n + kNB - 1) / kNB;
  for (int64_t bi = nb - 1; bi >= 0; --bi) {
    const int64_t j = bi * kNB;
    const int64_t jb = (n - j) < kNB ? (n - j) : kNB;
    const double *Lb = Linv + bi * kNB * kNB;
    launch_dgemm(1, 0, jb, nrhs, jb, 1.0, Lb, kNB, B + j, ldb, 0.0, B + j, ldb, 0, c.status, c.st);
    if (j > 0)
      launch_dgemm(1, 0, j, nrhs, jb, -1.0, L + j, lda, B + j, ldb, 1.0, B, ldb, 0, c.status, c.st);
  }
}

// X <- L^-1 for a lower-triangular jb x jb block L (ld lda) by recursive
// doubling, from the inverses Linv of its kNB-wide diagonal blocks:
//   [[P, 0], [Q, R]]^-1 = [[P^-1, 0], [-R^-1 Q P^-1, R^-1]].
// The kNB-block inverses go on the diagonal of X (zeros elsewhere); then for
// b = kNB, 2 kNB, ... every pair of b-blocks gets T = Q P^-1 and its lower
// left block -R^-1 T, each one batched product over the pairs (a last pair
// whose second block is shorter than b gets its own two products).  log2 of
// the block count steps instead of one per block row; T (scratch) holds
// (kNBS/2)^2 doubles.  On stream st; with fixed the float64 products skip
// the tile autotuner (which synchronises), as work on a second stream must.
void trinv_doubling(Call &c, const double *L, int64_t jb, int64_t lda, const double *Linv,
                    double *X, int64_t ldx, double *T, cudaStream_t st, bool fixed) {
  auto gemm = fixed ? launch_dgemm_fixed : launch_dgemm;
  launch_place_diag_inverses(Linv, jb, X, ldx, st);
  for (int64_t b = kNB; b < jb; b *= 2) {
    const int64_t full = jb / (2 * b);  // pairs with both blocks b long
    if (full > 0) {
      const int64_t sL = 2 * b + 2 * b * lda, sX = 2 * b + 2 * b * ldx;
      launch_dgemm_batched(0, 0, b, b, b, 1.0, L + b, lda, sL, X, ldx, sX, 0.0, T, b, b * b,
                           (int)full, c.status, st);
      launch_dgemm_batched(0, 0, b, b, b, -1.0, X + b + b * ldx, ldx, sX, T, b, b * b, 0.0, X + b,
                           ldx, sX, (int)full, c.status, st);
    }
    const int64_t r0 = full * 2 * b, b2 = jb - r0 - b;  // a last pair with a short R
    if (b2 > 0) {
      gemm(0, 0, b2, b, b, 1.0, L + (r0 + b) + r0 * lda, lda, X + r0 + r0 * ldx, ldx, 0.0, T, b2,
           0, c.status, st);
      gemm(0, 0, b2, b, b2, -1.0, X + (r0 + b) + (r0 + b) * ldx, ldx, T, b2, 0.0,
           X + (r0 + b) + r0 * ldx, ldx, 0, c.status, st);
    }
  }
}

// C = Y Lambda(cl) Y^T + N (lower triangle) from a scratch Y buffer (n x k),
// which is left holding G = Y L_Lambda.
void build_C(Call &c, const Staged &s, const Dims &d, double *Y, double *C) {
  double *lamL = c.alloc<double>((size_t)d.nl * d.nc * d.nc, "lambda factors");
  if (!lamL) return;
  launch_ybuild(s.y, Y, d.n, c.st);
  launch_lambda_factor(s.cl, d.lmin, d.lmax, d.nc, d.comps, lamL, c.st);
  launch_mix_lambda(Y, d.n, d.n, d.nc, d.k0, d.lmin, d.lmax, lamL, c.st);
  launch_copy_lower(s.N, d.n, C, d.n, d.n, c.st);
  launch_dgemm(0, 1, d.n, d.n, d.k, 1.0, Y, d.n, Y, d.n, 1.0, C, d.n, 1, c.status, c.st);
}

// ------------------------------------------------ split-precision drivers --
// Panels of kNBS columns: the diagonal block is factored in float64 (64-wide
// blocks), its explicit inverse formed by a float64 solve of the identity, and
// the panel solve and trailing update run as split-precision products with
// K = kNBS.
constexpr int64_t kNBS = 512;

struct Split {
  Call *c;
  int nslices;
  // SMs the split kernel leaves free (for float64 work on a second stream)
  int reserve_sms = 0;
  void *ws = nullptr;
  size_t ws_bytes = 0;
  double *tinv = nullptr;  // (kNBS/2)^2 scratch of the block-inverse doubling
  // the doubling scratch, allocated on first use unless preset
  double *tinv_scratch() {
    if (!tinv) tinv = c->alloc<double>((size_t)(kNBS / 2) * (kNBS / 2), "inverse scratch");
    return tinv;
  }
  // use a caller-provided workspace (no allocation later)
  void preset(void *p, size_t bytes) {
    ws = p;
    ws_bytes = bytes;
  }
  // make sure the digit workspace holds a product of this shape
  bool reserve(int64_t M, int64_t N, int64_t K, bool shared) {
    size_t need = ozaki_workspace_bytes(M, N, K, nslices, shared);
    if (need <= ws_bytes) return true;
    ws = c->alloc<unsigned char>(need, "split workspace");
    ws_bytes = ws ? need : 0;
    return ws != nullptr;
  }
  void gemm(int ta, int tb, int64_t M, int64_t N, int64_t K, double alpha, const double *A,
            int64_t lda, const double *B, int64_t ldb, double beta, double *C, int64_t ldc,
            int lower) {
    if (c->err != QML_OK || M <= 0 || N <= 0) return;
    const bool shared = (A == B && lda == ldb && ta != tb && M == N);
    if (!reserve(M, N, K, shared)) return;
    c->cuda_ok(ozaki_gemm(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, lower, nslices,
                          ws, c->status, c->st, reserve_sms),
               "split-precision gemm");
  }
};

// The float64 part of the split Cholesky for the panel of columns j .. j + jb
// of A (its diagonal block already updated by every earlier panel), on stream
// st: the diagonal block factored 64 columns at a time (the 64-block factor
// leaves the coefficients of its row solve in the slot of its inverse; the
// rows below are solved by forward substitution, in place and into T (m2 x 64
// <= (kNBS - kNB) x kNB), whose product with itself updates the rest, out of
// place so it can take small tiles), then the inverses of the 64-blocks (one
// launch, a CTA each) and the explicit inverse of the whole block into
// LinvB's slot (float64, recursive doubling).  With split_diag_df the
// 64-blocks and their row solves run in float-float instead (about 2^-46 per
// operation; the factor goes to the inverse slot, the coefficients to S behind
// T's panel part).  fixed: float64 products without the tile autotuner.
void panel_chain(Call &c, Split &sp, double *A, int64_t lda, int64_t j, int64_t jb,
                 double *Linv64, double *LinvB, double *ldparts, bool dfdiag, cudaStream_t st,
                 bool fixed) {
  auto gemm = fixed ? launch_dgemm_fixed : launch_dgemm;
  double *Ajj = A + j + j * lda;
  double *T = sp.tinv_scratch();  // (kNBS/2)^2 doubles: the panel block below, then the doubling
  if (!T) return;
  double *S = T + (int64_t)(kNBS - kNB) * kNB;
  for (int64_t i = 0; i < jb; i += kNB) {
    const int64_t ib = (jb - i) < kNB ? (jb - i) : kNB;
    double *Lb = Linv64 + ((j + i) / kNB) * kNB * kNB;
    double *Ab = A + (j + i) + (j + i) * lda;
    if (dfdiag)
      launch_potrf_diag_df(Ab, lda, j + jb, j + i, Lb, S, c.status, st);
    else
      launch_potrf_diag_factor(Ab, lda, j + jb, j + i, Lb, ldparts + (j + i) / kNB, c.status, st);
    if (i + ib < jb) {
      const int64_t m2 = jb - i - ib;
      double *A21 = Ajj + (i + ib) + i * lda;
      double *A22 = Ajj + (i + ib) + (i + ib) * lda;
      if (dfdiag)
        launch_trsm_rows_df(S, ib, A21, lda, m2, T, m2, c.status, st);
      else
        launch_trsm_rows(Lb, ib, A21, lda, m2, T, m2, c.status, st);
      gemm(0, 1, m2, m2, ib, -1.0, T, m2, T, m2, 1.0, A22, lda, 1, c.status, st);
    }
  }
  if (dfdiag)
    launch_trtri_blocks_df(Ajj, lda, jb, Linv64 + (j / kNB) * kNB * kNB, ldparts + j / kNB,
                           c.status, st);
  else
    launch_trtri_blocks(Ajj, lda, jb, Linv64 + (j / kNB) * kNB * kNB, c.status, st);
  trinv_doubling(c, Ajj, jb, lda, Linv64 + (j / kNB) * kNB * kNB, LinvB + (j / kNBS) * kNBS * kNBS,
                 kNBS, T, st, fixed);
}

// Cholesky A = L L^T (lower, in place).  Linv64: inverses of the 64-blocks
// (n/64 blocks of 64x64); LinvB: explicit inverses of the kNBS diagonal blocks
// (ceil(n/kNBS) blocks of kNBS x kNBS, ld kNBS).  Panels of kNBS columns: the
// float64 chain of the diagonal block (panel_chain), then the panel solve
// A21 <- A21 L_jj^-T (a product with the explicit inverse) and the trailing
// update A22 <- A22 - A21 A21^T (lower) as split-precision products.  With a
// right-hand side B (n x nrhs, ld ldb) the forward substitution B <- L^-1 B
// runs panel by panel in the same loop: B_j <- L_jj^-1 B_j and
// B_below <- B_below - A21 B_j as soon as panel j is final.
//
// Lookahead (tuning key split_lookahead, default 1; off while the stream is
// being captured): the trailing update is split into the next panel's columns
// and the rest; right after the first part, the next panel's float64 chain
// starts on a second, high-priority stream, while the main stream runs the
// rest of the trailing update and panel j's substitution on B with
// split_lookahead_sms SMs (default 8) left free for the chain.  The float64
// chain (about 0.8 ms a panel at n = 5952) then hides behind split products.
// Every output is the same product as without lookahead (the split product
// of an element depends only on its own row and column), so the results are
// bit-identical.
void potrf_split(Call &c, Split &sp, double *A, int64_t n, int64_t lda, double *Linv64,
                 double *LinvB, double *ldparts, double *logdet, double *B = nullptr,
                 int64_t nrhs = 0, int64_t ldb = 0) {
  const bool dfdiag = tune_get("split_diag_df", 0) != 0;
  if (!sp.tinv_scratch()) return;  // allocated on the main stream before any use
  bool look = tune_get("split_lookahead", 1) != 0 && n > kNBS;
  if (look) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(c.st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
      look = false;
  }
  cudaStream_t s2 = nullptr;
  cudaEvent_t e_next = nullptr, e_diag = nullptr;
  if (look) {
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    look = cudaStreamCreateWithPriority(&s2, cudaStreamNonBlocking, hi) == cudaSuccess &&
           cudaEventCreateWithFlags(&e_next, cudaEventDisableTiming) == cudaSuccess &&
           cudaEventCreateWithFlags(&e_diag, cudaEventDisableTiming) == cudaSuccess;
  }
  const int reserve = look ? (int)tune_get("split_lookahead_sms", 8) : 0;
  panel_chain(c, sp, A, lda, 0, n < kNBS ? n : kNBS, Linv64, LinvB, ldparts, dfdiag, c.st, false);
  for (int64_t j = 0; j < n && c.err == QML_OK; j += kNBS) {
    const int64_t jb = (n - j) < kNBS ? (n - j) : kNBS;
    const double *Xinv = LinvB + (j / kNBS) * kNBS * kNBS;
    // panel j's chain ran on the second stream
    if (look && j > 0) c.cuda_ok(cudaStreamWaitEvent(c.st, e_diag, 0), "lookahead");
    double *A21 = A + (j + jb) + j * lda;
    const int64_t m2 = n - j - jb;
    if (m2 > 0) {
      double *A22 = A + (j + jb) + (j + jb) * lda;
      const int64_t jb2 = m2 < kNBS ? m2 : kNBS;
      // panel: A21 <- A21 L_jj^-T
      sp.gemm(0, 1, m2, jb, jb, 1.0, A21, lda, Xinv, kNBS, 0.0, A21, lda, 0);
      if (look) {
        // the next panel's columns first: its diagonal block (lower) and the
        // rows below it; then its chain starts on the second stream
        sp.gemm(0, 1, jb2, jb2, jb, -1.0, A21, lda, A21, lda, 1.0, A22, lda, 1);
        if (m2 > jb2)
          sp.gemm(0, 1, m2 - jb2, jb2, jb, -1.0, A21 + jb2, lda, A21, lda, 1.0, A22 + jb2, lda,
                  0);
        c.cuda_ok(cudaEventRecord(e_next, c.st), "lookahead");
        c.cuda_ok(cudaStreamWaitEvent(s2, e_next, 0), "lookahead");
        panel_chain(c, sp, A, lda, j + jb, jb2, Linv64, LinvB, ldparts, dfdiag, s2, true);
        c.cuda_ok(cudaEventRecord(e_diag, s2), "lookahead");
        sp.reserve_sms = reserve;
        if (m2 > jb2)
          sp.gemm(0, 1, m2 - jb2, m2 - jb2, jb, -1.0, A21 + jb2, lda, A21 + jb2, lda, 1.0,
                  A22 + jb2 + jb2 * lda, lda, 1);
      } else {
        sp.gemm(0, 1, m2, m2, jb, -1.0, A21, lda, A21, lda, 1.0, A22, lda, 1);
      }
    }
    if (B) {
      // forward substitution, panel j: B_j <- L_jj^-1 B_j ; B_below -= A21 B_j
      sp.gemm(0, 0, jb, nrhs, jb, 1.0, Xinv, kNBS, B + j, ldb, 0.0, B + j, ldb, 0);
      if (m2 > 0)
        sp.gemm(0, 0, m2, nrhs, jb, -1.0, A21, lda, B + j, ldb, 1.0, B + j + jb, ldb, 0);
    }
    sp.reserve_sms = 0;
    if (!look && m2 > 0)
      panel_chain(c, sp, A, lda, j + jb, m2 < kNBS ? m2 : kNBS, Linv64, LinvB, ldparts, dfdiag,
                  c.st, false);
  }
  if (look) {
    // nothing of the second stream outlives this call: the main stream waits
    // for all of it (the last chain was waited for already; this covers an
    // early exit on error)
    if (cudaEventRecord(e_diag, s2) == cudaSuccess) cudaStreamWaitEvent(c.st, e_diag, 0);
    cudaEventDestroy(e_next);
    cudaEventDestroy(e_diag);
    cudaStreamDestroy(s2);
  }
  if (logdet) launch_sum_logdet(ldparts, (int)((n + kNB - 1) / kNB), logdet, c.st);
}

// B <- L^-1 B with the explicit kNBS block inverses (split products).
void trsm_split(Call &c, Split &sp, const double *L, int64_t n, int64_t lda, const double *LinvB,
                double *B, int64_t nrhs, int64_t ldb) {
  for (int64_t j = 0; j < n; j += kNBS) {
    const int64_t jb = (n - j) < kNBS ? (n - j) : kNBS;
    const double *Xinv = LinvB + (j / kNBS) * kNBS * kNBS;
    sp.gemm(0, 0, jb, nrhs, jb, 1.0, Xinv, kNBS, B + j, ldb, 0.0, B + j, ldb, 0);
    if (j + jb < n)
      sp.gemm(0, 0, n - j - jb, nrhs, jb, -1.0, L + (j + jb) + j * lda, lda, B + j, ldb, 1.0,
              B + j + jb, ldb, 0);
  }
}

// C = Y Lambda Y^T + N with the split product for G G^T.
void build_C_split(Call &c, Split &sp, const Staged &s, const Dims &d, double *Y, double *C) {
  double *lamL = c.alloc<double>((size_t)d.nl * d.nc * d.nc, "lambda factors");
  if (!lamL) return;
  launch_ybuild(s.y, Y, d.n, c.st);
  launch_lambda_factor(s.cl, d.lmin, d.lmax, d.nc, d.comps, lamL, c.st);
  launch_mix_lambda(Y, d.n, d.n, d.nc, d.k0, d.lmin, d.lmax, lamL, c.st);
  launch_copy_lower(s.N, d.n, C, d.n, d.n, c.st);
  sp.gemm(0, 1, d.n, d.n, d.k, 1.0, Y, d.n, Y, d.n, 1.0, C, d.n, 1);
}

// C += Y_b Lambda_b Y_b^T (lower triangle) for the multipoles l0 .. l1 of the
// fiducial spectra s.cl ([6][ldcl]): Y_b built into the scratch Y (n x
// nc band_k0(l0, l1)), mixed by the per-(l, m) factors of Lambda, and one
// lower-triangle product (split precision when spl is given).  The pixel-basis
// C over a signal band wider than the window, and the fixed-signal terms of
// N_eff (Eq. N_eff), are sums of such bands.
void add_band_signal(Call &c, Split *spl, const Staged &s, const Dims &d, int l0, int l1,
                     int ldcl, double *Y, double *C) {
  const int k0b = band_k0(l0, l1), kb = d.nc * k0b;
  double *lamL = c.alloc<double>((size_t)(l1 - l0 + 1) * d.nc * d.nc, "lambda factors");
  if (!lamL) return;
  YArgs ya = s.y;
  ya.lmin = l0;
  ya.lmax = l1;
  launch_ybuild(ya, Y, d.n, c.st);
  launch_lambda_factor(s.cl, l0, l1, d.nc, d.comps, lamL, c.st, ldcl);
  launch_mix_lambda(Y, d.n, d.n, d.nc, k0b, l0, l1, lamL, c.st);
  if (spl)
    spl->gemm(0, 1, d.n, d.n, kb, 1.0, Y, d.n, Y, d.n, 1.0, C, d.n, 1);
  else
    launch_dgemm(0, 1, d.n, d.n, kb, 1.0, Y, d.n, Y, d.n, 1.0, C, d.n, 1, c.status, c.st);
}

}  // namespace

// ======================================================================
// Bin edges of a problem (Sect. 2.4): empty for one bin per multipole.
qml_status check_bins(const qml_problem *p, const Dims &d, std::vector<int> &edges) {
  edges.clear();
  if (p->nbins < 0) return fail(QML_EINVAL, "nbins must be >= 0");
  if (p->nbins == 0) return QML_OK;
  if (!p->bin_edges) return fail(QML_EINVAL, "nbins > 0 needs bin_edges");
  if (p->nbins > d.nl) return fail(QML_EINVAL, "more bins than multipoles");
  edges.assign(p->bin_edges, p->bin_edges + p->nbins + 1);
  if (edges.front() != d.lmin || edges.back() != d.lmax + 1)
    return fail(QML_EINVAL, "bin_edges must run from lmin to lmax + 1");
  for (int b = 0; b < p->nbins; ++b)
    if (edges[b + 1] <= edges[b]) return fail(QML_EINVAL, "bin_edges must increase strictly");
  return QML_OK;
}

struct qml_plan {
  Dims d;
  int nspec = 0;
  int spec[6];
  int na = 0;
  cudaStream_t st = nullptr;
  std::vector<void *> mem;
  double *L = nullptr, *Linv = nullptr, *X = nullptr;
  double *LinvB = nullptr;  // kNBS-block inverses (split precision)
  bool split = false;
  int nslices = 0;
  double *F = nullptr, *b = nullptr, *Finv = nullptr, *Fm12 = nullptr;
  int *uv = nullptr;
  // native binning (Sect. 2.4): na = nspec x bins is the size of F and of
  // every estimate; na_l = nspec x multipoles that of the per-l sums, which
  // the device arrays bstart / bcount (na entries) gather into bins
  int na_l = 0;
  bool binned = false;
  int *bstart = nullptr, *bcount = nullptr;
  // harmonic basis (Sect. 2.3.2): L holds the factor of N (or N_eff), X holds
  // U = L_N^-1 Y; LK the float64 factor of Kt = I + L_Lambda^T M L_Lambda with
  // its 64-block inverses, lamL / lamLi the per-l factors of Lambda and their
  // inverses
  bool harmonic = false;
  double *LK = nullptr, *LKinv = nullptr, *lamL = nullptr, *lamLi = nullptr;
};

namespace {

// Harmonic basis: W (k x k) holds M = Y^T N^-1 Y on entry and W = M (I +
// Lambda M)^-1 = L_Lambda^-T Kt^-1 L_Lambda^T M (Eq. smw_stable) on return;
// T is k x k scratch.
void harmonic_W_from_M(Call &c, const qml_plan *plan, double *W, double *T) {
  const Dims &d = plan->d;
  launch_lambda_t_apply(W, d.k, d.nc, d.k0, d.lmin, plan->lamL, d.k, T, d.k, c.st);
  trsm_blocked(c, plan->LK, d.k, d.k, plan->LKinv, T, d.k, d.k);
  trsm_blocked_t(c, plan->LK, d.k, d.k, plan->LKinv, T, d.k, d.k);
  launch_lambda_t_apply(T, d.k, d.nc, d.k0, d.lmin, plan->lamLi, d.k, W, d.k, c.st);
  launch_symmetrize_avg(W, d.k, d.k, c.st);
}

// W = Y^T C^-1 Y (symmetric, k x k) from a plan's factors: X^T X (pixel
// basis), or M = U^T U followed by the harmonic step above; T is k x k
// scratch for the harmonic basis.
void plan_W(Call &c, const qml_plan *plan, double *W, double *T) {
  const Dims &d = plan->d;
  if (plan->split) {
    Split spl{&c, plan->nslices};
    spl.gemm(1, 0, d.k, d.k, d.n, 1.0, plan->X, d.n, plan->X, d.n, 0.0, W, d.k, 1);
  } else {
    launch_dgemm(1, 0, d.k, d.k, d.n, 1.0, plan->X, d.n, plan->X, d.n, 0.0, W, d.k, 1, c.status,
                 c.st);
  }
  launch_symmetrize_lower(W, d.k, d.k, c.st);
  if (plan->harmonic) harmonic_W_from_M(c, plan, W, T);
}

// w = Y^T C^-1 d for nsims maps D (device, n x nsims) through a plan; U is
// n x nsims scratch (overwritten).  Pixel basis: w = X^T (L^-1 d).  Harmonic
// basis: v = U_Y^T (L_N^-1 d) = Y^T N^-1 d, then w = (I + M Lambda)^-1 v =
// L_Lambda^-T Kt^-1 L_Lambda^T v (Eq. smw_stable_data).
void weighted_data(Call &c, const qml_plan *plan, const double *D, int nsims, double *U,
                   double *w) {
  const Dims &d = plan->d;
  double *wv = plan->harmonic ? c.alloc<double>((size_t)d.k * nsims, "v") : w;
  if (c.err != QML_OK) return;
  launch_copy_matrix(D, d.n, U, d.n, d.n, nsims, c.st);
  if (plan->split) {
    Split spl{&c, plan->nslices};
    trsm_split(c, spl, plan->L, d.n, d.n, plan->LinvB, U, nsims, d.n);
    spl.gemm(1, 0, d.k, nsims, d.n, 1.0, plan->X, d.n, U, d.n, 0.0, wv, d.k, 0);
  } else {
    trsm_blocked(c, plan->L, d.n, d.n, plan->Linv, U, nsims, d.n);
    launch_dgemm(1, 0, d.k, nsims, d.n, 1.0, plan->X, d.n, U, d.n, 0.0, wv, d.k, 0, c.status,
                 c.st);
  }
  if (plan->harmonic) {
    launch_lambda_t_apply(wv, d.k, d.nc, d.k0, d.lmin, plan->lamL, nsims, wv, d.k, c.st);
    trsm_blocked(c, plan->LK, d.k, d.k, plan->LKinv, wv, nsims, d.k);
    trsm_blocked_t(c, plan->LK, d.k, d.k, plan->LKinv, wv, nsims, d.k);
    launch_lambda_t_apply(wv, d.k, d.nc, d.k0, d.lmin, plan->lamLi, nsims, w, d.k, c.st);
  }
}

}  // namespace

extern "C" {

int32_t qml_version(void) { return 100; }

int64_t qml_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

const char *qml_last_error(void) { return g_err.c_str(); }

qml_status qml_ybuild(const qml_problem *prob, double *Y, int64_t ldy, void *stream) {
  Dims d;
  qml_status s = check_problem(prob, d, false, false);
  if (s != QML_OK) return s;
  if (!Y || ldy < d.n) return fail(QML_EINVAL, "Y is NULL or ldy < n");
  Call c(stream);
  Staged sp;
  if (!stage_problem(c, prob, d, sp, nullptr, false)) return c.finish();
  double *Yd = c.out(Y, (size_t)ldy * d.k, "Y");
  if (!Yd) return c.finish();
  launch_ybuild(sp.y, Yd, ldy, c.st);
  return c.finish();
}

qml_status qml_synthesize(const qml_problem *prob, const double *alm, const double *noise,
                          int32_t nsims, double *maps, void *stream) {
  Dims d;
  qml_status s = check_problem(prob, d, false, false);
  if (s != QML_OK) return s;
  if (nsims < 0 || !alm || !noise || !maps) return fail(QML_EINVAL, "bad synthesize arguments");
  if (nsims == 0) return QML_OK;
  Call c(stream);
  Staged sp;
  if (!stage_problem(c, prob, d, sp, nullptr, false)) return c.finish();
  const double *a = c.in(alm, (size_t)d.k * nsims, "alm");
  const double *nz = c.in(noise, (size_t)d.n * nsims, "noise");
  double *out = c.out(maps, (size_t)d.n * nsims, "maps");
  double *Y = c.alloc<double>((size_t)d.n * d.k, "Y");
  if (!c.make_status() || !Y || !out) return c.finish();
  launch_ybuild(sp.y, Y, d.n, c.st);
  launch_copy_matrix(nz, d.n, out, d.n, d.n, nsims, c.st);
  launch_dgemm(0, 0, d.n, nsims, d.k, 1.0, Y, d.n, a, d.k, 1.0, out, d.n, 0, c.status, c.st);
  return c.finish();
}

int32_t qml_plan_basis(const qml_plan *plan) {
  if (!plan) return -1;
  return plan->harmonic ? QML_BASIS_HARMONIC : QML_BASIS_PIXEL;
}

void qml_plan_free(qml_plan *plan) {
  if (!plan) return;
  for (void *p : plan->mem) cudaFreeAsync(p, plan->st);
  cudaStreamSynchronize(plan->st);
  delete plan;
}

qml_status qml_fisher(const qml_problem *prob, double *F, qml_plan **plan_out, void *stream) {
  Dims d;
  qml_status s = check_problem(prob, d, true, true);
  if (s != QML_OK) return s;
  if (!F) return fail(QML_EINVAL, "F is NULL");
  if (plan_out) *plan_out = nullptr;
  std::vector<int> edges;
  s = check_bins(prob, d, edges);
  if (s != QML_OK) return s;
  const bool binned = !edges.empty();
  const int na_l = prob->nspec * d.nl;  // per-multipole entries
  const int nb = binned ? prob->nbins : d.nl;
  const int na = prob->nspec * nb;      // entries of F and of the estimates
  const int naf = d.nspec_full * d.nl;
  if (na_l + (na_l & 1) > 2048)
    return fail(QML_EINVAL, "Fisher matrix larger than 2048 (nspec x (lmax - lmin + 1))");
  Call c(stream);
  Staged sp;
  if (!stage_problem(c, prob, d, sp, prob->cl_fid, true, (size_t)d.lsig1 + 1))
    return c.finish();
  double *Fout = c.out(F, (size_t)na * na, "F");
  if (!c.make_status()) return c.finish();

  // plan-owned buffers are allocated outside the per-call list
  qml_plan *plan = new qml_plan();
  plan->d = d;
  plan->nspec = prob->nspec;
  for (int i = 0; i < 6; ++i) plan->spec[i] = prob->spec[i];
  plan->na = na;
  plan->na_l = na_l;
  plan->binned = binned;
  plan->st = c.st;
  auto palloc = [&](size_t count) -> double * {
    void *p = nullptr;
    if (c.err != QML_OK) return nullptr;
    if (!c.cuda_ok(cudaMallocAsync(&p, count * sizeof(double), c.st), "plan buffers")) return nullptr;
    plan->mem.push_back(p);
    return (double *)p;
  };
  const int64_t nblocks = (d.n + kNB - 1) / kNB;
  plan->split = (prob->precision == QML_SPLIT_BF16);
  plan->nslices = prob->nslices;
  // basis: the harmonic (SMW) route costs n^3/3 + n^2 k + n k^2 + 7 k^3 / 3
  // flops, the pixel route n^3/3 + n^2 k_sig + n^2 k + n k^2 (the fixed-signal
  // terms, n^2 (k_sig - k), are common): harmonic is cheaper when 3 n^2 > 7 k^2
  int basis = prob->basis;
  if (basis == QML_BASIS_AUTO)
    basis = (3.0 * (double)d.n * d.n > 7.0 * (double)d.k * d.k) ? QML_BASIS_HARMONIC
                                                                  : QML_BASIS_PIXEL;
  plan->harmonic = (basis == QML_BASIS_HARMONIC);
  const int ldcl = d.lsig1 + 1;
  plan->L = palloc((size_t)d.n * d.n);
  plan->Linv = palloc((size_t)nblocks * kNB * kNB);
  if (plan->split) plan->LinvB = palloc((size_t)((d.n + kNBS - 1) / kNBS) * kNBS * kNBS);
  plan->X = palloc((size_t)d.n * d.k);
  if (plan->harmonic) {
    plan->LK = palloc((size_t)d.k * d.k);
    plan->LKinv = palloc((size_t)((d.k + kNB - 1) / kNB) * kNB * kNB);
    plan->lamL = palloc((size_t)d.nl * d.nc * d.nc);
    plan->lamLi = palloc((size_t)d.nl * d.nc * d.nc);
  }
  plan->F = palloc((size_t)na * na);
  plan->b = palloc(na);
  plan->Finv = palloc((size_t)na * na);
  plan->Fm12 = palloc((size_t)na * na);
  {
    void *p = nullptr;
    if (c.err == QML_OK && c.cuda_ok(cudaMallocAsync(&p, 4 * 6 * sizeof(int), c.st), "plan"))
      plan->mem.push_back(p);
    plan->uv = (int *)p;
  }
  std::vector<int> h_bins;  // bstart then bcount, kept alive until the copy completes
  if (binned) {
    h_bins.resize(2 * (size_t)na);
    for (int sp = 0; sp < prob->nspec; ++sp)
      for (int bb = 0; bb < nb; ++bb) {
        h_bins[sp * nb + bb] = sp * d.nl + (edges[bb] - d.lmin);
        h_bins[na + sp * nb + bb] = edges[bb + 1] - edges[bb];
      }
    void *p = nullptr;
    if (c.err == QML_OK &&
        c.cuda_ok(cudaMallocAsync(&p, h_bins.size() * sizeof(int), c.st), "plan bins")) {
      plan->mem.push_back(p);
      plan->bstart = (int *)p;
      plan->bcount = plan->bstart + na;
      c.cuda_ok(cudaMemcpyAsync(p, h_bins.data(), h_bins.size() * sizeof(int),
                                cudaMemcpyHostToDevice, c.st),
                "plan bins");
    }
  }
  // per-multipole F and noise bias (the plan's own when not binned)
  double *Fl = binned ? c.alloc<double>((size_t)na_l * na_l, "per-l F") : plan->F;
  double *bl = binned ? c.alloc<double>(na_l, "per-l b") : plan->b;
  double *ldparts = c.alloc<double>(nblocks);
  double *W = c.alloc<double>((size_t)d.k * d.k, "W");
  const int NP = d.nc * d.nc, NU = NP * (NP + 1) / 2;
  const int nblk = d.nl * (d.nl + 1) / 2;
  double *parts = c.alloc<double>((size_t)nblk * NU);
  double *diag = c.alloc<double>((size_t)d.nl * NP);
  double *Ffull = c.alloc<double>((size_t)naf * naf);
  double *tfull = c.alloc<double>(naf);
  double *eigw = c.alloc<double>(fisher_eig_work_doubles(na));
  double *minmax = c.alloc<double>(2);
  int h_uv_full[24], h_uv[24], h_sel[6];
  for (int i = 0; i < d.nspec_full; ++i) spec_uv(d, d.full_ids[i], h_uv_full + 4 * i);
  for (int i = 0; i < prob->nspec; ++i) {
    spec_uv(d, prob->spec[i], h_uv + 4 * i);
    for (int j = 0; j < d.nspec_full; ++j)
      if (d.full_ids[j] == prob->spec[i]) h_sel[i] = j;
  }
  int *uv_full = upload(c, h_uv_full, 4 * d.nspec_full, "spectra");
  int *ids_full = upload(c, d.full_ids, d.nspec_full, "spectra");
  int *sel = upload(c, h_sel, prob->nspec, "spectra");
  if (c.err == QML_OK)
    c.cuda_ok(cudaMemcpyAsync(plan->uv, h_uv, 4 * prob->nspec * sizeof(int),
                              cudaMemcpyHostToDevice, c.st), "spectra");
  if (c.err != QML_OK) {
    qml_status e = c.finish();
    qml_plan_free(plan);
    return e;
  }

  Split spl{&c, prob->nslices};
  Split *sp_or_null = plan->split ? &spl : nullptr;
  // Signal-band pieces: the whole band for the pixel basis; for the harmonic
  // basis the fixed signal below and above the window (Eq. N_eff).  They are
  // built in a scratch Y of their own width, or in plan->X when that fits.
  auto scratch_for = [&](int kb) -> double * {
    return kb <= d.k ? plan->X : c.alloc<double>((size_t)d.n * kb, "signal-band Y");
  };
  launch_copy_lower(sp.N, d.n, plan->L, d.n, d.n, c.st);
  if (!plan->harmonic) {
    // C = Y_sig Lambda Y_sig^T + N ; L L^T = C ; X = L^-1 Y_win ; W = X^T X
    add_band_signal(c, sp_or_null, sp, d, d.lsig0, d.lsig1, ldcl,
                    scratch_for(d.nc * band_k0(d.lsig0, d.lsig1)), plan->L);
    launch_ybuild(sp.y, plan->X, d.n, c.st);  // X no longer holds the band signal
    if (plan->split) {
      // factor and X = L^-1 Y in one panel loop (the forward substitution
      // runs beside the next panel's float64 chain)
      potrf_split(c, spl, plan->L, d.n, d.n, plan->Linv, plan->LinvB, ldparts, nullptr, plan->X,
                  d.k, d.n);
      spl.gemm(1, 0, d.k, d.k, d.n, 1.0, plan->X, d.n, plan->X, d.n, 0.0, W, d.k, 1);
    } else {
      potrf_blocked(c, plan->L, d.n, d.n, plan->Linv, ldparts, nullptr);
      trsm_blocked(c, plan->L, d.n, d.n, plan->Linv, plan->X, d.k, d.n);
      launch_dgemm(1, 0, d.k, d.k, d.n, 1.0, plan->X, d.n, plan->X, d.n, 0.0, W, d.k, 1,
                   c.status, c.st);
    }
    launch_symmetrize_lower(W, d.k, d.k, c.st);
  } else {
    // N_eff = N + fixed signal outside the window ; L_N L_N^T = N_eff
    if (d.lsig0 < d.lmin)
      add_band_signal(c, sp_or_null, sp, d, d.lsig0, d.lmin - 1, ldcl,
                      scratch_for(d.nc * band_k0(d.lsig0, d.lmin - 1)), plan->L);
    if (d.lsig1 > d.lmax)
      add_band_signal(c, sp_or_null, sp, d, d.lmax + 1, d.lsig1, ldcl,
                      scratch_for(d.nc * band_k0(d.lmax + 1, d.lsig1)), plan->L);
    // U = L_N^-1 Y_win ; M = U^T U (the noise-weighted Gramian Y^T N^-1 Y)
    launch_ybuild(sp.y, plan->X, d.n, c.st);
    if (plan->split) {
      potrf_split(c, spl, plan->L, d.n, d.n, plan->Linv, plan->LinvB, ldparts, nullptr, plan->X,
                  d.k, d.n);
      spl.gemm(1, 0, d.k, d.k, d.n, 1.0, plan->X, d.n, plan->X, d.n, 0.0, W, d.k, 1);
    } else {
      potrf_blocked(c, plan->L, d.n, d.n, plan->Linv, ldparts, nullptr);
      trsm_blocked(c, plan->L, d.n, d.n, plan->Linv, plan->X, d.k, d.n);
      launch_dgemm(1, 0, d.k, d.k, d.n, 1.0, plan->X, d.n, plan->X, d.n, 0.0, W, d.k, 1,
                   c.status, c.st);
    }
    launch_symmetrize_lower(W, d.k, d.k, c.st);
    // Kt = I + L_Lambda^T M L_Lambda, factored in float64 (the SMW inner
    // matrix); then W = L_Lambda^-T Kt^-1 L_Lambda^T M = M (I + Lambda M)^-1
    // (Eq. smw_stable) by two triangular solves and two per-(l, m) mixes
    double *T = c.alloc<double>((size_t)d.k * d.k, "SMW product");
    double *ldk = c.alloc<double>((size_t)((d.k + kNB - 1) / kNB));
    if (c.err == QML_OK) {
      launch_lambda_factor(sp.cl, d.lmin, d.lmax, d.nc, d.comps, plan->lamL, c.st, ldcl);
      launch_lambda_inverse(plan->lamL, d.nl, d.nc, d.lmin, plan->lamLi, c.status, c.st);
      launch_form_ktilde(W, d.k, d.nc, d.k0, d.lmin, plan->lamL, plan->LK, d.k, c.st);
      potrf_blocked(c, plan->LK, d.k, d.k, plan->LKinv, ldk, nullptr);
      harmonic_W_from_M(c, plan, W, T);
    }
  }
  // block sums -> F, noise bias
  launch_fisher_blocksum(W, d.k, d.nc, d.k0, d.lmin, d.lmax, parts, diag, c.st);
  launch_fisher_assemble(parts, diag, d.nc, d.nl, d.nspec_full, uv_full, Ffull, tfull, c.st);
  launch_fisher_select(Ffull, tfull, sp.cl, d.lmin, d.lmax, d.nspec_full, ids_full, prob->nspec,
                       sel, Fl, bl, c.st, ldcl);
  if (binned) {  // P_b = sum_{l in b} P_l: F and the noise bias summed over bins
    launch_bin_fisher(Fl, na_l, plan->bstart, plan->bcount, na, plan->F, c.st);
    launch_bin_rows(bl, na_l, 1, plan->bstart, plan->bcount, na, plan->b, c.st);
  }
  c.cuda_ok(run_fisher_eig(plan->F, na, eigw, plan->Finv, plan->Fm12, minmax, c.status, c.st),
            "eigendecomposition");
  launch_copy_matrix(plan->F, na, Fout, na, na, na, c.st);
  qml_status e = c.finish();
  if (e != QML_OK || !plan_out) {
    qml_plan_free(plan);
    return e;
  }
  *plan_out = plan;
  return QML_OK;
}

qml_status qml_estimate(qml_plan *plan, const double *maps, int32_t nsims, double *y, double *b,
                        double *cl_deconv, double *cl_decorr, double *q_conv, void *stream) {
  if (!plan) return fail(QML_EINVAL, "plan is NULL");
  if (nsims < 0 || (nsims > 0 && !maps)) return fail(QML_EINVAL, "need maps and nsims >= 0");
  const Dims &d = plan->d;
  const int na = plan->na;
  Call c(stream);
  if (nsims == 0) {  // no maps: only the noise bias, which belongs to the plan
    double *bd = c.out(b, na, "b");
    if (bd) c.cuda_ok(cudaMemcpyAsync(bd, plan->b, na * sizeof(double), cudaMemcpyDeviceToDevice, c.st), "b");
    return c.finish();
  }
  const double *D = c.in(maps, (size_t)d.n * nsims, "maps");
  double *U = c.alloc<double>((size_t)d.n * nsims, "U");
  double *w = c.alloc<double>((size_t)d.k * nsims, "w");
  double *yd = c.out(y, (size_t)na * nsims, "y");
  if (!yd) yd = c.alloc<double>((size_t)na * nsims, "y");
  double *q = c.out(q_conv, (size_t)na * nsims, "q");
  if (!q) q = c.alloc<double>((size_t)na * nsims, "q");
  double *bd = c.out(b, na, "b");
  double *dec = c.out(cl_deconv, (size_t)na * nsims, "cl_deconv");
  double *dcr = c.out(cl_decorr, (size_t)na * nsims, "cl_decorr");
  if (!c.make_status()) return c.finish();
  // w = Y^T C^-1 d (pixel or harmonic basis)
  weighted_data(c, plan, D, nsims, U, w);
  if (plan->binned) {  // per-l y, then summed over bins
    double *yl = c.alloc<double>((size_t)plan->na_l * nsims, "per-l y");
    if (c.err != QML_OK) return c.finish();
    launch_quad_y(w, d.k, nsims, d.nc, d.k0, d.lmin, d.lmax, plan->nspec, plan->uv, yl, c.st);
    launch_bin_rows(yl, plan->na_l, nsims, plan->bstart, plan->bcount, na, yd, c.st);
  } else {
    launch_quad_y(w, d.k, nsims, d.nc, d.k0, d.lmin, d.lmax, plan->nspec, plan->uv, yd, c.st);
  }
  launch_sub_bias(yd, plan->b, na, nsims, q, c.st);
  if (bd) launch_copy_matrix(plan->b, na, bd, na, na, 1, c.st);
  if (dec) launch_dgemm(0, 0, na, nsims, na, 1.0, plan->Finv, na, q, na, 0.0, dec, na, 0, c.status, c.st);
  if (dcr) launch_dgemm(0, 0, na, nsims, na, 1.0, plan->Fm12, na, q, na, 0.0, dcr, na, 0, c.status, c.st);
  return c.finish();
}

qml_status pix_loglike(const qml_problem *prob, const double *cl_theta, const double *maps,
                       int32_t nmaps, double *lnL, double *chi2, double *logdet, void *stream) {
  Dims d;
  qml_status s = check_problem(prob, d, false, true);
  if (s != QML_OK) return s;
  if (!cl_theta || !maps || nmaps <= 0) return fail(QML_EINVAL, "need cl_theta, maps, nmaps > 0");
  Call c(stream);
  Staged sp;
  if (!stage_problem(c, prob, d, sp, cl_theta, true)) return c.finish();
  const double *D = c.in(maps, (size_t)d.n * nmaps, "maps");
  double *o_lnl = c.out(lnL, nmaps, "lnL");
  double *o_chi = c.out(chi2, nmaps, "chi2");
  double *o_ld = c.out(logdet, 1, "logdet");
  if (!o_chi) o_chi = c.alloc<double>(nmaps);
  if (!o_ld) o_ld = c.alloc<double>(1);
  const int64_t nblocks = (d.n + kNB - 1) / kNB;
  double *Y = c.alloc<double>((size_t)d.n * d.k, "Y");
  double *C = c.alloc<double>((size_t)d.n * d.n, "C");
  double *Linv = c.alloc<double>((size_t)nblocks * kNB * kNB);
  double *ldparts = c.alloc<double>(nblocks);
  double *U = c.alloc<double>((size_t)d.n * nmaps, "U");
  if (!c.make_status()) return c.finish();
  if (prob->precision == QML_SPLIT_BF16) {
    Split spl{&c, prob->nslices};
    double *LinvB = c.alloc<double>((size_t)((d.n + kNBS - 1) / kNBS) * kNBS * kNBS);
    if (!LinvB) return c.finish();
    build_C_split(c, spl, sp, d, Y, C);
    launch_copy_matrix(D, d.n, U, d.n, d.n, nmaps, c.st);
    potrf_split(c, spl, C, d.n, d.n, Linv, LinvB, ldparts, o_ld, U, nmaps, d.n);
  } else {
    build_C(c, sp, d, Y, C);
    potrf_blocked(c, C, d.n, d.n, Linv, ldparts, o_ld);
    launch_copy_matrix(D, d.n, U, d.n, d.n, nmaps, c.st);
    trsm_blocked(c, C, d.n, d.n, Linv, U, nmaps, d.n);
  }
  launch_colnorm2(U, d.n, d.n, nmaps, o_chi, c.st);
  if (o_lnl) launch_loglike_finish(o_chi, o_ld, nmaps, o_lnl, c.st);
  return c.finish();
}

qml_status pix_loglike_batch(const lnl_mask *masks, int32_t nmask, int32_t nitems,
                             const int32_t *item_mask, const double *item_cl, int32_t ld_out,
                             double *lnL, double *chi2, double *logdet, void *stream) {
  if (!masks || nmask < 1) return fail(QML_EINVAL, "need nmask >= 1 masks");
  if (nitems < 0 || (nitems > 0 && (!item_mask || !item_cl)))
    return fail(QML_EINVAL, "need item_mask and item_cl for nitems > 0");
  std::vector<Dims> dims(nmask);
  int maxmaps = 0;
  for (int m = 0; m < nmask; ++m) {
    qml_status st = check_problem(&masks[m].prob, dims[m], false, true);
    if (st != QML_OK) return fail(st, "mask " + std::to_string(m) + ": " + g_err);
    if (!masks[m].maps || masks[m].nmaps < 1)
      return fail(QML_EINVAL, "mask " + std::to_string(m) + ": need maps and nmaps >= 1");
    if (dims[m].lmin != dims[0].lmin || dims[m].lmax != dims[0].lmax ||
        dims[m].nc != dims[0].nc || masks[m].prob.has_T != masks[0].prob.has_T)
      return fail(QML_EINVAL, "all masks need the same fields and multipole band");
    maxmaps = masks[m].nmaps > maxmaps ? masks[m].nmaps : maxmaps;
  }
  if (ld_out < maxmaps) return fail(QML_EINVAL, "ld_out < largest nmaps");
  if (nitems == 0) return QML_OK;
  const Dims &d0 = dims[0];
  const size_t L = (size_t)d0.lmax + 1;
  // item -> mask on the host (the schedule is built there)
  std::vector<int32_t> imask(nitems);
  if (is_device_ptr(item_mask)) {
    if (cudaMemcpy(imask.data(), item_mask, nitems * sizeof(int32_t), cudaMemcpyDeviceToHost) !=
        cudaSuccess)
      return fail(QML_ECUDA, "item_mask copy");
  } else {
    memcpy(imask.data(), item_mask, nitems * sizeof(int32_t));
  }
  for (int i = 0; i < nitems; ++i)
    if (imask[i] < 0 || imask[i] >= nmask) return fail(QML_EINVAL, "item_mask out of range");

  Call c(stream);
  const double *cl_d = c.in(item_cl, (size_t)nitems * 6 * L, "item_cl");
  double *o_lnl = c.out(lnL, (size_t)nitems * ld_out, "lnL");
  double *o_chi = c.out(chi2, (size_t)nitems * ld_out, "chi2");
  double *o_ld = c.out(logdet, (size_t)nitems, "logdet");
  if (!c.make_status()) return c.finish();

  // ---- per-mask setup: L_N, M = Y^T N^-1 Y, v = Y^T N^-1 d, d^T N^-1 d, ln|N|
  struct MaskState {
    double *M = nullptr, *v = nullptr, *dnd = nullptr, *lnN = nullptr;
  };
  std::vector<MaskState> ms(nmask);
  const int k = d0.k;
  for (int m = 0; m < nmask; ++m) {
    const Dims &d = dims[m];
    const qml_problem *pr = &masks[m].prob;
    const int nm = masks[m].nmaps;
    Staged sp;
    if (!stage_problem(c, pr, d, sp, nullptr, true)) return c.finish();
    const double *D = c.in(masks[m].maps, (size_t)d.n * nm, "maps");
    const int64_t nb = (d.n + kNB - 1) / kNB;
    double *U = c.alloc<double>((size_t)d.n * k, "Y");
    double *LN = c.alloc<double>((size_t)d.n * d.n, "L_N");
    double *Linv = c.alloc<double>((size_t)nb * kNB * kNB);
    double *ldp = c.alloc<double>(nb);
    double *u = c.alloc<double>((size_t)d.n * nm);
    ms[m].M = c.alloc<double>((size_t)k * k, "M");
    ms[m].v = c.alloc<double>((size_t)k * nm);
    ms[m].dnd = c.alloc<double>(nm);
    ms[m].lnN = c.alloc<double>(1);
    if (c.err != QML_OK) return c.finish();
    launch_ybuild(sp.y, U, d.n, c.st);
    launch_copy_lower(sp.N, d.n, LN, d.n, d.n, c.st);
    launch_copy_matrix(D, d.n, u, d.n, d.n, nm, c.st);
    if (pr->precision == QML_SPLIT_BF16) {
      Split spl{&c, pr->nslices};
      double *LinvB = c.alloc<double>((size_t)((d.n + kNBS - 1) / kNBS) * kNBS * kNBS);
      if (!LinvB) return c.finish();
      potrf_split(c, spl, LN, d.n, d.n, Linv, LinvB, ldp, ms[m].lnN);
      trsm_split(c, spl, LN, d.n, d.n, LinvB, U, k, d.n);
      trsm_split(c, spl, LN, d.n, d.n, LinvB, u, nm, d.n);
      spl.gemm(1, 0, k, k, d.n, 1.0, U, d.n, U, d.n, 0.0, ms[m].M, k, 1);
      spl.gemm(1, 0, k, nm, d.n, 1.0, U, d.n, u, d.n, 0.0, ms[m].v, k, 0);
    } else {
      potrf_blocked(c, LN, d.n, d.n, Linv, ldp, ms[m].lnN);
      trsm_blocked(c, LN, d.n, d.n, Linv, U, k, d.n);
      trsm_blocked(c, LN, d.n, d.n, Linv, u, nm, d.n);
      launch_dgemm(1, 0, k, k, d.n, 1.0, U, d.n, U, d.n, 0.0, ms[m].M, k, 1, c.status, c.st);
      launch_dgemm(1, 0, k, nm, d.n, 1.0, U, d.n, u, d.n, 0.0, ms[m].v, k, 0, c.status, c.st);
    }
    launch_symmetrize_lower(ms[m].M, k, k, c.st);
    launch_colnorm2(u, d.n, d.n, nm, ms[m].dnd, c.st);
  }

  // ---- per-item work, round-robin over worker streams
  const int ns_max = (int)std::max<int64_t>(1, std::min<int64_t>(16, tune_get("batch_streams", 4)));
  const int NS = nitems < ns_max ? nitems : ns_max;
  // CUDA graphs: item 0 runs as plain launches (so that the tile autotuner
  // can time its shapes), then each (worker, mask) pair captures its per-item
  // sequence once -- reading the spectrum from a fixed per-worker slot and
  // writing its results to fixed slots -- and replays it for every later item
  bool graphs = tune_get("batch_graphs", 1) != 0 && nitems > NS;
  // Split precision covers the per-mask products (L_N, U = L_N^-1 Y, M, v);
  // the per-item inner factor Kt (the SMW inner inverse and ln|Kt|) stays in
  // native float64 unless the tuning key batch_split_kt asks for its trailing
  // updates and panel products in split precision too.
  const bool split_kt = tune_get("batch_split_kt", 0) != 0;
  bool any_split = false;
  for (int m = 0; m < nmask; ++m)
    any_split |= (split_kt && masks[m].prob.precision == QML_SPLIT_BF16);
  struct Worker {
    cudaStream_t st = nullptr;
    cudaEvent_t done = nullptr;
    double *K, *lamL, *z, *rr, *Linv, *LinvB, *ldp;
    double *cl, *lnK, *lnl, *chi, *ld;  // fixed slots of the captured sequence
    double *tinv;                       // block-inverse scratch (split)
    void *ws;
    size_t ws_bytes;
  };
  std::vector<Worker> wk(NS);
  const int64_t nbk = (k + kNB - 1) / kNB, nbbk = (k + kNBS - 1) / kNBS;
  size_t wsb = 0;
  if (any_split) {
    wsb = ozaki_workspace_bytes(k, k, kNBS, 0, true);
    size_t b2 = ozaki_workspace_bytes(k, kNBS, kNBS, 0, false);
    size_t b3 = ozaki_workspace_bytes(k, maxmaps, kNBS, 0, false);
    if (b2 > wsb) wsb = b2;
    if (b3 > wsb) wsb = b3;
  }
  double *lnK = c.alloc<double>(nitems);
  for (int w = 0; w < NS; ++w) {
    wk[w].K = c.alloc<double>((size_t)k * k, "Kt");
    wk[w].lamL = c.alloc<double>((size_t)d0.nl * d0.nc * d0.nc);
    wk[w].z = c.alloc<double>((size_t)k * maxmaps);
    wk[w].rr = c.alloc<double>(maxmaps);
    wk[w].Linv = c.alloc<double>((size_t)nbk * kNB * kNB);
    wk[w].LinvB = any_split ? c.alloc<double>((size_t)nbbk * kNBS * kNBS) : nullptr;
    wk[w].ldp = c.alloc<double>(nbk);
    wk[w].cl = c.alloc<double>(6 * L);
    wk[w].lnK = c.alloc<double>(1);
    wk[w].lnl = c.alloc<double>(maxmaps);
    wk[w].chi = c.alloc<double>(maxmaps);
    wk[w].ld = c.alloc<double>(1);
    wk[w].ws = any_split ? (void *)c.alloc<unsigned char>(wsb, "split workspace") : nullptr;
    wk[w].tinv = any_split ? c.alloc<double>((size_t)(kNBS / 2) * (kNBS / 2)) : nullptr;
    wk[w].ws_bytes = wsb;
  }
  if (c.err != QML_OK) return c.finish();
  cudaEvent_t setup_done;
  if (!c.cuda_ok(cudaEventCreateWithFlags(&setup_done, cudaEventDisableTiming), "event"))
    return c.finish();
  c.cuda_ok(cudaEventRecord(setup_done, c.st), "event");
  for (int w = 0; w < NS && c.err == QML_OK; ++w) {
    c.cuda_ok(cudaStreamCreateWithFlags(&wk[w].st, cudaStreamNonBlocking), "worker stream");
    c.cuda_ok(cudaEventCreateWithFlags(&wk[w].done, cudaEventDisableTiming), "event");
    if (wk[w].st) c.cuda_ok(cudaStreamWaitEvent(wk[w].st, setup_done, 0), "event wait");
  }
  std::vector<Call *> wc(NS, nullptr);
  for (int w = 0; w < NS; ++w) {
    wc[w] = new Call(wk[w].st);
    wc[w]->status = c.status;
  }
  // the per-item sequence of worker w on mask m: spectrum cl, outputs
  auto item_body = [&](int w, int m, const double *cl, double *lnKp, double *ol, double *oc,
                       double *od) {
    Call &cw = *wc[w];
    Worker &W = wk[w];
    const int nm = masks[m].nmaps;
    launch_lambda_factor(cl, d0.lmin, d0.lmax, d0.nc, d0.comps, W.lamL, W.st);
    launch_form_ktilde(ms[m].M, k, d0.nc, d0.k0, d0.lmin, W.lamL, W.K, k, W.st);
    launch_lambda_t_apply(ms[m].v, k, d0.nc, d0.k0, d0.lmin, W.lamL, nm, W.z, k, W.st);
    if (split_kt && masks[m].prob.precision == QML_SPLIT_BF16) {
      Split spl{&cw, masks[m].prob.nslices};
      spl.preset(W.ws, W.ws_bytes);
      spl.tinv = W.tinv;
      potrf_split(cw, spl, W.K, k, k, W.Linv, W.LinvB, W.ldp, lnKp);
      trsm_split(cw, spl, W.K, k, k, W.LinvB, W.z, nm, k);
    } else {
      potrf_blocked(cw, W.K, k, k, W.Linv, W.ldp, lnKp);
      trsm_blocked(cw, W.K, k, k, W.Linv, W.z, nm, k);
    }
    launch_colnorm2(W.z, k, k, nm, W.rr, W.st);
    launch_batch_finish(W.rr, ms[m].dnd, ms[m].lnN, lnKp, nm, ol, oc, od, W.st);
  };
  std::vector<cudaGraphExec_t> gexec((size_t)NS * nmask, nullptr);
  std::vector<long long> glaunch((size_t)NS * nmask, 0);
  for (int i = 0; i < nitems && c.err == QML_OK; ++i) {
    const int w = i % NS, m = imask[i];
    Worker &W = wk[w];
    const int nm = masks[m].nmaps;
    double *ol = o_lnl ? o_lnl + (size_t)i * ld_out : nullptr;
    double *oc = o_chi ? o_chi + (size_t)i * ld_out : nullptr;
    double *od = o_ld ? o_ld + i : nullptr;
    const double *cli = cl_d + (size_t)i * 6 * L;
    const size_t g = (size_t)w * nmask + m;
    if (graphs && i > 0 && !gexec[g]) {
      const long long before = qml_launch_count();
      cudaGraph_t graph = nullptr;
      bool ok = cudaStreamBeginCapture(W.st, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      if (ok) {
        item_body(w, m, W.cl, W.lnK, W.lnl, W.chi, W.ld);
        ok = cudaStreamEndCapture(W.st, &graph) == cudaSuccess && graph != nullptr;
      }
      const long long captured = qml_launch_count() - before;
      count_launch((int)-captured);  // recorded, not launched
      if (ok && cudaGraphInstantiate(&gexec[g], graph, 0) == cudaSuccess) {
        glaunch[g] = captured;
      } else {
        gexec[g] = nullptr;
        graphs = false;  // plain launches from here on
        cudaGetLastError();
      }
      if (graph) cudaGraphDestroy(graph);
      if (wc[w]->err != QML_OK) {  // an error while recording: report it
        c.err = wc[w]->err;
        break;
      }
    }
    if (graphs && gexec[g]) {
      c.cuda_ok(cudaMemcpyAsync(W.cl, cli, 6 * L * sizeof(double), cudaMemcpyDeviceToDevice, W.st),
                "item spectrum");
      c.cuda_ok(cudaGraphLaunch(gexec[g], W.st), "graph launch");
      count_launch((int)glaunch[g]);
      c.cuda_ok(cudaMemcpyAsync(lnK + i, W.lnK, sizeof(double), cudaMemcpyDeviceToDevice, W.st),
                "item result");
      if (ol)
        c.cuda_ok(cudaMemcpyAsync(ol, W.lnl, nm * sizeof(double), cudaMemcpyDeviceToDevice, W.st),
                  "item result");
      if (oc)
        c.cuda_ok(cudaMemcpyAsync(oc, W.chi, nm * sizeof(double), cudaMemcpyDeviceToDevice, W.st),
                  "item result");
      if (od)
        c.cuda_ok(cudaMemcpyAsync(od, W.ld, sizeof(double), cudaMemcpyDeviceToDevice, W.st),
                  "item result");
    } else {
      item_body(w, m, cli, lnK + i, ol, oc, od);
    }
    if (wc[w]->err != QML_OK && c.err == QML_OK) c.err = wc[w]->err;
  }
  for (int w = 0; w < NS; ++w) {
    if (wk[w].st && wk[w].done) {
      cudaEventRecord(wk[w].done, wk[w].st);
      cudaStreamWaitEvent(c.st, wk[w].done, 0);
    }
  }
  qml_status res = c.finish();
  for (cudaGraphExec_t ge : gexec)
    if (ge) cudaGraphExecDestroy(ge);
  for (int w = 0; w < NS; ++w) {
    delete wc[w];
    if (wk[w].done) cudaEventDestroy(wk[w].done);
    if (wk[w].st) cudaStreamDestroy(wk[w].st);
  }
  cudaEventDestroy(setup_done);
  return res;
}

qml_status qml_cross(qml_plan *plan1, qml_plan *plan2, const double *maps1, const double *maps2,
                     int32_t nsims, double *Wx, double *q, double *cl, void *stream) {
  if (!plan1 || !plan2 || !Wx) return fail(QML_EINVAL, "qml_cross needs two plans and Wx");
  if (nsims < 0 || (nsims > 0 && (!maps1 || !maps2)))
    return fail(QML_EINVAL, "qml_cross needs maps1, maps2 and nsims >= 0");
  const Dims &d = plan1->d, &d2 = plan2->d;
  if (d.n != d2.n || d.nc != d2.nc || d.lmin != d2.lmin || d.lmax != d2.lmax ||
      plan1->nspec != plan2->nspec || d.nT != d2.nT)
    return fail(QML_EINVAL, "qml_cross: the plans need the same pixels, fields, window and spectra");
  for (int i = 0; i < plan1->nspec; ++i)
    if (plan1->spec[i] != plan2->spec[i])
      return fail(QML_EINVAL, "qml_cross: the plans need the same spectra");
  if (plan1->binned || plan2->binned)
    return fail(QML_EINVAL, "qml_cross: per-multipole plans only (no bins)");
  const int na = plan1->na;
  Call c(stream);
  double *Wxd = c.out(Wx, (size_t)na * na, "Wx");
  double *W1 = c.alloc<double>((size_t)d.k * d.k, "W1");
  double *W2 = c.alloc<double>((size_t)d.k * d.k, "W2");
  double *T = (plan1->harmonic || plan2->harmonic) ? c.alloc<double>((size_t)d.k * d.k, "SMW product")
                                                   : nullptr;
  const int NP = d.nc * d.nc;
  double *parts = c.alloc<double>((size_t)d.nl * (d.nl + 1) / 2 * NP * NP, "cross sums");
  if (!c.make_status()) return c.finish();
  // Wx_ab = 1/2 tr[W1 E_a W2 E_b] (Eq. q_cross)
  plan_W(c, plan1, W1, T);
  plan_W(c, plan2, W2, T);
  launch_cross_blocksum(W1, W2, d.k, d.nc, d.k0, d.lmin, d.lmax, parts, c.st);
  launch_cross_assemble(parts, d.nc, d.nl, plan1->nspec, plan1->uv, Wxd, c.st);
  if (nsims > 0) {
    const double *D1 = c.in(maps1, (size_t)d.n * nsims, "maps1");
    const double *D2 = c.in(maps2, (size_t)d.n * nsims, "maps2");
    double *U = c.alloc<double>((size_t)d.n * nsims, "U");
    double *w1 = c.alloc<double>((size_t)d.k * nsims, "w1");
    double *w2 = c.alloc<double>((size_t)d.k * nsims, "w2");
    double *qd = c.out(q, (size_t)na * nsims, "q");
    if (!qd) qd = c.alloc<double>((size_t)na * nsims, "q");
    double *cld = c.out(cl, (size_t)na * nsims, "cl");
    double *A = cld ? c.alloc<double>((size_t)na * na, "Wx factors") : nullptr;
    if (c.err != QML_OK) return c.finish();
    weighted_data(c, plan1, D1, nsims, U, w1);
    weighted_data(c, plan2, D2, nsims, U, w2);
    launch_quad_cross(w1, w2, d.k, nsims, d.nc, d.k0, d.lmin, d.lmax, plan1->nspec, plan1->uv,
                      qd, c.st);
    if (cld) {  // C_x = Wx^-1 q_x
      launch_copy_matrix(Wxd, na, A, na, na, na, c.st);
      launch_copy_matrix(qd, na, cld, na, na, nsims, c.st);
      launch_lu_solve(A, na, cld, nsims, c.status, c.st);
    }
  }
  return c.finish();
}

qml_status qml_potrf(int64_t n, double *A, int64_t lda, double *logdet, int32_t precision,
                     void *stream) {
  if (n <= 0 || !A || lda < n) return fail(QML_EINVAL, "bad potrf arguments");
  if (precision != QML_FP64 && precision != QML_SPLIT_BF16)
    return fail(QML_EINVAL, "precision must be QML_FP64 or QML_SPLIT_BF16");
  Call c(stream);
  double *Ad = c.out(A, (size_t)lda * n, "A");
  if (Ad != A && Ad) {
    c.cuda_ok(cudaMemcpyAsync(Ad, A, (size_t)lda * n * sizeof(double), cudaMemcpyHostToDevice, c.st),
              "A");
  }
  double *ld = c.out(logdet, 1, "logdet");
  const int64_t nblocks = (n + kNB - 1) / kNB;
  double *Linv = c.alloc<double>((size_t)nblocks * kNB * kNB);
  double *ldparts = c.alloc<double>(nblocks);
  if (!c.make_status()) return c.finish();
  if (precision == QML_SPLIT_BF16) {
    double *LinvB = c.alloc<double>((size_t)((n + kNBS - 1) / kNBS) * kNBS * kNBS);
    if (!LinvB) return c.finish();
    Split spl{&c, 0};
    potrf_split(c, spl, Ad, n, lda, Linv, LinvB, ldparts, ld);
  } else {
    potrf_blocked(c, Ad, n, lda, Linv, ldparts, ld);
  }
  return c.finish();
}

qml_status qml_trsm(int64_t n, int64_t nrhs, const double *L, int64_t lda, double *B, int64_t ldb,
                    int32_t precision, void *stream) {
  if (n <= 0 || nrhs < 0 || !L || !B || lda < n || ldb < n)
    return fail(QML_EINVAL, "bad trsm arguments");
  if (precision != QML_FP64 && precision != QML_SPLIT_BF16)
    return fail(QML_EINVAL, "precision must be QML_FP64 or QML_SPLIT_BF16");
  if (nrhs == 0) return QML_OK;
  Call c(stream);
  const double *Ld = c.in(L, (size_t)lda * n, "L");
  double *Bd = c.out(B, (size_t)ldb * nrhs, "B");
  if (Bd != B && Bd)
    c.cuda_ok(cudaMemcpyAsync(Bd, B, (size_t)ldb * nrhs * sizeof(double), cudaMemcpyHostToDevice,
                              c.st), "B");
  const int64_t nblocks = (n + kNB - 1) / kNB;
  double *Linv = c.alloc<double>((size_t)nblocks * kNB * kNB);
  if (!c.make_status()) return c.finish();
  launch_trtri_blocks(Ld, lda, n, Linv, c.status, c.st);
  if (precision == QML_SPLIT_BF16) {
    // explicit inverses of the kNBS diagonal blocks (float64), then split products
    double *LinvB = c.alloc<double>((size_t)((n + kNBS - 1) / kNBS) * kNBS * kNBS);
    if (!LinvB) return c.finish();
    Split spl{&c, 0};
    double *T = spl.tinv_scratch();
    if (!T) return c.finish();
    for (int64_t j = 0; j < n; j += kNBS) {
      const int64_t jb = (n - j) < kNBS ? (n - j) : kNBS;
      double *Xinv = LinvB + (j / kNBS) * kNBS * kNBS;
      trinv_doubling(c, Ld + j + j * lda, jb, lda, Linv + (j / kNB) * kNB * kNB, Xinv, kNBS, T,
                     c.st, false);
    }
    trsm_split(c, spl, Ld, n, lda, LinvB, Bd, nrhs, ldb);
  } else {
    trsm_blocked(c, Ld, n, lda, Linv, Bd, nrhs, ldb);
  }
  return c.finish();
}

qml_status qml_gemm(int32_t transA, int32_t transB, int64_t m, int64_t nn, int64_t kk,
                    double alpha, const double *A, int64_t lda, const double *B, int64_t ldb,
                    double beta, double *C, int64_t ldc, int32_t lower, int32_t precision,
                    void *stream) {
  if (m < 0 || nn < 0 || kk < 0) return fail(QML_EINVAL, "bad gemm arguments");
  if (precision != QML_FP64 && precision != QML_SPLIT_BF16)
    return fail(QML_EINVAL, "precision must be QML_FP64 or QML_SPLIT_BF16");
  if (m == 0 || nn == 0) return QML_OK;
  if (!C || (kk > 0 && (!A || !B))) return fail(QML_EINVAL, "bad gemm arguments");
  const int64_t ar = transA ? kk : m, ac = transA ? m : kk;
  const int64_t br = transB ? nn : kk, bc = transB ? kk : nn;
  if (lda < (ar > 0 ? ar : 1) || ldb < (br > 0 ? br : 1) || ldc < (m > 0 ? m : 1))
    return fail(QML_EINVAL, "leading dimension too small");
  if (lower && m != nn) return fail(QML_EINVAL, "lower needs a square C");
  Call c(stream);
  const double *Ad = c.in(A, (size_t)lda * ac, "A");
  const double *Bd = c.in(B, (size_t)ldb * bc, "B");
  double *Cd = c.out(C, (size_t)ldc * nn, "C");
  if (Cd != C && Cd && beta != 0.0)
    c.cuda_ok(cudaMemcpyAsync(Cd, C, (size_t)ldc * nn * sizeof(double), cudaMemcpyHostToDevice, c.st),
              "C");
  if (!c.make_status()) return c.finish();
  if (precision == QML_SPLIT_BF16 && kk > 0) {  // (kk == 0: C <- beta C, no digits)
    const bool shared = (A == B && lda == ldb && transA != transB && m == nn);
    void *ws = c.alloc<unsigned char>(ozaki_workspace_bytes(m, nn, kk, 0, shared), "split workspace");
    if (!ws) return c.finish();
    c.cuda_ok(ozaki_gemm(transA, transB, m, nn, kk, alpha, Ad, lda, Bd, ldb, beta, Cd, ldc, lower,
                         0, ws, c.status, c.st),
              "split-precision gemm");
    return c.finish();
  }
  launch_dgemm(transA, transB, m, nn, kk, alpha, Ad, lda, Bd, ldb, beta, Cd, ldc, lower, c.status,
               c.st);
  return c.finish();
}

}  // extern "C"
