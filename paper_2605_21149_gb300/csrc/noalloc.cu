// qml_potrf_noalloc: the blocked Cholesky of qml_potrf for callers that
// cannot allocate device memory.
//
// Who needs it: code embedded in a host runtime that owns every byte of the
// GPU (a framework's custom-call or plugin interface that hands the callee
// pre-allocated buffers and forbids it from allocating), and hot loops where
// the implicit device synchronisation of cudaMalloc / cudaFree, or a call into
// another allocator, is not acceptable.  This entry point calls no
// cudaMalloc, cudaMallocAsync, cudaFree or allocating library routine, and it
// never runs the float64 GEMM tile autotuner (which allocates a timing buffer
// and synchronises): each product takes the tuning table's measured tile for
// its shape when one is there, else the heuristic tile.
//
// Its scratch (the inverses of the 64 x 64 diagonal blocks, the per-block
// log-determinants and the status word) lives in the file-scope array below,
// sized for n <= kNoAllocMaxN.  Every GPU that loads the library holds the
// array (2.1 MB) until the process exits.  Every call shares it and it keeps
// the previous call's contents: the status word is cleared at the start of
// each call, everything else is fully overwritten before it is read.  Calls
// whose execution overlaps on the GPU (different streams, or threads sharing
// a device) race on the array and must be serialised by the caller.
//
// Host code may not use the array's name as a device address (in host code
// it names a host-side shadow); the device address comes from
// cudaGetSymbolAddress, taken once per device with that device current, on
// the first call on that device.  Every call reads the status word back and
// synchronises `stream` before it returns.
#include "qmlgb.h"
#include "internal.cuh"

#include <cuda_runtime.h>

#include <mutex>
#include <string>

namespace qmlgb {
void set_last_error(const std::string &msg);
}

using namespace qmlgb;

namespace {

constexpr int64_t kNoAllocMaxN = 4096;
constexpr int64_t kMaxBlocks = kNoAllocMaxN / kNB;          // 64 diagonal blocks
constexpr int64_t kStatusDoubles = 32;                      // 256 bytes for the status word
constexpr int64_t kScratchDoubles = kStatusDoubles + kMaxBlocks + kMaxBlocks * kNB * kNB;

static_assert(sizeof(DevStatus) <= kStatusDoubles * sizeof(double), "status slot too small");

// status | per-block log-determinants | diagonal-block inverses
static __device__ __align__(256) double g_potrf_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_scratch_ptr[kMaxDevices] = {nullptr};

// device address of the scratch array for the current device (set-up once)
double *scratch_for_current_device(std::string &err) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
    return nullptr;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    err = "device index out of range";
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_potrf_scratch);
    if (e != cudaSuccess || !p) {
      err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
      return nullptr;
    }
    g_scratch_ptr[dev] = (double *)p;
  }
  return g_scratch_ptr[dev];
}

bool device_pointer(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

qml_status fail_na(qml_status s, const std::string &msg) {
  set_last_error(msg);
  return s;
}

}  // namespace

extern "C" qml_status qml_potrf_noalloc(int64_t n, double *A, int64_t lda, double *logdet,
                                        void *stream) {
  if (n <= 0 || !A || lda < n) return fail_na(QML_EINVAL, "bad potrf_noalloc arguments");
  if (n > kNoAllocMaxN)
    return fail_na(QML_EINVAL, "n = " + std::to_string(n) +
                                   " exceeds the static scratch limit of qml_potrf_noalloc (n <= " +
                                   std::to_string(kNoAllocMaxN) + ")");
  if (!device_pointer(A) || (logdet && !device_pointer(logdet)))
    return fail_na(QML_EINVAL, "qml_potrf_noalloc needs device pointers for A and logdet");
  std::string err;
  double *base = scratch_for_current_device(err);
  if (!base) return fail_na(QML_ECUDA, err);
  cudaStream_t st = (cudaStream_t)stream;
  DevStatus *status = (DevStatus *)base;
  double *ldparts = base + kStatusDoubles;
  double *Linv = ldparts + kMaxBlocks;
  cudaError_t e = cudaMemsetAsync(status, 0, sizeof(DevStatus), st);
  if (e != cudaSuccess) return fail_na(QML_ECUDA, std::string("status: ") + cudaGetErrorString(e));
  // right-looking blocked Cholesky, the same kernels and order as qml_potrf
  for (int64_t j = 0; j < n; j += kNB) {
    const int64_t jb = (n - j) < kNB ? (n - j) : kNB;
    double *Lb = Linv + (j / kNB) * kNB * kNB;
    launch_potrf_diag(A + j + j * lda, lda, n, j, Lb, ldparts + j / kNB, status, st);
    if (j + jb < n) {
      const int64_t m2 = n - j - jb;
      double *A21 = A + (j + jb) + j * lda;
      double *A22 = A + (j + jb) + (j + jb) * lda;
      // never the tile autotuner: it allocates a timing buffer and synchronises
      launch_dgemm_fixed(0, 1, m2, jb, jb, 1.0, A21, lda, Lb, kNB, 0.0, A21, lda, 0, status, st);
      launch_dgemm_fixed(0, 1, m2, m2, jb, -1.0, A21, lda, A21, lda, 1.0, A22, lda, 1, status, st);
    }
  }
  if (logdet) launch_sum_logdet(ldparts, (int)((n + kNB - 1) / kNB), logdet, st);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail_na(QML_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
  DevStatus hs{};
  e = cudaMemcpyAsync(&hs, status, sizeof(hs), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail_na(QML_ECUDA, std::string("synchronize: ") + cudaGetErrorString(e));
  if (hs.code == QML_ENOTSPD)
    return fail_na(QML_ENOTSPD, "matrix not positive definite (Cholesky pivot at column " +
                                    std::to_string(hs.info - 1) + ")");
  if (hs.code != 0) return fail_na(QML_ECUDA, "device status " + std::to_string(hs.code));
  return QML_OK;
}
