// hss_matvec_noalloc: the HSS matvec without any device allocation.
//
// For callers that must not allocate device memory when they call us -- a host
// application that reserves the whole device up front for its own pool, or a
// latency-critical loop where a cudaMalloc (which may synchronize the device)
// is not allowed.  The caller passes the generators, x and y in its own device
// memory; the intermediate per-level vectors live in one file-scope static
// device array of fixed size instead of an allocated workspace.
#include <algorithm>
#include <mutex>

#include "../../include/hss.h"
#include "common.cuh"

namespace {

// 2^21 doubles = 16 MiB, held by every device that loads the library until exit.
constexpr size_t kScratchDoubles = size_t(1) << 21;
constexpr int kMaxCols = 32;
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

// device address of g_noalloc_scratch per device, looked up once with that
// device current (the host-side name is only a stand-in for the symbol)
double* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

int scratch_address(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return HSS_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return HSS_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return HSS_ERR_CUDA;
    }
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return HSS_OK;
}

}  // namespace

extern "C" int hss_matvec_noalloc(const hss_shape* shape, const double* D, const double* U,
                                  const double* E, const double* S, const double* x, double* y,
                                  int32_t nrhs, int32_t ld, void* stream) {
  if (!shape || !D || !U || !S || !x || !y || x == y || nrhs < 0) return HSS_ERR_INVALID_ARG;
  if (shape->node_sizes) return HSS_ERR_INVALID_ARG;   // uniform trees only
  const int L = shape->levels, leaf = shape->leaf, r = shape->rank;
  if (L < 1 || L > 24 || leaf < 1 || r < 1 || r > leaf) return HSS_ERR_INVALID_ARG;
  if ((long long)leaf << L != (long long)shape->n || ld < shape->n) return HSS_ERR_INVALID_ARG;
  if (L >= 2 && !E) return HSS_ERR_INVALID_ARG;
  // doubles per right-hand-side column: x̂ and ŷ of every level 1..L
  const long long per_col = 2LL * ((2LL << L) - 2) * r;
  if (per_col > (long long)kScratchDoubles) return HSS_ERR_TOO_LARGE;
  if (nrhs == 0) return HSS_OK;
  double* scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc) return rc;
  const int cols = (int)std::min<long long>(kMaxCols, (long long)kScratchDoubles / per_col);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const long long rr = (long long)r * r;
  const int nL = 1 << L;

  // packed offsets of E (levels 1..L-1) and S (levels 1..L)
  long long eoff[32] = {0}, soff[32] = {0};
  for (long long l = 1, acc = 0; l <= L - 1; ++l) {
    eoff[l] = acc;
    acc += (1LL << l) * 2 * rr;
  }
  for (long long l = 1, acc = 0; l <= L; ++l) {
    soff[l] = acc;
    acc += (1LL << (l - 1)) * rr;
  }

  for (int j0 = 0; j0 < nrhs; j0 += cols) {
    const int nc = std::min(cols, nrhs - j0);
    const double* xc = x + (long long)j0 * ld;
    double* yc = y + (long long)j0 * ld;
    // x̂_l at scratch + base, ŷ_l right after it: (2^l r) x nc each, ld = 2^l r.
    // Every element is written (beta = 0) before it is read, so nothing is cleared.
    double* xh[32] = {nullptr};
    double* yh[32] = {nullptr};
    long long off = 0;
    for (int l = 1; l <= L; ++l) {
      const long long sz = (1LL << l) * r * nc;
      xh[l] = scratch + off;
      yh[l] = scratch + off + sz;
      off += 2 * sz;
    }
    gemm_batched<double>(true, false, r, nc, leaf, 1.0, U, leaf, (long long)leaf * r, xc, ld, leaf,
                         0.0, xh[L], nL * r, r, nL, st);
    for (int l = L - 1; l >= 1; --l)
      gemm_batched<double>(true, false, r, nc, 2 * r, 1.0, E + eoff[l], 2 * r, 2 * rr, xh[l + 1],
                           (2 << l) * r, 2 * r, 0.0, xh[l], (1 << l) * r, r, 1 << l, st);
    for (int l = 1; l <= L; ++l) {
      const int ldl = (1 << l) * r;
      gemm_batched<double>(false, false, r, nc, r, 1.0, S + soff[l], r, rr, xh[l], ldl, 2 * r, 0.0,
                           yh[l] + r, ldl, 2 * r, 1 << (l - 1), st);
      gemm_batched<double>(true, false, r, nc, r, 1.0, S + soff[l], r, rr, xh[l] + r, ldl, 2 * r,
                           0.0, yh[l], ldl, 2 * r, 1 << (l - 1), st);
    }
    for (int l = 1; l <= L - 1; ++l)
      gemm_batched<double>(false, false, 2 * r, nc, r, 1.0, E + eoff[l], 2 * r, 2 * rr, yh[l],
                           (1 << l) * r, r, 1.0, yh[l + 1], (2 << l) * r, 2 * r, 1 << l, st);
    gemm_batched<double>(false, false, leaf, nc, leaf, 1.0, D, leaf, (long long)leaf * leaf, xc, ld,
                         leaf, 0.0, yc, ld, leaf, nL, st);
    gemm_batched<double>(false, false, leaf, nc, r, 1.0, U, leaf, (long long)leaf * r, yh[L],
                         nL * r, r, 1.0, yc, ld, leaf, nL, st);
    if (cudaGetLastError() != cudaSuccess) return HSS_ERR_CUDA;
  }
  return HSS_OK;
}
