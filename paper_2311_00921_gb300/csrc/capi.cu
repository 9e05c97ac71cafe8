// C ABI of the HSS-ULV library: the device-resident object, its arena, and the
// level schedule of Alg. 2 (factor), the solve of Sec. 3.2 and the HSS matvec.
//
// Per level l the work is batched over the 2^l nodes of the level; each step is
// one launch (batched GEMM / SYR2K / per-node kernel), so a level costs a fixed
// handful of launches whatever its node count.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "../../include/hss.h"
#include "common.cuh"
#include "ulv_kernels.cuh"

namespace {

constexpr int kMaxCols = 32;      // right-hand-side columns per matvec pass
constexpr int kSolveCols = 16;    // columns per triangular-sweep pass

struct Level {
  int n = 0, b = 0, r = 0, c = 0;
  double* V = nullptr;   // n x b x r
  double* T = nullptr;   // n x r x r
  double* LB = nullptr;  // n x r x r
  double* M = nullptr;   // n x b x b factored blocks (leaves: own buffer; else = A)
  double* A = nullptr;   // n x b x b merged blocks (levels < L), 1 block at the root
  double* B = nullptr;   // n x b x r bases fed to the QL (levels 1 .. L-1)
  double* yv = nullptr;  // level vector for the solve: (n b) x kSolveCols
  double* xh = nullptr;  // matvec up-sweep: (n r) x kMaxCols
  double* yh = nullptr;  // matvec down-sweep: (n r) x kMaxCols
};

}  // namespace

struct hss_s {
  int n = 0, leaf = 0, rank = 0, L = 0;
  int device = 0;
  double *D = nullptr, *U = nullptr, *E = nullptr, *S = nullptr;
  std::vector<long long> Eoff, Soff;   // element offset of level l in E / S
  std::vector<Level> lv;               // index = level (0 = root)
  double *W = nullptr, *Y = nullptr;   // n_L x b x r scratch
  double *X = nullptr, *Z = nullptr;   // n_L x r x r scratch
  double *t1 = nullptr, *t2 = nullptr; // n_L x r x kMaxCols scratch
  double* logdet_part = nullptr;       // 2^(L+1) - 1 node contributions
  double* logdet_val = nullptr;
  int* status = nullptr;
  void* arena = nullptr;
  size_t arena_bytes = 0;
  int factorized = 0;
  int precision = HSS_FP64;
  cudaStream_t last_stream = nullptr;
  int ir_iters = 0;
  double ir_resid = 0.0;
  // launch accounting and the optional per-launch event log
  long long launches = 0;
  int tracing = 0;
  struct Rec {
    int kind;
    double flops;
    cudaEvent_t a, b;
  };
  std::vector<Rec> trace;
};

namespace {

struct Bump {
  char* base;
  size_t off = 0;
  size_t cap;
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = reinterpret_cast<T*>(base + off);
    off += count * sizeof(T);
    return p;
  }
};

// lays the object out in [base, base + cap); with base = nullptr only measures
size_t layout(hss_s* h, char* base) {
  Bump bp{base, 0, 0};
  const int L = h->L, r = h->rank, leaf = h->leaf;
  const long long nL = 1LL << L;
  h->D = bp.take<double>(nL * leaf * leaf);
  h->U = bp.take<double>(nL * leaf * r);
  long long esz = 0, ssz = 0;
  h->Eoff.assign(L + 1, 0);
  h->Soff.assign(L + 1, 0);
  for (int l = 1; l <= L - 1; ++l) {
    h->Eoff[l] = esz;
    esz += (1LL << l) * 2 * r * r;
  }
  for (int l = 1; l <= L; ++l) {
    h->Soff[l] = ssz;
    ssz += (1LL << (l - 1)) * r * r;
  }
  h->E = bp.take<double>(std::max<long long>(esz, 1));
  h->S = bp.take<double>(ssz);
  h->lv.assign(L + 1, Level());
  for (int l = 0; l <= L; ++l) {
    Level& P = h->lv[l];
    P.n = 1 << l;
    P.b = (l == L) ? leaf : 2 * r;
    P.r = (l == 0) ? 0 : r;
    P.c = P.b - P.r;
    if (l >= 1) {
      P.V = bp.take<double>((size_t)P.n * P.b * r);
      P.T = bp.take<double>((size_t)P.n * r * r);
      P.LB = bp.take<double>((size_t)P.n * r * r);
    }
    if (l < L) {
      P.A = bp.take<double>((size_t)P.n * P.b * P.b);
      P.M = P.A;
    } else {
      P.M = bp.take<double>((size_t)P.n * P.b * P.b);
    }
    if (l >= 1 && l < L) P.B = bp.take<double>((size_t)P.n * P.b * r);
    if (l < L) P.yv = bp.take<double>((size_t)P.n * P.b * kSolveCols);
    if (l >= 1) {
      P.xh = bp.take<double>((size_t)P.n * r * kMaxCols);
      P.yh = bp.take<double>((size_t)P.n * r * kMaxCols);
    }
  }
  h->W = bp.take<double>((size_t)nL * leaf * r);
  h->Y = bp.take<double>((size_t)nL * leaf * r);
  h->X = bp.take<double>((size_t)nL * r * r);
  h->Z = bp.take<double>((size_t)nL * r * r);
  h->t1 = bp.take<double>((size_t)nL * r * kMaxCols);
  h->t2 = bp.take<double>((size_t)nL * r * kMaxCols);
  h->logdet_part = bp.take<double>((size_t)(2 * nL - 1));
  h->logdet_val = bp.take<double>(1);
  h->status = bp.take<int>(8);
  return bp.off + 256;
}

int cuda_err(cudaError_t e) { return e == cudaSuccess ? HSS_OK : HSS_ERR_CUDA; }

// Brackets one kernel launch: counts it and, when tracing, logs two events.
struct Launch {
  hss_s* h;
  cudaStream_t st;
  hss_s::Rec rec{};
  bool on = false;
  Launch(hss_s* h_, int kind, double flops, cudaStream_t st_) : h(h_), st(st_) {
    ++h->launches;
    if (h->tracing) {
      rec.kind = kind;
      rec.flops = flops;
      if (cudaEventCreate(&rec.a) == cudaSuccess && cudaEventCreate(&rec.b) == cudaSuccess) {
        cudaEventRecord(rec.a, st);
        on = true;
      }
    }
  }
  ~Launch() {
    if (on) {
      cudaEventRecord(rec.b, st);
      h->trace.push_back(rec);
    }
  }
};

void clear_trace(hss_s* h) {
  for (auto& r : h->trace) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  h->trace.clear();
}

double gemm_flops(int m, int n, int k, int batch) { return 2.0 * m * n * (double)k * batch; }

void gemm(hss_s* h, bool ta, bool tb, int m, int n, int k, double alpha, const double* A, int lda,
          long long sA, const double* B, int ldb, long long sB, double beta, double* C, int ldc,
          long long sC, int batch, cudaStream_t st) {
  if (m <= 0 || n <= 0 || k <= 0 || batch <= 0) return;
  Launch l(h, n <= 32 ? HSS_K_GEMM_SKINNY : HSS_K_GEMM, gemm_flops(m, n, k, batch), st);
  gemm_batched<double>(ta, tb, m, n, k, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, batch,
                       st);
}

int check_launch() {
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HSS_OK : HSS_ERR_CUDA;
}

// partial Cholesky of the first c of b columns: POTRF c x c, TRSM (b-c) x c,
// SYRK (b-c) x (b-c) with depth c
double pchol_flops(int b, int c) {
  const double r = b - c;
  return (double)c * c * c / 3.0 + r * c * c + r * (r + 1.0) * c;
}

// triangular sweep of one node: c x c triangle plus the (b-c) x c block
double trsv_flops(int b, int c, int nrhs) {
  return ((double)c * c + 2.0 * (b - c) * c) * nrhs;
}

// Q application on a level vector: vec_seg := vec_seg - V op(T) (Vᵀ vec_seg)
// (op(T) = Tᵀ for Qᵀ, T for Q), nc <= kMaxCols columns
void apply_q(hss_s* h, const Level& P, double* vec, int ldv, int nc, bool transpose,
             cudaStream_t st) {
  const int b = P.b, r = P.r, n = P.n;
  const long long s1 = (long long)r * kMaxCols;
  gemm(h, true, false, r, nc, b, 1.0, P.V, b, (long long)b * r, vec, ldv, b, 0.0,
                       h->t1, r, s1, n, st);
  gemm(h, transpose, false, r, nc, r, 1.0, P.T, r, (long long)r * r, h->t1, r, s1,
                       0.0, h->t2, r, s1, n, st);
  gemm(h, false, false, b, nc, r, -1.0, P.V, b, (long long)b * r, h->t2, r, s1, 1.0,
                       vec, ldv, b, n, st);
}

int factorize_fp64(hss_s* h, cudaStream_t st) {
  const int L = h->L, r = h->rank;
  const long long rr = (long long)r * r;
  cudaMemsetAsync(h->status, 0, 8 * sizeof(int), st);
  for (int l = L; l >= 1; --l) {
    Level& P = h->lv[l];
    Level& Q = h->lv[l - 1];
    const int b = P.b, n = P.n, c = P.c;
    const long long br = (long long)b * r, bb = (long long)b * b;
    // (a) basis completion (Eq. 2-3)
    const double* Bsrc = (l == L) ? h->U : P.B;
    {
      Launch k(h, HSS_K_QL, (2.0 * b * r * r - 2.0 / 3.0 * r * r * r + 1.0 * b * r * r) * n, st);
      launch_ql_basis<double>(Bsrc, b, br, P.V, br, P.T, rr, P.LB, rr, b, r, n, st);
    }
    // (d, first half) merge: rescaled coupling Ŝ = L_B(c2) S L_B(c1)ᵀ into the
    // parent's off-diagonal blocks, parent basis blkdiag(L_B(c1), L_B(c2)) E_p
    const int np = n / 2;
    const double* Sl = h->S + h->Soff[l];
    const int ldq = 2 * r;
    const long long sq = 4 * rr;
    gemm(h, false, false, r, r, r, 1.0, P.LB + rr, r, 2 * rr, Sl, r, rr, 0.0, h->Z, r,
                         rr, np, st);
    gemm(h, false, true, r, r, r, 1.0, h->Z, r, rr, P.LB, r, 2 * rr, 0.0, Q.A + r, ldq,
                         sq, np, st);
    gemm(h, false, true, r, r, r, 1.0, P.LB, r, 2 * rr, h->Z, r, rr, 0.0,
                         Q.A + (long long)r * ldq, ldq, sq, np, st);
    if (l - 1 >= 1) {
      const double* Ep = h->E + h->Eoff[l - 1];
      gemm(h, false, false, r, r, r, 1.0, P.LB, r, 2 * rr, Ep, 2 * r, 2 * rr, 0.0,
                           Q.B, 2 * r, 2 * rr, np, st);
      gemm(h, false, false, r, r, r, 1.0, P.LB + rr, r, 2 * rr, Ep + r, 2 * r, 2 * rr,
                           0.0, Q.B + r, 2 * r, 2 * rr, np, st);
    }
    // (b) diagonal product Â = Qᵀ A Q with Q = I - V T Vᵀ, in the symmetric
    // compact-WY form Â = A - Y'Vᵀ - V Y'ᵀ, Y' = A V T - ½ V Tᵀ Vᵀ A V T
    const double* Ain = (l == L) ? h->D : P.A;
    gemm(h, false, false, b, r, b, 1.0, Ain, b, bb, P.V, b, br, 0.0, h->W, b, br, n,
                         st);
    gemm(h, false, false, b, r, r, 1.0, h->W, b, br, P.T, r, rr, 0.0, h->Y, b, br, n,
                         st);
    gemm(h, true, false, r, r, b, 1.0, P.V, b, br, h->Y, b, br, 0.0, h->X, r, rr, n,
                         st);
    gemm(h, true, false, r, r, r, 1.0, P.T, r, rr, h->X, r, rr, 0.0, h->Z, r, rr, n,
                         st);
    gemm(h, false, false, b, r, r, -0.5, P.V, b, br, h->Z, r, rr, 1.0, h->Y, b, br, n,
                         st);
    {
      Launch k(h, HSS_K_SYR2K, 2.0 * r * b * (b + 1.0) * n, st);
      syr2k_lower_batched<double>(b, r, Ain, b, bb, h->Y, b, br, P.V, b, br, P.M, b, bb, n, st);
    }
    // (c) partial Cholesky + (d, second half) Schur complements into the parent
    {
      Launch k(h, HSS_K_PCHOL, pchol_flops(b, c) * n, st);
      launch_pchol<double>(P.M, b, bb, b, c, Q.A, ldq, sq, h->logdet_part + ((1LL << l) - 1), l,
                           0, h->status, n, st);
    }
    int rc = check_launch();
    if (rc) return rc;
  }
  // root Cholesky (Alg. 2 line 6)
  Level& R0 = h->lv[0];
  {
    Launch k(h, HSS_K_PCHOL, pchol_flops(R0.b, R0.b), st);
    launch_pchol<double>(R0.A, R0.b, (long long)R0.b * R0.b, R0.b, R0.b, nullptr, 0, 0,
                         h->logdet_part, 0, 0, h->status, 1, st);
  }
  {
    Launch k(h, HSS_K_OTHER, (double)((2LL << L) - 1), st);
    launch_logdet_reduce(h->logdet_part, (int)((2LL << L) - 1), h->logdet_val, st);
  }
  return check_launch();
}

int solve_fp64(hss_s* h, double* x, int nrhs, int ld, cudaStream_t st) {
  const int L = h->L, r = h->rank;
  for (int j0 = 0; j0 < nrhs; j0 += kSolveCols) {
    const int nc = std::min(kSolveCols, nrhs - j0);
    double* xc = x + (long long)j0 * ld;
    // forward sweep, leaves -> root
    for (int l = L; l >= 1; --l) {
      Level& P = h->lv[l];
      Level& Q = h->lv[l - 1];
      double* vec = (l == L) ? xc : P.yv;
      const int ldv = (l == L) ? ld : P.n * P.b;
      apply_q(h, P, vec, ldv, nc, /*transpose=*/true, st);
      {
        Launch k(h, HSS_K_TRSV_FWD, trsv_flops(P.b, P.c, nc) * P.n, st);
        launch_trsv_fwd<double>(P.M, P.b, (long long)P.b * P.b, P.b, P.c, vec, ldv, P.b, nc, Q.yv,
                                Q.n * Q.b, r, P.n, st);
      }
    }
    Level& R0 = h->lv[0];
    {
      Launch k(h, HSS_K_TRSV_FWD, trsv_flops(R0.b, R0.b, nc), st);
      launch_trsv_fwd<double>(R0.A, R0.b, 0, R0.b, R0.b, R0.yv, R0.b, 0, nc, nullptr, 0, 0, 1,
                              st);
    }
    {
      Launch k(h, HSS_K_TRSV_BWD, trsv_flops(R0.b, R0.b, nc), st);
      launch_trsv_bwd<double>(R0.A, R0.b, 0, R0.b, R0.b, R0.yv, R0.b, 0, nc, nullptr, 0, 0, 1,
                              st);
    }
    // backward sweep, root -> leaves
    for (int l = 1; l <= L; ++l) {
      Level& P = h->lv[l];
      Level& Q = h->lv[l - 1];
      double* vec = (l == L) ? xc : P.yv;
      const int ldv = (l == L) ? ld : P.n * P.b;
      {
        Launch k(h, HSS_K_TRSV_BWD, trsv_flops(P.b, P.c, nc) * P.n, st);
        launch_trsv_bwd<double>(P.M, P.b, (long long)P.b * P.b, P.b, P.c, vec, ldv, P.b, nc, Q.yv,
                                Q.n * Q.b, r, P.n, st);
      }
      apply_q(h, P, vec, ldv, nc, /*transpose=*/false, st);
    }
    int rc = check_launch();
    if (rc) return rc;
  }
  return HSS_OK;
}

int matvec_fp64(hss_s* h, const double* x, double* y, int nrhs, int ld, cudaStream_t st) {
  const int L = h->L, r = h->rank, leaf = h->leaf;
  const long long rr = (long long)r * r;
  const int nL = 1 << L;
  for (int j0 = 0; j0 < nrhs; j0 += kMaxCols) {
    const int nc = std::min(kMaxCols, nrhs - j0);
    const double* xc = x + (long long)j0 * ld;
    double* yc = y + (long long)j0 * ld;
    // up-sweep: x̂_L = Uᵀ x, x̂_l = E_lᵀ [x̂_{l+1}(2p); x̂_{l+1}(2p+1)]
    gemm(h, true, false, r, nc, leaf, 1.0, h->U, leaf, (long long)leaf * r, xc, ld,
                         leaf, 0.0, h->lv[L].xh, nL * r, r, nL, st);
    for (int l = L - 1; l >= 1; --l) {
      Level& P = h->lv[l];
      Level& C = h->lv[l + 1];
      gemm(h, true, false, r, nc, 2 * r, 1.0, h->E + h->Eoff[l], 2 * r, 2 * rr, C.xh,
                           C.n * r, 2 * r, 0.0, P.xh, P.n * r, r, P.n, st);
    }
    // sibling couplings of every level
    for (int l = 1; l <= L; ++l) {
      Level& P = h->lv[l];
      const double* Sl = h->S + h->Soff[l];
      const int ldl = P.n * r;
      gemm(h, false, false, r, nc, r, 1.0, Sl, r, rr, P.xh, ldl, 2 * r, 0.0, P.yh + r,
                           ldl, 2 * r, P.n / 2, st);
      gemm(h, true, false, r, nc, r, 1.0, Sl, r, rr, P.xh + r, ldl, 2 * r, 0.0, P.yh,
                           ldl, 2 * r, P.n / 2, st);
    }
    // down-sweep: ŷ_{l+1}(children) += E_l ŷ_l
    for (int l = 1; l <= L - 1; ++l) {
      Level& P = h->lv[l];
      Level& C = h->lv[l + 1];
      gemm(h, false, false, 2 * r, nc, r, 1.0, h->E + h->Eoff[l], 2 * r, 2 * rr, P.yh,
                           P.n * r, r, 1.0, C.yh, C.n * r, 2 * r, P.n, st);
    }
    // leaves: y = D x + U ŷ
    gemm(h, false, false, leaf, nc, leaf, 1.0, h->D, leaf, (long long)leaf * leaf, xc,
                         ld, leaf, 0.0, yc, ld, leaf, nL, st);
    gemm(h, false, false, leaf, nc, r, 1.0, h->U, leaf, (long long)leaf * r,
                         h->lv[L].yh, nL * r, r, 1.0, yc, ld, leaf, nL, st);
    int rc = check_launch();
    if (rc) return rc;
  }
  return HSS_OK;
}

int read_status(hss_s* h, int* st_host) {
  cudaError_t e = cudaMemcpy(st_host, h->status, 8 * sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return HSS_ERR_CUDA;
  return st_host[ST_CODE];
}

}  // namespace

extern "C" {

const char* hss_strerror(int code) {
  switch (code) {
    case HSS_OK: return "ok";
    case HSS_ERR_INVALID_ARG: return "invalid argument";
    case HSS_ERR_NOT_FACTORIZED: return "not factorized";
    case HSS_ERR_NOT_SPD: return "matrix not positive definite (non-positive Cholesky pivot)";
    case HSS_ERR_CUDA: return "CUDA error";
    case HSS_ERR_OOM: return "out of device memory";
    case HSS_ERR_TIMEOUT: return "device wait timed out";
    case HSS_ERR_NO_CONVERGENCE: return "iterative refinement did not converge";
    case HSS_ERR_TOO_LARGE: return "problem exceeds the fixed scratch of hss_matvec_noalloc";
    default: return "unknown error";
  }
}

int hss_create(const hss_shape* shape, const double* D, const double* U, const double* E,
               const double* S, int on_device, hss_t* out) {
  if (!shape || !out || !D || !U || !S) return HSS_ERR_INVALID_ARG;
  *out = nullptr;
  const int L = shape->levels, leaf = shape->leaf, r = shape->rank;
  if (L < 1 || L > 24 || leaf < 1 || leaf > 768 || r < 1 || r > leaf || r > 256)
    return HSS_ERR_INVALID_ARG;
  if ((long long)leaf << L != (long long)shape->n) return HSS_ERR_INVALID_ARG;
  if (L >= 2 && !E) return HSS_ERR_INVALID_ARG;
  hss_s* h = new (std::nothrow) hss_s();
  if (!h) return HSS_ERR_OOM;
  h->n = shape->n;
  h->leaf = leaf;
  h->rank = r;
  h->L = L;
  cudaGetDevice(&h->device);
  const size_t bytes = layout(h, nullptr);
  void* mem = nullptr;
  if (cudaMalloc(&mem, bytes) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return HSS_ERR_OOM;
  }
  h->arena = mem;
  h->arena_bytes = bytes;
  layout(h, static_cast<char*>(mem));
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const long long nL = 1LL << L;
  cudaError_t e = cudaSuccess;
  e = e ? e : cudaMemcpy(h->D, D, sizeof(double) * nL * leaf * leaf, kind);
  e = e ? e : cudaMemcpy(h->U, U, sizeof(double) * nL * leaf * r, kind);
  if (L >= 2) {
    const long long esz = h->Eoff[L - 1] + (1LL << (L - 1)) * 2 * r * r;
    e = e ? e : cudaMemcpy(h->E, E, sizeof(double) * esz, kind);
  }
  const long long ssz = h->Soff[L] + (1LL << (L - 1)) * (long long)r * r;
  e = e ? e : cudaMemcpy(h->S, S, sizeof(double) * ssz, kind);
  e = e ? e : cudaMemset(h->status, 0, 8 * sizeof(int));
  if (e != cudaSuccess) {
    cudaFree(mem);
    delete h;
    return HSS_ERR_CUDA;
  }
  *out = h;
  return HSS_OK;
}

void hss_destroy(hss_t h) {
  if (!h) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(h->device);
  clear_trace(h);
  cudaFree(h->arena);
  cudaSetDevice(cur);
  delete h;
}

int hss_factorize(hss_t h, const hss_options* opt, void* stream) {
  if (!h) return HSS_ERR_INVALID_ARG;
  const int prec = opt ? opt->precision : HSS_FP64;
  if (prec != HSS_FP64) return HSS_ERR_INVALID_ARG;   // mixed modes: not built yet
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  h->factorized = 0;
  int rc = factorize_fp64(h, st);
  if (rc) return rc;
  h->precision = prec;
  h->factorized = 1;
  h->last_stream = st;
  return HSS_OK;
}

int hss_solve(hss_t h, const double* b, double* x, int32_t nrhs, int32_t ld, void* stream) {
  if (!h || !b || !x || nrhs < 0 || ld < h->n) return HSS_ERR_INVALID_ARG;
  if (!h->factorized) return HSS_ERR_NOT_FACTORIZED;
  if (nrhs == 0) return HSS_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (x != b) {
    cudaError_t e = cudaMemcpy2DAsync(x, sizeof(double) * ld, b, sizeof(double) * ld,
                                      sizeof(double) * h->n, nrhs, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return HSS_ERR_CUDA;
  }
  h->last_stream = st;
  return solve_fp64(h, x, nrhs, ld, st);
}

int hss_matvec(hss_t h, const double* x, double* y, int32_t nrhs, int32_t ld, void* stream) {
  if (!h || !x || !y || nrhs < 0 || ld < h->n || x == y) return HSS_ERR_INVALID_ARG;
  if (nrhs == 0) return HSS_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  h->last_stream = st;
  return matvec_fp64(h, x, y, nrhs, ld, st);
}

int hss_sync(hss_t h) {
  if (!h) return HSS_ERR_INVALID_ARG;
  if (cudaStreamSynchronize(h->last_stream) != cudaSuccess) return HSS_ERR_CUDA;
  int s[8];
  return read_status(h, s);
}

int hss_logdet(hss_t h, double* out) {
  if (!h || !out) return HSS_ERR_INVALID_ARG;
  if (!h->factorized) return HSS_ERR_NOT_FACTORIZED;
  int rc = hss_sync(h);
  if (rc) return rc;
  if (cudaMemcpy(out, h->logdet_val, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
    return HSS_ERR_CUDA;
  return HSS_OK;
}

int hss_last_info(hss_t h, int32_t* level, int32_t* node, int32_t* col, int32_t* ir_iters,
                  double* ir_resid) {
  if (!h) return HSS_ERR_INVALID_ARG;
  if (cudaStreamSynchronize(h->last_stream) != cudaSuccess) return HSS_ERR_CUDA;
  int s[8];
  int rc = read_status(h, s);
  if (rc < 0 && rc != HSS_ERR_CUDA) {
    if (level) *level = s[ST_LEVEL];
    if (node) *node = s[ST_NODE];
    if (col) *col = s[ST_COL];
  } else {
    if (level) *level = -1;
    if (node) *node = -1;
    if (col) *col = -1;
  }
  if (ir_iters) *ir_iters = h->ir_iters;
  if (ir_resid) *ir_resid = h->ir_resid;
  return rc;
}

int hss_trace(hss_t h, int32_t enable) {
  if (!h) return HSS_ERR_INVALID_ARG;
  if (enable) {
    for (auto& r : h->trace) cudaEventSynchronize(r.b);
    clear_trace(h);
  }
  h->tracing = enable ? 1 : 0;
  return HSS_OK;
}

int hss_trace_read(hss_t h, int32_t kind, double* ms, int64_t* launches, double* flops) {
  if (!h || kind < 0 || kind >= HSS_K_COUNT) return HSS_ERR_INVALID_ARG;
  double tot = 0.0, fl = 0.0;
  long long cnt = 0;
  for (auto& r : h->trace) {
    if (r.kind != kind) continue;
    if (cudaEventSynchronize(r.b) != cudaSuccess) return HSS_ERR_CUDA;
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) return HSS_ERR_CUDA;
    tot += t;
    fl += r.flops;
    ++cnt;
  }
  if (ms) *ms = tot;
  if (launches) *launches = cnt;
  if (flops) *flops = fl;
  return HSS_OK;
}

int hss_launch_count(hss_t h, int64_t* out) {
  if (!h || !out) return HSS_ERR_INVALID_ARG;
  *out = h->launches;
  return HSS_OK;
}

int hss_export(hss_t h, int32_t what, int32_t level, double* dst, size_t count) {
  if (!h || !dst || level < 0 || level > h->L) return HSS_ERR_INVALID_ARG;
  if (!h->factorized) return HSS_ERR_NOT_FACTORIZED;
  if (h->precision != HSS_FP64) return HSS_ERR_INVALID_ARG;
  const Level& P = h->lv[level];
  const double* src = nullptr;
  size_t n = 0;
  const size_t r = h->rank;
  switch (what) {
    case 0: src = P.V; n = (size_t)P.n * P.b * r; break;
    case 1: src = P.T; n = (size_t)P.n * r * r; break;
    case 2: src = P.LB; n = (size_t)P.n * r * r; break;
    case 3: src = P.M; n = (size_t)P.n * P.b * P.b; break;
    case 4: src = P.B; n = (size_t)P.n * P.b * r; break;
    default: return HSS_ERR_INVALID_ARG;
  }
  if (!src || n > count) return HSS_ERR_INVALID_ARG;
  if (cudaStreamSynchronize(h->last_stream) != cudaSuccess) return HSS_ERR_CUDA;
  return cuda_err(cudaMemcpy(dst, src, n * sizeof(double), cudaMemcpyDeviceToHost));
}

}  // extern "C"
