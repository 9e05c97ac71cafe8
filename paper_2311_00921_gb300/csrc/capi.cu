// C ABI of the HSS-ULV library: the device-resident object, its arenas, and the
// level schedule of Alg. 2 (factor), the solve of Sec. 3.2, the HSS matvec and
// iterative refinement for the mixed-precision factor.
//
// Per level l the work is batched over the 2^l nodes of the level; each step is
// one launch (batched GEMM / SYR2K / per-node kernel), so a level costs a fixed
// handful of launches whatever its node count.  The schedule is written once,
// templated on the arithmetic type: double for HSS_FP64, float for the mixed
// modes (whose root Cholesky, residual and update stay in double).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "../../include/hss.h"
#include "basis.cuh"
#include "common.cuh"
#include "dfgemm.cuh"
#include "ir_kernels.cuh"
#include "tc_gemm.cuh"
#include "ulv_kernels.cuh"
#include "uneven.cuh"

#include <type_traits>

namespace {

constexpr int kMaxCols = 32;      // right-hand-side columns per matvec pass
constexpr int kSolveCols = 16;    // columns per triangular-sweep / refinement pass
constexpr int kPanel = 32;        // columns per blocked-Cholesky panel (the panel kernel's limit)
constexpr int kRootPanels = 16;
constexpr int kFuseNodes = 64;    // levels up to this many nodes apply Q inside the sweep kernel
constexpr int kTreeTop = 6;       // levels 1 .. 6 (<= 64 nodes): one tree launch per direction

template <typename T>
struct LevelT {
  int n = 0, b = 0, r = 0, c = 0;
  T* V = nullptr;   // n x b x r Householder vectors
  T* T_ = nullptr;  // n x r x r compact-WY factor
  T* LB = nullptr;  // n x r x r, L_B = Q^Sᵀ B
  T* M = nullptr;   // n x b x b factored blocks (leaves: own buffer; else = A)
  T* A = nullptr;   // n x b x b merged blocks (levels < L), 1 block at the root
  T* B = nullptr;   // n x b x r bases fed to the QL (levels 1 .. L-1)
  T* yv = nullptr;  // level vector of the solve: (n b) x kSolveCols
};

template <typename T>
struct Factor {
  std::vector<LevelT<T>> lv;   // index = level (0 = root)
  T *W = nullptr, *Y = nullptr, *X = nullptr, *Z = nullptr;
  T *t1 = nullptr, *t2 = nullptr;   // r x kSolveCols per node: Q application of wide levels
  const T *D = nullptr, *U = nullptr, *E = nullptr, *S = nullptr;   // generators in T
  T *Dc = nullptr, *Uc = nullptr, *Ec = nullptr, *Sc = nullptr;     // converted copies (float)
  T* d = nullptr;               // n x kSolveCols refinement correction (float)
  BasisScratch<T> bs;           // scratch of the basis completion chain
  void* arena = nullptr;
  size_t bytes = 0;
};

// One refinement lane: the right-hand-side columns [col0, col0 + nc) of a pass
// refine on their own stream with their own slice of every scratch vector, so
// that two lanes overlap (one lane's FP32 sweeps beside the other's FP64
// matvec).  Lane 0 runs on the caller's stream.
struct Lane {
  cudaStream_t st = nullptr;        // lane 1 only (lane 0 uses the caller's)
  cudaStream_t ms = nullptr;        // the matvec's leaf product D x
  cudaEvent_t mv_start = nullptr, mv_dx = nullptr, norm_ready = nullptr;
  int* tcnt = nullptr;              // arrival counts of the tree forward sweep
  int* tready = nullptr;            // ready flags of the tree backward sweep
  int epoch = 0;
};

}  // namespace

struct hss_s {
  int n = 0, leaf = 0, rank = 0, L = 0;   // n: order of the (padded) uniform tree
  int n_user = 0;                      // order of the caller's matrix (= n unless uneven)
  int uneven = 0;                      // an uneven tree embedded in the uniform one
  int* pmap = nullptr;                 // n entries: caller's row of each padded row, or -1
  double *vin = nullptr, *vout = nullptr;   // padded vectors (n x kMaxCols) of uneven calls
  int device = 0;
  double *D = nullptr, *U = nullptr, *E = nullptr, *S = nullptr;
  long long esz = 0, ssz = 0;
  std::vector<long long> Eoff, Soff;   // element offset of level l in E / S
  Factor<double> f64;
  Factor<float> f32;
  std::vector<double*> xh, yh;         // matvec up / down sweep per level: (2^l r) x kMaxCols
  double* R0 = nullptr;                // FP64 root block of a mixed factor (2r x 2r)
  double* root_vec = nullptr;          // FP64 root vector of a mixed solve (2r x kSolveCols)
  double* root_vec2 = nullptr;
  double* A0inv = nullptr;             // FP64 inverse of the root block (mixed solves)
  int a0inv_valid = 0;
  double* rbuf = nullptr;              // n x kSolveCols residual
  double* bbuf = nullptr;              // n x kSolveCols copy of b (x aliasing b)
  double* norms = nullptr;             // 6 x kSolveCols: |b|, 1/|b|, |r|, 1/|r|, |x|, 1/|x|
  double* norm_part = nullptr;         // 64 x kSolveCols partial sums of the column norms
  double* logdet_part = nullptr;       // 2^(L+1) - 1 node contributions
  double* logdet_val = nullptr;
  int* status = nullptr;
  void* arena = nullptr;
  size_t arena_bytes = 0;
  int factorized = 0;
  int precision = HSS_FP64;
  int use_tc = 0;                      // tensor-core contractions in the FP32 factor
  void* tc_ws = nullptr;               // packed tensor-core operands (allocated on first use)
  size_t tc_ws_bytes = 0;
  TcMode tc_mode = TcMode::TF32x3;
  int ir_max_it = 30;
  double ir_tol = 1e-12;
  long long wait_budget = 0;           // polls of a device pipeline wait (0 = default)
  int residual = HSS_RESIDUAL_FP64;    // arithmetic of the refinement residual
  int basis_method = HSS_BASIS_HOUSEHOLDER;   // method of the basis completion
  int schedule = HSS_SCHEDULE_ASYNC;   // launches of the solve's upper levels
  int staging = 0;                     // panel staging of the sweep kernels (see launch_ulv_fwd)
  int tuned = 0;                       // hss_tune has chosen the following
  int tuned_basis = HSS_BASIS_HOUSEHOLDER, tuned_schedule = HSS_SCHEDULE_ASYNC, tuned_staging = 0;
  int tuned_panel = 0, tuned_lanes = 1;
  int ql_panel = 0;                    // register panel of the Householder basis kernel (0 = default)

  // pair-of-FP32 generators (hi parts are the FP32 factor's converted copies)
  // and the pair matvec's vectors, in the FP32 arena
  float *Dl = nullptr, *Ul = nullptr, *El = nullptr, *Sl = nullptr;
  float *xs_h = nullptr, *xs_l = nullptr, *yt_h = nullptr, *yt_l = nullptr;
  std::vector<float*> xp_h, xp_l, yp_h, yp_l;
  int pairs_valid = 0;
  cudaStream_t last_stream = nullptr;
  // basis-completion chain runs ahead on its own stream; one event per level
  cudaStream_t qstream = nullptr;
  std::vector<cudaEvent_t> ev_level;
  cudaEvent_t ev_start = nullptr;
  Lane lane[2];                        // refinement lanes (lane 0 also serves every other call)
  cudaEvent_t ev_ir_fork = nullptr, ev_ir_join = nullptr;
  double* hnorm = nullptr;             // pinned host: |b|, |r| of the kSolveCols columns, then
                                       // each refinement lane's status words (8 ints a lane)
  int ir_lanes = 1;                    // refinement lanes (2: one lane's FP32 sweeps beside
                                       // the other's FP64 matvec), the tuner's choice
  double* zq64 = nullptr;              // merge scratch of the basis chain (n_L/2 x r x r)
  float* zq32 = nullptr;
  int ir_iters = 0;
  double ir_resid = 0.0;
  // launch accounting and the optional per-launch event log
  long long launches = 0;
  int tracing = 0;
  int serialize = 0;                   // run the basis chain, the matvec and both
                                       // refinement lanes on the caller's stream only
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
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

template <typename T>
void layout_factor(Bump& bp, Factor<T>& f, int L, int leaf, int r) {
  f.lv.assign(L + 1, LevelT<T>());
  const size_t nL = size_t(1) << L;
  for (int l = 0; l <= L; ++l) {
    LevelT<T>& P = f.lv[l];
    P.n = 1 << l;
    P.b = (l == L) ? leaf : 2 * r;
    P.r = (l == 0) ? 0 : r;
    P.c = P.b - P.r;
    if (l >= 1) {
      P.V = bp.take<T>((size_t)P.n * P.b * r);
      P.T_ = bp.take<T>((size_t)P.n * r * r);
      P.LB = bp.take<T>((size_t)P.n * r * r);
    }
    if (l < L) {
      P.A = bp.take<T>((size_t)P.n * P.b * P.b);
      P.M = P.A;
    } else {
      P.M = bp.take<T>((size_t)P.n * P.b * P.b);
    }
    if (l >= 1 && l < L) P.B = bp.take<T>((size_t)P.n * P.b * r);
    if (l < L) P.yv = bp.take<T>((size_t)P.n * P.b * kSolveCols);
  }
  f.W = bp.take<T>(nL * leaf * r);
  f.Y = bp.take<T>(nL * leaf * r);
  f.X = bp.take<T>(nL * r * r);
  f.Z = bp.take<T>(nL * r * r);
  f.t1 = bp.take<T>(nL * r * kSolveCols);
  f.t2 = bp.take<T>(nL * r * kSolveCols);
  // the basis chain runs concurrently with the main chain: its own scratch
  f.bs.X = bp.take<T>(nL * leaf * r);
  for (T** p : {&f.bs.G, &f.bs.R1, &f.bs.R, &f.bs.P, &f.bs.U, &f.bs.Ui})
    *p = bp.take<T>(nL * r * r);
  f.bs.fail = bp.take<int>(nL);
}

// the object's main arena: FP64 generators, FP64 factor, matvec and refinement
size_t layout_main(hss_s* h, char* base) {
  Bump bp{base};
  const int L = h->L, r = h->rank, leaf = h->leaf;
  const long long nL = 1LL << L;
  h->D = bp.take<double>(nL * leaf * leaf);
  h->U = bp.take<double>(nL * leaf * r);
  h->Eoff.assign(L + 1, 0);
  h->Soff.assign(L + 1, 0);
  h->esz = h->ssz = 0;
  for (int l = 1; l <= L - 1; ++l) {
    h->Eoff[l] = h->esz;
    h->esz += (1LL << l) * 2 * r * r;
  }
  for (int l = 1; l <= L; ++l) {
    h->Soff[l] = h->ssz;
    h->ssz += (1LL << (l - 1)) * r * r;
  }
  h->E = bp.take<double>(std::max<long long>(h->esz, 1));
  h->S = bp.take<double>(h->ssz);
  layout_factor<double>(bp, h->f64, L, leaf, r);
  h->f64.D = h->D;
  h->f64.U = h->U;
  h->f64.E = h->E;
  h->f64.S = h->S;
  h->xh.assign(L + 1, nullptr);
  h->yh.assign(L + 1, nullptr);
  for (int l = 1; l <= L; ++l) {
    h->xh[l] = bp.take<double>((size_t(1) << l) * r * kMaxCols);
    h->yh[l] = bp.take<double>((size_t(1) << l) * r * kMaxCols);
  }
  h->zq64 = bp.take<double>((size_t)nL * r * r);
  h->R0 = bp.take<double>((size_t)4 * r * r);
  h->A0inv = bp.take<double>((size_t)4 * r * r);
  h->root_vec = bp.take<double>((size_t)2 * r * kSolveCols);
  h->root_vec2 = bp.take<double>((size_t)2 * r * kSolveCols);
  h->rbuf = bp.take<double>((size_t)h->n * kSolveCols);
  h->bbuf = bp.take<double>((size_t)h->n * kSolveCols);
  h->norms = bp.take<double>(6 * kSolveCols);
  h->norm_part = bp.take<double>(64 * kSolveCols);
  h->logdet_part = bp.take<double>((size_t)(2 * nL - 1) + kRootPanels);
  h->logdet_val = bp.take<double>(1);
  h->status = bp.take<int>(8);
  for (Lane& ln : h->lane) {
    ln.tcnt = bp.take<int>(size_t(2) << kTreeTop);
    ln.tready = bp.take<int>(size_t(2) << kTreeTop);
  }
  if (h->uneven) {
    h->pmap = bp.take<int>((size_t)h->n);
    h->vin = bp.take<double>((size_t)h->n * kMaxCols);
    h->vout = bp.take<double>((size_t)h->n * kMaxCols);
  }
  return bp.off + 256;
}

// the FP32 arena of the mixed modes: converted generators, factor, correction
size_t layout_f32(hss_s* h, char* base) {
  Bump bp{base};
  const int L = h->L, r = h->rank, leaf = h->leaf;
  const long long nL = 1LL << L;
  Factor<float>& f = h->f32;
  f.Dc = bp.take<float>(nL * leaf * leaf);
  f.Uc = bp.take<float>(nL * leaf * r);
  f.Ec = bp.take<float>(std::max<long long>(h->esz, 1));
  f.Sc = bp.take<float>(h->ssz);
  layout_factor<float>(bp, f, L, leaf, r);
  f.d = bp.take<float>((size_t)h->n * kSolveCols);
  h->zq32 = bp.take<float>((size_t)nL * r * r);
  h->Dl = bp.take<float>(nL * leaf * leaf);
  h->Ul = bp.take<float>(nL * leaf * r);
  h->El = bp.take<float>(std::max<long long>(h->esz, 1));
  h->Sl = bp.take<float>(h->ssz);
  h->xs_h = bp.take<float>((size_t)h->n * kSolveCols);
  h->xs_l = bp.take<float>((size_t)h->n * kSolveCols);
  h->yt_h = bp.take<float>((size_t)h->n * kSolveCols);
  h->yt_l = bp.take<float>((size_t)h->n * kSolveCols);
  for (auto* v : {&h->xp_h, &h->xp_l, &h->yp_h, &h->yp_l}) {
    v->assign(L + 1, nullptr);
    for (int l = 1; l <= L; ++l) (*v)[l] = bp.take<float>((size_t(1) << l) * r * kSolveCols);
  }
  f.D = f.Dc;
  f.U = f.Uc;
  f.E = f.Ec;
  f.S = f.Sc;
  return bp.off + 256;
}

int cuda_err(cudaError_t e) { return e == cudaSuccess ? HSS_OK : HSS_ERR_CUDA; }

// a launcher's error: shared memory the device cannot give is a size problem,
// anything else a CUDA failure
#define HSS_TRY(call)                                                                  \
  do {                                                                                 \
    const cudaError_t e_ = (call);                                                     \
    if (e_ != cudaSuccess)                                                             \
      return e_ == cudaErrorInvalidConfiguration ? HSS_ERR_INVALID_ARG : HSS_ERR_CUDA; \
  } while (0)

int check_launch() {
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HSS_OK : HSS_ERR_CUDA;
}

// Brackets one kernel launch: counts it and, when tracing, logs two events.
struct Launch {
  hss_s* h;
  cudaStream_t st;
  hss_s::Rec rec{};
  bool on = false;
  Launch(hss_s* h_, int kind, double flops, cudaStream_t st_, bool f32 = false)
      : h(h_), st(st_) {
    ++h->launches;
    if (f32) kind += HSS_K_FP32;
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

// Hooks of the basis completion chain: the same accounting as Launch, opened
// before and closed after each of its launches.
struct BasisTrace {
  hss_s* h;
  cudaStream_t st;
  bool f32;
  hss_s::Rec rec{};
  bool on = false;
};

void basis_before(void* ctx, int kind, double flops) {
  BasisTrace* t = static_cast<BasisTrace*>(ctx);
  ++t->h->launches;
  t->on = false;
  if (!t->h->tracing) return;
  static const int cls[4] = {HSS_K_BASIS_GEMM, HSS_K_BASIS_NODE, HSS_K_OTHER, HSS_K_QL};
  t->rec.kind = cls[kind] + (t->f32 ? HSS_K_FP32 : 0);
  t->rec.flops = flops;
  if (cudaEventCreate(&t->rec.a) == cudaSuccess && cudaEventCreate(&t->rec.b) == cudaSuccess) {
    cudaEventRecord(t->rec.a, t->st);
    t->on = true;
  }
}

void basis_after(void* ctx) {
  BasisTrace* t = static_cast<BasisTrace*>(ctx);
  if (!t->on) return;
  cudaEventRecord(t->rec.b, t->st);
  t->h->trace.push_back(t->rec);
  t->on = false;
}

void clear_trace(hss_s* h) {
  for (auto& r : h->trace) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  h->trace.clear();
}

template <typename T>
void gemm(hss_s* h, bool ta, bool tb, int m, int n, int k, T alpha, const T* A, int lda,
          long long sA, const T* B, int ldb, long long sB, T beta, T* C, int ldc, long long sC,
          int batch, cudaStream_t st) {
  if (m <= 0 || n <= 0 || k <= 0 || batch <= 0) return;
  Launch l(h, n <= 32 ? HSS_K_GEMM_SKINNY : HSS_K_GEMM, 2.0 * m * n * (double)k * batch, st,
           sizeof(T) == 4);
  gemm_batched<T>(ta, tb, m, n, k, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, batch, st);
}

// partial Cholesky of the first c of b columns: POTRF c x c, TRSM (b-c) x c,
// SYRK (b-c) x (b-c) with depth c
// one Cholesky panel: kb x kb POTRF plus the (rows - kb) x kb TRSM
double panel_flops(int rows, int kb) {
  return (double)kb * kb * kb / 3.0 + (double)(rows - kb) * kb * kb;
}

// triangular sweep of one node: c x c triangle plus the (b-c) x c block
double trsv_flops(int b, int c, int nrhs) { return ((double)c * c + 2.0 * (b - c) * c) * nrhs; }

// (I - V op(T) Vᵀ) on b x nrhs: two b x r products and one r x r
double qapply_flops(int b, int r, int nrhs) { return (4.0 * b * r + 2.0 * r * r) * nrhs; }

enum { SPLIT_D = 1, SPLIT_U = 2, SPLIT_E = 4, SPLIT_S = 8, SPLIT_ALL = 15 };
cudaError_t split_generators(hss_s* h, cudaStream_t st, int which, bool lo);

// levels L .. 1 of Alg. 2; leaves the merged root block in f.lv[0].A.
// Two chains: the basis chain (basis completion of level l, then the merge's
// rescaled coupling Ŝ and the parent basis, which need only L_B of level l) runs
// ahead on h->qstream; the main chain (diagonal product and partial Cholesky of
// level l) waits for level l's basis event.  The levels' basis completions,
// latency-bound at the top of the tree, thus overlap the main chain.  With
// split_d the FP32 copy of D is made on the main chain once the basis chain has
// started (only the leaves' diagonal product needs it).
template <typename T>
int factor_levels(hss_s* h, Factor<T>& f, T* zq, cudaStream_t st, bool split_d) {
  const int L = h->L, r = h->rank;
  const long long rr = (long long)r * r;
  cudaStream_t qs = h->serialize ? st : h->qstream;
  if (cudaEventRecord(h->ev_start, st) != cudaSuccess) return HSS_ERR_CUDA;
  if (cudaStreamWaitEvent(qs, h->ev_start, 0) != cudaSuccess) return HSS_ERR_CUDA;
  if constexpr (std::is_same<T, float>::value) {
    if (split_d && split_generators(h, st, SPLIT_D, h->residual == HSS_RESIDUAL_PAIR32) !=
                       cudaSuccess)
      return HSS_ERR_CUDA;
  }
  // basis chain
  for (int l = L; l >= 1; --l) {
    LevelT<T>& P = f.lv[l];
    LevelT<T>& Q = f.lv[l - 1];
    const int b = P.b, n = P.n;
    const long long br = (long long)b * r;
    // (a) basis completion (Eq. 2-3)
    const T* Bsrc = (l == L) ? f.U : P.B;
    if (h->basis_method == HSS_BASIS_CHOLQR && r <= basis_max_rank<T>()) {
      // Cholesky QR twice + Householder reconstruction; Householder kernel for
      // the nodes it flags
      BasisTrace bt{h, qs, sizeof(T) == 4};
      BasisHook hook;
      hook.before = basis_before;
      hook.after = basis_after;
      hook.ctx = &bt;
      HSS_TRY(launch_basis_completion<T>(Bsrc, br, P.V, br, P.T_, rr, P.LB, rr, b, r, n, f.bs,
                                         hook, qs));
    } else {
      Launch k(h, HSS_K_QL, (2.0 * b * r * r - 2.0 / 3.0 * r * r * r + 1.0 * b * r * r) * n, qs,
               sizeof(T) == 4);
      HSS_TRY(launch_ql_basis<T>(Bsrc, b, br, P.V, br, P.T_, rr, P.LB, rr, b, r, n, qs, nullptr,
                                 h->ql_panel));
    }
    // (d, first half) merge: Ŝ = L_B(c2) S L_B(c1)ᵀ and Ŝᵀ into the parent's
    // off-diagonal blocks, parent basis blkdiag(L_B(c1), L_B(c2)) E_p
    const int np = n / 2;
    const T* Sl = f.S + h->Soff[l];
    const int ldq = 2 * r;
    const long long sq = 4 * rr;
    gemm<T>(h, false, false, r, r, r, T(1), P.LB + rr, r, 2 * rr, Sl, r, rr, T(0), zq, r, rr, np,
            qs);
    gemm<T>(h, false, true, r, r, r, T(1), zq, r, rr, P.LB, r, 2 * rr, T(0), Q.A + r, ldq, sq, np,
            qs);
    gemm<T>(h, false, true, r, r, r, T(1), P.LB, r, 2 * rr, zq, r, rr, T(0),
            Q.A + (long long)r * ldq, ldq, sq, np, qs);
    if (l - 1 >= 1) {
      const T* Ep = f.E + h->Eoff[l - 1];
      gemm<T>(h, false, false, r, r, r, T(1), P.LB, r, 2 * rr, Ep, 2 * r, 2 * rr, T(0), Q.B, 2 * r,
              2 * rr, np, qs);
      gemm<T>(h, false, false, r, r, r, T(1), P.LB + rr, r, 2 * rr, Ep + r, 2 * r, 2 * rr, T(0),
              Q.B + r, 2 * r, 2 * rr, np, qs);
    }
    if (cudaEventRecord(h->ev_level[l], qs) != cudaSuccess) return HSS_ERR_CUDA;
    int rc = check_launch();
    if (rc) return rc;
  }
  // main chain
  for (int l = L; l >= 1; --l) {
    LevelT<T>& P = f.lv[l];
    LevelT<T>& Q = f.lv[l - 1];
    const int b = P.b, n = P.n, c = P.c;
    const long long br = (long long)b * r, bb = (long long)b * b;
    const int ldq = 2 * r;
    const long long sq = 4 * rr;
    if (cudaStreamWaitEvent(st, h->ev_level[l], 0) != cudaSuccess) return HSS_ERR_CUDA;
    // (b) diagonal product Â = Qᵀ A Q with Q = I - V T Vᵀ, in the symmetric
    // compact-WY form Â = A - Y'Vᵀ - V Y'ᵀ, Y' = A V T - ½ V Tᵀ Vᵀ A V T
    const T* Ain = (l == L) ? f.D : P.A;
    bool tc = false;
    if constexpr (std::is_same<T, float>::value) {
      if (h->use_tc) {
        tc = true;
        Launch k(h, HSS_K_TC_GEMM, 2.0 * b * r * (double)b * n, st);
        // W (b x r) = A V: rows of A against columns of V, both along K = b
        const TcOperand a{Ain, b, bb, nullptr, 0, 0, 0, false};
        const TcOperand v{P.V, b, br, nullptr, 0, 0, 0, true};
        if (tc_gemm(h->tc_mode, b, r, b, a, v, f.W, b, br, n, h->tc_ws, h->tc_ws_bytes,
                    h->status, h->wait_budget, st) != cudaSuccess)
          return HSS_ERR_CUDA;
      }
    }
    if (!tc)
      gemm<T>(h, false, false, b, r, b, T(1), Ain, b, bb, P.V, b, br, T(0), f.W, b, br, n, st);
    gemm<T>(h, false, false, b, r, r, T(1), f.W, b, br, P.T_, r, rr, T(0), f.Y, b, br, n, st);
    gemm<T>(h, true, false, r, r, b, T(1), P.V, b, br, f.Y, b, br, T(0), f.X, r, rr, n, st);
    gemm<T>(h, true, false, r, r, r, T(1), P.T_, r, rr, f.X, r, rr, T(0), f.Z, r, rr, n, st);
    gemm<T>(h, false, false, b, r, r, T(-0.5), P.V, b, br, f.Z, r, rr, T(1), f.Y, b, br, n, st);
    if (tc) {
      if constexpr (std::is_same<T, float>::value) {
        Launch k(h, HSS_K_TC_SYR2K, 2.0 * r * b * (b + 1.0) * n, st);
        if (tc_syr2k_lower(h->tc_mode, b, r, Ain, b, bb, f.Y, b, br, P.V, b, br, P.M, b, bb, n,
                           h->tc_ws, h->tc_ws_bytes, h->status, h->wait_budget, st) != cudaSuccess)
          return HSS_ERR_CUDA;
      }
    } else {
      Launch k(h, HSS_K_SYR2K, 2.0 * r * b * (b + 1.0) * n, st, sizeof(T) == 4);
      syr2k_lower_batched<T>(b, r, Ain, b, bb, f.Y, b, br, P.V, b, br, P.M, b, bb, n, st);
    }
    // (c) partial Cholesky of the first c columns, blocked over the whole level:
    // per panel of kPanel columns a per-node panel kernel (diagonal block and
    // the rows below it) and one SYRK of every node's trailing lower triangle
    double* slots = h->logdet_part + ((1LL << l) - 1);
    if (c == 0 && cudaMemsetAsync(slots, 0, sizeof(double) * n, st) != cudaSuccess)
      return HSS_ERR_CUDA;
    for (int k0 = 0; k0 < c; k0 += kPanel) {
      const int kb = std::min(kPanel, c - k0), rows = b - k0, nt = rows - kb;
      T* Mk = P.M + k0 + (long long)k0 * b;
      {
        Launch k(h, HSS_K_PCHOL, panel_flops(rows, kb) * n, st, sizeof(T) == 4);
        HSS_TRY(launch_chol_panel<T>(Mk, b, bb, rows, kb, slots, l, 0, k0, h->status, n, k0 > 0,
                                     st));
      }
      if (nt > 0) {
        Launch k(h, HSS_K_SYR2K, (double)nt * (nt + 1.0) * kb * n, st, sizeof(T) == 4);
        T* Tr = Mk + kb + (long long)kb * b;
        if (k0 + kb == c)   // the last update leaves Â^SS: its epilogue is the merge
          syrk_lower_merge_batched<T>(nt, kb, Tr, b, bb, Mk + kb, b, bb, Tr, b, bb, Q.A, ldq, sq,
                                      n, st);
        else
          syrk_lower_batched<T>(nt, kb, Tr, b, bb, Mk + kb, b, bb, Tr, b, bb, n, st);
      }
    }
    // (d, second half) with nothing eliminated (c = 0) Â^SS is the whole block:
    // copied into the parents' diagonal blocks by its own pass
    if (c == 0) {
      Launch k(h, HSS_K_OTHER, 0.0, st, sizeof(T) == 4);
      HSS_TRY(launch_scatter_ss<T>(P.M, b, bb, c, r, Q.A, ldq, sq, n, st));
    }
    int rc = check_launch();
    if (rc) return rc;
  }
  return HSS_OK;
}

// Blocked right-looking Cholesky of the FP64 root block (last step of Alg. 2):
// per 32-column panel, the diagonal block and the rows below it with the rows
// split over CTAs of 32 rows, then the trailing update as a batch of 16-column
// blocks, so that neither step queues on one SM's FP64 pipe.
int root_cholesky(hss_s* h, double* R, int b0, cudaStream_t st) {
  double* slots = h->logdet_part + ((2LL << h->L) - 1);
  if (cudaMemsetAsync(slots, 0, kRootPanels * sizeof(double), st) != cudaSuccess ||
      cudaMemsetAsync(h->logdet_part, 0, sizeof(double), st) != cudaSuccess)
    return HSS_ERR_CUDA;
  for (int k0 = 0, p = 0; k0 < b0; k0 += kPanel, ++p) {
    const int kb = std::min(kPanel, b0 - k0), rows = b0 - k0;
    double* Mk = R + k0 + (long long)k0 * b0;
    {
      Launch k(h, HSS_K_PCHOL, panel_flops(rows, kb), st);
      HSS_TRY(launch_chol_panel<double>(Mk, b0, 0, rows, kb, slots + p, 0, 0, k0, h->status, 1,
                                        false, st, std::max(1, (rows - kb + 31) / 32)));
    }
    const int nt = rows - kb;
    if (nt > 0) {
      double* P = Mk + kb;   // rows below the panel
      double* C = R + (k0 + kb) + (long long)(k0 + kb) * b0;
      // column block j (16 columns) of the trailing matrix: C_j -= P P_jᵀ, all
      // blocks in one batched launch; a last partial block on its own
      const int nb16 = nt / 16, tail = nt - 16 * nb16;
      if (nb16 > 0)
        gemm<double>(h, false, true, nt, 16, kb, -1.0, P, b0, 0, P, b0, 16, 1.0, C, b0,
                     16LL * b0, nb16, st);
      if (tail > 0)
        gemm<double>(h, false, true, nt, tail, kb, -1.0, P, b0, 0, P + 16 * nb16, b0, 0, 1.0,
                     C + 16LL * nb16 * b0, b0, 0, 1, st);
    }
  }
  return check_launch();
}

int factorize(hss_s* h, int prec, cudaStream_t st) {
  const int L = h->L, r = h->rank;
  cudaMemsetAsync(h->status, 0, 8 * sizeof(int), st);
  double* root = nullptr;
  if (prec == HSS_FP64) {
    int rc = factor_levels<double>(h, h->f64, h->zq64, st, false);
    if (rc) return rc;
    root = h->f64.lv[0].A;
  } else {
    Factor<float>& f = h->f32;
    // the generators in FP32 (part of every factorization), with their
    // low-order FP32 parts when the residual is the pair-arithmetic one: U, E
    // and S before the basis chain starts, D (the large one) on the main chain
    // after it
    const bool lo = h->residual == HSS_RESIDUAL_PAIR32;
    h->pairs_valid = 0;
    HSS_TRY(split_generators(h, st, SPLIT_U | SPLIT_E | SPLIT_S, lo));
    int rc = factor_levels<float>(h, f, h->zq32, st, /*split_d=*/true);
    if (rc) return rc;
    h->pairs_valid = lo ? 1 : 0;
    {   // the root block goes to FP64 for the root Cholesky
      Launch k(h, HSS_K_OTHER, 0.0, st);
      launch_f32_to_f64(f.lv[0].A, h->R0, 4LL * r * r, st);
    }
    root = h->R0;
  }
  // root Cholesky (last step of Alg. 2), FP64 in every mode
  const int b0 = 2 * r;
  int rc = root_cholesky(h, root, b0, st);
  if (rc) return rc;
  {
    Launch k(h, HSS_K_OTHER, (double)((2LL << L) - 1), st);
    launch_logdet_reduce(h->logdet_part, (int)((2LL << L) - 1) + kRootPanels, h->logdet_val, st);
  }
  // mixed modes: the root solve of every refinement pass multiplies by the FP64
  // inverse of the root block, formed here from its Cholesky factor with the
  // triangular sweeps run on the identity, 16 columns per CTA
  h->a0inv_valid = 0;
  if (prec != HSS_FP64 && b0 % kSolveCols == 0) {
    {
      Launch k(h, HSS_K_OTHER, 0.0, st);
      launch_eye(h->A0inv, b0, st);
    }
    const int chunks = b0 / kSolveCols;
    const long long sx = (long long)kSolveCols * b0;
    {
      Launch k(h, HSS_K_TRSV_FWD, trsv_flops(b0, b0, b0), st);
      HSS_TRY(launch_trsv_fwd<double>(root, b0, 0, b0, b0, h->A0inv, b0, sx, kSolveCols, nullptr,
                                      0, 0, chunks, st));
    }
    {
      Launch k(h, HSS_K_TRSV_BWD, trsv_flops(b0, b0, b0), st);
      HSS_TRY(launch_trsv_bwd<double>(root, b0, 0, b0, b0, h->A0inv, b0, sx, kSolveCols, nullptr,
                                      0, 0, chunks, st));
    }
    h->a0inv_valid = 1;
  }
  return check_launch();
}

// the ULV sweeps on nc <= kSolveCols columns of x (in place), arithmetic T;
// the root solve is FP64 in every mode
// vec_seg := vec_seg - V op(T) (Vᵀ vec_seg), op(T) = Tᵀ for Qᵀ and T for Q, as
// three batched GEMMs over the level (used where the level has many nodes)
template <typename T>
void apply_q(hss_s* h, Factor<T>& f, const LevelT<T>& P, T* vec, int ldv, int nc, bool transpose,
             cudaStream_t st, int col0) {
  const int b = P.b, r = P.r, n = P.n;
  const long long s1 = (long long)r * kSolveCols;
  T* t1 = f.t1 + (long long)col0 * r;   // this lane's columns of the scratch
  T* t2 = f.t2 + (long long)col0 * r;
  gemm<T>(h, true, false, r, nc, b, T(1), P.V, b, (long long)b * r, vec, ldv, b, T(0), t1, r, s1,
          n, st);
  gemm<T>(h, transpose, false, r, nc, r, T(1), P.T_, r, (long long)r * r, t1, r, s1, T(0), t2, r,
          s1, n, st);
  gemm<T>(h, false, false, b, nc, r, T(-1), P.V, b, (long long)b * r, t2, r, s1, T(1), vec, ldv,
          b, n, st);
}

// The ULV sweeps on nc <= kSolveCols columns of x (in place), arithmetic T;
// the root solve is FP64 in every mode.  Lane g uses columns col0 .. col0+nc-1
// of every level vector and scratch block, and its own tree flags.
template <typename T>
int solve_sweeps(hss_s* h, Factor<T>& f, T* x, int nc, int ld, cudaStream_t st, int g = 0,
                 int col0 = 0) {
  const int L = h->L, r = h->rank;
  Lane& ln = h->lane[g];
  // level l's vector, this lane's columns
  auto lvec = [&](int l) { return f.lv[l].yv + (long long)col0 * f.lv[l].n * f.lv[l].b; };
  // levels lo .. 1 (the narrow top of the tree) run as one launch per direction
  // where the tree kernels' shared memory fits
  const int lo = (h->schedule == HSS_SCHEDULE_ASYNC && tree_fits<T>(2 * r, nc, r))
                     ? std::min(L - 1, kTreeTop)
                     : 0;
  TreeLevels<T> tl{};
  double tree_flops = 0.0;
  for (int l = 0; l <= lo; ++l) {
    tl.M[l] = f.lv[l].M;
    tl.V[l] = f.lv[l].V;
    tl.Tm[l] = f.lv[l].T_;
    tl.vec[l] = lvec(l);
    if (l >= 1) tree_flops += (trsv_flops(2 * r, r, nc) + qapply_flops(2 * r, r, nc)) * (1 << l);
  }
  for (int l = L; l > lo; --l) {
    LevelT<T>& P = f.lv[l];
    LevelT<T>& Q = f.lv[l - 1];
    T* vec = (l == L) ? x : lvec(l);
    const int ldv = (l == L) ? ld : P.n * P.b;
    // Qᵀ then the forward triangular sweep: fused in one launch where the level
    // is narrow (the launches, not the flops, set its time) and the fused
    // kernel's shared memory fits, else three batched GEMMs and the sweep
    const bool fused = P.n <= kFuseNodes && ulv_fused_fits<T>(P.b, nc, r, false);
    if (!fused) apply_q<T>(h, f, P, vec, ldv, nc, /*transpose=*/true, st, col0);
    Launch k(h, HSS_K_TRSV_FWD,
             (trsv_flops(P.b, P.c, nc) + (fused ? qapply_flops(P.b, r, nc) : 0.0)) * P.n, st,
             sizeof(T) == 4);
    HSS_TRY(launch_ulv_fwd<T>(P.M, P.b, (long long)P.b * P.b, P.b, P.c, vec, ldv, P.b, nc,
                              lvec(l - 1), Q.n * Q.b, r, fused ? P.V : nullptr,
                              (long long)P.b * r, P.T_, (long long)r * r, r, P.n, st,
                              h->staging));
  }
  if (lo >= 1) {
    Launch k(h, HSS_K_TRSV_FWD, tree_flops, st, sizeof(T) == 4);
    HSS_TRY(launch_tree_fwd<T>(tl, lo, 2 * r, r, r, nc, ln.tcnt, st));
  }
  const int b0 = 2 * r;
  const long long rc0 = (long long)col0 * b0;
  double* rootA;
  double* rv;
  if (sizeof(T) == sizeof(double)) {
    rootA = reinterpret_cast<double*>(f.lv[0].A);
    rv = reinterpret_cast<double*>(lvec(0));
  } else {
    rootA = h->R0;
    rv = h->root_vec + rc0;
    Launch k(h, HSS_K_OTHER, 0.0, st);
    launch_f32_to_f64(reinterpret_cast<const float*>(lvec(0)), rv, (long long)b0 * nc, st);
  }
  if (sizeof(T) != sizeof(double) && h->a0inv_valid) {
    gemm<double>(h, false, false, b0, nc, b0, 1.0, h->A0inv, b0, 0, rv, b0, 0, 0.0,
                 h->root_vec2 + rc0, b0, 0, 1, st);
    rv = h->root_vec2 + rc0;
  } else {
    {
      Launch k(h, HSS_K_TRSV_FWD, trsv_flops(b0, b0, nc), st);
      HSS_TRY(launch_trsv_fwd<double>(rootA, b0, 0, b0, b0, rv, b0, 0, nc, nullptr, 0, 0, 1, st));
    }
    {
      Launch k(h, HSS_K_TRSV_BWD, trsv_flops(b0, b0, nc), st);
      HSS_TRY(launch_trsv_bwd<double>(rootA, b0, 0, b0, b0, rv, b0, 0, nc, nullptr, 0, 0, 1, st));
    }
  }
  if (sizeof(T) != sizeof(double)) {
    Launch k(h, HSS_K_OTHER, 0.0, st);
    launch_f64_to_f32(rv, reinterpret_cast<float*>(lvec(0)), (long long)b0 * nc, st);
  }
  if (lo >= 1) {
    const long long wl = h->wait_budget > 0 ? h->wait_budget : (h->wait_budget < 0 ? 0 : 1LL << 24);
    if (++ln.epoch <= 0) ln.epoch = 1;
    Launch k(h, HSS_K_TRSV_BWD, tree_flops, st, sizeof(T) == 4);
    HSS_TRY(launch_tree_bwd<T>(tl, lo, 2 * r, r, r, nc, ln.tready, ln.epoch, wl, h->status, st));
  }
  for (int l = lo + 1; l <= L; ++l) {
    LevelT<T>& P = f.lv[l];
    LevelT<T>& Q = f.lv[l - 1];
    T* vec = (l == L) ? x : lvec(l);
    const int ldv = (l == L) ? ld : P.n * P.b;
    // the backward triangular sweep then Q (fused where the level is narrow and
    // the fused kernel fits)
    const bool fused = P.n <= kFuseNodes && ulv_fused_fits<T>(P.b, nc, r, true);
    {
      Launch k(h, HSS_K_TRSV_BWD,
               (trsv_flops(P.b, P.c, nc) + (fused ? qapply_flops(P.b, r, nc) : 0.0)) * P.n, st,
               sizeof(T) == 4);
      HSS_TRY(launch_ulv_bwd<T>(P.M, P.b, (long long)P.b * P.b, P.b, P.c, vec, ldv, P.b, nc,
                                lvec(l - 1), Q.n * Q.b, r, fused ? P.V : nullptr,
                                (long long)P.b * r, P.T_, (long long)r * r, r, P.n, st,
                                h->staging));
    }
    if (!fused) apply_q<T>(h, f, P, vec, ldv, nc, /*transpose=*/false, st, col0);
  }
  return check_launch();
}

// y = A x in FP64 on lane g's streams, using columns col0 .. of the per-level
// scratch (nrhs <= kMaxCols - col0 when col0 > 0)
int matvec_fp64(hss_s* h, const double* x, int ldx, double* y, int ldy, int nrhs,
                cudaStream_t st, int g = 0, int col0 = 0) {
  const int L = h->L, r = h->rank, leaf = h->leaf;
  const long long rr = (long long)r * r;
  const int nL = 1 << L;
  Lane& ln = h->lane[g];
  const cudaStream_t ms = h->serialize ? st : ln.ms;
  // this lane's columns of the level vectors x̂_l, ŷ_l ((2^l r) x kMaxCols each)
  auto xh = [&](int l) { return h->xh[l] + (long long)col0 * ((1LL << l) * r); };
  auto yh = [&](int l) { return h->yh[l] + (long long)col0 * ((1LL << l) * r); };
  for (int j0 = 0, nc = 0; j0 < nrhs; j0 += nc) {
    nc = std::min(kMaxCols - col0, nrhs - j0);   // passes of at most kMaxCols - col0 columns
    const double* xc = x + (long long)j0 * ldx;
    double* yc = y + (long long)j0 * ldy;
    // leaves, first part: y = D x, which needs nothing else, on the second
    // stream while the basis sweeps below run on the caller's
    if (cudaEventRecord(ln.mv_start, st) != cudaSuccess ||
        cudaStreamWaitEvent(ms, ln.mv_start, 0) != cudaSuccess)
      return HSS_ERR_CUDA;
    gemm<double>(h, false, false, leaf, nc, leaf, 1.0, h->D, leaf, (long long)leaf * leaf, xc, ldx,
                 leaf, 0.0, yc, ldy, leaf, nL, ms);
    if (cudaEventRecord(ln.mv_dx, ms) != cudaSuccess) return HSS_ERR_CUDA;
    // up-sweep: x̂_L = Uᵀ x, x̂_l = E_lᵀ [x̂_{l+1}(2p); x̂_{l+1}(2p+1)]
    gemm<double>(h, true, false, r, nc, leaf, 1.0, h->U, leaf, (long long)leaf * r, xc, ldx, leaf,
                 0.0, xh(L), nL * r, r, nL, st);
    for (int l = L - 1; l >= 1; --l)
      gemm<double>(h, true, false, r, nc, 2 * r, 1.0, h->E + h->Eoff[l], 2 * r, 2 * rr, xh(l + 1),
                   (2 << l) * r, 2 * r, 0.0, xh(l), (1 << l) * r, r, 1 << l, st);
    // sibling couplings of every level (these initialise ŷ)
    for (int l = 1; l <= L; ++l) {
      const double* Sl = h->S + h->Soff[l];
      const int ldl = (1 << l) * r;
      gemm<double>(h, false, false, r, nc, r, 1.0, Sl, r, rr, xh(l), ldl, 2 * r, 0.0, yh(l) + r,
                   ldl, 2 * r, 1 << (l - 1), st);
      gemm<double>(h, true, false, r, nc, r, 1.0, Sl, r, rr, xh(l) + r, ldl, 2 * r, 0.0, yh(l),
                   ldl, 2 * r, 1 << (l - 1), st);
    }
    // down-sweep: ŷ_{l+1}(children) += E_l ŷ_l
    for (int l = 1; l <= L - 1; ++l)
      gemm<double>(h, false, false, 2 * r, nc, r, 1.0, h->E + h->Eoff[l], 2 * r, 2 * rr, yh(l),
                   (1 << l) * r, r, 1.0, yh(l + 1), (2 << l) * r, 2 * r, 1 << l, st);
    // leaves, second part: y += U ŷ once D x is done
    if (cudaStreamWaitEvent(st, ln.mv_dx, 0) != cudaSuccess) return HSS_ERR_CUDA;
    gemm<double>(h, false, false, leaf, nc, r, 1.0, h->U, leaf, (long long)leaf * r, yh(L),
                 nL * r, r, 1.0, yc, ldy, leaf, nL, st);
    int rc = check_launch();
    if (rc) return rc;
  }
  return HSS_OK;
}

// hi = fl32(g) into the FP32 factor's generator copies and, with `lo`, the
// low-order parts fl32(g - hi) of the pair representation (used only by the
// pair-arithmetic matvec); `which` selects D, U, E, S (SPLIT_*)
cudaError_t split_generators(hss_s* h, cudaStream_t st, int which, bool lo) {
  const int L = h->L, r = h->rank;
  Factor<float>& f = h->f32;
  const long long nL = 1LL << L;
  cudaError_t e = cudaSuccess;
  if (which & SPLIT_D) {
    Launch k(h, HSS_K_OTHER, 0.0, st);
    e = launch_df_split(h->D, f.Dc, lo ? h->Dl : nullptr, nL * h->leaf * h->leaf, st);
  }
  if (e == cudaSuccess && (which & SPLIT_U)) {
    Launch k(h, HSS_K_OTHER, 0.0, st);
    e = launch_df_split(h->U, f.Uc, lo ? h->Ul : nullptr, nL * h->leaf * r, st);
  }
  if (e == cudaSuccess && h->esz && (which & SPLIT_E)) {
    Launch k(h, HSS_K_OTHER, 0.0, st);
    e = launch_df_split(h->E, f.Ec, lo ? h->El : nullptr, h->esz, st);
  }
  if (e == cudaSuccess && (which & SPLIT_S)) {
    Launch k(h, HSS_K_OTHER, 0.0, st);
    e = launch_df_split(h->S, f.Sc, lo ? h->Sl : nullptr, h->ssz, st);
  }
  return e;
}

// The FP32 arena (converted generators, FP32 factor, pair matvec buffers),
// allocated on first use.
int ensure_f32_arena(hss_s* h) {
  if (h->f32.arena) return HSS_OK;
  const size_t bytes = layout_f32(h, nullptr);
  void* mem = nullptr;
  if (cudaMalloc(&mem, bytes) != cudaSuccess) {
    cudaGetLastError();
    return HSS_ERR_OOM;
  }
  h->f32.arena = mem;
  h->f32.bytes = bytes;
  layout_f32(h, static_cast<char*>(mem));
  return HSS_OK;
}

#define DF_TRY(call)                                  \
  do {                                                \
    if ((call) != cudaSuccess) return HSS_ERR_CUDA;   \
  } while (0)

// y = A x (nc <= kSolveCols columns) with the same up-sweep / coupling /
// down-sweep / leaf structure as matvec_fp64, every product in pair-of-FP32
// arithmetic (dfgemm.cu).  x enters scaled per column by a power of two near
// 1 / |x_j| so that its pairs stay in range; y leaves scaled back, in FP64.
int matvec_pair(hss_s* h, const double* x, int ldx, double* y, int ldy, int nc, cudaStream_t st) {
  const int L = h->L, r = h->rank, leaf = h->leaf, n = h->n;
  const long long rr = (long long)r * r;
  const int nL = 1 << L;
  const Factor<float>& f = h->f32;
  double* xn = h->norms + 4 * kSolveCols;
  {
    Launch k(h, HSS_K_OTHER, 2.0 * n * nc, st);
    launch_col_norms(x, ldx, n, nc, xn, xn + kSolveCols, h->norm_part, st);
  }
  {
    Launch k(h, HSS_K_OTHER, 0.0, st);
    DF_TRY(launch_df_split_cols(x, ldx, n, nc, xn, h->xs_h, h->xs_l, n, st));
  }
  auto df = [&](bool ta, int m, int k, const float* Ah, const float* Al, int lda, long long sA,
                const float* Bh, const float* Bl, int ldb, long long sB, bool acc, float* Ch,
                float* Cl, double* C64, int ldc64, int ldc, long long sC, int batch) {
    Launch kk(h, HSS_K_PAIR_GEMM, 2.0 * m * nc * (double)k * batch, st, true);
    return df_gemm(ta, m, nc, k, Ah, Al, lda, sA, Bh, Bl, ldb, sB, acc, Ch, Cl, C64, ldc64, xn,
                   ldc, sC, batch, st);
  };
  // up-sweep: x̂_L = Uᵀ x, x̂_l = E_lᵀ [x̂_{l+1}(2p); x̂_{l+1}(2p+1)]
  DF_TRY(df(true, r, leaf, f.Uc, h->Ul, leaf, (long long)leaf * r, h->xs_h, h->xs_l, n, leaf,
            false, h->xp_h[L], h->xp_l[L], nullptr, 0, nL * r, r, nL));
  for (int l = L - 1; l >= 1; --l)
    DF_TRY(df(true, r, 2 * r, f.Ec + h->Eoff[l], h->El + h->Eoff[l], 2 * r, 2 * rr, h->xp_h[l + 1],
              h->xp_l[l + 1], (2 << l) * r, 2 * r, false, h->xp_h[l], h->xp_l[l], nullptr, 0,
              (1 << l) * r, r, 1 << l));
  // sibling couplings of every level (these initialise ŷ)
  for (int l = 1; l <= L; ++l) {
    const float* Sh = f.Sc + h->Soff[l];
    const float* Sl = h->Sl + h->Soff[l];
    const int ldl = (1 << l) * r;
    DF_TRY(df(false, r, r, Sh, Sl, r, rr, h->xp_h[l], h->xp_l[l], ldl, 2 * r, false,
              h->yp_h[l] + r, h->yp_l[l] + r, nullptr, 0, ldl, 2 * r, 1 << (l - 1)));
    DF_TRY(df(true, r, r, Sh, Sl, r, rr, h->xp_h[l] + r, h->xp_l[l] + r, ldl, 2 * r, false,
              h->yp_h[l], h->yp_l[l], nullptr, 0, ldl, 2 * r, 1 << (l - 1)));
  }
  // down-sweep: ŷ_{l+1}(children) += E_l ŷ_l
  for (int l = 1; l <= L - 1; ++l)
    DF_TRY(df(false, 2 * r, r, f.Ec + h->Eoff[l], h->El + h->Eoff[l], 2 * r, 2 * rr, h->yp_h[l],
              h->yp_l[l], (1 << l) * r, r, true, h->yp_h[l + 1], h->yp_l[l + 1], nullptr, 0,
              (2 << l) * r, 2 * r, 1 << l));
  // leaves: y = D x + U ŷ, the second product writing FP64
  DF_TRY(df(false, leaf, leaf, f.Dc, h->Dl, leaf, (long long)leaf * leaf, h->xs_h, h->xs_l, n,
            leaf, false, h->yt_h, h->yt_l, nullptr, 0, n, leaf, nL));
  DF_TRY(df(false, leaf, r, f.Uc, h->Ul, leaf, (long long)leaf * r, h->yp_h[L], h->yp_l[L], nL * r,
            r, true, h->yt_h, h->yt_l, y, ldy, n, leaf, nL));
  return check_launch();
}

int read_status(hss_s* h, int* st_host) {
  cudaError_t e = cudaMemcpy(st_host, h->status, 8 * sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return HSS_ERR_CUDA;
  return st_host[ST_CODE];
}

// Iterative refinement with the FP32 factor: x_0 = M⁻¹ b; r_k = b - A x_k in
// FP64; stop when every column's |r_k| / |b| <= tol; x_{k+1} = x_k + M⁻¹ r_k.
// Right-hand sides enter the FP32 sweeps scaled to unit norm.
int solve_ir(hss_s* h, const double* b, double* x, int nrhs, int ld, cudaStream_t st) {
  const int n = h->n;
  Factor<float>& f = h->f32;
  double* nb = h->norms;                    // |b|
  double* ib = h->norms + kSolveCols;       // 1 / |b|
  double* nr = h->norms + 2 * kSolveCols;   // |r|
  double* ir = h->norms + 3 * kSolveCols;   // 1 / |r|
  // pinned host copies: |b|, |r| per column, then each lane's status word
  double* hnb = h->hnorm;
  double* hnr = h->hnorm + kSolveCols;
  int* hst = reinterpret_cast<int*>(h->hnorm + 2 * kSolveCols);
  int worst_it = 0;
  double worst_res = 0.0;
  int result = HSS_OK;
  // one refinement lane: columns c0 .. c0+nc-1 of the pass on stream ls
  struct IrLane {
    int g, c0, nc;
    cudaStream_t ls;
    int it = 0;
    double rel = 0.0;
    bool active = false;
  };
  for (int j0 = 0; j0 < nrhs; j0 += kSolveCols) {
    const int nc = std::min(kSolveCols, nrhs - j0);
    const double* bc = b + (long long)j0 * ld;
    double* xc = x + (long long)j0 * ld;
    int ldb = ld;
    if (bc == xc) {   // keep b: x is overwritten by the iterates
      if (cudaMemcpy2DAsync(h->bbuf, sizeof(double) * n, bc, sizeof(double) * ld,
                            sizeof(double) * n, nc, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return HSS_ERR_CUDA;
      bc = h->bbuf;
      ldb = n;
    }
    // two lanes over the columns when there are two columns or more (the pair
    // residual's split buffers are shared: one lane); a serialized trace runs
    // both lanes' launches on the caller's stream, one after the other
    const int lanes = (nc >= 2 && h->ir_lanes == 2 && h->residual == HSS_RESIDUAL_FP64) ? 2 : 1;
    IrLane lane[2];
    lane[0].g = 0;
    lane[0].c0 = 0;
    lane[0].nc = lanes == 2 ? (nc + 1) / 2 : nc;
    lane[0].ls = st;
    lane[1].g = 1;
    lane[1].c0 = lane[0].nc;
    lane[1].nc = nc - lane[0].nc;
    lane[1].ls = h->serialize ? st : h->lane[1].st;
    // residual r = b - A x of a lane, its norms and the status word to the host
    auto residual_step = [&](IrLane& q) -> int {
      const long long o = (long long)q.c0 * n;
      int rc = h->residual == HSS_RESIDUAL_PAIR32
                   ? matvec_pair(h, xc, ld, h->rbuf, n, q.nc, q.ls)
                   : matvec_fp64(h, xc + (long long)q.c0 * ld, ld, h->rbuf + o, n, q.nc, q.ls,
                                 q.g, q.c0);
      if (rc) return rc;
      {
        Launch k(h, HSS_K_OTHER, (double)n * q.nc, q.ls);
        launch_residual(bc + (long long)q.c0 * ldb, ldb, h->rbuf + o, n, n, q.nc, q.ls);
      }
      {
        Launch k(h, HSS_K_OTHER, 2.0 * n * q.nc, q.ls);
        launch_col_norms(h->rbuf + o, n, n, q.nc, nr + q.c0, ir + q.c0,
                         h->norm_part + 64LL * q.c0, q.ls);
      }
      if (cudaMemcpyAsync(hnr + q.c0, nr + q.c0, sizeof(double) * q.nc, cudaMemcpyDeviceToHost,
                          q.ls) != cudaSuccess ||
          cudaMemcpyAsync(hst + 8 * q.g, h->status, 8 * sizeof(int), cudaMemcpyDeviceToHost,
                          q.ls) != cudaSuccess ||
          cudaEventRecord(h->lane[q.g].norm_ready, q.ls) != cudaSuccess)
        return HSS_ERR_CUDA;
      return HSS_OK;
    };
    // d = M⁻¹ v in FP32 (v scaled by scale), x = x (+)= d unscaled
    auto correction = [&](IrLane& q, const double* v, int ldv, const double* scale,
                          const double* unscale, int accumulate) -> int {
      const long long o = (long long)q.c0 * n;
      {
        Launch k(h, HSS_K_OTHER, 0.0, q.ls);
        launch_cols_to_f32(v, ldv, f.d + o, n, n, q.nc, scale, q.ls);
      }
      int rc = solve_sweeps<float>(h, f, f.d + o, q.nc, n, q.ls, q.g, q.c0);
      if (rc) return rc;
      Launch k(h, HSS_K_OTHER, accumulate ? (double)n * q.nc : 0.0, q.ls);
      launch_cols_update(xc + (long long)q.c0 * ld, ld, f.d + o, n, n, q.nc, unscale, accumulate,
                         q.ls);
      return HSS_OK;
    };
    for (int g = 0; g < lanes; ++g) {   // x_0 = M⁻¹ b, then the first residual
      IrLane& q = lane[g];
      {
        Launch k(h, HSS_K_OTHER, 2.0 * n * q.nc, q.ls);
        launch_col_norms(bc + (long long)q.c0 * ldb, ldb, n, q.nc, nb + q.c0, ib + q.c0,
                         h->norm_part + 64LL * q.c0, q.ls);
      }
      if (cudaMemcpyAsync(hnb + q.c0, nb + q.c0, sizeof(double) * q.nc, cudaMemcpyDeviceToHost,
                          q.ls) != cudaSuccess)
        return HSS_ERR_CUDA;
      int rc = correction(q, bc + (long long)q.c0 * ldb, ldb, ib + q.c0, nb + q.c0, 0);
      if (rc) return rc;
      // lane 1 starts once lane 0's first sweeps are done: from then on one
      // lane's FP32 sweeps run beside the other lane's FP64 matvec
      if (g == 0 && lanes == 2 &&
          (cudaEventRecord(h->ev_ir_fork, q.ls) != cudaSuccess ||
           cudaStreamWaitEvent(lane[1].ls, h->ev_ir_fork, 0) != cudaSuccess))
        return HSS_ERR_CUDA;
      rc = residual_step(q);
      if (rc) return rc;
      q.active = true;
    }
    // each lane: wait for its own residual norms only, then queue its next
    // correction and residual; the other lane's work stays in flight
    for (bool any = true; any;) {
      any = false;
      for (int g = 0; g < lanes; ++g) {
        IrLane& q = lane[g];
        if (!q.active) continue;
        if (cudaEventSynchronize(h->lane[g].norm_ready) != cudaSuccess) return HSS_ERR_CUDA;
        if (hst[8 * g + ST_CODE]) return hst[8 * g + ST_CODE];
        q.rel = 0.0;
        for (int j = q.c0; j < q.c0 + q.nc; ++j)
          q.rel = std::max(q.rel, hnb[j] > 0 ? hnr[j] / hnb[j] : hnr[j]);
        if (!(q.rel > h->ir_tol) || q.it >= h->ir_max_it) {
          q.active = false;
          continue;
        }
        ++q.it;
        int rc = correction(q, h->rbuf + (long long)q.c0 * n, n, ir + q.c0, nr + q.c0, 1);
        if (rc) return rc;
        rc = residual_step(q);
        if (rc) return rc;
        any = true;
      }
    }
    if (lanes == 2) {
      if (cudaEventRecord(h->ev_ir_join, lane[1].ls) != cudaSuccess ||
          cudaStreamWaitEvent(st, h->ev_ir_join, 0) != cudaSuccess)
        return HSS_ERR_CUDA;
    }
    for (int g = 0; g < lanes; ++g) {
      worst_it = std::max(worst_it, lane[g].it);
      worst_res = std::max(worst_res, lane[g].rel);
      if (lane[g].rel > h->ir_tol || !(lane[g].rel == lane[g].rel)) result = HSS_ERR_NO_CONVERGENCE;
    }
  }
  h->ir_iters = worst_it;
  h->ir_resid = worst_res;
  return result;
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
  if (L < 1 || L > 24 || leaf < 1 || leaf > 1024 || r < 1 || r > leaf || r > 256)
    return HSS_ERR_INVALID_ARG;
  if (L >= 2 && !E) return HSS_ERR_INVALID_ARG;
  // an uneven tree: its generators embedded in the uniform (leaf, rank) ones
  UnevenPad pad;
  if (shape->node_sizes) {
    if (on_device || (long long)leaf << L > 0x7fffffffLL) return HSS_ERR_INVALID_ARG;
    const int rc = pad_uneven(*shape, D, U, E, S, &pad);
    if (rc) return rc;
    D = pad.D.data();
    U = pad.U.data();
    E = pad.E.data();
    S = pad.S.data();
  } else if ((long long)leaf << L != (long long)shape->n) {
    return HSS_ERR_INVALID_ARG;
  }
  hss_s* h = new (std::nothrow) hss_s();
  if (!h) return HSS_ERR_OOM;
  h->n = (int)((long long)leaf << L);
  h->n_user = shape->n;
  h->uneven = shape->node_sizes ? 1 : 0;
  h->leaf = leaf;
  h->rank = r;
  h->L = L;
  cudaGetDevice(&h->device);
  const size_t bytes = layout_main(h, nullptr);
  void* mem = nullptr;
  if (cudaMalloc(&mem, bytes) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return HSS_ERR_OOM;
  }
  h->arena = mem;
  h->arena_bytes = bytes;
  layout_main(h, static_cast<char*>(mem));
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const long long nL = 1LL << L;
  cudaError_t e = cudaSuccess;
  e = e ? e : cudaMemcpy(h->D, D, sizeof(double) * nL * leaf * leaf, kind);
  e = e ? e : cudaMemcpy(h->U, U, sizeof(double) * nL * leaf * r, kind);
  if (L >= 2) e = e ? e : cudaMemcpy(h->E, E, sizeof(double) * h->esz, kind);
  e = e ? e : cudaMemcpy(h->S, S, sizeof(double) * h->ssz, kind);
  e = e ? e : cudaMemset(h->status, 0, 8 * sizeof(int));
  for (Lane& ln : h->lane)
    e = e ? e : cudaMemset(ln.tready, 0, sizeof(int) << (kTreeTop + 1));
  if (h->uneven)
    e = e ? e : cudaMemcpy(h->pmap, pad.pmap.data(), sizeof(int) * h->n, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(mem);
    delete h;
    return HSS_ERR_CUDA;
  }
  h->ev_level.assign(L + 1, nullptr);
  e = cudaStreamCreateWithFlags(&h->qstream, cudaStreamNonBlocking);
  e = e ? e : cudaEventCreateWithFlags(&h->ev_start, cudaEventDisableTiming);
  e = e ? e : cudaEventCreateWithFlags(&h->ev_ir_fork, cudaEventDisableTiming);
  e = e ? e : cudaEventCreateWithFlags(&h->ev_ir_join, cudaEventDisableTiming);
  for (int g = 0; g < 2 && e == cudaSuccess; ++g) {
    Lane& ln = h->lane[g];
    if (g == 1) e = cudaStreamCreateWithFlags(&ln.st, cudaStreamNonBlocking);
    e = e ? e : cudaStreamCreateWithFlags(&ln.ms, cudaStreamNonBlocking);
    e = e ? e : cudaEventCreateWithFlags(&ln.mv_start, cudaEventDisableTiming);
    e = e ? e : cudaEventCreateWithFlags(&ln.mv_dx, cudaEventDisableTiming);
    e = e ? e : cudaEventCreateWithFlags(&ln.norm_ready, cudaEventDisableTiming);
  }
  if (e == cudaSuccess && cudaMallocHost(&h->hnorm, sizeof(double) * 2 * kSolveCols + 16 * sizeof(int)) != cudaSuccess)
    e = cudaErrorMemoryAllocation;
  for (int l = 1; l <= L && e == cudaSuccess; ++l)
    e = cudaEventCreateWithFlags(&h->ev_level[l], cudaEventDisableTiming);
  if (e != cudaSuccess) {
    hss_destroy(h);
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
  if (h->qstream) cudaStreamSynchronize(h->qstream);
  for (cudaEvent_t ev : h->ev_level)
    if (ev) cudaEventDestroy(ev);
  if (h->ev_start) cudaEventDestroy(h->ev_start);
  if (h->ev_ir_fork) cudaEventDestroy(h->ev_ir_fork);
  if (h->ev_ir_join) cudaEventDestroy(h->ev_ir_join);
  for (Lane& ln : h->lane) {
    for (cudaStream_t s : {ln.st, ln.ms})
      if (s) cudaStreamSynchronize(s);
    for (cudaEvent_t ev : {ln.mv_start, ln.mv_dx, ln.norm_ready})
      if (ev) cudaEventDestroy(ev);
    if (ln.st) cudaStreamDestroy(ln.st);
    if (ln.ms) cudaStreamDestroy(ln.ms);
  }
  if (h->hnorm) cudaFreeHost(h->hnorm);
  if (h->qstream) cudaStreamDestroy(h->qstream);
  cudaFree(h->arena);
  if (h->f32.arena) cudaFree(h->f32.arena);
  if (h->tc_ws) cudaFree(h->tc_ws);
  cudaSetDevice(cur);
  delete h;
}

int hss_factorize(hss_t h, const hss_options* opt, void* stream) {
  if (!h) return HSS_ERR_INVALID_ARG;
  const int prec = opt ? opt->precision : HSS_FP64;
  if (prec != HSS_FP64 && prec != HSS_MIXED_FP32 && prec != HSS_MIXED_TF32 &&
      prec != HSS_MIXED_BF16)
    return HSS_ERR_INVALID_ARG;
  if (opt && (opt->ir_max_it < 0 || !(opt->ir_tol >= 0.0))) return HSS_ERR_INVALID_ARG;
  if (opt && opt->residual != HSS_RESIDUAL_FP64 && opt->residual != HSS_RESIDUAL_PAIR32)
    return HSS_ERR_INVALID_ARG;
  if (opt && (opt->basis < HSS_BASIS_HOUSEHOLDER || opt->basis > HSS_BASIS_AUTO))
    return HSS_ERR_INVALID_ARG;
  if (opt && (opt->schedule < HSS_SCHEDULE_ASYNC || opt->schedule > HSS_SCHEDULE_AUTO))
    return HSS_ERR_INVALID_ARG;
  if (opt && opt->ql_panel != 0 && opt->ql_panel != 16 && opt->ql_panel != 32)
    return HSS_ERR_INVALID_ARG;
  if (opt && (opt->ir_lanes < 0 || opt->ir_lanes > 2)) return HSS_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  h->factorized = 0;
  if (prec != HSS_FP64) {
    const int rc = ensure_f32_arena(h);
    if (rc) return rc;
  }
  if (opt) {
    h->ir_max_it = opt->ir_max_it;
    h->ir_tol = opt->ir_tol;
    h->residual = opt->residual;
    h->wait_budget = opt->wait_budget;
    h->basis_method = opt->basis == HSS_BASIS_AUTO
                          ? (h->tuned ? h->tuned_basis : HSS_BASIS_HOUSEHOLDER)
                          : opt->basis;
    h->ql_panel = opt->basis == HSS_BASIS_AUTO && h->tuned ? h->tuned_panel : opt->ql_panel;
    const bool sauto = opt->schedule == HSS_SCHEDULE_AUTO;
    h->schedule = sauto ? (h->tuned ? h->tuned_schedule : HSS_SCHEDULE_ASYNC) : opt->schedule;
    h->staging = sauto && h->tuned ? h->tuned_staging : 0;
    h->ir_lanes = opt->ir_lanes ? opt->ir_lanes : (sauto && h->tuned ? h->tuned_lanes : 1);
  } else {
    h->wait_budget = 0;
    h->basis_method = HSS_BASIS_HOUSEHOLDER;
    h->ql_panel = 0;
    h->schedule = HSS_SCHEDULE_ASYNC;
    h->staging = 0;
    h->ir_lanes = 1;
  }
  h->use_tc = (prec == HSS_MIXED_TF32 || prec == HSS_MIXED_BF16) ? 1 : 0;
  h->tc_mode = (prec == HSS_MIXED_BF16) ? TcMode::BF16x3 : TcMode::TF32x3;
  if (h->use_tc) {   // packing workspace of the largest level's contractions
    size_t need = 0;
    for (int l = h->L; l >= 1; --l) {
      const int b = (l == h->L) ? h->leaf : 2 * h->rank, n = 1 << l;
      need = std::max(need, tc_workspace_bytes(h->tc_mode, b, h->rank, b, n));
      need = std::max(need, tc_workspace_bytes(h->tc_mode, b, b, 2 * h->rank, n));
    }
    if (need > h->tc_ws_bytes) {
      if (h->tc_ws) cudaFree(h->tc_ws);
      h->tc_ws = nullptr;
      h->tc_ws_bytes = 0;
      if (cudaMalloc(&h->tc_ws, need) != cudaSuccess) {
        cudaGetLastError();
        return HSS_ERR_OOM;
      }
      h->tc_ws_bytes = need;
    }
  }
  int rc = factorize(h, prec, st);
  if (rc) return rc;
  h->precision = prec;
  h->factorized = 1;
  h->last_stream = st;
  return HSS_OK;
}

}  // extern "C"

namespace {

// the solve of a uniform tree (or of the padded one, on padded vectors)
int solve_uniform(hss_t h, const double* b, double* x, int nrhs, int ld, cudaStream_t st) {
  if (h->precision != HSS_FP64) return solve_ir(h, b, x, nrhs, ld, st);
  if (x != b) {
    cudaError_t e = cudaMemcpy2DAsync(x, sizeof(double) * ld, b, sizeof(double) * ld,
                                      sizeof(double) * h->n, nrhs, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return HSS_ERR_CUDA;
  }
  for (int j0 = 0; j0 < nrhs; j0 += kSolveCols) {
    const int nc = std::min(kSolveCols, nrhs - j0);
    int rc = solve_sweeps<double>(h, h->f64, x + (long long)j0 * ld, nc, ld, st);
    if (rc) return rc;
  }
  return HSS_OK;
}

// Runs op(in, out, nc) on the padded vectors of an uneven tree, cols columns
// per pass: the caller's rows of x scattered in (zero padded rows), out
// gathered back into y.  A no-convergence result is carried to the end.
template <typename Op>
int on_padded(hss_t h, const double* x, double* y, int nrhs, int ld, int cols, cudaStream_t st,
              Op op) {
  int result = HSS_OK, worst_it = 0;
  double worst_res = 0.0;
  for (int j0 = 0; j0 < nrhs; j0 += cols) {
    const int nc = std::min(cols, nrhs - j0);
    launch_pad_rows(x + (long long)j0 * ld, ld, h->vin, h->n, h->pmap, h->n, nc, 1, st);
    const int rc = op(h->vin, h->vout, nc);
    if (rc && rc != HSS_ERR_NO_CONVERGENCE) return rc;
    if (rc) result = rc;
    worst_it = std::max(worst_it, h->ir_iters);
    worst_res = std::max(worst_res, h->ir_resid);
    launch_pad_rows(y + (long long)j0 * ld, ld, h->vout, h->n, h->pmap, h->n, nc, 0, st);
    if (cudaGetLastError() != cudaSuccess) return HSS_ERR_CUDA;
  }
  h->ir_iters = worst_it;
  h->ir_resid = worst_res;
  return result;
}

}  // namespace

extern "C" {

int hss_solve(hss_t h, const double* b, double* x, int32_t nrhs, int32_t ld, void* stream) {
  if (!h || !b || !x || nrhs < 0 || ld < h->n_user) return HSS_ERR_INVALID_ARG;
  if (!h->factorized) return HSS_ERR_NOT_FACTORIZED;
  if (nrhs == 0) return HSS_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  h->last_stream = st;
  if (!h->uneven) return solve_uniform(h, b, x, nrhs, ld, st);
  return on_padded(h, b, x, nrhs, ld, kSolveCols, st, [&](const double* in, double* out, int nc) {
    return solve_uniform(h, in, out, nc, h->n, st);
  });
}

int hss_matvec(hss_t h, const double* x, double* y, int32_t nrhs, int32_t ld, void* stream) {
  if (!h || !x || !y || nrhs < 0 || ld < h->n_user || x == y) return HSS_ERR_INVALID_ARG;
  if (nrhs == 0) return HSS_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  h->last_stream = st;
  if (!h->uneven) return matvec_fp64(h, x, ld, y, ld, nrhs, st);
  return on_padded(h, x, y, nrhs, ld, kMaxCols, st, [&](const double* in, double* out, int nc) {
    return matvec_fp64(h, in, h->n, out, h->n, nc, st);
  });
}

int hss_matvec_pair(hss_t h, const double* x, double* y, int32_t nrhs, int32_t ld,
                    void* stream) {
  if (!h || !x || !y || nrhs < 0 || ld < h->n_user || x == y) return HSS_ERR_INVALID_ARG;
  if (nrhs == 0) return HSS_OK;
  int rc = ensure_f32_arena(h);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  h->last_stream = st;
  if (!h->pairs_valid) {
    if (split_generators(h, st, SPLIT_ALL, true) != cudaSuccess) return HSS_ERR_CUDA;
    h->pairs_valid = 1;
  }
  if (h->uneven)
    return on_padded(h, x, y, nrhs, ld, kSolveCols, st, [&](const double* in, double* out, int nc) {
      return matvec_pair(h, in, h->n, out, h->n, nc, st);
    });
  for (int j0 = 0; j0 < nrhs; j0 += kSolveCols) {
    const int nc = std::min(kSolveCols, nrhs - j0);
    rc = matvec_pair(h, x + (long long)j0 * ld, ld, y + (long long)j0 * ld, ld, nc, st);
    if (rc) return rc;
  }
  return HSS_OK;
}

int hss_tune(hss_t h, const hss_options* opt, int32_t nrhs, const char* cache_path, void* stream,
             hss_tuning* out) {
  if (!h || !opt || nrhs < 1) return HSS_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int nc = std::min<int>(nrhs, kSolveCols);
  hss_tuning best{};
  // cache key
  char key[512];
  {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, h->device) != cudaSuccess) return HSS_ERR_CUDA;
    char dev[256];
    int q = 0;
    for (const char* c = prop.name; *c && q < 255; ++c) dev[q++] = (*c == ' ' ? '_' : *c);
    dev[q] = 0;
    snprintf(key, sizeof key, "%s p%d res%d n%d leaf%d rank%d L%d cols%d", dev, opt->precision,
             opt->residual, h->n_user, h->leaf, h->rank, h->L, nc);
  }
  bool found = false;
  if (cache_path) {
    if (FILE* f = fopen(cache_path, "r")) {
      char line[1024];
      const size_t kl = strlen(key);
      while (fgets(line, sizeof line, f)) {
        if (strncmp(line, key, kl) != 0 || line[kl] != ' ') continue;
        hss_tuning t{};
        if (sscanf(line + kl,
                   " basis %d panel %d schedule %d staging %d lanes %d factor_ms %lf solve_ms %lf",
                   &t.basis, &t.ql_panel, &t.schedule, &t.staging, &t.ir_lanes, &t.factor_ms,
                   &t.solve_ms) == 7 &&
            (t.ir_lanes == 1 || t.ir_lanes == 2) &&
            t.basis >= HSS_BASIS_HOUSEHOLDER && t.basis <= HSS_BASIS_CHOLQR &&
            (t.ql_panel == 16 || t.ql_panel == 32) &&
            t.schedule >= HSS_SCHEDULE_ASYNC && t.schedule <= HSS_SCHEDULE_LEVELS &&
            (t.staging == 0 || t.staging == 1)) {
          best = t;
          best.from_cache = 1;
          found = true;
        }
      }
      fclose(f);
    }
  }
  hss_options o = *opt;
  if (!found) {
    double* buf = nullptr;
    if (cudaMalloc(&buf, sizeof(double) * 2 * (size_t)h->n_user * kSolveCols) != cudaSuccess) {
      cudaGetLastError();
      return HSS_ERR_OOM;
    }
    double* b = buf;
    double* x = buf + (size_t)h->n_user * kSolveCols;
    launch_fill_test(b, h->n_user, nc, st);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess)
                 ? HSS_OK
                 : HSS_ERR_CUDA;
    // best of two timed runs of fn (after one untimed run)
    auto timed = [&](auto&& fn, double* ms) -> int {
      int r = fn();
      if (r && r != HSS_ERR_NO_CONVERGENCE) return r;
      *ms = 1e30;
      for (int t = 0; t < 2; ++t) {
        if (cudaEventRecord(e0, st) != cudaSuccess) return HSS_ERR_CUDA;
        r = fn();
        if (r && r != HSS_ERR_NO_CONVERGENCE) return r;
        float v = 0.f;
        if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&v, e0, e1) != cudaSuccess)
          return HSS_ERR_CUDA;
        *ms = std::min(*ms, (double)v);
      }
      return hss_sync(h);
    };
    best.factor_ms = 1e30;
    const bool cholqr_ok = o.precision == HSS_FP64 ? h->rank <= basis_max_rank<double>()
                                                  : h->rank <= basis_max_rank<float>();
    // candidates: the Householder kernel with each panel width (FP32 has 16
    // and 32 columns, FP64 16), then Cholesky QR; through the tuned path of
    // hss_factorize so that each runs exactly as it will be used
    struct Cand { int basis, panel; };
    const Cand cands[3] = {{HSS_BASIS_HOUSEHOLDER, 32}, {HSS_BASIS_HOUSEHOLDER, 16},
                           {HSS_BASIS_CHOLQR, 16}};
    for (const Cand& cd : cands) {
      if (rc != HSS_OK) break;
      if (cd.basis == HSS_BASIS_CHOLQR && !cholqr_ok) continue;
      if (cd.panel == 32 && o.precision == HSS_FP64) continue;
      h->tuned = 1;
      h->tuned_basis = cd.basis;
      h->tuned_panel = cd.panel;
      o.basis = HSS_BASIS_AUTO;
      o.schedule = HSS_SCHEDULE_ASYNC;
      double ms = 0.0;
      rc = timed([&] { return hss_factorize(h, &o, st); }, &ms);
      if (rc != HSS_OK) break;
      double& by_basis = best.factor_ms_by_basis[cd.basis];
      by_basis = by_basis > 0 ? std::min(by_basis, ms) : ms;
      if (cd.basis == HSS_BASIS_HOUSEHOLDER) best.factor_ms_by_panel[cd.panel == 32] = ms;
      if (ms < best.factor_ms) {
        best.factor_ms = ms;
        best.basis = cd.basis;
        best.ql_panel = cd.panel;
      }
    }
    h->tuned = 0;
    if (rc == HSS_OK) {   // leave the object factorized with the choice
      h->tuned_panel = best.ql_panel;
      h->tuned = 1;
      h->tuned_basis = best.basis;
      o.basis = HSS_BASIS_AUTO;
      rc = hss_factorize(h, &o, st);
      h->tuned = 0;
    }
    best.solve_ms = 1e30;
    // refinement lanes: two only where they apply (a mixed factor with the FP64
    // residual and at least two columns)
    const int max_lanes =
        (o.precision != HSS_FP64 && o.residual == HSS_RESIDUAL_FP64 && nc >= 2) ? 2 : 1;
    for (int lanes = 1; rc == HSS_OK && lanes <= max_lanes; ++lanes) {
      h->ir_lanes = lanes;
      double lane_best = 1e30;
      for (int sched = HSS_SCHEDULE_ASYNC; rc == HSS_OK && sched <= HSS_SCHEDULE_LEVELS;
           ++sched) {
        for (int stg = 0; rc == HSS_OK && stg <= 1; ++stg) {
          h->schedule = sched;
          h->staging = stg;
          double ms = 0.0;
          rc = timed([&] { return hss_solve(h, b, x, nc, h->n_user, st); }, &ms);
          if (rc != HSS_OK) break;
          lane_best = std::min(lane_best, ms);
          if (lanes == 1) best.solve_ms_by_config[sched][stg] = ms;
          if (ms < best.solve_ms) {
            best.solve_ms = ms;
            best.schedule = sched;
            best.staging = stg;
            best.ir_lanes = lanes;
          }
        }
      }
      if (rc == HSS_OK) best.solve_ms_by_lanes[lanes - 1] = lane_best;
    }
    h->ir_lanes = 1;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(st);
    cudaFree(buf);
    if (rc) return rc;
    if (cache_path) {
      if (FILE* f = fopen(cache_path, "a")) {
        fprintf(f,
                "%s basis %d panel %d schedule %d staging %d lanes %d factor_ms %.4f "
                "solve_ms %.4f\n",
                key, best.basis, best.ql_panel, best.schedule, best.staging, best.ir_lanes,
                best.factor_ms, best.solve_ms);
        fclose(f);
      }
    }
  }
  h->tuned = 1;
  h->tuned_basis = best.basis;
  h->tuned_panel = best.ql_panel;
  h->tuned_schedule = best.schedule;
  h->tuned_staging = best.staging;
  h->tuned_lanes = best.ir_lanes;
  o.basis = HSS_BASIS_AUTO;
  o.schedule = HSS_SCHEDULE_AUTO;
  const int rc = hss_factorize(h, &o, st);
  if (rc) return rc;
  if (out) *out = best;
  return HSS_OK;
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
  if (!h || enable < 0 || enable > 2) return HSS_ERR_INVALID_ARG;
  if (enable) {
    for (auto& r : h->trace) cudaEventSynchronize(r.b);
    clear_trace(h);
  }
  h->tracing = enable ? 1 : 0;
  h->serialize = enable == 2 ? 1 : 0;
  return HSS_OK;
}

int hss_trace_read(hss_t h, int32_t kind, double* ms, int64_t* launches, double* flops) {
  if (!h || kind < 0 || kind >= 2 * HSS_K_COUNT) return HSS_ERR_INVALID_ARG;
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
  const bool f32 = (h->precision != HSS_FP64);
  const size_t r = h->rank;
  size_t n = 0;
  const void* src = nullptr;
  const int lb = (level == h->L) ? h->leaf : 2 * h->rank;
  const size_t nodes = size_t(1) << level;
  switch (what) {
    case 0: n = nodes * lb * r; break;
    case 1: n = nodes * r * r; break;
    case 2: n = nodes * r * r; break;
    case 3: n = nodes * lb * lb; break;
    case 4: n = nodes * lb * r; break;
    default: return HSS_ERR_INVALID_ARG;
  }
  if (f32) {
    const LevelT<float>& P = h->f32.lv[level];
    const float* ps[5] = {P.V, P.T_, P.LB, P.M, P.B};
    src = ps[what];
  } else {
    const LevelT<double>& P = h->f64.lv[level];
    const double* ps[5] = {P.V, P.T_, P.LB, P.M, P.B};
    src = ps[what];
  }
  if (!src || n > count) return HSS_ERR_INVALID_ARG;
  if (cudaStreamSynchronize(h->last_stream) != cudaSuccess) return HSS_ERR_CUDA;
  if (!f32) return cuda_err(cudaMemcpy(dst, src, n * sizeof(double), cudaMemcpyDeviceToHost));
  std::vector<float> tmp(n);
  if (cudaMemcpy(tmp.data(), src, n * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
    return HSS_ERR_CUDA;
  for (size_t i = 0; i < n; ++i) dst[i] = (double)tmp[i];
  return HSS_OK;
}

}  // extern "C"
