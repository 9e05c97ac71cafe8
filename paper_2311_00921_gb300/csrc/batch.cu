// Batched factorization and solve of many independent HSS matrices of uneven
// order, leaf size, rank and depth (FP64).
//
// Layout ("forest"): matrices are grouped by (leaf, rank); inside a group they
// are sorted by depth L, deepest first, and every per-level array is the
// concatenation, by height above the leaves, of the members' arrays.  At
// height h the members with L > h are active and their nodes form one
// contiguous batch of identical shape (b = leaf at h = 0, 2 rank above), so a
// whole height of all members is one launch per step of Alg. 2 -- the same
// kernels as the single-matrix path.  Parent of node g is g / 2, except for the
// members whose root lies at height h + 1: sorted last, their nodes are a
// contiguous suffix whose parents are the members' root blocks (one root array
// per group, factored in one batched launch at the end).  Groups run on their
// own streams (each with a second stream for the basis chain, as in the single
// path), joined to the caller's stream.
#include <math.h>

#include <algorithm>
#include <new>
#include <numeric>
#include <vector>

#include "../../include/hss.h"
#include "common.cuh"
#include "ulv_kernels.cuh"
#include "uneven.cuh"

namespace {

constexpr int kCols = 16;   // right-hand-side columns per sweep pass

struct Height {
  long long nodes = 0;   // N_h
  long long split = 0;   // nodes [0, split) have a parent at h + 1; the rest have roots
  int mfirst = 0;        // first member (group order) whose root is at height h + 1
  int b = 0, c = 0;
  double *V = nullptr, *T = nullptr, *LB = nullptr, *M = nullptr, *A = nullptr, *B = nullptr;
  double *E = nullptr, *S = nullptr, *yv = nullptr, *ldp = nullptr;
};

struct Group {
  int leaf = 0, r = 0, H = 0;
  std::vector<int> member;     // user index of each member, deepest first
  std::vector<int> L;          // depth of each member
  std::vector<Height> ht;      // heights 0 .. H-1
  double *D = nullptr, *U = nullptr;
  double *R = nullptr, *rootvec = nullptr, *ldroot = nullptr;
  double *W = nullptr, *Y = nullptr, *X = nullptr, *Z = nullptr, *Zq = nullptr;
  double *t1 = nullptr, *t2 = nullptr, *xg = nullptr;
  long long rows = 0;          // leaf-level rows of the group
  std::vector<long long> row_off;   // member -> row offset in xg
  cudaStream_t st = nullptr, qs = nullptr;
  std::vector<cudaEvent_t> ev;      // per height: basis chain done
  cudaEvent_t ev_start = nullptr, ev_done = nullptr;
};

}  // namespace

struct hss_batch_s {
  int count = 0;
  std::vector<int> n;          // order of each matrix (user order)
  std::vector<Group> groups;
  // per member logdet ranges: device table of (offset into ldp_all, count)
  long long* ranges = nullptr;
  int* range_start = nullptr;   // count + 1
  double* ldp_all = nullptr;
  double* logdet = nullptr;     // count
  int* status = nullptr;
  const double** ptr_tab = nullptr;   // device pointer table for gather / scatter
  long long* ptr_rows = nullptr;      // device: (rows, row offset) per matrix, then group lds
  // uneven members: device row maps (padded row -> caller's row or -1), a table of
  // them (null for uniform members) and the callers' orders
  void* map_mem = nullptr;
  const int** map_tab = nullptr;
  long long* user_n = nullptr;
  void* arena = nullptr;
  int factorized = 0;
  cudaEvent_t ev_join = nullptr;
  std::vector<cudaEvent_t> ev_group;
  // optional CUDA graph of the whole factorization (captured on cap_stream)
  int use_graph = 0;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  cudaEvent_t ev_cap_in = nullptr, ev_cap_out = nullptr;
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

size_t layout(hss_batch_s* bt, char* base) {
  Bump bp{base};
  long long ldp_total = 0;
  for (Group& g : bt->groups) {
    const int r = g.r, leaf = g.leaf;
    const long long rr = (long long)r * r;
    const int nm = (int)g.member.size();
    g.H = g.L[0];
    g.ht.assign(g.H, Height());
    for (int h = 0; h < g.H; ++h) {
      Height& t = g.ht[h];
      for (int m = 0; m < nm; ++m)
        if (g.L[m] > h) t.nodes += 1LL << (g.L[m] - h);
      for (int m = 0; m < nm; ++m)
        if (g.L[m] > h + 1) t.split += 1LL << (g.L[m] - h);
      t.mfirst = 0;
      while (t.mfirst < nm && g.L[t.mfirst] > h + 1) ++t.mfirst;
      t.b = (h == 0) ? leaf : 2 * r;
      t.c = t.b - r;
      t.V = bp.take<double>(t.nodes * t.b * r);
      t.T = bp.take<double>(t.nodes * rr);
      t.LB = bp.take<double>(t.nodes * rr);
      if (h == 0) {
        t.M = bp.take<double>(t.nodes * t.b * t.b);
      } else {
        t.A = bp.take<double>(t.nodes * t.b * t.b);
        t.M = t.A;
        t.B = bp.take<double>(t.nodes * t.b * r);
        t.E = bp.take<double>(t.nodes * 2 * rr);
        t.yv = bp.take<double>(t.nodes * t.b * kCols);
      }
      t.S = bp.take<double>((t.nodes / 2) * rr);
      ldp_total += t.nodes;
    }
    const long long n0 = g.ht[0].nodes;
    g.rows = n0 * leaf;
    g.D = bp.take<double>(n0 * leaf * leaf);
    g.U = bp.take<double>(n0 * leaf * r);
    g.R = bp.take<double>((size_t)nm * 4 * rr);
    g.rootvec = bp.take<double>((size_t)nm * 2 * r * kCols);
    g.W = bp.take<double>(n0 * leaf * r);
    g.Y = bp.take<double>(n0 * leaf * r);
    g.X = bp.take<double>(n0 * rr);
    g.Z = bp.take<double>(n0 * rr);
    g.Zq = bp.take<double>(n0 * rr);
    g.t1 = bp.take<double>(n0 * r * kCols);
    g.t2 = bp.take<double>(n0 * r * kCols);
    g.xg = bp.take<double>(g.rows * kCols);
    ldp_total += nm;
  }
  bt->ldp_all = bp.take<double>(ldp_total);
  bt->logdet = bp.take<double>(bt->count);
  bt->status = bp.take<int>(8);
  bt->ptr_tab = bp.take<const double*>(2 * bt->count);
  bt->ptr_rows = bp.take<long long>(3 * bt->count);   // (rows, offset) pairs, then group lds
  // per-member logdet ranges: one per height the member spans, plus its root
  long long nr = 0;
  for (Group& g : bt->groups)
    for (int L : g.L) nr += L + 1;
  bt->ranges = bp.take<long long>(2 * nr);
  bt->range_start = bp.take<int>(bt->count + 1);
  // per-height logdet slices and root slices inside ldp_all
  if (base) {
    long long o = 0;
    for (Group& g : bt->groups) {
      for (int h = 0; h < g.H; ++h) {
        g.ht[h].ldp = bt->ldp_all + o;
        o += g.ht[h].nodes;
      }
      g.ldroot = bt->ldp_all + o;
      o += (long long)g.member.size();
    }
  }
  return bp.off + 256;
}

void gemm(bool ta, bool tb, int m, int n, int k, double alpha, const double* A, int lda,
          long long sA, const double* B, int ldb, long long sB, double beta, double* C, int ldc,
          long long sC, long long batch, cudaStream_t st) {
  if (batch > 0) gemm_batched<double>(ta, tb, m, n, k, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc,
                                      sC, (int)batch, st);
}

#define TRY(call)                                                                      \
  do {                                                                                 \
    const cudaError_t e_ = (call);                                                     \
    if (e_ != cudaSuccess)                                                             \
      return e_ == cudaErrorInvalidConfiguration ? HSS_ERR_INVALID_ARG : HSS_ERR_CUDA; \
  } while (0)

int factor_group(hss_batch_s* bt, Group& g) {
  const int r = g.r;
  const long long rr = (long long)r * r;
  cudaStream_t st = g.st, qs = g.qs;
  TRY(cudaEventRecord(g.ev_start, st));
  TRY(cudaStreamWaitEvent(qs, g.ev_start, 0));
  // basis chain: completion of every height, then the merge's coupling and bases
  for (int h = 0; h < g.H; ++h) {
    Height& t = g.ht[h];
    const int b = t.b;
    const long long br = (long long)b * r;
    const double* Bsrc = (h == 0) ? g.U : t.B;
    TRY(launch_ql_basis<double>(Bsrc, b, br, t.V, br, t.T, rr, t.LB, rr, b, r, (int)t.nodes, qs));
    const long long np = t.split / 2, nq = (t.nodes - t.split) / 2;
    // pairs with a regular parent at h + 1
    if (np > 0) {
      Height& u = g.ht[h + 1];
      gemm(false, false, r, r, r, 1.0, t.LB + rr, r, 2 * rr, t.S, r, rr, 0.0, g.Zq, r, rr, np, qs);
      gemm(false, true, r, r, r, 1.0, g.Zq, r, rr, t.LB, r, 2 * rr, 0.0, u.A + r, 2 * r, 4 * rr, np,
           qs);
      gemm(false, true, r, r, r, 1.0, t.LB, r, 2 * rr, g.Zq, r, rr, 0.0, u.A + (long long)r * 2 * r,
           2 * r, 4 * rr, np, qs);
      gemm(false, false, r, r, r, 1.0, t.LB, r, 2 * rr, u.E, 2 * r, 2 * rr, 0.0, u.B, 2 * r, 2 * rr,
           np, qs);
      gemm(false, false, r, r, r, 1.0, t.LB + rr, r, 2 * rr, u.E + r, 2 * r, 2 * rr, 0.0, u.B + r,
           2 * r, 2 * rr, np, qs);
    }
    // pairs whose parent is a member's root
    if (nq > 0) {
      const double* LBq = t.LB + t.split * rr;
      const double* Sq = t.S + (t.split / 2) * rr;
      double* Rq = g.R + (long long)t.mfirst * 4 * rr;
      gemm(false, false, r, r, r, 1.0, LBq + rr, r, 2 * rr, Sq, r, rr, 0.0, g.Zq, r, rr, nq, qs);
      gemm(false, true, r, r, r, 1.0, g.Zq, r, rr, LBq, r, 2 * rr, 0.0, Rq + r, 2 * r, 4 * rr, nq,
           qs);
      gemm(false, true, r, r, r, 1.0, LBq, r, 2 * rr, g.Zq, r, rr, 0.0, Rq + (long long)r * 2 * r,
           2 * r, 4 * rr, nq, qs);
    }
    TRY(cudaEventRecord(g.ev[h], qs));
    TRY(cudaGetLastError());
  }
  // main chain: diagonal product and partial Cholesky of every height
  for (int h = 0; h < g.H; ++h) {
    Height& t = g.ht[h];
    const int b = t.b, c = t.c;
    const long long br = (long long)b * r, bb = (long long)b * b, n = t.nodes;
    TRY(cudaStreamWaitEvent(st, g.ev[h], 0));
    const double* Ain = (h == 0) ? g.D : t.A;
    gemm(false, false, b, r, b, 1.0, Ain, b, bb, t.V, b, br, 0.0, g.W, b, br, n, st);
    gemm(false, false, b, r, r, 1.0, g.W, b, br, t.T, r, rr, 0.0, g.Y, b, br, n, st);
    gemm(true, false, r, r, b, 1.0, t.V, b, br, g.Y, b, br, 0.0, g.X, r, rr, n, st);
    gemm(true, false, r, r, r, 1.0, t.T, r, rr, g.X, r, rr, 0.0, g.Z, r, rr, n, st);
    gemm(false, false, b, r, r, -0.5, t.V, b, br, g.Z, r, rr, 1.0, g.Y, b, br, n, st);
    syr2k_lower_batched<double>(b, r, Ain, b, bb, g.Y, b, br, t.V, b, br, t.M, b, bb, (int)n, st);
    if (t.split > 0)
      TRY(launch_pchol<double>(t.M, b, bb, b, c, g.ht[h + 1].A, 2 * r, 4 * rr, t.ldp, h, 0,
                               bt->status, (int)t.split, st));
    if (t.nodes > t.split)
      TRY(launch_pchol<double>(t.M + t.split * bb, b, bb, b, c, g.R + (long long)t.mfirst * 4 * rr,
                               2 * r, 4 * rr, t.ldp, h, (int)t.split, bt->status,
                               (int)(t.nodes - t.split), st));
    TRY(cudaGetLastError());
  }
  // every member's root Cholesky in one launch
  const int nm = (int)g.member.size();
  TRY(launch_pchol<double>(g.R, 2 * r, 4 * rr, 2 * r, 2 * r, nullptr, 0, 0, g.ldroot, g.H, 0,
                           bt->status, nm, st));
  return HSS_OK;
}

void apply_q(Group& g, const Height& t, double* vec, int ldv, int nc, bool transpose,
             cudaStream_t st) {
  const int b = t.b, r = g.r;
  const long long s1 = (long long)r * kCols;
  gemm(true, false, r, nc, b, 1.0, t.V, b, (long long)b * r, vec, ldv, b, 0.0, g.t1, r, s1, t.nodes,
       st);
  gemm(transpose, false, r, nc, r, 1.0, t.T, r, (long long)r * r, g.t1, r, s1, 0.0, g.t2, r, s1,
       t.nodes, st);
  gemm(false, false, b, nc, r, -1.0, t.V, b, (long long)b * r, g.t2, r, s1, 1.0, vec, ldv, b,
       t.nodes, st);
}

int solve_group(Group& g, int nc) {
  const int r = g.r, nm = (int)g.member.size();
  cudaStream_t st = g.st;
  const int ldroot = nm * 2 * r;
  for (int h = 0; h < g.H; ++h) {
    Height& t = g.ht[h];
    double* vec = (h == 0) ? g.xg : t.yv;
    const int ldv = (h == 0) ? (int)g.rows : (int)(t.nodes * t.b);
    const long long bb = (long long)t.b * t.b;
    apply_q(g, t, vec, ldv, nc, true, st);
    if (t.split > 0) {
      Height& u = g.ht[h + 1];
      TRY(launch_trsv_fwd<double>(t.M, t.b, bb, t.b, t.c, vec, ldv, t.b, nc, u.yv,
                                  (int)(u.nodes * u.b), r, (int)t.split, st));
    }
    if (t.nodes > t.split)
      TRY(launch_trsv_fwd<double>(t.M + t.split * bb, t.b, bb, t.b, t.c, vec + t.split * t.b, ldv,
                                  t.b, nc, g.rootvec + (long long)t.mfirst * 2 * r, ldroot, r,
                                  (int)(t.nodes - t.split), st));
  }
  TRY(launch_trsv_fwd<double>(g.R, 2 * r, 4LL * r * r, 2 * r, 2 * r, g.rootvec, ldroot, 2 * r, nc,
                              nullptr, 0, 0, nm, st));
  TRY(launch_trsv_bwd<double>(g.R, 2 * r, 4LL * r * r, 2 * r, 2 * r, g.rootvec, ldroot, 2 * r, nc,
                              nullptr, 0, 0, nm, st));
  for (int h = g.H - 1; h >= 0; --h) {
    Height& t = g.ht[h];
    double* vec = (h == 0) ? g.xg : t.yv;
    const int ldv = (h == 0) ? (int)g.rows : (int)(t.nodes * t.b);
    const long long bb = (long long)t.b * t.b;
    if (t.split > 0) {
      Height& u = g.ht[h + 1];
      TRY(launch_trsv_bwd<double>(t.M, t.b, bb, t.b, t.c, vec, ldv, t.b, nc, u.yv,
                                  (int)(u.nodes * u.b), r, (int)t.split, st));
    }
    if (t.nodes > t.split)
      TRY(launch_trsv_bwd<double>(t.M + t.split * bb, t.b, bb, t.b, t.c, vec + t.split * t.b, ldv,
                                  t.b, nc, g.rootvec + (long long)t.mfirst * 2 * r, ldroot, r,
                                  (int)(t.nodes - t.split), st));
    apply_q(g, t, vec, ldv, nc, false, st);
  }
  TRY(cudaGetLastError());
  return HSS_OK;
}

// one CTA per matrix: copy nc columns between the matrix's own column-major
// buffer (ld = its order) and its rows (n_i of the uniform tree) of its group's
// leaf vector; an uneven member maps each padded row to its own row (or to none:
// zero going in, dropped coming out)
__global__ void gather_scatter_kernel(const double* const* ptrs, const long long* rows,
                                      const double* const* group_vec, const long long* group_ld,
                                      const int* const* maps, const long long* user_n, int nc,
                                      int col0, int scatter) {
  const int i = blockIdx.x;
  const long long n = rows[2 * i], off = rows[2 * i + 1];
  double* gv = const_cast<double*>(group_vec[i]);
  const long long ldg = group_ld[i], un = user_n[i];
  const int* map = maps[i];
  double* user = const_cast<double*>(ptrs[i]);
  for (long long e = threadIdx.x; e < n * nc; e += blockDim.x) {
    const long long k = e % n, j = e / n;
    const long long q = map ? map[k] : k;
    double* g = gv + off + k + j * ldg;
    if (scatter) {
      if (q >= 0) user[q + (long long)(col0 + j) * un] = *g;
    } else {
      *g = q >= 0 ? user[q + (long long)(col0 + j) * un] : 0.0;
    }
  }
}

// per-matrix log det: fixed-order sum of the matrix's node contributions
__global__ void batch_logdet_kernel(const double* ldp_all, const long long* ranges,
                                    const int* range_start, double* out) {
  __shared__ double red[32];
  const int i = blockIdx.x;
  double s = 0.0;
  for (int q = range_start[i]; q < range_start[i + 1]; ++q) {
    const long long o = ranges[2 * q], cnt = ranges[2 * q + 1];
    for (long long k = threadIdx.x; k < cnt; k += blockDim.x) s += ldp_all[o + k];
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) out[i] = s;
}

// fork every group's streams off the caller's stream, run fn per group, join back
template <typename F>
int fork_join(hss_batch_s* bt, cudaStream_t st, F fn) {
  if (cudaEventRecord(bt->ev_join, st) != cudaSuccess) return HSS_ERR_CUDA;
  for (Group& g : bt->groups)
    if (cudaStreamWaitEvent(g.st, bt->ev_join, 0) != cudaSuccess) return HSS_ERR_CUDA;
  int rc = HSS_OK;
  for (Group& g : bt->groups) {
    rc = fn(g);
    if (rc) break;
  }
  for (Group& g : bt->groups) {
    if (cudaEventRecord(g.ev_done, g.st) != cudaSuccess) return HSS_ERR_CUDA;
    if (cudaStreamWaitEvent(st, g.ev_done, 0) != cudaSuccess) return HSS_ERR_CUDA;
  }
  return rc;
}

int enqueue_factorize(hss_batch_s* bt, cudaStream_t st) {
  if (cudaMemsetAsync(bt->status, 0, 8 * sizeof(int), st) != cudaSuccess) return HSS_ERR_CUDA;
  int rc = fork_join(bt, st, [&](Group& g) { return factor_group(bt, g); });
  if (rc) return rc;
  batch_logdet_kernel<<<bt->count, 256, 0, st>>>(bt->ldp_all, bt->ranges, bt->range_start,
                                                 bt->logdet);
  return cudaGetLastError() == cudaSuccess ? HSS_OK : HSS_ERR_CUDA;
}

}  // namespace

extern "C" {

int hss_batch_create(int32_t count, const hss_shape* shapes, const double* const* D,
                     const double* const* U, const double* const* E, const double* const* S,
                     hss_batch_t* out) {
  if (!out || count <= 0 || !shapes || !D || !U || !S || !E) return HSS_ERR_INVALID_ARG;
  *out = nullptr;
  // uneven members: generators embedded in the uniform (leaf, rank) layout
  std::vector<UnevenPad> pads(count);
  std::vector<const double*> Dp(D, D + count), Up(U, U + count), Ep(E, E + count),
      Sp(S, S + count);
  for (int i = 0; i < count; ++i) {
    const hss_shape& s = shapes[i];
    if (s.levels < 1 || s.levels > 24 || s.leaf < 1 || s.leaf > 768 || s.rank < 1 ||
        s.rank > s.leaf || s.rank > 256)
      return HSS_ERR_INVALID_ARG;
    if (!D[i] || !U[i] || !S[i] || (s.levels >= 2 && !E[i])) return HSS_ERR_INVALID_ARG;
    if (s.node_sizes) {
      if (pad_uneven(s, D[i], U[i], E[i], S[i], &pads[i]) != HSS_OK) return HSS_ERR_INVALID_ARG;
      Dp[i] = pads[i].D.data();
      Up[i] = pads[i].U.data();
      Ep[i] = pads[i].E.data();
      Sp[i] = pads[i].S.data();
    } else if ((long long)s.leaf << s.levels != (long long)s.n) {
      return HSS_ERR_INVALID_ARG;
    }
  }
  D = Dp.data();
  U = Up.data();
  E = Ep.data();
  S = Sp.data();
  hss_batch_s* bt = new (std::nothrow) hss_batch_s();
  if (!bt) return HSS_ERR_OOM;
  bt->count = count;
  bt->n.resize(count);
  // groups by (leaf, rank), members deepest first
  std::vector<int> order(count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    const hss_shape &x = shapes[a], &y = shapes[b];
    if (x.leaf != y.leaf) return x.leaf < y.leaf;
    if (x.rank != y.rank) return x.rank < y.rank;
    return x.levels > y.levels;
  });
  for (int q = 0; q < count; ++q) {
    const int i = order[q];
    bt->n[i] = shapes[i].n;
    if (bt->groups.empty() || bt->groups.back().leaf != shapes[i].leaf ||
        bt->groups.back().r != shapes[i].rank) {
      bt->groups.emplace_back();
      bt->groups.back().leaf = shapes[i].leaf;
      bt->groups.back().r = shapes[i].rank;
    }
    bt->groups.back().member.push_back(i);
    bt->groups.back().L.push_back(shapes[i].levels);
  }
  const size_t bytes = layout(bt, nullptr);
  void* mem = nullptr;
  if (cudaMalloc(&mem, bytes) != cudaSuccess) {
    cudaGetLastError();
    delete bt;
    return HSS_ERR_OOM;
  }
  bt->arena = mem;
  for (Group& g : bt->groups) g.ht.clear();
  layout(bt, static_cast<char*>(mem));
  // copy the generators into the concatenated per-height arrays
  cudaError_t e = cudaSuccess;
  std::vector<long long> rstart(1, 0), rtab;
  std::vector<const double*> ptab;
  std::vector<long long> prow(2 * count, 0);
  std::vector<double*> gvec(count, nullptr);
  std::vector<long long> gld(count, 0);
  for (Group& g : bt->groups) {
    const int r = g.r, leaf = g.leaf;
    const long long rr = (long long)r * r;
    std::vector<long long> node_off(g.H, 0);   // running node offset per height
    g.row_off.assign(g.member.size(), 0);
    for (size_t m = 0; m < g.member.size(); ++m) {
      const int i = g.member[m], L = g.L[m];
      const hss_shape& s = shapes[i];
      const long long nl = 1LL << L;
      g.row_off[m] = node_off[0] * leaf;
      prow[2 * i] = nl * leaf;   // rows of the (padded) uniform tree
      prow[2 * i + 1] = g.row_off[m];
      gvec[i] = g.xg;
      gld[i] = g.rows;
      e = e ? e : cudaMemcpy(g.D + node_off[0] * leaf * leaf, D[i], sizeof(double) * nl * leaf * leaf,
                             cudaMemcpyHostToDevice);
      e = e ? e : cudaMemcpy(g.U + node_off[0] * leaf * r, U[i], sizeof(double) * nl * leaf * r,
                             cudaMemcpyHostToDevice);
      // E and S of the member: level l = L - h, packed level 1 first
      long long eoff = 0, soff = 0;
      std::vector<long long> Eo(L + 1, 0), So(L + 1, 0);
      for (int l = 1; l <= L - 1; ++l) {
        Eo[l] = eoff;
        eoff += (1LL << l) * 2 * rr;
      }
      for (int l = 1; l <= L; ++l) {
        So[l] = soff;
        soff += (1LL << (l - 1)) * rr;
      }
      for (int h = 0; h < L; ++h) {
        const int l = L - h;
        Height& t = g.ht[h];
        const long long nn = 1LL << l;
        if (h >= 1)
          e = e ? e : cudaMemcpy(t.E + node_off[h] * 2 * rr, E[i] + Eo[l], sizeof(double) * nn * 2 * rr,
                                 cudaMemcpyHostToDevice);
        e = e ? e : cudaMemcpy(t.S + (node_off[h] / 2) * rr, S[i] + So[l], sizeof(double) * (nn / 2) * rr,
                               cudaMemcpyHostToDevice);
        rtab.push_back((t.ldp - bt->ldp_all) + node_off[h]);
        rtab.push_back(nn);
        node_off[h] += nn;
      }
      rtab.push_back((g.ldroot - bt->ldp_all) + (long long)m);
      rtab.push_back(1);
      rstart.push_back((long long)rtab.size() / 2);
      (void)i;
    }
  }
  // range table in user order
  std::vector<long long> ranges_user;
  std::vector<int> start_user(count + 1, 0);
  {
    // rstart is in group order; map members back to user order
    std::vector<std::pair<long long, long long>> seg(count);
    int q = 0;
    for (Group& g : bt->groups)
      for (size_t m = 0; m < g.member.size(); ++m, ++q) seg[g.member[m]] = {rstart[q], rstart[q + 1]};
    for (int i = 0; i < count; ++i) {
      start_user[i] = (int)(ranges_user.size() / 2);
      for (long long k = seg[i].first; k < seg[i].second; ++k) {
        ranges_user.push_back(rtab[2 * k]);
        ranges_user.push_back(rtab[2 * k + 1]);
      }
    }
    start_user[count] = (int)(ranges_user.size() / 2);
  }
  e = e ? e : cudaMemcpy(bt->ranges, ranges_user.data(), sizeof(long long) * ranges_user.size(),
                         cudaMemcpyHostToDevice);
  e = e ? e : cudaMemcpy(bt->range_start, start_user.data(), sizeof(int) * (count + 1),
                         cudaMemcpyHostToDevice);
  e = e ? e : cudaMemcpy(bt->ptr_rows, prow.data(), sizeof(long long) * 2 * count,
                         cudaMemcpyHostToDevice);
  // second half of ptr_tab / ptr_rows: each matrix's group vector and its leading dimension
  e = e ? e : cudaMemcpy(bt->ptr_tab + count, gvec.data(), sizeof(double*) * count,
                         cudaMemcpyHostToDevice);
  e = e ? e : cudaMemcpy(bt->ptr_rows + 2 * count, gld.data(), sizeof(long long) * count,
                         cudaMemcpyHostToDevice);
  e = e ? e : cudaMemset(bt->status, 0, 8 * sizeof(int));
  {   // row maps of uneven members, their table, the callers' orders
    long long map_ints = 0;
    for (int i = 0; i < count; ++i) map_ints += (long long)pads[i].pmap.size();
    const size_t tab = sizeof(int*) * count, un = sizeof(long long) * count;
    if (e == cudaSuccess && cudaMalloc(&bt->map_mem, tab + un + sizeof(int) * (map_ints + 1)) !=
                                cudaSuccess) {
      cudaGetLastError();
      hss_batch_destroy(bt);
      return HSS_ERR_OOM;
    }
    if (e == cudaSuccess) {
      char* base = static_cast<char*>(bt->map_mem);
      bt->map_tab = reinterpret_cast<const int**>(base);
      bt->user_n = reinterpret_cast<long long*>(base + tab);
      int* maps = reinterpret_cast<int*>(base + tab + un);
      std::vector<const int*> mt(count, nullptr);
      std::vector<long long> nn(count);
      long long o = 0;
      for (int i = 0; i < count; ++i) {
        nn[i] = shapes[i].n;
        if (pads[i].pmap.empty()) continue;
        mt[i] = maps + o;
        e = e ? e : cudaMemcpy(maps + o, pads[i].pmap.data(), sizeof(int) * pads[i].pmap.size(),
                               cudaMemcpyHostToDevice);
        o += (long long)pads[i].pmap.size();
      }
      e = e ? e : cudaMemcpy(bt->map_tab, mt.data(), tab, cudaMemcpyHostToDevice);
      e = e ? e : cudaMemcpy(bt->user_n, nn.data(), un, cudaMemcpyHostToDevice);
    }
  }
  for (Group& g : bt->groups) {
    g.ev.assign(g.H, nullptr);
    e = e ? e : cudaStreamCreateWithFlags(&g.st, cudaStreamNonBlocking);
    e = e ? e : cudaStreamCreateWithFlags(&g.qs, cudaStreamNonBlocking);
    e = e ? e : cudaEventCreateWithFlags(&g.ev_start, cudaEventDisableTiming);
    e = e ? e : cudaEventCreateWithFlags(&g.ev_done, cudaEventDisableTiming);
    for (int h = 0; h < g.H && e == cudaSuccess; ++h)
      e = cudaEventCreateWithFlags(&g.ev[h], cudaEventDisableTiming);
  }
  e = e ? e : cudaEventCreateWithFlags(&bt->ev_join, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    hss_batch_destroy(bt);
    return HSS_ERR_CUDA;
  }
  *out = bt;
  return HSS_OK;
}

void hss_batch_destroy(hss_batch_t bt) {
  if (!bt) return;
  for (Group& g : bt->groups) {
    if (g.st) cudaStreamSynchronize(g.st);
    if (g.qs) cudaStreamSynchronize(g.qs);
    for (cudaEvent_t ev : g.ev)
      if (ev) cudaEventDestroy(ev);
    if (g.ev_start) cudaEventDestroy(g.ev_start);
    if (g.ev_done) cudaEventDestroy(g.ev_done);
    if (g.st) cudaStreamDestroy(g.st);
    if (g.qs) cudaStreamDestroy(g.qs);
  }
  if (bt->ev_join) cudaEventDestroy(bt->ev_join);
  if (bt->cap_stream) cudaStreamSynchronize(bt->cap_stream);
  if (bt->graph_exec) cudaGraphExecDestroy(bt->graph_exec);
  if (bt->ev_cap_in) cudaEventDestroy(bt->ev_cap_in);
  if (bt->ev_cap_out) cudaEventDestroy(bt->ev_cap_out);
  if (bt->cap_stream) cudaStreamDestroy(bt->cap_stream);
  cudaFree(bt->arena);
  if (bt->map_mem) cudaFree(bt->map_mem);
  delete bt;
}

int hss_batch_set_graph(hss_batch_t bt, int32_t enable) {
  if (!bt) return HSS_ERR_INVALID_ARG;
  bt->use_graph = enable ? 1 : 0;
  return HSS_OK;
}

int hss_batch_factorize(hss_batch_t bt, const hss_options* opt, void* stream) {
  if (!bt) return HSS_ERR_INVALID_ARG;
  if (opt && opt->precision != HSS_FP64) return HSS_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  bt->factorized = 0;
  if (!bt->use_graph) {
    int rc = enqueue_factorize(bt, st);
    if (rc) return rc;
    bt->factorized = 1;
    return HSS_OK;
  }
  if (!bt->graph_exec) {
    // one plain run first (kernel attributes, module loading), then capture the
    // same launches on the object's own stream
    int rc = enqueue_factorize(bt, st);
    if (rc) return rc;
    if (cudaStreamSynchronize(st) != cudaSuccess) return HSS_ERR_CUDA;
    cudaError_t e = cudaSuccess;
    if (!bt->cap_stream) {
      e = e ? e : cudaStreamCreateWithFlags(&bt->cap_stream, cudaStreamNonBlocking);
      e = e ? e : cudaEventCreateWithFlags(&bt->ev_cap_in, cudaEventDisableTiming);
      e = e ? e : cudaEventCreateWithFlags(&bt->ev_cap_out, cudaEventDisableTiming);
      if (e) return HSS_ERR_CUDA;
    }
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(bt->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return HSS_ERR_CUDA;
    rc = enqueue_factorize(bt, bt->cap_stream);
    e = cudaStreamEndCapture(bt->cap_stream, &graph);
    if (rc || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return rc ? rc : HSS_ERR_CUDA;
    }
    e = cudaGraphInstantiate(&bt->graph_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      bt->graph_exec = nullptr;
      return HSS_ERR_CUDA;
    }
  }
  cudaError_t e = cudaEventRecord(bt->ev_cap_in, st);
  e = e ? e : cudaStreamWaitEvent(bt->cap_stream, bt->ev_cap_in, 0);
  e = e ? e : cudaGraphLaunch(bt->graph_exec, bt->cap_stream);
  e = e ? e : cudaEventRecord(bt->ev_cap_out, bt->cap_stream);
  e = e ? e : cudaStreamWaitEvent(st, bt->ev_cap_out, 0);
  if (e != cudaSuccess) return HSS_ERR_CUDA;
  bt->factorized = 1;
  return HSS_OK;
}

int hss_batch_solve(hss_batch_t bt, const double* const* b, double* const* x, int32_t nrhs,
                    void* stream) {
  if (!bt || !b || !x || nrhs < 0) return HSS_ERR_INVALID_ARG;
  if (!bt->factorized) return HSS_ERR_NOT_FACTORIZED;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int count = bt->count;
  for (int i = 0; i < count; ++i)
    if (!b[i] || !x[i]) return HSS_ERR_INVALID_ARG;
  // device pointer tables: b then x (the group vectors follow in ptr_tab + count)
  std::vector<const double*> bp(b, b + count), xp(x, x + count);
  for (int j0 = 0; j0 < nrhs; j0 += kCols) {
    const int nc = std::min(kCols, nrhs - j0);
    if (cudaMemcpyAsync(bt->ptr_tab, bp.data(), sizeof(double*) * count, cudaMemcpyHostToDevice,
                        st) != cudaSuccess)
      return HSS_ERR_CUDA;
    gather_scatter_kernel<<<count, 256, 0, st>>>(bt->ptr_tab, bt->ptr_rows,
                                                 bt->ptr_tab + count,
                                                 bt->ptr_rows + 2 * count, bt->map_tab,
                                                 bt->user_n, nc, j0, 0);
    int rc = fork_join(bt, st, [&](Group& g) { return solve_group(g, nc); });
    if (rc) return rc;
    if (cudaMemcpyAsync(bt->ptr_tab, xp.data(), sizeof(double*) * count, cudaMemcpyHostToDevice,
                        st) != cudaSuccess)
      return HSS_ERR_CUDA;
    gather_scatter_kernel<<<count, 256, 0, st>>>(bt->ptr_tab, bt->ptr_rows,
                                                 bt->ptr_tab + count,
                                                 bt->ptr_rows + 2 * count, bt->map_tab,
                                                 bt->user_n, nc, j0, 1);
    if (cudaGetLastError() != cudaSuccess) return HSS_ERR_CUDA;
    // the pointer table is reused by the next pass: keep the host copies alive until then
    if (cudaStreamSynchronize(st) != cudaSuccess) return HSS_ERR_CUDA;
  }
  return HSS_OK;
}

int hss_batch_logdet(hss_batch_t bt, double* out) {
  if (!bt || !out) return HSS_ERR_INVALID_ARG;
  if (!bt->factorized) return HSS_ERR_NOT_FACTORIZED;
  if (cudaDeviceSynchronize() != cudaSuccess) return HSS_ERR_CUDA;
  int s[8];
  if (cudaMemcpy(s, bt->status, sizeof(s), cudaMemcpyDeviceToHost) != cudaSuccess)
    return HSS_ERR_CUDA;
  if (s[ST_CODE]) return s[ST_CODE];
  return cudaMemcpy(out, bt->logdet, sizeof(double) * bt->count, cudaMemcpyDeviceToHost) ==
                 cudaSuccess
             ? HSS_OK
             : HSS_ERR_CUDA;
}

}  // extern "C"
