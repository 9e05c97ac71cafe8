// Per-node ULV step kernels (one CTA per tree node).
//
//  * ql_basis_kernel   -- basis completion, Eq. 2-3 (Sec. 2): Householder QL of
//                         the node basis B (b x r) as the QR of its row- and
//                         column-reversed copy (LAPACK dlarfg signs), giving
//                         Q = I - V T Vᵀ = [Q^R Q^S] with the redundant part first,
//                         and L_B = Q^Sᵀ B (r x r, lower triangular).
//  * chol_panel_kernel -- one 32-column panel of the partial Cholesky, Eq.
//                         partial-Cholesky (Alg. 2), for every node of a
//                         level: POTRF of the diagonal block and TRSM of the rows
//                         below it; the trailing SYRK is a level-wide launch
//                         (gemm.cu).  With c = b it is the panel of the root
//                         Cholesky (the last step of Alg. 2).
//  * scatter_ss_kernel -- the merge (Alg. 2) as its own pass: Â^SS of each node
//                         into its parent's diagonal block.  Used only where a
//                         level eliminates nothing (rank = block order); otherwise
//                         the last Schur update writes the parent block itself
//                         (syrk_lower_merge_batched, gemm.cu).
//  * pchol_kernel      -- the whole partial Cholesky of a node in one CTA, with
//                         the merge as its epilogue (the batched forest path).
//  * trsv_fwd_kernel /
//    trsv_bwd_kernel   -- one level of the ULV solve (Sec. 3.2): forward
//                         y := Qᵀ y (optionally), z^R = L^RR⁻¹ y^R, y^S -= L^SR z^R
//                         (pushed to the parent's vector); backward
//                         x^R = L^RR⁻ᵀ (z^R - L^SRᵀ x^S), then x := Q x (optionally).
//  * logdet_reduce_kernel -- 2 Σ log diag over all nodes, fixed summation order.
#include <math.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

#include "common.cuh"
#include "ulv_kernels.cuh"

namespace {

constexpr int NT = 256;
constexpr int NB = 32;   // panel width of the blocked Cholesky / triangular solves

// ------------------------------------------------------------------ QL
// Sum over the 32 lanes of acc[k] lands in lane k (k < NV; NV = 16 or 32):
// a transposing butterfly, NV - 1 (+ NV for NV = 16) shuffles instead of NV * 5.
template <typename T, int NV>
HSS_DEVINL T warp_transpose_reduce(T (&acc)[NV], int lane) {
  if (NV == 16) {
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], 16);
  }
#pragma unroll
  for (int s = NV / 2; s >= 1; s >>= 1) {
    const bool upper = (lane & s) != 0;
#pragma unroll
    for (int i = 0; i < s; ++i) {
      const T send = upper ? acc[i] : acc[i + s];
      const T keep = upper ? acc[i + s] : acc[i];
      acc[i] = keep + __shfl_xor_sync(0xffffffffu, send, s);
    }
  }
  return acc[0];
}

// CTA-level product O(q, c) = Σ_{i >= i0} Pt(q, i) A(i, c) for q < NBP and the
// ncols columns of A (column c at A + c * lda): the panel's reflectors (Pt,
// transposed in shared memory with row pitch NBP + 1) against 64-row slabs of A
// staged in shared memory.  Thread t owns reflector q = t % NBP and NBP / 8
// consecutive columns of each 32-column chunk.  O(q, c) lands at Out[q * os1 + c * os2].
template <typename T, int NBP>
HSS_DEVINL void cta_vt_times(const T* Pt, const T* A, long long lda, int ncols, int i0, int b,
                             T* As, T* Out, int os1, int os2) {
  constexpr int CPT = NBP / 8;   // columns per thread per chunk
  const int tid = threadIdx.x;
  const int q = tid % NBP, cg = tid / NBP;
  for (int c0 = 0; c0 < ncols; c0 += 32) {
    T acc[CPT];
#pragma unroll
    for (int u = 0; u < CPT; ++u) acc[u] = T(0);
    for (int s0 = i0; s0 < b; s0 += 64) {
      for (int e = tid; e < 64 * 32; e += NT) {
        const int ii = e % 64, cc = e / 64;
        const int i = s0 + ii, c = c0 + cc;
        As[ii * 33 + cc] = (i < b && c < ncols) ? A[i + (long long)c * lda] : T(0);
      }
      __syncthreads();
      const int rows = min(64, b - s0);
      for (int ii = 0; ii < rows; ++ii) {
        const T v = Pt[q + (s0 + ii) * (NBP + 1)];
#pragma unroll
        for (int u = 0; u < CPT; ++u) acc[u] = fma(v, As[ii * 33 + cg * CPT + u], acc[u]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < CPT; ++u) {
      const int c = c0 + cg * CPT + u;
      if (c < ncols) Out[q * os1 + c * os2] = acc[u];
    }
  }
}

// Blocked Householder QR of the reversed basis (= QL of the basis).  Panels of
// NBP columns are factored in registers: thread t holds rows j0 + t + NT s of the
// panel, and column j costs one CTA-wide reduction of the Gram row
// g_k = Σ_{i>j} x_ij x_ik (k >= j): its first entry is the squared norm below the
// pivot, and with the pivot row it gives every v_jᵀ x_k, so the reflector and
// its application to the rest of the panel need no second reduction.  The
// trailing columns get the panel's block reflector, A -= Ṽ_p (T_pᵀ (Ṽ_pᵀ A)),
// as two CTA-level products; the compact-WY T is assembled block by block,
// T(0:j0, p) = -T(0:j0, 0:j0) (Ṽ_{0:j0}ᵀ Ṽ_p) T_p, with T(0:j0, 0:j0) streamed
// through shared memory in 64 x 32 slabs.
template <typename T, int NBP, int RPT>
__global__ void __launch_bounds__(NT)
ql_basis_kernel(const T* __restrict__ Bsrc, int ldb_src, long long sB, T* V, long long sV, T* Tm,
                long long sT, T* LB, long long sL, int b, int r, const int* __restrict__ only_if) {
  if (only_if && only_if[blockIdx.x] == 0) return;   // node completed by another path
  extern __shared__ unsigned char smem_raw[];
  T* Pt = reinterpret_cast<T*>(smem_raw);       // panel reflectors, transposed: (NBP+1) x b
  T* Ws = Pt + (size_t)b * (NBP + 1);           // NBP x r : Ṽ_pᵀ A_trail
  T* Xs = Ws + (size_t)NBP * r;                 // r x NBP : Ṽ_{0:j0}ᵀ Ṽ_p
  T* Ys = Xs + (size_t)r * NBP;                 // r x NBP
  T* As = Ys + (size_t)r * NBP;                 // 64 x 33 staging slab
  constexpr int NW = NT / 32;
  __shared__ T red[2][NW][NBP];
  __shared__ T prow[2][NBP];
  __shared__ T tau_s[256];
  __shared__ T Tp[NBP][NBP + 1];
  __shared__ T Gp[NBP][NBP + 1];
  const long long node = blockIdx.x;
  const T* B = Bsrc + node * sB;
  T* W = V + node * sV;   // working matrix, reversed coordinates during the QR
  T* Tn = Tm + node * sT;
  T* Ln = LB + node * sL;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;

  for (long long e = tid; e < (long long)b * r; e += NT) {
    const int i = (int)(e % b), j = (int)(e / b);
    W[i + (long long)j * b] = B[(b - 1 - i) + (long long)(r - 1 - j) * ldb_src];
  }
  for (int e = tid; e < r * r; e += NT) Tn[e] = T(0);
  __syncthreads();

  for (int j0 = 0; j0 < r; j0 += NBP) {
    const int nbw = min(NBP, r - j0);
    T x[RPT][NBP];
#pragma unroll
    for (int s = 0; s < RPT; ++s) {
      const int i = j0 + tid + NT * s;
#pragma unroll
      for (int k = 0; k < NBP; ++k)
        x[s][k] = (i < b && k < nbw) ? W[i + (long long)(j0 + k) * b] : T(0);
    }
#pragma unroll
    for (int jj = 0; jj < NBP; ++jj) {
      if (jj >= nbw) break;
      const int j = j0 + jj;
      const int buf = jj & 1;
      if (tid == jj) {   // the pivot row (row j is thread jj's first row)
#pragma unroll
        for (int k = 0; k < NBP; ++k) prow[buf][k] = x[0][k];
      }
      T g[NBP];
#pragma unroll
      for (int k = 0; k < NBP; ++k) g[k] = T(0);
#pragma unroll
      for (int s = 0; s < RPT; ++s) {
        const int i = j0 + tid + NT * s;
        if (i > j && i < b) {
          const T a = x[s][jj];
#pragma unroll
          for (int k = jj; k < NBP; ++k) g[k] = fma(a, x[s][k], g[k]);
        }
      }
      const T gw = warp_transpose_reduce<T, NBP>(g, lane);
      if (lane < NBP) red[buf][wid][lane] = gw;
      __syncthreads();
      T gk = T(0);   // Σ_{i>j} x_ij x_ik for k = lane
      if (lane < NBP) {
#pragma unroll
        for (int w = 0; w < NW; ++w) gk += red[buf][w][lane];
      }
      const T sigma = __shfl_sync(0xffffffffu, gk, jj);
      const T alpha = prow[buf][jj];
      T tau, beta, scale;
      if (sigma == T(0)) {
        tau = T(0);
        beta = alpha;
        scale = T(1);
      } else {
        const T nrm = sqrt(alpha * alpha + sigma);
        beta = alpha >= T(0) ? -nrm : nrm;
        tau = (beta - alpha) / beta;
        scale = T(1) / (alpha - beta);
      }
      if (tid == 0) tau_s[j] = tau;
      // v_jᵀ x_k = x_jk + scale g_k, held by lane k; then x_k -= tau (v_jᵀ x_k) v_j
      const T tw = lane < NBP ? tau * fma(scale, gk, prow[buf][lane]) : T(0);
#pragma unroll
      for (int s = 0; s < RPT; ++s) {
        const int i = j0 + tid + NT * s;
        const bool below = i > j && i < b;
        const T v = below ? x[s][jj] * scale : (i == j ? T(1) : T(0));
#pragma unroll
        for (int k = jj + 1; k < NBP; ++k) {
          const T twk = __shfl_sync(0xffffffffu, tw, k);
          x[s][k] = fma(-twk, v, x[s][k]);
        }
        if (below) x[s][jj] = v;
        if (i == j) x[s][jj] = beta;   // R(j, j)
      }
    }
    // write the panel back (R on and above the diagonal, reflectors below) and
    // keep the reflectors, with their unit diagonal and zeros above, transposed
#pragma unroll
    for (int s = 0; s < RPT; ++s) {
      const int i = j0 + tid + NT * s;
      if (i < b) {
#pragma unroll
        for (int k = 0; k < NBP; ++k) {
          if (k < nbw) W[i + (long long)(j0 + k) * b] = x[s][k];
          const int d = j0 + k;
          T v = T(0);
          if (k < nbw) v = i > d ? x[s][k] : (i == d ? T(1) : T(0));
          Pt[k + i * (NBP + 1)] = v;
        }
      }
    }
    for (int e = tid; e < j0 * NBP; e += NT) Pt[(e % NBP) + (e / NBP) * (NBP + 1)] = T(0);
    __syncthreads();
    // panel Gram Gp(a, c) = v_aᵀ v_c (a < c) from the register panel: the
    // columns c and NBP - c share one transposing warp reduction (c + (NBP - c)
    // = NBP products), then the warps' partials are summed through shared memory
    {
      T* Gs = Ws;   // NW x NBP x (NBP + 1) partials; the product buffers are free here
#pragma unroll
      for (int c = 1; c <= NBP / 2; ++c) {
        const int c2 = NBP - c;   // partner column (c2 == c for c = NBP / 2)
        T g[NBP];
#pragma unroll
        for (int q = 0; q < NBP; ++q) g[q] = T(0);
#pragma unroll
        for (int s = 0; s < RPT; ++s) {
          const int i = j0 + tid + NT * s;
          if (i < b) {
            auto vref = [&](int k) -> T {
              const int d = j0 + k;
              return i > d ? x[s][k] : (i == d ? T(1) : T(0));
            };
            const T vc = vref(c), vc2 = vref(c2);
#pragma unroll
            for (int q = 0; q < NBP; ++q) {
              if (q < c) g[q] = fma(vref(q), vc, g[q]);                   // (a = q, c)
              else if (c2 != c) g[q] = fma(vref(q - c), vc2, g[q]);       // (a = q - c, c2)
            }
          }
        }
        const T gw = warp_transpose_reduce<T, NBP>(g, lane);
        if (lane < NBP) {
          if (lane < c) Gs[(wid * NBP + c) * (NBP + 1) + lane] = gw;
          else if (c2 != c && lane - c < c2) Gs[(wid * NBP + c2) * (NBP + 1) + (lane - c)] = gw;
        }
      }
      __syncthreads();
      for (int e = tid; e < NBP * NBP; e += NT) {
        const int a = e % NBP, c = e / NBP;
        if (a < c) {
          T v = T(0);
#pragma unroll
          for (int w = 0; w < NW; ++w) v += Gs[(w * NBP + c) * (NBP + 1) + a];
          Gp[a][c] = v;
        }
      }
      __syncthreads();
    }
    // panel T (forward dlarft): T_p(0:c, c) = -tau_c T_p(0:c, 0:c) Gp(0:c, c),
    // lane a keeps row a of T_p in registers
    if (wid == 0) {
      T tp[NBP];
#pragma unroll
      for (int m = 0; m < NBP; ++m) tp[m] = T(0);
#pragma unroll
      for (int c = 0; c < NBP; ++c) {
        if (c < nbw) {
          const T tc = tau_s[j0 + c];
          T v = T(0);
#pragma unroll
          for (int m = 0; m < c; ++m) v = fma(tp[m], Gp[m][c], v);
          tp[c] = lane < c ? -tc * v : (lane == c ? tc : T(0));
        }
      }
      if (lane < NBP) {
#pragma unroll
        for (int m = 0; m < NBP; ++m) Tp[lane][m] = (lane < nbw && m < nbw) ? tp[m] : T(0);
      }
    }
    __syncthreads();
    // T(0:j0, panel) = -T(0:j0, 0:j0) (Ṽ_{0:j0}ᵀ Ṽ_p) T_p ; T(panel, panel) = T_p
    if (j0 > 0) {
      // Xs(a, q) = v_aᵀ v_q over rows >= j0 (where v_a, a < j0, is below its diagonal)
      cta_vt_times<T, NBP>(Pt, W, b, j0, j0, b, As, Xs, 1, NBP);
      __syncthreads();
      // Ys(a, q) = Σ_{m >= a} T(a, m) Xs(m, q): thread owns row a0 + tid % 64 and
      // columns tid / 64 + (NT / 64) t of each 64-row block
      constexpr int QT = NBP / (NT / 64);
      const int aa = tid % 64, qb = tid / 64;
      for (int a0 = 0; a0 < j0; a0 += 64) {
        T acc[QT];
#pragma unroll
        for (int t = 0; t < QT; ++t) acc[t] = T(0);
        for (int m0 = a0; m0 < j0; m0 += 32) {
          for (int e = tid; e < 64 * 32; e += NT) {
            const int ra = e % 64, mm = e / 64;
            const int ga = a0 + ra, gm = m0 + mm;
            As[ra * 33 + mm] = (ga < j0 && gm < j0) ? Tn[ga + (long long)gm * r] : T(0);
          }
          __syncthreads();
          for (int mm = 0; mm < 32; ++mm) {
            const T tv = As[aa * 33 + mm];
            const int m = m0 + mm;
            if (m >= j0) break;
#pragma unroll
            for (int t = 0; t < QT; ++t) acc[t] = fma(tv, Xs[(qb + (NT / 64) * t) + m * NBP], acc[t]);
          }
          __syncthreads();
        }
        const int a = a0 + aa;
        if (a < j0) {
#pragma unroll
          for (int t = 0; t < QT; ++t) {
            const int q = qb + (NT / 64) * t;
            if (q < nbw) Ys[a + q * r] = acc[t];
          }
        }
      }
      __syncthreads();
      for (int e = tid; e < j0 * nbw; e += NT) {   // T(0:j0, panel) = -Y T_p
        const int a = e % j0, q = e / j0;
        T v = T(0);
        for (int m = 0; m <= q; ++m) v += Ys[a + m * r] * Tp[m][q];
        Tn[a + (long long)(j0 + q) * r] = -v;
      }
    }
    for (int e = tid; e < nbw * nbw; e += NT) {
      const int a = e % nbw, q = e / nbw;
      Tn[(j0 + a) + (long long)(j0 + q) * r] = Tp[a][q];
    }
    // trailing columns k >= j0 + nbw: A_k -= Ṽ_p T_pᵀ (Ṽ_pᵀ A_k)
    const int k0 = j0 + nbw, nk = r - k0;
    if (nk > 0) {
      cta_vt_times<T, NBP>(Pt, W + (long long)k0 * b, b, nk, j0, b, As, Ws, 1, NBP);
      __syncthreads();
      // Ys(:, k) = T_pᵀ Ws(:, k)
      for (int e = tid; e < nk * NBP; e += NT) {
        const int c = e % NBP, k = e / NBP;
        T v = T(0);
        for (int a = 0; a <= c; ++a) v += Tp[a][c] * Ws[a + k * NBP];
        Ys[c + k * NBP] = v;
      }
      __syncthreads();
      // A(i, k) -= Σ_q v_q(i) Ys(q, k): thread owns a row and 8 columns per pass
      const int rows = b - j0;
      for (int c0 = 0; c0 < nk; c0 += 8 * (NT / 64)) {
        const int cb = c0 + (tid / 64) * 8;
        for (int ii = tid % 64; ii < rows; ii += 64) {
          const int i = j0 + ii;
          T acc[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) acc[u] = T(0);
#pragma unroll 4
          for (int q = 0; q < NBP; ++q) {
            const T v = Pt[q + i * (NBP + 1)];
#pragma unroll
            for (int u = 0; u < 8; ++u) acc[u] = fma(v, Ys[q + (cb + u) * NBP], acc[u]);
          }
#pragma unroll
          for (int u = 0; u < 8; ++u)
            if (cb + u < nk) W[i + (long long)(k0 + cb + u) * b] -= acc[u];
        }
      }
    }
    __syncthreads();
  }

  // One pass over row pairs (i, b-1-i) of the reversed working matrix: L_B(a, c)
  // = R(r-1-a, r-1-c) from its upper triangle, and V = F_b Ṽ with Ṽ's unit
  // diagonal and zeros above written in, each pair read and written by one thread.
  const int half = (b + 1) / 2;
  for (long long e = tid; e < (long long)half * r; e += NT) {
    const int i = (int)(e % half), j = (int)(e / half);
    const int i2 = b - 1 - i;
    const T w1 = W[i + (long long)j * b];
    const T w2 = W[i2 + (long long)j * b];
    if (i < r) Ln[(r - 1 - i) + (long long)(r - 1 - j) * r] = i <= j ? w1 : T(0);
    if (i2 != i && i2 < r) Ln[(r - 1 - i2) + (long long)(r - 1 - j) * r] = i2 <= j ? w2 : T(0);
    const T v1 = i > j ? w1 : (i == j ? T(1) : T(0));     // Ṽ(i, j)  -> V(b-1-i, j)
    const T v2 = i2 > j ? w2 : (i2 == j ? T(1) : T(0));   // Ṽ(i2, j) -> V(i, j)
    W[i + (long long)j * b] = v2;
    if (i2 != i) W[i2 + (long long)j * b] = v1;
  }
}

// ------------------------------------------------------------------ partial Cholesky
template <typename T>
__global__ void __launch_bounds__(NT)
pchol_kernel(T* Mb, int ldm, long long sM, int b, int c, T* PA, int ldpa, long long sPA,
             double* logdet_part, int level, int node0, int* status) {
  extern __shared__ unsigned char smem_raw[];
  T* P = reinterpret_cast<T*>(smem_raw);   // panel: b rows x NB, column-major ld = b
  __shared__ int fail;
  __shared__ double ld_acc;
  const int node = blockIdx.x;
  T* M = Mb + (long long)node * sM;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) {
    fail = 0;
    ld_acc = 0.0;
  }
  __syncthreads();

  for (int k0 = 0; k0 < c; k0 += NB) {
    const int kb = min(NB, c - k0);
    const int n1 = b - k0;
    // load panel M[k0:b, k0:k0+kb]
    for (int e = tid; e < n1 * kb; e += NT) {
      const int i = e % n1, jj = e / n1;
      P[i + jj * b] = M[(k0 + i) + (long long)(k0 + jj) * ldm];
    }
    __syncthreads();
    // diagonal block: one warp, lane i owns row i
    if (wid == 0) {
      double lsum = 0.0;
      for (int jj = 0; jj < kb; ++jj) {
        const T d = P[jj + jj * b];
        if (!(d > T(0))) {
          if (lane == 0) {
            fail = 1;
            report_failure(status, -3 /*NOT_SPD*/, level, node0 + node, k0 + jj);
          }
          break;
        }
        const T s = sqrt(d);
        lsum += log((double)s);
        __syncwarp();
        if (lane > jj && lane < kb) P[lane + jj * b] /= s;
        if (lane == jj) P[jj + jj * b] = s;
        __syncwarp();
        if (lane > jj && lane < kb) {
          const T lij = P[lane + jj * b];
          for (int t = jj + 1; t <= lane; ++t) P[lane + t * b] -= lij * P[t + jj * b];
        }
        __syncwarp();
      }
      if (lane == 0) ld_acc += lsum;
    }
    __syncthreads();
    if (fail) return;
    // panel TRSM: rows kb..n1-1 solve x L_diagᵀ = m, right-looking on a row held
    // in registers (critical path kb steps, independent updates within a step)
    for (int i = kb + tid; i < n1; i += NT) {
      T x[NB];
#pragma unroll
      for (int jj = 0; jj < NB; ++jj) x[jj] = jj < kb ? P[i + jj * b] : T(0);
#pragma unroll
      for (int jj = 0; jj < NB; ++jj) {
        if (jj < kb) {
          x[jj] = x[jj] / P[jj + jj * b];
#pragma unroll
          for (int t = jj + 1; t < NB; ++t)
            if (t < kb) x[t] = fma(-x[jj], P[t + jj * b], x[t]);
        }
      }
#pragma unroll
      for (int jj = 0; jj < NB; ++jj)
        if (jj < kb) P[i + jj * b] = x[jj];
    }
    __syncthreads();
    // write the panel back (lower part of the diagonal block and everything below)
    for (int e = tid; e < n1 * kb; e += NT) {
      const int i = e % n1, jj = e / n1;
      if (i >= jj) M[(k0 + i) + (long long)(k0 + jj) * ldm] = P[i + jj * b];
    }
    // trailing update of the lower triangle, rows/cols >= k0 + kb
    const int base = kb;   // panel row of the first trailing index
    const int n2 = n1 - kb;
    if (n2 > 0) {
      const int nt = (n2 + 63) / 64;
      const int tx = tid & 15, ty = tid >> 4;
      for (int tp = 0; tp < nt * (nt + 1) / 2; ++tp) {
        int t = tp, ti = 0;
        while (t > ti) { t -= ti + 1; ++ti; }
        const int tj = t;
        T acc[4][4];
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[p][q] = T(0);
        for (int kk = 0; kk < kb; ++kk) {
          T a[4], bb[4];
#pragma unroll
          for (int s = 0; s < 4; ++s) {
            const int ri = ti * 64 + tx + 16 * s;
            const int rj = tj * 64 + ty + 16 * s;
            a[s] = ri < n2 ? P[base + ri + kk * b] : T(0);
            bb[s] = rj < n2 ? P[base + rj + kk * b] : T(0);
          }
#pragma unroll
          for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[p][q] = fma(a[p], bb[q], acc[p][q]);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int rj = tj * 64 + ty + 16 * q;
          if (rj >= n2) continue;
#pragma unroll
          for (int p = 0; p < 4; ++p) {
            const int ri = ti * 64 + tx + 16 * p;
            if (ri >= n2 || ri < rj) continue;
            T* m = M + (k0 + kb + ri) + (long long)(k0 + kb + rj) * ldm;
            *m -= acc[p][q];
          }
        }
      }
    }
    __syncthreads();
  }
  if (tid == 0 && logdet_part) logdet_part[node0 + node] = 2.0 * ld_acc;
  // merge epilogue: Â^SS (r x r, lower) -> parent diagonal block at (off, off)
  if (PA) {
    const int r = b - c;
    const int p = node >> 1;
    const int off = (node & 1) * r;
    T* A = PA + (long long)p * sPA;
    for (int e = tid; e < r * r; e += NT) {
      const int i = e % r, j = e / r;
      if (i < j) continue;
      const T v = M[(c + i) + (long long)(c + j) * ldm];
      A[(off + i) + (long long)(off + j) * ldpa] = v;
      A[(off + j) + (long long)(off + i) * ldpa] = v;
    }
  }
}

// a[i] for a run-time i (a static-index select keeps the array in registers)
template <typename T>
HSS_DEVINL T reg_select(const T (&a)[NB], int i) {
  T v = T(0);
#pragma unroll
  for (int t = 0; t < NB; ++t)
    if (t == i) v = a[t];
  return v;
}

// ------------------------------------------------------------------ Cholesky panel
// One panel (kb <= NB columns) of a right-looking blocked Cholesky, one CTA per
// node (blockIdx.x) and row split (blockIdx.y); the trailing update is a
// separate level-wide SYRK.  Warp 0 factors the kb x kb diagonal block in
// registers (lane i holds row i, the pivot and the column entries travel by
// shuffles), then every thread solves rows of X L_11ᵀ = M_21 below it in
// registers against the block kept in shared memory.  With several row splits
// (a lone node, e.g. the root, whose row solves would otherwise queue on one
// SM's FP64 pipe) each CTA factors the diagonal block itself and solves its own
// share of the rows; split 0 alone writes the block, the log-det and a failure.
// The node's log-det slot gets (or, with accumulate, adds) 2 Σ log L_jj.
template <typename T>
__global__ void __launch_bounds__(NT)
chol_panel_kernel(T* Mb, int ldm, long long sM, int rows, int kb, double* logdet_part, int level,
                  int node0, int col0, int* status, int accumulate) {
  __shared__ T Ls[NB][NB + 1];   // Ls[t][j] = L(t, j) of the diagonal block
  __shared__ T dinv[NB];
  __shared__ int fail;
  const int node = blockIdx.x;
  const bool lead = blockIdx.y == 0;
  T* M = Mb + (long long)node * sM;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (wid == 0) {
    T a[NB];
#pragma unroll
    for (int t = 0; t < NB; ++t)
      a[t] = (lane < kb && t <= lane) ? M[lane + (long long)t * ldm] : T(0);
    int bad = -1;
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      if (j >= kb) break;
      const T d = __shfl_sync(0xffffffffu, a[j], j);   // updated A(j, j)
      if (bad < 0 && !(d > T(0))) bad = j;
      const T s = sqrt(d);
      const T inv = T(1) / s;
      if (lane == j) a[j] = s;
      if (lane > j) a[j] *= inv;
      // a[t] -= L(lane, j) L(t, j) for j < t <= lane; L(t, j) is lane t's a[j]
#pragma unroll
      for (int t = j + 1; t < NB; ++t) {
        const T ltj = __shfl_sync(0xffffffffu, a[j], t);
        if (t <= lane) a[t] = fma(-a[j], ltj, a[t]);
      }
    }
    if (lane == 0) fail = bad >= 0;
    if (bad >= 0) {
      if (lane == 0 && lead)
        report_failure(status, -3 /*NOT_SPD*/, level, node0 + node, col0 + bad);
    } else {
#pragma unroll
      for (int t = 0; t < NB; ++t)
        if (lane < kb && t <= lane) {
          if (lead) M[lane + (long long)t * ldm] = a[t];
          Ls[lane][t] = a[t];
        }
      const T dg = reg_select(a, lane);
      if (lane < kb) dinv[lane] = T(1) / dg;
      double ld = lane < kb ? log((double)dg) : 0.0;
      ld = warp_sum(ld);
      if (lane == 0 && logdet_part && lead) {
        if (accumulate)
          logdet_part[node] += 2.0 * ld;
        else
          logdet_part[node] = 2.0 * ld;
      }
    }
  }
  __syncthreads();
  if (fail) return;
  // this split's rows: [kb + per y, kb + per (y + 1))
  const int per = (rows - kb + gridDim.y - 1) / gridDim.y;
  const int i0 = kb + per * blockIdx.y, i1 = min(rows, i0 + per);
  for (int i = i0 + tid; i < i1; i += NT) {
    T x[NB];
#pragma unroll
    for (int t = 0; t < NB; ++t) x[t] = t < kb ? M[i + (long long)t * ldm] : T(0);
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      if (j >= kb) break;
      x[j] *= dinv[j];
#pragma unroll
      for (int t = j + 1; t < NB; ++t) x[t] = fma(-x[j], Ls[t][j], x[t]);
    }
#pragma unroll
    for (int t = 0; t < NB; ++t)
      if (t < kb) M[i + (long long)t * ldm] = x[t];
  }
}

// ------------------------------------------------------------------ triangular sweeps
// Both sweeps walk the factored columns in blocks of CB (<= NB): the block's
// panel (rows k0 .. b-1 of columns k0 .. k0+kb-1, the diagonal block and the
// L^RR / L^SR rows below it) is staged into shared memory with cp.async, the
// next block's copy in flight while the current one is used (NBUF = 2), so the
// global-memory latency stays out of the dependent chains.  Panel pitch P = b|1
// (odd) keeps both row-wise and column-wise lane access free of bank conflicts.
HSS_DEVINL uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
HSS_DEVINL void cp_async_elem(float* s, const float* g) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_addr(s)), "l"(g) : "memory");
}
HSS_DEVINL void cp_async_elem(double* s, const double* g) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_addr(s)), "l"(g) : "memory");
}
HSS_DEVINL void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
HSS_DEVINL void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// 8 consecutive values from 16-byte aligned shared memory, in 128-bit loads
HSS_DEVINL void load8(const float* p, float (&v)[8]) {
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const float4 f = reinterpret_cast<const float4*>(p)[q];
    v[4 * q] = f.x;
    v[4 * q + 1] = f.y;
    v[4 * q + 2] = f.z;
    v[4 * q + 3] = f.w;
  }
}
HSS_DEVINL void load8(const double* p, double (&v)[8]) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const double2 f = reinterpret_cast<const double2*>(p)[q];
    v[2 * q] = f.x;
    v[2 * q + 1] = f.y;
  }
}

// 16 consecutive values from 16-byte aligned shared memory, in 128-bit loads
HSS_DEVINL void load16(const float* p, float (&v)[16]) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float4 f = reinterpret_cast<const float4*>(p)[q];
    v[4 * q] = f.x;
    v[4 * q + 1] = f.y;
    v[4 * q + 2] = f.z;
    v[4 * q + 3] = f.w;
  }
}
HSS_DEVINL void load16(const double* p, double (&v)[16]) {
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const double2 f = reinterpret_cast<const double2*>(p)[q];
    v[2 * q] = f.x;
    v[2 * q + 1] = f.y;
  }
}

// rows [row0, row0+nrows) of columns [col0, col0+ncols) of src (leading
// dimension ld) into dst[(i - row0) + (c - col0) * P], one commit group
template <typename T>
HSS_DEVINL void stage_block(const T* src, int ld, int row0, int nrows, int col0, int ncols, T* dst,
                            int P) {
  const T* s0 = src + row0 + (long long)col0 * ld;
  for (int cc = 0; cc < ncols; ++cc)
    for (int ii = threadIdx.x; ii < nrows; ii += NT)
      cp_async_elem(dst + ii + cc * P, s0 + ii + (long long)cc * ld);
  cp_async_commit();
}

// rows k0 .. b-1 of columns k0 .. k0+kb-1 of M into Lp (pitch P)
template <typename T>
HSS_DEVINL void stage_panel(const T* M, int ldm, int k0, int kb, int b, T* Lp, int P) {
  stage_block(M, ldm, k0, b - k0, k0, kb, Lp, P);
}

// Padded pitch of the partial-sum scratch (conflict-free scalar stores)
constexpr int ZP = 17;

// y (b x nrhs in shared memory, ld b) := (I - V op(T) Vᵀ) y, op(T) = Tᵀ for the
// forward sweep (Qᵀ y) and T for the backward one (Q y).  V (b x r) and T
// (r x r) of the node stream through the panel buffers in CB-column slabs.  yr
// holds y row by row (pitch 16, zero past nrhs; filled here when fill is set),
// t1, t2 hold r x 16 row by row, zp NT x ZP partial sums.  The products read a
// row of 16 right-hand sides with 128-bit loads that every lane shares, so
// each FMA costs about a third of a shared load.  Called by every thread with
// y visible; returns with no copy in flight.  y = null: the vector lives only
// in yr (row by row), and the update goes there.
template <typename T>
HSS_DEVINL void q_apply(T* y, T* yr, bool fill, int b, int nrhs, const T* V, const T* Tm, int r,
                        bool transpose, T* Lbuf, int P, int CB, int NBUF, T* zp, T* t1, T* t2) {
  const int tid = threadIdx.x;
  const int ns = (r + CB - 1) / CB;
  auto buf = [&](int sl) { return Lbuf + (size_t)(NBUF == 2 ? (sl & 1) : 0) * P * CB; };
  if (fill) {
    for (int e = tid; e < b * 16; e += NT) {
      const int i = e / 16, j = e % 16;
      yr[e] = j < nrhs ? y[i + j * b] : T(0);
    }
  }
  __syncthreads();
  const int q = tid % CB, g = tid / CB, NG = NT / CB;   // slab column, row group
  T acc2[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) acc2[j] = T(0);
  // (0) t1 = Vᵀ y and (2) y -= V t2 stream V; (1) t2 = op(T) t1 streams T
  for (int phase = 0; phase < 3; ++phase) {
    const T* src = phase == 1 ? Tm : V;
    const int rows = phase == 1 ? r : b;
    stage_block(src, rows, 0, rows, 0, min(CB, r), buf(0), P);
    for (int sl = 0; sl < ns; ++sl) {
      const int q0 = sl * CB, qn = min(CB, r - q0);
      const bool next = sl + 1 < ns;
      if (NBUF == 2 && next) {
        stage_block(src, rows, 0, rows, q0 + CB, min(CB, r - q0 - CB), buf(sl + 1), P);
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      __syncthreads();
      const T* S = buf(sl);
      if (phase == 0 || (phase == 1 && transpose)) {
        // out row (q0 + q) = Σ_i S(i, q) in row i: row groups g, then summed
        const T* in = phase == 0 ? yr : t1;
        T* out = phase == 0 ? t1 : t2;
        T a[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) a[j] = T(0);
        if (q < qn) {
          for (int i = g; i < rows; i += NG) {
            const T sv = S[i + q * P];
            T v[16];
            load16(in + i * 16, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) a[j] = fma(sv, v[j], a[j]);
          }
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) zp[(g * CB + q) * ZP + j] = a[j];
        __syncthreads();
        for (int e = tid; e < qn * 16; e += NT) {
          const int qq = e / 16, j = e % 16;
          T sum = T(0);
          for (int gg = 0; gg < NG; ++gg) sum += zp[(gg * CB + qq) * ZP + j];
          out[(q0 + qq) * 16 + j] = sum;
        }
      } else if (phase == 1) {
        // t2 row (tid) += Σ_{p in slab} T(tid, p) t1 row p
        if (tid < r) {
          for (int pp = 0; pp < qn; ++pp) {
            const T tv = S[tid + pp * P];
            T v[16];
            load16(t1 + (q0 + pp) * 16, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) acc2[j] = fma(tv, v[j], acc2[j]);
          }
        }
      } else {
        // y(i, :) -= Σ_{q in slab} V(i, q) t2 row q
        for (int i = tid; i < b; i += NT) {
          T a[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) a[j] = T(0);
          for (int qq = 0; qq < qn; ++qq) {
            const T sv = S[i + qq * P];
            T v[16];
            load16(t2 + (q0 + qq) * 16, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) a[j] = fma(sv, v[j], a[j]);
          }
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (j < nrhs) {
              if (y)
                y[i + j * b] -= a[j];
              else
                yr[i * 16 + j] -= a[j];
            }
        }
      }
      __syncthreads();
      if (NBUF == 1 && next)
        stage_block(src, rows, 0, rows, q0 + CB, min(CB, r - q0 - CB), buf(sl + 1), P);
    }
    if (phase == 1 && !transpose && tid < r) {
#pragma unroll
      for (int j = 0; j < 16; ++j) t2[tid * 16 + j] = acc2[j];
    }
    __syncthreads();
  }
}

// The same Q application with all of V resident in shared memory (Vs, b x r,
// pitch Pv odd, staged by the caller; T read through L1): no slab staging and
// no barriers inside a phase.  Phase (0) t1 = Vᵀ y and (1) t2 = op(T) t1 give
// each thread one row of t1 / t2 and 8 of the 16 right-hand sides (two
// threads a row); phase (2) y -= V t2 gives each thread rows of y.  Called by
// every thread with yr (and y when fill) visible and the staging of Vs
// committed; returns with yr (or y) updated and visible.
constexpr int kVres = 4;   // flag in the NBUF argument: V resident in shared memory

template <typename T>
HSS_DEVINL void q_apply_res(T* y, T* yr, bool fill, int b, int nrhs, const T* Vs, int Pv,
                            const T* Tm, int r, bool transpose, T* t1, T* t2) {
  const int tid = threadIdx.x;
  if (fill) {
    for (int e = tid; e < b * 16; e += NT) {
      const int i = e / 16, j = e % 16;
      yr[e] = j < nrhs ? y[i + j * b] : T(0);
    }
  }
  cp_async_wait<0>();
  __syncthreads();
  const int j0 = (tid & 1) * 8;
  // (0) t1 row q = Σ_i V(i, q) yr row i
  for (int q = tid >> 1; q < r; q += NT / 2) {
    T a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = T(0);
    const T* vq = Vs + (size_t)q * Pv;
    for (int i = 0; i < b; ++i) {
      const T v = vq[i];
      T yv[8];
      load8(yr + i * 16 + j0, yv);
#pragma unroll
      for (int j = 0; j < 8; ++j) a[j] = fma(v, yv[j], a[j]);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) t1[q * 16 + j0 + j] = a[j];
  }
  __syncthreads();
  // (1) t2 row p = Σ_q op(T)(p, q) t1 row q; op(T) = Tᵀ (forward) reads
  // column p of T, T (backward) row p
  for (int p = tid >> 1; p < r; p += NT / 2) {
    T a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = T(0);
    for (int q = 0; q < r; ++q) {
      const T tv = transpose ? __ldg(Tm + q + (size_t)p * r) : __ldg(Tm + p + (size_t)q * r);
      T tq[8];
      load8(t1 + q * 16 + j0, tq);
#pragma unroll
      for (int j = 0; j < 8; ++j) a[j] = fma(tv, tq[j], a[j]);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) t2[p * 16 + j0 + j] = a[j];
  }
  __syncthreads();
  // (2) y row i -= Σ_q V(i, q) t2 row q
  for (int i = tid; i < b; i += NT) {
    T a[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) a[j] = T(0);
    for (int q = 0; q < r; ++q) {
      const T v = Vs[i + (size_t)q * Pv];
      T tv[16];
      load16(t2 + q * 16, tv);
#pragma unroll
      for (int j = 0; j < 16; ++j) a[j] = fma(v, tv[j], a[j]);
    }
#pragma unroll
    for (int j = 0; j < 16; ++j)
      if (j < nrhs) {
        if (y)
          y[i + j * b] -= a[j];
        else
          yr[i * 16 + j] -= a[j];
      }
  }
  __syncthreads();
}

// a load of a vector that another CTA of the same kernel may have written:
// through L2 (CG) so that no stale L1 line is read
template <bool CG, typename T>
HSS_DEVINL T ldv(const T* p) {
  if (CG) return __ldcg(p);
  return *p;
}

// forward: y (b x nrhs, smem) := [L^RR⁻¹ y^R ; y^S - L^SR L^RR⁻¹ y^R], for node
// `node` of the batch (one CTA)
template <typename T, bool CG>
HSS_DEVINL void fwd_node(int node, const T* __restrict__ Mb, int ldm, long long sM, int b, int c,
                         T* X, int ldx, long long sX, int nrhs, T* Par, int ldpar, long long sPar,
                         const T* Vb, long long sV, const T* Tb, long long sT, int r, int CB,
                         int NBUF) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(16) T zt[NB * 16];
  T* y = reinterpret_cast<T*>(smem_raw);   // b x nrhs, ld = b
  const int P = b | 1;
  const bool vres = (NBUF & kVres) && Vb;   // V resident in the panel region
  NBUF &= ~kVres;
  // Q application (Vb given): y row by row, partial sums, t1 and t2 (r x 16)
  const size_t qsz = Vb ? (size_t)b * 16 + (size_t)NT * ZP + (size_t)32 * r : 0;
  T* yr = y + (((size_t)b * nrhs + 15) & ~size_t(15));
  T* zpq = yr + (size_t)b * 16;
  T* t1 = zpq + (size_t)NT * ZP;
  T* t2 = t1 + (size_t)16 * r;
  T* Lbuf = yr + qsz;                      // NBUF panels of P x CB
  const T* M = Mb + (long long)node * sM;
  T* x = X + (long long)node * sX;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = NT / 32;
  const int nblk = (c + CB - 1) / CB;
  if (!Vb && nblk > 0) stage_panel(M, ldm, 0, min(CB, c), b, Lbuf, P);
  if (vres) stage_block(Vb + (long long)node * sV, b, 0, b, 0, r, Lbuf, P);
  for (int e = tid; e < b * nrhs; e += NT) {
    const int i = e % b, j = e / b;
    y[i + j * b] = ldv<CG>(x + i + (long long)j * ldx);
  }
  if (Vb) {   // y := Qᵀ y, then the first panel
    __syncthreads();
    if (vres)
      q_apply_res(y, yr, true, b, nrhs, Lbuf, P, Tb + (long long)node * sT, r, true, t1, t2);
    else
      q_apply(y, yr, true, b, nrhs, Vb + (long long)node * sV, Tb + (long long)node * sT, r, true,
              Lbuf, P, CB, NBUF, zpq, t1, t2);
    if (nblk > 0) stage_panel(M, ldm, 0, min(CB, c), b, Lbuf, P);
  }
  for (int bi = 0; bi < nblk; ++bi) {
    const int k0 = bi * CB;
    const int kb = min(CB, c - k0);
    const T* L = Lbuf + (size_t)(NBUF == 2 ? (bi & 1) : 0) * P * CB;
    const bool next = bi + 1 < nblk;
    if (NBUF == 2 && next) {
      stage_panel(M, ldm, k0 + CB, min(CB, c - k0 - CB), b, Lbuf + (size_t)((bi + 1) & 1) * P * CB,
                  P);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    // diagonal block: warp w handles right-hand sides w, w + nw, ...; lane i
    // keeps row i of the block in registers
    {
      T lrow[NB];
#pragma unroll
      for (int t = 0; t < NB; ++t) lrow[t] = (lane < kb && t <= lane) ? L[lane + t * P] : T(0);
      const T inv = lane < kb ? T(1) / reg_select(lrow, lane) : T(0);
      for (int j = wid; j < nrhs; j += nw) {
        T* yj = y + j * b + k0;
        T v = lane < kb ? yj[lane] : T(0);
#pragma unroll
        for (int t = 0; t < NB; ++t) {
          if (t >= kb) break;
          if (lane == t) v *= inv;
          const T zt = __shfl_sync(0xffffffffu, v, t);
          if (lane > t) v = fma(-lrow[t], zt, v);
        }
        if (lane < kb) yj[lane] = v;
      }
    }
    __syncthreads();
    // the solved block transposed (zt[t][j], zero past nrhs) for vector loads
    for (int e = tid; e < NB * 16; e += NT) {
      const int t = e / 16, j = e % 16;
      zt[e] = (t < kb && j < nrhs) ? y[(k0 + t) + j * b] : T(0);
    }
    __syncthreads();
    // every row below the block (the S rows included: L^SR lives there)
    for (int i = k0 + kb + tid; i < b; i += NT) {
      const int ii = i - k0;
      T acc[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) acc[j] = T(0);
#pragma unroll
      for (int t = 0; t < NB; ++t) {
        if (t < kb) {
          const T l = L[ii + t * P];
          T zv[16];
          load16(zt + t * 16, zv);
#pragma unroll
          for (int j = 0; j < 16; ++j) acc[j] = fma(l, zv[j], acc[j]);
        }
      }
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (j < nrhs) y[i + j * b] -= acc[j];
    }
    __syncthreads();
    if (NBUF == 1 && next) stage_panel(M, ldm, k0 + CB, min(CB, c - k0 - CB), b, Lbuf, P);
  }
  cp_async_wait<0>();
  for (int e = tid; e < b * nrhs; e += NT) {
    const int i = e % b, j = e / b;
    x[i + (long long)j * ldx] = y[i + j * b];
  }
  if (Par) {
    const int r = b - c;
    T* pv = Par + (long long)node * sPar;
    for (int e = tid; e < r * nrhs; e += NT) {
      const int i = e % r, j = e / r;
      pv[i + (long long)j * ldpar] = y[(c + i) + j * b];
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(NT)
trsv_fwd_kernel(const T* __restrict__ Mb, int ldm, long long sM, int b, int c, T* X, int ldx,
                long long sX, int nrhs, T* Par, int ldpar, long long sPar, const T* Vb,
                long long sV, const T* Tb, long long sT, int r, int CB, int NBUF) {
  fwd_node<T, false>(blockIdx.x, Mb, ldm, sM, b, c, X, ldx, sX, nrhs, Par, ldpar, sPar, Vb, sV,
                     Tb, sT, r, CB, NBUF);
}

// backward: x^S from the parent's vector (or in place when Par is null),
// x^R = L^RR⁻ᵀ (z^R - L^SRᵀ x^S); the node segment becomes [x^R; x^S]
template <typename T, bool CG>
HSS_DEVINL void bwd_node(int node, const T* __restrict__ Mb, int ldm, long long sM, int b, int c,
                         T* X, int ldx, long long sX, int nrhs, const T* Par, int ldpar,
                         long long sPar, const T* Vb, long long sV, const T* Tb, long long sT,
                         int r, int CB, int NBUF) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // the node vector row by row (pitch 16, zero past nrhs; 16-byte aligned for
  // vector loads): the only copy of it in shared memory
  T* xt = reinterpret_cast<T*>(smem_raw);
  T* zp = xt + (size_t)b * 16;             // NT x ZP partial sums
  T* t1 = zp + (size_t)NT * ZP;
  T* t2 = t1 + (size_t)16 * (Vb ? r : 0);
  T* Lbuf = t2 + (size_t)16 * (Vb ? r : 0);
  const int P = b | 1;
  const bool vres = (NBUF & kVres) && Vb;   // V resident in the panel region for Q
  NBUF &= ~kVres;
  const T* M = Mb + (long long)node * sM;
  T* x = X + (long long)node * sX;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = NT / 32;
  const int nblk = (c + CB - 1) / CB;
  if (nblk > 0) {
    const int k0 = (nblk - 1) * CB;
    stage_panel(M, ldm, k0, c - k0, b, Lbuf + (size_t)(NBUF == 2 ? ((nblk - 1) & 1) : 0) * P * CB,
                P);
  }
  // x^S (rows c .. b-1) from the parent's vector, z^R from this level's
  for (int e = tid; e < b * 16; e += NT) {
    const int i = e % b, j = e / b;
    T v = T(0);
    if (j < nrhs) {
      if (i >= c && Par)
        v = ldv<CG>(Par + (long long)node * sPar + (i - c) + (long long)j * ldpar);
      else
        v = ldv<CG>(x + i + (long long)j * ldx);
    }
    xt[i * 16 + j] = v;
  }
  for (int bi = nblk - 1; bi >= 0; --bi) {
    const int k0 = bi * CB;
    const int kb = min(CB, c - k0);
    const T* L = Lbuf + (size_t)(NBUF == 2 ? (bi & 1) : 0) * P * CB;
    const bool next = bi > 0;
    if (NBUF == 2 && next) {
      stage_panel(M, ldm, k0 - CB, CB, b, Lbuf + (size_t)((bi - 1) & 1) * P * CB, P);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    // z_t -= Σ_{i >= k0+kb} L(i, t) x_i: thread (t = lane, rows i ≡ warp mod nw)
    // accumulates every right-hand side, then the warps' partial sums are added
    {
      T acc[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) acc[j] = T(0);
      if (lane < kb) {
        for (int i = k0 + kb + wid; i < b; i += nw) {
          const T l = L[(i - k0) + lane * P];
          T xv[16];
          load16(xt + i * 16, xv);
#pragma unroll
          for (int j = 0; j < 16; ++j) acc[j] = fma(l, xv[j], acc[j]);
        }
      }
#pragma unroll
      for (int j = 0; j < 16; ++j) zp[(wid * NB + lane) * ZP + j] = acc[j];
    }
    __syncthreads();
    for (int e = tid; e < kb * 16; e += NT) {
      const int t = e / 16, j = e % 16;
      if (j < nrhs) {
        T sum = T(0);
#pragma unroll
        for (int w = 0; w < NT / 32; ++w) sum += zp[(w * NB + t) * ZP + j];
        xt[(k0 + t) * 16 + j] -= sum;
      }
    }
    __syncthreads();
    // diagonal block, transposed back substitution; lane i keeps column i of
    // the block (L(t, i), t >= i) in registers
    {
      T lcol[NB];
#pragma unroll
      for (int t = 0; t < NB; ++t)
        lcol[t] = (lane < kb && t >= lane && t < kb) ? L[t + lane * P] : T(0);
      const T inv = lane < kb ? T(1) / reg_select(lcol, lane) : T(0);
      for (int j = wid; j < nrhs; j += nw) {
        T v = lane < kb ? xt[(k0 + lane) * 16 + j] : T(0);
#pragma unroll
        for (int tt = NB - 1; tt >= 0; --tt) {
          if (tt >= kb) continue;
          if (lane == tt) v *= inv;
          const T xs = __shfl_sync(0xffffffffu, v, tt);
          if (lane < tt) v = fma(-lcol[tt], xs, v);
        }
        if (lane < kb) xt[(k0 + lane) * 16 + j] = v;
      }
    }
    __syncthreads();
    if (NBUF == 1 && next) stage_panel(M, ldm, k0 - CB, CB, b, Lbuf, P);
  }
  cp_async_wait<0>();
  if (Vb) {   // x := Q x, on the row-major vector
    __syncthreads();
    if (vres) {
      stage_block(Vb + (long long)node * sV, b, 0, b, 0, r, Lbuf, P);
      q_apply_res<T>(nullptr, xt, false, b, nrhs, Lbuf, P, Tb + (long long)node * sT, r, false,
                     t1, t2);
    } else {
      q_apply<T>(nullptr, xt, false, b, nrhs, Vb + (long long)node * sV,
                 Tb + (long long)node * sT, r, false, Lbuf, P, CB, NBUF, zp, t1, t2);
    }
  }
  __syncthreads();
  for (int e = tid; e < b * nrhs; e += NT) {
    const int i = e % b, j = e / b;
    x[i + (long long)j * ldx] = xt[i * 16 + j];
  }
}

template <typename T>
__global__ void __launch_bounds__(NT)
trsv_bwd_kernel(const T* __restrict__ Mb, int ldm, long long sM, int b, int c, T* X, int ldx,
                long long sX, int nrhs, const T* Par, int ldpar, long long sPar, const T* Vb,
                long long sV, const T* Tb, long long sT, int r, int CB, int NBUF) {
  bwd_node<T, false>(blockIdx.x, Mb, ldm, sM, b, c, X, ldx, sX, nrhs, Par, ldpar, sPar, Vb, sV,
                     Tb, sT, r, CB, NBUF);
}

// ------------------------------------------------------------------ upper tree in one launch
// Levels lo .. 1 of the solve (block order b = 2r at every level) in one
// launch each way, without a barrier between levels: a node's step starts as
// soon as the nodes it depends on are done (the asynchronous execution of the
// tree of Sec. 4.2, within one GPU).
//
// Forward (leaves towards the root): CTA k starts with node k of level lo.
// After a node, the CTA counts itself in at the parent; the CTA that arrives
// second runs the parent (its sibling's results are already in memory), the
// first one retires.  Nothing waits.
template <typename T>
__global__ void __launch_bounds__(NT)
tree_fwd_kernel(TreeLevels<T> lv, int lo, int b, int c, int r, int nrhs, int* __restrict__ cnt,
                int CB, int NBUF) {
  __shared__ int go;
  int l = lo, i = blockIdx.x;
  for (;;) {
    const int n = 1 << l;
    fwd_node<T, true>(i, lv.M[l], b, (long long)b * b, b, c, lv.vec[l], n * b, b, nrhs,
                      lv.vec[l - 1], (n / 2) * b, r, lv.V[l], (long long)b * r, lv.Tm[l],
                      (long long)r * r, r, CB, NBUF);
    if (l == 1) break;
    __threadfence();   // this node's results before the arrival count
    __syncthreads();
    if (threadIdx.x == 0) {
      go = atomicAdd(cnt + (1 << (l - 1)) - 1 + (i >> 1), 1) == 1;
      __threadfence();
    }
    __syncthreads();
    if (!go) break;
    --l;
    i >>= 1;
  }
}

HSS_DEVINL int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
HSS_DEVINL void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Backward (root towards the leaves), a cooperative launch of 2^lo CTAs: CTA k
// runs node k >> (lo - l) of every level l whose node it is the leftmost
// descendant of, waiting for the parent's ready flag (= epoch of this call).
// The wait polls at most wait_limit times; on expiry the CTA records
// HSS_ERR_TIMEOUT (with the level and node) in status and returns, and the
// CTAs below it then give up the same way.
template <typename T>
__global__ void __launch_bounds__(NT)
tree_bwd_kernel(TreeLevels<T> lv, int lo, int b, int c, int r, int nrhs, int* __restrict__ ready,
                int epoch, long long wait_limit, int* status, int CB, int NBUF) {
  __shared__ int ok;
  const int k = blockIdx.x;
  for (int l = 1; l <= lo; ++l) {
    const int shift = lo - l;
    if (k & ((1 << shift) - 1)) continue;   // another CTA runs this level's node
    const int i = k >> shift;
    if (l > 1) {
      if (threadIdx.x == 0) {
        const int* f = ready + (1 << (l - 1)) - 1 + (i >> 1);
        int got = 0;
        for (long long it = 0; it < wait_limit; ++it) {
          if (ld_acquire(f) == epoch) {
            got = 1;
            break;
          }
          __nanosleep(64);
        }
        ok = got;
      }
      __syncthreads();
      if (!ok) {
        if (threadIdx.x == 0) report_failure(status, -6 /*TIMEOUT*/, l, i, -1);
        return;
      }
    }
    const int n = 1 << l;
    bwd_node<T, true>(i, lv.M[l], b, (long long)b * b, b, c, lv.vec[l], n * b, b, nrhs,
                      lv.vec[l - 1], (n / 2) * b, r, lv.V[l], (long long)b * r, lv.Tm[l],
                      (long long)r * r, r, CB, NBUF);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) st_release(ready + (1 << l) - 1 + i, epoch);
  }
}

__global__ void logdet_reduce_kernel(const double* part, int n, double* out) {
  // fixed-order pairwise sum in one CTA: deterministic for a given n
  __shared__ double s[1024];
  const int tid = threadIdx.x;
  double acc = 0.0;
  for (int i = tid; i < n; i += blockDim.x) acc += part[i];
  s[tid] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (tid < w) s[tid] += s[tid + w];
    __syncthreads();
  }
  if (tid == 0) *out = s[0];
}

}  // namespace

// ------------------------------------------------------------------ launchers
// opt a kernel into `bytes` of dynamic shared memory (plus its static part);
// false if the device cannot give that much
// (the 48 KB default holds static + dynamic shared memory together)
// The answers are remembered per (device, kernel, bytes): the queries and the
// attribute change cost microseconds of host time, and the sweeps ask before
// every launch.
template <typename K>
bool smem_opt_in(K kernel, size_t bytes) {
  static std::mutex mu;
  static std::map<std::tuple<int, const void*, size_t>, bool> memo;
  int dev = 0;
  cudaGetDevice(&dev);
  const auto key = std::make_tuple(dev, reinterpret_cast<const void*>(kernel), bytes);
  {
    std::lock_guard<std::mutex> g(mu);
    const auto it = memo.find(key);
    if (it != memo.end()) return it->second;
  }
  bool ok = false;
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, kernel) == cudaSuccess) {
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (bytes + fa.sharedSizeBytes <= 48 * 1024)
      ok = true;
    else if (bytes + fa.sharedSizeBytes <= (size_t)optin)
      ok = (size_t)fa.maxDynamicSharedSizeBytes >= bytes ||
           cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)bytes) == cudaSuccess;
  } else {
    cudaGetLastError();
    return false;
  }
  std::lock_guard<std::mutex> g(mu);
  memo[key] = ok;
  return ok;
}

template <typename T>
size_t ql_smem(int b, int r, int NBP) {
  // transposed panel, then the product buffers (which also hold the warps'
  // partial panel Gram matrices)
  const size_t region = std::max<size_t>((size_t)3 * NBP * r + 64 * 33,
                                         (size_t)(NT / 32) * NBP * (NBP + 1));
  return ((size_t)b * (NBP + 1) + region) * sizeof(T);
}

template <typename T, int NBP, int RPT>
cudaError_t launch_ql_rows(const T* Bsrc, int ldb_src, long long sB, T* V, long long sV, T* Tm,
                           long long sT, T* LB, long long sL, int b, int r, int nodes,
                           cudaStream_t st, const int* only_if) {
  const size_t sm = ql_smem<T>(b, r, NBP);
  if (!smem_opt_in(ql_basis_kernel<T, NBP, RPT>, sm)) return cudaErrorInvalidConfiguration;
  ql_basis_kernel<T, NBP, RPT><<<nodes, NT, sm, st>>>(Bsrc, ldb_src, sB, V, sV, Tm, sT, LB, sL,
                                                      b, r, only_if);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_ql_basis(const T* Bsrc, int ldb_src, long long sB, T* V, long long sV, T* Tm,
                            long long sT, T* LB, long long sL, int b, int r, int nodes,
                            cudaStream_t st, const int* only_if, int panel) {
  // panel width: 16 columns in FP64; 32 (default) or 16 in FP32.  RPT panel
  // rows per thread (b <= RPT NT); four rows a thread hold a 16-column panel
  // only, so the register panel stays within the register file.
  if (b > 4 * NT || r > 256) return cudaErrorInvalidValue;
#define QL_RUN(NBP_)                                                                            \
  do {                                                                                          \
    if (b <= NT)                                                                                \
      return launch_ql_rows<T, NBP_, 1>(Bsrc, ldb_src, sB, V, sV, Tm, sT, LB, sL, b, r, nodes,  \
                                        st, only_if);                                           \
    if (b <= 2 * NT)                                                                            \
      return launch_ql_rows<T, NBP_, 2>(Bsrc, ldb_src, sB, V, sV, Tm, sT, LB, sL, b, r, nodes,  \
                                        st, only_if);                                           \
    if (b <= 3 * NT || NBP_ > 16)                                                               \
      return launch_ql_rows<T, NBP_, 3>(Bsrc, ldb_src, sB, V, sV, Tm, sT, LB, sL, b, r, nodes,  \
                                        st, only_if);                                           \
    return launch_ql_rows<T, 16, 4>(Bsrc, ldb_src, sB, V, sV, Tm, sT, LB, sL, b, r, nodes, st,  \
                                    only_if);                                                   \
  } while (0)
  if constexpr (sizeof(T) == 4) {
    if (panel != 16 && b <= 3 * NT) QL_RUN(32);
  }
  QL_RUN(16);
#undef QL_RUN
}

template <typename T>
size_t pchol_smem(int b) { return (size_t)b * NB * sizeof(T); }

template <typename T>
cudaError_t launch_pchol(T* M, int ldm, long long sM, int b, int c, T* PA, int ldpa, long long sPA,
                         double* logdet_part, int level, int node0, int* status, int nodes,
                         cudaStream_t st) {
  const size_t sm = pchol_smem<T>(b);
  if (!smem_opt_in(pchol_kernel<T>, sm)) return cudaErrorInvalidConfiguration;
  pchol_kernel<T><<<nodes, NT, sm, st>>>(M, ldm, sM, b, c, PA, ldpa, sPA, logdet_part, level,
                                         node0, status);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_chol_panel(T* M, int ldm, long long sM, int rows, int kb, double* logdet_part,
                              int level, int node0, int col0, int* status, int nodes,
                              bool accumulate, cudaStream_t st, int splits) {
  if (kb < 1 || kb > NB || rows < kb || splits < 1 || splits > 65535)
    return cudaErrorInvalidValue;
  chol_panel_kernel<T><<<dim3(nodes, splits), NT, 0, st>>>(M, ldm, sM, rows, kb, logdet_part,
                                                           level, node0, col0, status,
                                                           accumulate ? 1 : 0);
  return cudaGetLastError();
}

// Â^SS of every node (lower triangle at M[c:, c:]) into its parent's diagonal
// block at (off, off), both triangles (the merge step of Alg. 2)
template <typename T>
__global__ void scatter_ss_kernel(const T* __restrict__ Mb, int ldm, long long sM, int c, int r,
                                  T* PA, int ldpa, long long sPA) {
  const int node = blockIdx.x;
  const T* M = Mb + (long long)node * sM;
  T* A = PA + (long long)(node >> 1) * sPA;
  const int off = (node & 1) * r;
  // CTA y takes columns y, y + gridDim.y, ...
  const int ncol = (r - (int)blockIdx.y + (int)gridDim.y - 1) / (int)gridDim.y;
  for (int e = threadIdx.x; e < r * ncol; e += blockDim.x) {
    const int i = e % r, j = (int)blockIdx.y + (e / r) * (int)gridDim.y;
    if (i < j) continue;
    const T v = M[(c + i) + (long long)(c + j) * ldm];
    A[(off + i) + (long long)(off + j) * ldpa] = v;
    A[(off + j) + (long long)(off + i) * ldpa] = v;
  }
}

template <typename T>
cudaError_t launch_scatter_ss(const T* M, int ldm, long long sM, int c, int r, T* PA, int ldpa,
                              long long sPA, int nodes, cudaStream_t st) {
  if (r <= 0 || nodes <= 0) return cudaSuccess;
  scatter_ss_kernel<T><<<dim3(nodes, std::min(r, 16)), NT, 0, st>>>(M, ldm, sM, c, r, PA, ldpa,
                                                                    sPA);
  return cudaGetLastError();
}

// shared memory of a sweep: the node vector, the Q application's two r x 16
// buffers, and NBUF staged panels of P x CB
template <typename T>
size_t trsv_smem(int b, int nrhs, int r, int CB, int NBUF, bool bwd, bool vres = false) {
  // forward: the column-major vector (padded to 16 elements), plus its row-major
  // copy and the partial sums when Q is applied; backward: the row-major vector
  // and the partial sums only.  The panel region also holds all of V (pitch
  // b | 1) when V is resident.
  const size_t vec = bwd ? 0 : ((size_t)b * nrhs + 15) & ~size_t(15);
  const size_t rowmajor = (bwd || r > 0) ? (size_t)b * 16 + (size_t)NT * ZP : 0;
  size_t region = (size_t)NBUF * (b | 1) * CB;
  if (vres) region = std::max(region, (size_t)r * (b | 1));
  return (vec + rowmajor + (size_t)32 * r + region) * sizeof(T);
}

// Panel staging of a sweep launch of `nodes` CTAs.  staging = 0: the largest
// the device allows (two 32-column panels, else one, else 16- and 8-column
// panels).  staging = 1: the fewest waves of CTAs over the SMs (smaller panels
// let more CTAs share an SM), ties to the larger staging.
template <typename T, typename K>
cudaError_t trsv_config_uncached(K kernel, int b, int nrhs, int r, bool bwd, int* CB, int* NBUF,
                                 size_t* sm, int nodes, int staging);

// the choice, remembered per (device, kernel, shape, nodes, staging): it queries
// the occupancy calculator, which costs microseconds of host time per launch
template <typename T, typename K>
cudaError_t trsv_config(K kernel, int b, int nrhs, int r, bool bwd, int* CB, int* NBUF,
                        size_t* sm, int nodes = 1, int staging = 0) {
  struct Choice { cudaError_t e; int cb, nbuf; size_t sm; };
  static std::mutex mu;
  static std::map<std::tuple<int, const void*, int, int, int, int, int, int>, Choice> memo;
  int dev = 0;
  cudaGetDevice(&dev);
  const auto key = std::make_tuple(dev, reinterpret_cast<const void*>(kernel), b, nrhs, r,
                                   (int)bwd, staging == 1 ? nodes : 0, staging);
  {
    std::lock_guard<std::mutex> g(mu);
    const auto it = memo.find(key);
    if (it != memo.end()) {
      *CB = it->second.cb;
      *NBUF = it->second.nbuf;
      *sm = it->second.sm;
      return it->second.e;
    }
  }
  Choice c{cudaSuccess, 0, 0, 0};
  c.e = trsv_config_uncached<T>(kernel, b, nrhs, r, bwd, &c.cb, &c.nbuf, &c.sm, nodes, staging);
  std::lock_guard<std::mutex> g(mu);
  memo[key] = c;
  *CB = c.cb;
  *NBUF = c.nbuf;
  *sm = c.sm;
  return c.e;
}

template <typename T, typename K>
cudaError_t trsv_config_uncached(K kernel, int b, int nrhs, int r, bool bwd, int* CB, int* NBUF,
                                 size_t* sm, int nodes, int staging) {
  const int cbs[5] = {32, 32, 16, 16, 8}, bufs[5] = {2, 1, 2, 1, 1};
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || !sms)
      sms = 1;
  }
  long long best_waves = -1;
  // with Q fused (r > 0): first the layouts that keep all of V resident
  for (int q = 0; r > 0 && q < 5; ++q) {
    const size_t s = trsv_smem<T>(b, nrhs, r, cbs[q], bufs[q], bwd, true);
    if (!smem_opt_in(kernel, s)) continue;
    long long waves = 0;
    if (staging == 1) {
      int occ = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, NT, s) != cudaSuccess ||
          occ < 1)
        occ = 1;
      waves = (nodes + (long long)sms * occ - 1) / ((long long)sms * occ);
    }
    if (best_waves < 0 || waves < best_waves) {
      best_waves = waves;
      *CB = cbs[q];
      *NBUF = bufs[q] | kVres;
      *sm = s;
    }
    if (staging == 0) break;
  }
  if (best_waves >= 0) return cudaSuccess;
  for (int q = 0; q < 5; ++q) {
    const size_t s = trsv_smem<T>(b, nrhs, r, cbs[q], bufs[q], bwd);
    if (!smem_opt_in(kernel, s)) continue;
    long long waves = 0;
    if (staging == 1) {
      int occ = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, NT, s) != cudaSuccess ||
          occ < 1)
        occ = 1;
      waves = (nodes + (long long)sms * occ - 1) / ((long long)sms * occ);
    }
    if (best_waves < 0 || waves < best_waves) {
      best_waves = waves;
      *CB = cbs[q];
      *NBUF = bufs[q];
      *sm = s;
    }
    if (staging == 0) break;
  }
  return best_waves < 0 ? cudaErrorInvalidConfiguration : cudaSuccess;
}

template <typename T>
bool ulv_fused_fits(int b, int nrhs, int r, bool bwd) {
  int CB, NBUF;
  size_t sm;
  return bwd ? trsv_config<T>(trsv_bwd_kernel<T>, b, nrhs, r, true, &CB, &NBUF, &sm) ==
                   cudaSuccess
             : trsv_config<T>(trsv_fwd_kernel<T>, b, nrhs, r, false, &CB, &NBUF, &sm) ==
                   cudaSuccess;
}

template <typename T>
bool tree_fits(int b, int nrhs, int r) {
  int CB, NBUF;
  size_t sm;
  return trsv_config<T>(tree_fwd_kernel<T>, b, nrhs, r, false, &CB, &NBUF, &sm) == cudaSuccess &&
         trsv_config<T>(tree_bwd_kernel<T>, b, nrhs, r, true, &CB, &NBUF, &sm) == cudaSuccess;
}

template <typename T>
cudaError_t launch_ulv_fwd(const T* M, int ldm, long long sM, int b, int c, T* X, int ldx,
                           long long sX, int nrhs, T* Par, int ldpar, long long sPar, const T* V,
                           long long sV, const T* Tm, long long sT, int r, int nodes,
                           cudaStream_t st, int staging) {
  if (nrhs > 16 || (V && (r < 1 || r > NT || r > b))) return cudaErrorInvalidValue;
  int CB, NBUF;
  size_t sm;
  cudaError_t e = trsv_config<T>(trsv_fwd_kernel<T>, b, nrhs, V ? r : 0, false, &CB, &NBUF,
                                 &sm, nodes, staging);
  if (e != cudaSuccess) return e;
  trsv_fwd_kernel<T><<<nodes, NT, sm, st>>>(M, ldm, sM, b, c, X, ldx, sX, nrhs, Par, ldpar, sPar, V,
                                            sV, Tm, sT, V ? r : 0, CB, NBUF);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_ulv_bwd(const T* M, int ldm, long long sM, int b, int c, T* X, int ldx,
                           long long sX, int nrhs, const T* Par, int ldpar, long long sPar,
                           const T* V, long long sV, const T* Tm, long long sT, int r, int nodes,
                           cudaStream_t st, int staging) {
  if (nrhs > 16 || (V && (r < 1 || r > NT || r > b))) return cudaErrorInvalidValue;
  int CB, NBUF;
  size_t sm;
  cudaError_t e = trsv_config<T>(trsv_bwd_kernel<T>, b, nrhs, V ? r : 0, true, &CB, &NBUF,
                                 &sm, nodes, staging);
  if (e != cudaSuccess) return e;
  trsv_bwd_kernel<T><<<nodes, NT, sm, st>>>(M, ldm, sM, b, c, X, ldx, sX, nrhs, Par, ldpar, sPar, V,
                                            sV, Tm, sT, V ? r : 0, CB, NBUF);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_tree_fwd(const TreeLevels<T>& lv, int lo, int b, int c, int r, int nrhs,
                            int* cnt, cudaStream_t st) {
  if (lo < 1 || lo > 20 || nrhs > 16 || r < 1 || r > NT || r > b) return cudaErrorInvalidValue;
  int CB, NBUF;
  size_t sm;
  cudaError_t e = trsv_config<T>(tree_fwd_kernel<T>, b, nrhs, r, false, &CB, &NBUF, &sm);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(cnt, 0, sizeof(int) << lo, st);
  if (e != cudaSuccess) return e;
  tree_fwd_kernel<T><<<1 << lo, NT, sm, st>>>(lv, lo, b, c, r, nrhs, cnt, CB, NBUF);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_tree_bwd(const TreeLevels<T>& lv, int lo, int b, int c, int r, int nrhs,
                            int* ready, int epoch, long long wait_limit, int* status,
                            cudaStream_t st) {
  if (lo < 1 || lo > 20 || nrhs > 16 || r < 1 || r > NT || r > b) return cudaErrorInvalidValue;
  int CB, NBUF;
  size_t sm;
  cudaError_t e = trsv_config<T>(tree_bwd_kernel<T>, b, nrhs, r, true, &CB, &NBUF, &sm);
  if (e != cudaSuccess) return e;
  // the CTAs wait on one another: a cooperative launch, which the runtime
  // refuses unless all of them can be resident at once
  TreeLevels<T> lvc = lv;
  void* args[] = {&lvc, &lo, &b, &c, &r, &nrhs, &ready, &epoch, &wait_limit, &status, &CB, &NBUF};
  return cudaLaunchCooperativeKernel((const void*)tree_bwd_kernel<T>, dim3(1u << lo), dim3(NT),
                                     args, sm, st);
}

template <typename T>
cudaError_t launch_trsv_fwd(const T* M, int ldm, long long sM, int b, int c, T* X, int ldx,
                            long long sX, int nrhs, T* Par, int ldpar, long long sPar, int nodes,
                            cudaStream_t st) {
  return launch_ulv_fwd<T>(M, ldm, sM, b, c, X, ldx, sX, nrhs, Par, ldpar, sPar, nullptr, 0,
                           nullptr, 0, 0, nodes, st, 0);
}

template <typename T>
cudaError_t launch_trsv_bwd(const T* M, int ldm, long long sM, int b, int c, T* X, int ldx,
                            long long sX, int nrhs, const T* Par, int ldpar, long long sPar,
                            int nodes, cudaStream_t st) {
  return launch_ulv_bwd<T>(M, ldm, sM, b, c, X, ldx, sX, nrhs, Par, ldpar, sPar, nullptr, 0,
                           nullptr, 0, 0, nodes, st, 0);
}

void launch_logdet_reduce(const double* part, int n, double* out, cudaStream_t st) {
  logdet_reduce_kernel<<<1, 1024, 0, st>>>(part, n, out);
}

#define INST(T)                                                                                  \
  template cudaError_t launch_ql_basis<T>(const T*, int, long long, T*, long long, T*, long long,  \
                                          T*, long long, int, int, int, cudaStream_t,             \
                                          const int*, int);                                        \
  template cudaError_t launch_pchol<T>(T*, int, long long, int, int, T*, int, long long, double*, \
                                       int, int, int*, int, cudaStream_t);                        \
  template cudaError_t launch_trsv_fwd<T>(const T*, int, long long, int, int, T*, int, long long, \
                                          int, T*, int, long long, int, cudaStream_t);            \
  template cudaError_t launch_trsv_bwd<T>(const T*, int, long long, int, int, T*, int, long long, \
                                          int, const T*, int, long long, int, cudaStream_t);      \
  template cudaError_t launch_ulv_fwd<T>(const T*, int, long long, int, int, T*, int, long long,  \
                                         int, T*, int, long long, const T*, long long, const T*,  \
                                         long long, int, int, cudaStream_t, int);                 \
  template cudaError_t launch_ulv_bwd<T>(const T*, int, long long, int, int, T*, int, long long,  \
                                         int, const T*, int, long long, const T*, long long,      \
                                         const T*, long long, int, int, cudaStream_t, int);       \
  template size_t ql_smem<T>(int, int, int);                                                     \
  template cudaError_t launch_chol_panel<T>(T*, int, long long, int, int, double*, int, int, int,\
                                            int*, int, bool, cudaStream_t, int);                  \
  template cudaError_t launch_scatter_ss<T>(const T*, int, long long, int, int, T*, int,           \
                                            long long, int, cudaStream_t);                       \
  template cudaError_t launch_tree_fwd<T>(const TreeLevels<T>&, int, int, int, int, int, int*,    \
                                          cudaStream_t);                                         \
  template cudaError_t launch_tree_bwd<T>(const TreeLevels<T>&, int, int, int, int, int, int*,    \
                                          int, long long, int*, cudaStream_t);                   \
  template bool ulv_fused_fits<T>(int, int, int, bool);                                          \
  template bool tree_fits<T>(int, int, int);
INST(double)
INST(float)
