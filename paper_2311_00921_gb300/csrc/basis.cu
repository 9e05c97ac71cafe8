// Basis completion (Eq. 2-3, Sec. 2) without a serial Householder chain.
//
// The completion is the Householder QL factorization B = Q [0; L_B] of the
// node basis (b x r), computed as the Householder QR of the reversed basis
// Ã = F_b B F_r with LAPACK dlarfg signs: Q = F_b Q̃ F_b, L_B = F_r R̃ F_r.  The
// per-column reflector chain of a Householder kernel is a CTA-wide reduction
// per column; here the same factors are obtained from level-wide products:
//
//  1. Cholesky QR twice: G1 = ÃᵀÃ = R1ᵀR1, X = Ã R1⁻¹; G2 = XᵀX = R2ᵀR2, so
//     Q1 = X R2⁻¹ is orthonormal to working precision and Ã = Q1 R with
//     R = R2 R1 (Yamamoto, Nakatsukasa, Yanagisawa, Fukaya, "Roundoff error
//     analysis of the CholeskyQR2 algorithm", 2015).
//  2. Householder reconstruction (Ballard, Demmel, Grigori, Jacquelin, Knight,
//     Nguyen, "Reconstructing Householder vectors from tall-skinny QR", 2015):
//     with S = diag(±1) chosen column by column as -sign of the running
//     diagonal, the LU factorization without pivoting Q1 - [S; 0] = Y Ũ gives
//     the Householder vectors Y (unit lower trapezoidal), the compact-WY
//     factor T = -Ũ S Y1⁻ᵀ (Y1 the top r x r block of Y) and the triangular
//     factor S R of the Householder QR.  This sign choice is dlarfg's
//     β = -sign(α)‖x‖, so V = F_b Y, T and L_B = F_r (S R) F_r equal those of the
//     Householder kernel up to rounding.  Only the top r x r block is factored
//     (one CTA per node); the bottom block of Y is Q1_bottom Ũ⁻¹, a product.
//
// The level-wide products run in basis_gemm_kernel (many CTAs per node); the
// r x r Cholesky, LU and triangular inverses run one CTA per node in shared
// memory.  A node whose Gram Cholesky meets a non-positive pivot (a basis too
// ill-conditioned for Cholesky QR in this precision) is flagged and completed
// by the Householder kernel afterwards.
#include <math.h>

#include <algorithm>

#include "basis.cuh"
#include "common.cuh"
#include "ulv_kernels.cuh"

namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

// C (m x n) = alpha op(A) B for every node (blockIdx.y) of a batch.
//   TA    : op(A) = Aᵀ with A stored k x m (column-major), else A is m x k
//   BUP   : B (k x n) is upper triangular; the k loop of a tile stops at its
//           last column
//   LOWER : m = n and only tiles on or below the diagonal are computed
//           (blockIdx.x enumerates the pairs); the upper triangle of the
//           diagonal tiles is written too
//   REV   : row i of the product is stored in row m - 1 - i of C
template <typename T, bool TA, bool BUP, bool LOWER, bool REV>
__global__ void __launch_bounds__(NT)
basis_gemm_kernel(int m, int n, int k, T alpha, const T* __restrict__ A, int lda, long long sA,
                  const T* __restrict__ B, int ldb, long long sB, T* __restrict__ C, int ldc,
                  long long sC, int tiles_m) {
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const long long bz = blockIdx.y;
  A += bz * sA;
  B += bz * sB;
  C += bz * sC;
  int ti, tj;
  if (LOWER) {
    int t = blockIdx.x, i = 0;
    while (t > i) {
      t -= i + 1;
      ++i;
    }
    ti = i;
    tj = t;
  } else {
    ti = blockIdx.x % tiles_m;
    tj = blockIdx.x / tiles_m;
  }
  const int i0 = ti * BM, j0 = tj * BN;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int kend = BUP ? min(k, j0 + BN) : k;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[a][c] = T(0);

  for (int k0 = 0; k0 < kend; k0 += BK) {
#pragma unroll
    for (int e0 = 0; e0 < BM * BK; e0 += NT) {
      const int e = e0 + threadIdx.x;
      int i, kk;
      if (!TA) {
        i = e % BM;
        kk = e / BM;
      } else {
        kk = e % BK;
        i = e / BK;
      }
      const int gi = i0 + i, gk = k0 + kk;
      T v = T(0);
      if (gi < m && gk < kend) v = TA ? A[gk + (long long)gi * lda] : A[gi + (long long)gk * lda];
      As[kk][i] = v;
    }
#pragma unroll
    for (int e0 = 0; e0 < BN * BK; e0 += NT) {
      const int e = e0 + threadIdx.x;
      const int kk = e % BK, j = e / BK;
      const int gj = j0 + j, gk = k0 + kk;
      T v = T(0);
      if (gj < n && gk < kend && (!BUP || gk <= gj)) v = B[gk + (long long)gj * ldb];
      Bs[kk][j] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[4], bv[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        a[t] = As[kk][tx + 16 * t];
        bv[t] = Bs[kk][ty + 16 * t];
      }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fma(a[p], bv[q], acc[p][q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int gj = j0 + ty + 16 * q;
    if (gj >= n) continue;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int gi = i0 + tx + 16 * p;
      if (gi >= m) continue;
      const int row = REV ? m - 1 - gi : gi;
      C[row + (long long)gj * ldc] = alpha * acc[p][q];
    }
  }
}

template <typename T, bool TA, bool BUP, bool LOWER, bool REV>
void basis_gemm(int m, int n, int k, T alpha, const T* A, int lda, long long sA, const T* B,
                int ldb, long long sB, T* C, int ldc, long long sC, int batch, cudaStream_t st) {
  const int tm = (m + BM - 1) / BM, tn = (n + BN - 1) / BN;
  const int tiles = LOWER ? tm * (tm + 1) / 2 : tm * tn;
  dim3 g(tiles, batch);
  basis_gemm_kernel<T, TA, BUP, LOWER, REV><<<g, NT, 0, st>>>(m, n, k, alpha, A, lda, sA, B, ldb,
                                                               sB, C, ldc, sC, tm);
}

// Ã = F_b B F_r: Ã(i, j) = B(b-1-i, r-1-j), one node per blockIdx.y.
template <typename T>
__global__ void __launch_bounds__(NT)
reverse_basis_kernel(const T* __restrict__ B, long long sB, T* __restrict__ Out, long long sO,
                     int b, int r) {
  const long long node = blockIdx.y;
  const long long e = (long long)blockIdx.x * NT + threadIdx.x;
  if (e >= (long long)b * r) return;
  const int i = (int)(e % b), j = (int)(e / b);
  Out[node * sO + e] = B[node * sB + (b - 1 - i) + (long long)(r - 1 - j) * b];
}

}  // namespace

namespace {

// ---- per-node dense kernels on an r x r block in shared memory (row-major,
// pitch ld = r + 1), blocked by 32 columns.  Diagonal blocks are factored or
// inverted by one warp in registers; the rest of each panel step is spread
// over the CTA with every thread's FMAs independent.

constexpr int NBK = 32;
constexpr int NWARP = NT / 32;

// element (i, j) of the lower-triangular view: S itself, or its transpose (the
// upper triangle read as a lower one)
template <bool TRANS, typename T>
HSS_DEVINL T& el(T* S, int ld, int i, int j) {
  return TRANS ? S[j * ld + i] : S[i * ld + j];
}

// In-place Cholesky S = L Lᵀ of the lower triangle; returns (in every thread)
// whether a pivot was not positive or not finite (it is then taken as 1).
template <typename T>
HSS_DEVINL int chol_blocked(T* S, int ld, int r, int* bad_s) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int j0 = 0; j0 < r; j0 += NBK) {
    const int kb = min(NBK, r - j0);
    if (warp == 0) {   // diagonal block: lane i holds row j0 + i
      T a[NBK];
#pragma unroll
      for (int t = 0; t < NBK; ++t)
        a[t] = (lane < kb && t < kb && t <= lane) ? S[(j0 + lane) * ld + j0 + t] : T(0);
      int bad = 0;
#pragma unroll
      for (int t = 0; t < NBK; ++t) {
        T d = __shfl_sync(0xffffffffu, a[t], t);
        if (t < kb) {
          if (!(d > T(0)) || !(d <= T(3.0e38))) {
            bad = 1;
            d = T(1);
          }
          d = sqrt(d);
          if (lane == t) a[t] = d;
          if (lane > t) a[t] /= d;
        }
#pragma unroll
        for (int k = t + 1; k < NBK; ++k) {
          const T xk = __shfl_sync(0xffffffffu, a[t], k);
          if (t < kb && k < kb && k <= lane) a[k] = fma(-a[t], xk, a[k]);
        }
      }
      if (lane < kb) {
#pragma unroll
        for (int t = 0; t < NBK; ++t)
          if (t < kb && t <= lane) S[(j0 + lane) * ld + j0 + t] = a[t];
      }
      if (lane == 0 && bad) *bad_s = 1;
    }
    __syncthreads();
    // rows below: row_i(j0 : j0+kb) L_blk⁻ᵀ, forward substitution per row
    for (int i = j0 + kb + tid; i < r; i += NT) {
      T x[NBK];
#pragma unroll
      for (int t = 0; t < NBK; ++t) x[t] = t < kb ? S[i * ld + j0 + t] : T(0);
#pragma unroll
      for (int t = 0; t < NBK; ++t) {
        if (t < kb) {
          x[t] /= S[(j0 + t) * ld + j0 + t];
#pragma unroll
          for (int u = t + 1; u < NBK; ++u)
            if (u < kb) x[u] = fma(-x[t], S[(j0 + u) * ld + j0 + t], x[u]);
        }
      }
#pragma unroll
      for (int t = 0; t < NBK; ++t)
        if (t < kb) S[i * ld + j0 + t] = x[t];
    }
    __syncthreads();
    // trailing lower triangle: S(i, k) -= Σ_t L(i, t) L(k, t), k <= i
    const int m = r - j0 - kb;
    for (int e = tid; e < m * m; e += NT) {
      const int i = j0 + kb + e % m, k = j0 + kb + e / m;
      if (k > i) continue;
      T s0 = T(0), s1 = T(0);
      for (int t = 0; t < kb; t += 2) {
        s0 = fma(S[i * ld + j0 + t], S[k * ld + j0 + t], s0);
        if (t + 1 < kb) s1 = fma(S[i * ld + j0 + t + 1], S[k * ld + j0 + t + 1], s1);
      }
      S[i * ld + k] -= s0 + s1;
    }
    __syncthreads();
  }
  return *bad_s;
}

// In-place inverse of the lower-triangular matrix of the view (TRANS: the
// upper triangle of S read transposed, so its inverse is the inverse of the
// upper triangle).  UNIT: unit diagonal, implicit and left untouched.
template <bool TRANS, bool UNIT, typename T>
HSS_DEVINL void tri_inv_blocked(T* S, int ld, int r) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nb = (r + NBK - 1) / NBK;
  // diagonal blocks, one warp each: lane j solves L_blk x = e_j
  for (int p = warp; p < nb; p += NWARP) {
    const int j0 = p * NBK, kb = min(NBK, r - j0);
    T x[NBK];
#pragma unroll
    for (int t = 0; t < NBK; ++t) x[t] = (t == lane) ? T(1) : T(0);
#pragma unroll
    for (int t = 0; t < NBK; ++t) {
      if (t < kb) {
        if (!UNIT) x[t] /= el<TRANS>(S, ld, j0 + t, j0 + t);
#pragma unroll
        for (int u = t + 1; u < NBK; ++u)
          if (u < kb) x[u] = fma(-el<TRANS>(S, ld, j0 + u, j0 + t), x[t], x[u]);
      }
    }
    __syncwarp();
    if (lane < kb) {
#pragma unroll
      for (int t = 0; t < NBK; ++t)
        if (t < kb && (t > lane || (t == lane && !UNIT))) el<TRANS>(S, ld, j0 + t, j0 + lane) = x[t];
    }
  }
  __syncthreads();
  // block columns right to left: X(i, jb) = -(Σ_{k} Xinv(i, k) X(k, jb)) Xinv_jj
  for (int jb = nb - 2; jb >= 0; --jb) {
    const int j0 = jb * NBK;   // a full block (only the last one can be ragged)
    T acc[NBK];
    const int i = j0 + NBK + tid;
    const bool act = i < r;
    if (act) {
#pragma unroll
      for (int t = 0; t < NBK; ++t) acc[t] = T(0);
      for (int k = j0 + NBK; k <= i; ++k) {
        const T xik = (UNIT && k == i) ? T(1) : el<TRANS>(S, ld, i, k);
#pragma unroll
        for (int t = 0; t < NBK; ++t) acc[t] = fma(xik, el<TRANS>(S, ld, k, j0 + t), acc[t]);
      }
    }
    __syncthreads();
    if (act) {
      T out[NBK];
#pragma unroll
      for (int u = 0; u < NBK; ++u) {
        T v = T(0);
#pragma unroll
        for (int t = 0; t < NBK; ++t) {
          if (t < u) continue;   // Xinv_jj lower: t >= u
          const T w = (UNIT && t == u) ? T(1) : el<TRANS>(S, ld, j0 + t, j0 + u);
          v = fma(acc[t], w, v);
        }
        out[u] = -v;
      }
#pragma unroll
      for (int u = 0; u < NBK; ++u) el<TRANS>(S, ld, i, j0 + u) = out[u];
    }
    __syncthreads();
  }
}

// One CTA per node: Cholesky G = L Lᵀ of the Gram matrix (lower triangle read,
// r x r, stride sR) in shared memory, then L⁻¹ in place.  Writes R = Lᵀ and
// P = L⁻ᵀ = R⁻¹ (both upper, zeros below) and sets fail[node] when a pivot is
// not positive or not finite.  With accumulate (the second pass) the flag is
// ORed in, and it is also set when G is far from the identity (an entry of
// G - I above 1/2): the first pass then did not orthonormalise the basis well
// enough for one more pass to finish the job.  r <= NT.
template <typename T>
__global__ void __launch_bounds__(NT)
cholinv_kernel(const T* __restrict__ G, T* __restrict__ Rout, T* __restrict__ Pout, long long sR,
               int r, int* __restrict__ fail, int accumulate) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* S = reinterpret_cast<T*>(smem_raw);
  const int ld = r + 1;
  __shared__ int bad;
  const long long node = blockIdx.x;
  const T* g = G + node * sR;
  const int tid = threadIdx.x;
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int e = tid; e < r * r; e += NT) {
    const int i = e % r, j = e / r;
    const T v = (i >= j) ? g[e] : T(0);
    S[i * ld + j] = v;
    if (accumulate && i >= j && !(fabs(v - (i == j ? T(1) : T(0))) <= T(0.5))) bad = 1;
  }
  __syncthreads();
  chol_blocked(S, ld, r, &bad);
  T* Rn = Rout + node * sR;
  for (int e = tid; e < r * r; e += NT) {
    const int i = e % r, j = e / r;
    Rn[e] = (i <= j) ? S[j * ld + i] : T(0);
  }
  __syncthreads();
  tri_inv_blocked<false, false>(S, ld, r);
  T* Pn = Pout + node * sR;
  for (int e = tid; e < r * r; e += NT) {
    const int i = e % r, j = e / r;
    Pn[e] = (i <= j) ? S[j * ld + i] : T(0);
  }
  if (tid == 0) fail[node] = accumulate ? (fail[node] | bad) : bad;
}

// One CTA per node: the Householder reconstruction of the top r x r block Qt of
// the orthonormal factor (stride sR; U on exit).  LU without pivoting of
// Qt - diag(s), s_j = -sign of the running diagonal (+1 for a square basis's
// last column, where dlarfg leaves the column unreflected), blocked by 32
// columns; then
//   V(b-1-i, j) = Y1(i, j)            (unit lower, rows b-r .. b-1 of V)
//   L_B(r-1-i, r-1-j) = s_i R(i, j)   (i <= j; R the Cholesky QR factor)
//   Ui = U⁻¹, W = S Y1⁻ᵀ              (both upper)
template <typename T>
__global__ void __launch_bounds__(NT)
recon_lu_kernel(T* __restrict__ Qt, T* __restrict__ Ui, T* __restrict__ W,
                const T* __restrict__ R, long long sR, T* __restrict__ V, long long sV, int b,
                T* __restrict__ LB, long long sL, int r) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* S = reinterpret_cast<T*>(smem_raw);   // row-major, pitch r + 1
  const int ld = r + 1;
  __shared__ T sg[256];
  const long long node = blockIdx.x;
  T* q = Qt + node * sR;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int e = tid; e < r * r; e += NT) {
    const int i = e % r, j = e / r;
    S[i * ld + j] = q[e];
  }
  __syncthreads();
  for (int j0 = 0; j0 < r; j0 += NBK) {
    const int kb = min(NBK, r - j0);
    if (warp == 0) {   // diagonal block LU with the sign rule: lane i holds row j0 + i
      T a[NBK];
#pragma unroll
      for (int t = 0; t < NBK; ++t) a[t] = (lane < kb && t < kb) ? S[(j0 + lane) * ld + j0 + t] : T(0);
#pragma unroll
      for (int t = 0; t < NBK; ++t) {
        const T u = __shfl_sync(0xffffffffu, a[t], t);
        if (t < kb) {
          const bool last_sq = (b == r && j0 + t == r - 1);
          T s = u >= T(0) ? T(-1) : T(1);
          if (last_sq) s = -s;
          const T piv = last_sq ? T(0) : u - s;
          if (lane == 0) sg[j0 + t] = s;
          if (lane == t) a[t] = piv;
          if (lane > t) a[t] /= piv;
        }
#pragma unroll
        for (int k = t + 1; k < NBK; ++k) {
          const T ukt = __shfl_sync(0xffffffffu, a[k], t);
          if (t < kb && k < kb && lane > t) a[k] = fma(-a[t], ukt, a[k]);
        }
      }
      if (lane < kb) {
#pragma unroll
        for (int t = 0; t < NBK; ++t)
          if (t < kb) S[(j0 + lane) * ld + j0 + t] = a[t];
      }
    }
    __syncthreads();
    const int m = r - j0 - kb;
    // L panel rows (A U_blk⁻¹, row-wise) and U panel columns (L_blk⁻¹ A, unit lower)
    for (int task = tid; task < 2 * m; task += NT) {
      T x[NBK];
      if (task < m) {
        const int i = j0 + kb + task;
#pragma unroll
        for (int t = 0; t < NBK; ++t) x[t] = t < kb ? S[i * ld + j0 + t] : T(0);
#pragma unroll
        for (int t = 0; t < NBK; ++t) {
          if (t < kb) {
            x[t] /= S[(j0 + t) * ld + j0 + t];
#pragma unroll
            for (int u2 = t + 1; u2 < NBK; ++u2)
              if (u2 < kb) x[u2] = fma(-x[t], S[(j0 + t) * ld + j0 + u2], x[u2]);
          }
        }
#pragma unroll
        for (int t = 0; t < NBK; ++t)
          if (t < kb) S[i * ld + j0 + t] = x[t];
      } else {
        const int k = j0 + kb + (task - m);
#pragma unroll
        for (int t = 0; t < NBK; ++t) x[t] = t < kb ? S[(j0 + t) * ld + k] : T(0);
#pragma unroll
        for (int t = 0; t < NBK; ++t) {
          if (t < kb) {
#pragma unroll
            for (int u2 = t + 1; u2 < NBK; ++u2)
              if (u2 < kb) x[u2] = fma(-S[(j0 + u2) * ld + j0 + t], x[t], x[u2]);
          }
        }
#pragma unroll
        for (int t = 0; t < NBK; ++t)
          if (t < kb) S[(j0 + t) * ld + k] = x[t];
      }
    }
    __syncthreads();
    // trailing square: S(i, k) -= Σ_t L(i, t) U(t, k)
    for (int e = tid; e < m * m; e += NT) {
      const int i = j0 + kb + e % m, k = j0 + kb + e / m;
      T s0 = T(0), s1 = T(0);
      for (int t = 0; t < kb; t += 2) {
        s0 = fma(S[i * ld + j0 + t], S[(j0 + t) * ld + k], s0);
        if (t + 1 < kb) s1 = fma(S[i * ld + j0 + t + 1], S[(j0 + t + 1) * ld + k], s1);
      }
      S[i * ld + k] -= s0 + s1;
    }
    __syncthreads();
  }
  T* Vn = V + node * sV;
  T* Ln = LB + node * sL;
  const T* Rn = R + node * sR;
  for (int e = tid; e < r * r; e += NT) {
    const int i = e % r, j = e / r;
    const T sij = S[i * ld + j];
    Vn[(b - 1 - i) + (long long)j * b] = i > j ? sij : (i == j ? T(1) : T(0));
    q[e] = i <= j ? sij : T(0);
    Ln[(r - 1 - i) + (long long)(r - 1 - j) * r] = i <= j ? sg[i] * Rn[e] : T(0);
  }
  __syncthreads();
  tri_inv_blocked<true, false>(S, ld, r);   // U⁻¹ (upper triangle with the diagonal)
  tri_inv_blocked<false, true>(S, ld, r);   // Y1⁻¹ (strictly lower, unit diagonal)
  T* Un = Ui + node * sR;
  T* Wn = W + node * sR;
  for (int e = tid; e < r * r; e += NT) {
    const int i = e % r, j = e / r;
    Un[e] = i <= j ? S[i * ld + j] : T(0);
    // W(i, j) = s_i Y1⁻¹(j, i) for i <= j
    Wn[e] = i < j ? sg[i] * S[j * ld + i] : (i == j ? sg[i] : T(0));
  }
}

template <typename T>
size_t node_smem(int r) {
  return (size_t)r * (r + 1) * sizeof(T);
}

}  // namespace

template <typename T>
int basis_max_rank() {
  int r = 1;
  while (r + 1 <= NT && node_smem<T>(r + 1) <= 200 * 1024) ++r;
  return r;
}

template <typename T>
cudaError_t launch_basis_completion(const T* B, long long sB, T* V, long long sV, T* Tm,
                                   long long sT, T* LB, long long sL, int b, int r, int n,
                                   const BasisScratch<T>& s, const BasisHook& hook,
                                   cudaStream_t st) {
  if (r > basis_max_rank<T>() || r > b || n <= 0) return cudaErrorInvalidValue;
  const long long rr = (long long)r * r, br = (long long)b * r;
  const size_t smem = node_smem<T>(r);
  static size_t attr = 0;   // dynamic shared memory granted so far
  if (smem > attr) {
    if (cudaFuncSetAttribute(cholinv_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess ||
        cudaFuncSetAttribute(recon_lu_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
      return cudaErrorInvalidConfiguration;
    attr = smem;
  }
  auto pre = [&](int kind, double fl) {
    if (hook.before) hook.before(hook.ctx, kind, fl);
  };
  auto post = [&]() {
    if (hook.after) hook.after(hook.ctx);
  };
  const double r3 = (double)r * r * r;
  const double gram = (double)b * r * (r + 1) * n;   // lower triangle of a b-deep product
  // 1. Ã = F_b B F_r into V (free until the reconstruction writes it)
  pre(BASIS_COPY, 0.0);
  reverse_basis_kernel<T><<<dim3((unsigned)((br + NT - 1) / NT), n), NT, 0, st>>>(B, sB, V, sV, b,
                                                                               r);
  post();
  // 2-4. first Cholesky QR pass: G = ÃᵀÃ = R1ᵀR1, X = Ã R1⁻¹
  pre(BASIS_GEMM, gram);
  basis_gemm<T, true, false, true, false>(r, r, b, T(1), V, b, sV, V, b, sV, s.G, r, rr, n, st);
  post();
  pre(BASIS_NODE, 2.0 / 3.0 * r3 * n);
  cholinv_kernel<T><<<n, NT, smem, st>>>(s.G, s.R1, s.P, rr, r, s.fail, 0);
  post();
  pre(BASIS_GEMM, (double)b * r * (r + 1) * n);
  basis_gemm<T, false, true, false, false>(b, r, r, T(1), V, b, sV, s.P, r, rr, s.X, b, br, n, st);
  post();
  // 5-7. second pass: XᵀX = R2ᵀR2 (R2 into U, R2⁻¹ into P), R = R2 R1
  pre(BASIS_GEMM, gram);
  basis_gemm<T, true, false, true, false>(r, r, b, T(1), s.X, b, br, s.X, b, br, s.G, r, rr, n, st);
  post();
  pre(BASIS_NODE, 2.0 / 3.0 * r3 * n);
  cholinv_kernel<T><<<n, NT, smem, st>>>(s.G, s.U, s.P, rr, r, s.fail, 1);
  post();
  pre(BASIS_GEMM, r3 / 3.0 * n);
  basis_gemm<T, false, true, false, false>(r, r, r, T(1), s.U, r, rr, s.R1, r, rr, s.R, r, rr, n,
                                           st);
  post();
  // 8. top block of the orthonormal factor: X(0:r, :) R2⁻¹ into U
  pre(BASIS_GEMM, r3 * n);
  basis_gemm<T, false, true, false, false>(r, r, r, T(1), s.X, b, br, s.P, r, rr, s.U, r, rr, n,
                                           st);
  post();
  // 9. reconstruction: Y1, U, U⁻¹, S Y1⁻ᵀ, L_B
  pre(BASIS_NODE, 4.0 / 3.0 * r3 * n);
  recon_lu_kernel<T><<<n, NT, smem, st>>>(s.U, s.Ui, s.G, s.R, rr, V, sV, b, LB, sL, r);
  post();
  // 10. T = -U (S Y1⁻ᵀ)
  pre(BASIS_GEMM, r3 / 3.0 * n);
  basis_gemm<T, false, true, false, false>(r, r, r, T(-1), s.U, r, rr, s.G, r, rr, Tm, r, sT, n,
                                           st);
  post();
  if (b > r) {
    // 11-12. Y2 = X(r:b, :) R2⁻¹ U⁻¹, stored row-reversed into V(0 : b-r, :)
    pre(BASIS_GEMM, r3 / 3.0 * n);
    basis_gemm<T, false, true, false, false>(r, r, r, T(1), s.P, r, rr, s.Ui, r, rr, s.R1, r, rr,
                                             n, st);
    post();
    pre(BASIS_GEMM, (double)(b - r) * r * (r + 1) * n);
    basis_gemm<T, false, true, false, true>(b - r, r, r, T(1), s.X + r, b, br, s.R1, r, rr, V, b,
                                            sV, n, st);
    post();
  }
  // 13. nodes whose Gram Cholesky failed: the Householder kernel
  pre(BASIS_FALLBACK, 0.0);
  cudaError_t e = launch_ql_basis<T>(B, b, sB, V, sV, Tm, sT, LB, sL, b, r, n, st, s.fail);
  post();
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template int basis_max_rank<double>();
template int basis_max_rank<float>();
template cudaError_t launch_basis_completion<double>(const double*, long long, double*, long long,
                                                     double*, long long, double*, long long, int,
                                                     int, int, const BasisScratch<double>&,
                                                     const BasisHook&, cudaStream_t);
template cudaError_t launch_basis_completion<float>(const float*, long long, float*, long long,
                                                    float*, long long, float*, long long, int, int,
                                                    int, const BasisScratch<float>&,
                                                    const BasisHook&, cudaStream_t);
