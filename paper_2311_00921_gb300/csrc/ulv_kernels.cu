// Per-node ULV step kernels (one CTA per tree node).
//
//  * ql_basis_kernel   -- basis completion, Eq. 2-3 (Sec. 2): Householder QL of
//                         the node basis B (b x r) as the QR of its row- and
//                         column-reversed copy (LAPACK dlarfg signs), giving
//                         Q = I - V T Vᵀ = [Q^R Q^S] with the redundant part first,
//                         and L_B = Q^Sᵀ B (r x r, lower triangular).
//  * pchol_kernel      -- partial Cholesky, Eq. partial-Cholesky (Alg. 2 line 3):
//                         right-looking blocked Cholesky of the first c = b - r
//                         columns of Â (lower triangle).  It leaves L^RR, L^SR
//                         and the Schur complement Â^SS; its epilogue is the merge
//                         (Alg. 2 line 4): Â^SS is written straight into the
//                         parent's diagonal block (a gather, no separate pass).
//                         With c = b and no parent it is the root Cholesky (line 6).
//  * trsv_fwd_kernel /
//    trsv_bwd_kernel   -- the triangular parts of the ULV solve (Sec. 3.2): forward
//                         z^R = L^RR⁻¹ y^R, y^S -= L^SR z^R (pushed to the parent's
//                         vector), and backward x^R = L^RR⁻ᵀ (z^R - L^SRᵀ x^S).
//  * logdet_reduce_kernel -- 2 Σ log diag over all nodes, fixed summation order.
#include <math.h>

#include "common.cuh"
#include "ulv_kernels.cuh"

namespace {

constexpr int NT = 256;
constexpr int NB = 32;   // panel width of the blocked Cholesky / triangular solves

// ------------------------------------------------------------------ QL
template <typename T>
__global__ void __launch_bounds__(NT)
ql_basis_kernel(const T* __restrict__ Bsrc, int ldb_src, long long sB, T* V, long long sV, T* Tm,
                long long sT, T* LB, long long sL, int b, int r) {
  __shared__ T red[32];
  __shared__ T tau_s[512];
  __shared__ T beta_s;
  const long long node = blockIdx.x;
  const T* B = Bsrc + node * sB;
  T* W = V + node * sV;   // working matrix, reversed coordinates during the QR
  T* Tn = Tm + node * sT;
  T* Ln = LB + node * sL;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = NT / 32;

  // reversed copy: W(i, j) = B(b-1-i, r-1-j)
  for (long long e = tid; e < (long long)b * r; e += NT) {
    const int i = (int)(e % b), j = (int)(e / b);
    W[i + (long long)j * b] = B[(b - 1 - i) + (long long)(r - 1 - j) * ldb_src];
  }
  __syncthreads();

  // unblocked Householder QR of W (b x r)
  for (int j = 0; j < r; ++j) {
    T* wj = W + (long long)j * b;
    T s = T(0);
    for (int i = j + 1 + tid; i < b; i += NT) s += wj[i] * wj[i];
    const T sigma = block_sum(s, red);
    const T alpha = wj[j];
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
    if (tid == 0) {
      tau_s[j] = tau;
      beta_s = beta;
    }
    for (int i = j + 1 + tid; i < b; i += NT) wj[i] *= scale;
    __syncthreads();
    // apply H_j = I - tau v vᵀ (v_j = 1) to columns k > j, one warp per column
    if (tau != T(0)) {
      for (int k = j + 1 + wid; k < r; k += nw) {
        T* wk = W + (long long)k * b;
        T d = T(0);
        for (int i = j + 1 + lane; i < b; i += 32) d += wj[i] * wk[i];
        d = warp_sum(d) + wk[j];
        const T f = tau * d;
        for (int i = j + 1 + lane; i < b; i += 32) wk[i] -= f * wj[i];
        if (lane == 0) wk[j] -= f;
      }
    }
    __syncthreads();
    if (tid == 0) wj[j] = beta_s;   // R(j, j)
    __syncthreads();
  }

  // L_B(a, c) = R(r-1-a, r-1-c): R is the upper triangle of W
  for (int e = tid; e < r * r; e += NT) {
    const int a = e % r, c = e / r;
    T v = T(0);
    if (a >= c) v = W[(r - 1 - a) + (long long)(r - 1 - c) * b];
    Ln[a + (long long)c * r] = v;
  }
  __syncthreads();
  // explicit unit diagonal and zeros above it in the reversed reflectors
  for (int e = tid; e < r * r; e += NT) {
    const int i = e % r, j = e / r;
    if (i <= j) W[i + (long long)j * b] = (i == j) ? T(1) : T(0);
  }
  __syncthreads();
  // Gram G = Ṽᵀ Ṽ, upper part stored transposed in the strict lower triangle of T
  for (int e = wid; e < r * r; e += nw) {
    const int i = e % r, j = e / r;
    if (i >= j) continue;   // need G(i, j) for i < j
    const T* vi = W + (long long)i * b;
    const T* vj = W + (long long)j * b;
    T d = T(0);
    for (int t = j + lane; t < b; t += 32) d += vi[t] * vj[t];   // vj is zero above row j
    d = warp_sum(d);
    if (lane == 0) Tn[j + (long long)i * r] = d;   // G(i,j) at T(j,i)
  }
  __syncthreads();
  // forward columnwise T (dlarft): T(j,j) = tau_j, T(0:j, j) = -tau_j T(0:j,0:j) G(0:j, j)
  for (int j = 0; j < r; ++j) {
    const T tj = tau_s[j];
    T val = T(0);
    const int i = tid;
    if (i < j) {
      T acc = T(0);
      for (int m = i; m < j; ++m) acc += Tn[i + (long long)m * r] * Tn[j + (long long)m * r];
      val = -tj * acc;
    }
    __syncthreads();
    if (tid < j) Tn[tid + (long long)j * r] = val;   // r <= NT is checked by the host
    if (tid == 0) Tn[j + (long long)j * r] = tj;
    __syncthreads();
  }
  // zero the strict lower triangle (the Gram scratch)
  for (int e = tid; e < r * r; e += NT) {
    const int i = e % r, j = e / r;
    if (i > j) Tn[i + (long long)j * r] = T(0);
  }
  // back to natural row order: V = F_b Ṽ
  for (long long e = tid; e < (long long)(b / 2) * r; e += NT) {
    const int i = (int)(e % (b / 2)), j = (int)(e / (b / 2));
    T* col = W + (long long)j * b;
    const T x = col[i];
    col[i] = col[b - 1 - i];
    col[b - 1 - i] = x;
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
    // panel TRSM: rows kb..n1-1 : x L_diagᵀ = m
    for (int i = kb + tid; i < n1; i += NT) {
      for (int jj = 0; jj < kb; ++jj) {
        T x = P[i + jj * b];
        for (int t = 0; t < jj; ++t) x -= P[i + t * b] * P[jj + t * b];
        P[i + jj * b] = x / P[jj + jj * b];
      }
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

// ------------------------------------------------------------------ triangular sweeps
// forward: y (b x nrhs, smem) := [L^RR⁻¹ y^R ; y^S - L^SR L^RR⁻¹ y^R]
template <typename T>
__global__ void __launch_bounds__(NT)
trsv_fwd_kernel(const T* __restrict__ Mb, int ldm, long long sM, int b, int c, T* X, int ldx,
                long long sX, int nrhs, T* Par, int ldpar, long long sPar) {
  extern __shared__ unsigned char smem_raw[];
  T* y = reinterpret_cast<T*>(smem_raw);   // b x nrhs, ld = b
  const int node = blockIdx.x;
  const T* M = Mb + (long long)node * sM;
  T* x = X + (long long)node * sX;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = NT / 32;
  for (int e = tid; e < b * nrhs; e += NT) {
    const int i = e % b, j = e / b;
    y[i + j * b] = x[i + (long long)j * ldx];
  }
  __syncthreads();
  for (int k0 = 0; k0 < c; k0 += NB) {
    const int kb = min(NB, c - k0);
    // diagonal block: warp w handles right-hand sides w, w + nw, ...
    for (int j = wid; j < nrhs; j += nw) {
      T* yj = y + j * b + k0;
      T v = lane < kb ? yj[lane] : T(0);
      const T lii = lane < kb ? M[(k0 + lane) + (long long)(k0 + lane) * ldm] : T(1);
      for (int t = 0; t < kb; ++t) {
        T zt = __shfl_sync(0xffffffffu, v, t);
        zt = zt / __shfl_sync(0xffffffffu, lii, t);
        if (lane == t) v = zt;
        if (lane > t && lane < kb) v -= M[(k0 + lane) + (long long)(k0 + t) * ldm] * zt;
      }
      if (lane < kb) yj[lane] = v;
    }
    __syncthreads();
    // update every row below the block (the S rows included: L^SR lives there)
    for (int i = k0 + kb + tid; i < b; i += NT) {
      T acc[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) acc[j] = T(0);
      for (int t = 0; t < kb; ++t) {
        const T l = M[i + (long long)(k0 + t) * ldm];
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (j < nrhs) acc[j] = fma(l, y[(k0 + t) + j * b], acc[j]);
      }
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (j < nrhs) y[i + j * b] -= acc[j];
    }
    __syncthreads();
  }
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

// backward: x^S from the parent's vector (or in place when Par is null),
// x^R = L^RR⁻ᵀ (z^R - L^SRᵀ x^S); the node segment becomes [x^R; x^S]
template <typename T>
__global__ void __launch_bounds__(NT)
trsv_bwd_kernel(const T* __restrict__ Mb, int ldm, long long sM, int b, int c, T* X, int ldx,
                long long sX, int nrhs, const T* Par, int ldpar, long long sPar) {
  extern __shared__ unsigned char smem_raw[];
  T* y = reinterpret_cast<T*>(smem_raw);   // b x nrhs
  const int node = blockIdx.x;
  const T* M = Mb + (long long)node * sM;
  T* x = X + (long long)node * sX;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = NT / 32;
  const int r = b - c;
  for (int e = tid; e < b * nrhs; e += NT) {
    const int i = e % b, j = e / b;
    T v;
    if (i >= c && Par)
      v = Par[(long long)node * sPar + (i - c) + (long long)j * ldpar];
    else
      v = x[i + (long long)j * ldx];
    y[i + j * b] = v;
  }
  __syncthreads();
  const int nblk = (c + NB - 1) / NB;
  for (int bi = nblk - 1; bi >= 0; --bi) {
    const int k0 = bi * NB;
    const int kb = min(NB, c - k0);
    // z_t -= sum_{i >= k0+kb} L(i, t) x_i  for t in the block
    for (int e = tid; e < kb * nrhs; e += NT) {
      const int t = e % kb, j = e / kb;
      const T* lcol = M + (long long)(k0 + t) * ldm;
      T acc = T(0);
      for (int i = k0 + kb; i < b; ++i) acc = fma(lcol[i], y[i + j * b], acc);
      y[(k0 + t) + j * b] -= acc;
    }
    __syncthreads();
    // diagonal block, transposed back substitution
    for (int j = wid; j < nrhs; j += nw) {
      T* yj = y + j * b + k0;
      T v = lane < kb ? yj[lane] : T(0);
      for (int t = kb - 1; t >= 0; --t) {
        T xt = __shfl_sync(0xffffffffu, v, t);
        const T ltt = M[(k0 + t) + (long long)(k0 + t) * ldm];
        xt = xt / ltt;
        if (lane == t) v = xt;
        if (lane < t) v -= M[(k0 + t) + (long long)(k0 + lane) * ldm] * xt;
      }
      if (lane < kb) yj[lane] = v;
    }
    __syncthreads();
  }
  (void)r;
  for (int e = tid; e < b * nrhs; e += NT) {
    const int i = e % b, j = e / b;
    x[i + (long long)j * ldx] = y[i + j * b];
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
template <typename T>
void launch_ql_basis(const T* Bsrc, int ldb_src, long long sB, T* V, long long sV, T* Tm,
                     long long sT, T* LB, long long sL, int b, int r, int nodes, cudaStream_t st) {
  ql_basis_kernel<T><<<nodes, NT, 0, st>>>(Bsrc, ldb_src, sB, V, sV, Tm, sT, LB, sL, b, r);
}

template <typename T>
size_t pchol_smem(int b) { return (size_t)b * NB * sizeof(T); }

template <typename T>
void launch_pchol(T* M, int ldm, long long sM, int b, int c, T* PA, int ldpa, long long sPA,
                  double* logdet_part, int level, int node0, int* status, int nodes,
                  cudaStream_t st) {
  const size_t sm = pchol_smem<T>(b);
  static bool attr_set = false;   // per template instance
  if (!attr_set) {
    cudaFuncSetAttribute(pchol_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set = true;
  }
  pchol_kernel<T><<<nodes, NT, sm, st>>>(M, ldm, sM, b, c, PA, ldpa, sPA, logdet_part, level,
                                         node0, status);
}

template <typename T>
void launch_trsv_fwd(const T* M, int ldm, long long sM, int b, int c, T* X, int ldx, long long sX,
                     int nrhs, T* Par, int ldpar, long long sPar, int nodes, cudaStream_t st) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(trsv_fwd_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
    attr_set = true;
  }
  const size_t sm = (size_t)b * nrhs * sizeof(T);
  trsv_fwd_kernel<T><<<nodes, NT, sm, st>>>(M, ldm, sM, b, c, X, ldx, sX, nrhs, Par, ldpar, sPar);
}

template <typename T>
void launch_trsv_bwd(const T* M, int ldm, long long sM, int b, int c, T* X, int ldx, long long sX,
                     int nrhs, const T* Par, int ldpar, long long sPar, int nodes,
                     cudaStream_t st) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(trsv_bwd_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
    attr_set = true;
  }
  const size_t sm = (size_t)b * nrhs * sizeof(T);
  trsv_bwd_kernel<T><<<nodes, NT, sm, st>>>(M, ldm, sM, b, c, X, ldx, sX, nrhs, Par, ldpar, sPar);
}

void launch_logdet_reduce(const double* part, int n, double* out, cudaStream_t st) {
  logdet_reduce_kernel<<<1, 1024, 0, st>>>(part, n, out);
}

#define INST(T)                                                                                  \
  template void launch_ql_basis<T>(const T*, int, long long, T*, long long, T*, long long, T*,    \
                                   long long, int, int, int, cudaStream_t);                       \
  template void launch_pchol<T>(T*, int, long long, int, int, T*, int, long long, double*, int,   \
                                int, int*, int, cudaStream_t);                                    \
  template void launch_trsv_fwd<T>(const T*, int, long long, int, int, T*, int, long long, int,   \
                                   T*, int, long long, int, cudaStream_t);                        \
  template void launch_trsv_bwd<T>(const T*, int, long long, int, int, T*, int, long long, int,   \
                                   const T*, int, long long, int, cudaStream_t);
INST(double)
INST(float)
