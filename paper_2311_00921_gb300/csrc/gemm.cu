// Batched SIMT GEMM / SYR2K for the FP64 (and FP32) ULV path.
//
// On GB300 the FP64 pipe retires about 2 DFMA per clock per SM, so these
// kernels are bound by DFMA issue, not by memory: a 64x64 output tile with a
// 4x4 register micro-tile per thread keeps 16 independent DFMAs in flight per
// thread against 8 shared-memory loads, and the only other goal is enough
// CTAs to cover all 152 SMs.  Tall-skinny products (n <= 32 columns, the
// right-hand-side blocks of the solve and matvec) use a separate kernel whose
// warps own whole columns, so that no warp issues DFMAs on padding.  The FP32
// factor's wide products get their own 128 x 128 tile (sgemm128_kernel), since
// on the FP32 pipe the 4x4 micro-tile's shared-memory loads, not the FMAs, set
// the rate.  syr2k_lower_kernel also serves as the SYRK of the blocked partial
// Cholesky (template flag SYRK).
#include <type_traits>

#include "common.cuh"

namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

template <typename T, bool TA, bool TB, bool BETA>
__global__ void __launch_bounds__(NT)
gemm_tile_kernel(int m, int n, int k, T alpha, const T* __restrict__ A, int lda, long long sA,
                 const T* __restrict__ B, int ldb, long long sB, T beta, T* C, int ldc,
                 long long sC) {
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const long long bz = blockIdx.z;
  A += bz * sA;
  B += bz * sB;
  C += bz * sC;
  const int i0 = blockIdx.x * BM, j0 = blockIdx.y * BN;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);

  for (int k0 = 0; k0 < k; k0 += BK) {
#pragma unroll
    for (int e0 = 0; e0 < BM * BK; e0 += NT) {
      const int e = e0 + threadIdx.x;
      int i, kk;
      if (!TA) { i = e % BM; kk = e / BM; } else { kk = e % BK; i = e / BK; }
      const int gi = i0 + i, gk = k0 + kk;
      T v = T(0);
      if (gi < m && gk < k) v = TA ? A[gk + (long long)gi * lda] : A[gi + (long long)gk * lda];
      As[kk][i] = v;
    }
#pragma unroll
    for (int e0 = 0; e0 < BN * BK; e0 += NT) {
      const int e = e0 + threadIdx.x;
      int j, kk;
      if (!TB) { kk = e % BK; j = e / BK; } else { j = e % BN; kk = e / BN; }
      const int gj = j0 + j, gk = k0 + kk;
      T v = T(0);
      if (gj < n && gk < k) v = TB ? B[gj + (long long)gk * ldb] : B[gk + (long long)gj * ldb];
      Bs[kk][j] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        a[t] = As[kk][tx + 16 * t];
        b[t] = Bs[kk][ty + 16 * t];
      }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fma(a[p], b[q], acc[p][q]);
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
      T* c = C + gi + (long long)gj * ldc;
      *c = BETA ? fma(alpha, acc[p][q], beta * *c) : alpha * acc[p][q];
    }
  }
}

// tall-skinny: C (m x n, n <= 32) ; CTA = 64 rows x all n columns.
// warp w owns columns w, w + 8, w + 16, w + 24; lane owns rows lane, lane + 32.
template <typename T, bool TA, bool TB, bool BETA>
__global__ void __launch_bounds__(NT)
gemm_skinny_kernel(int m, int n, int k, T alpha, const T* __restrict__ A, int lda, long long sA,
                   const T* __restrict__ B, int ldb, long long sB, T beta, T* C, int ldc,
                   long long sC) {
  constexpr int SBK = 32;
  __shared__ T As[SBK][BM + 1];
  __shared__ T Bs[32][SBK + 1];   // Bs[j][kk]
  const long long bz = blockIdx.z;
  A += bz * sA;
  B += bz * sB;
  C += bz * sC;
  const int i0 = blockIdx.x * BM;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  T acc[4][2];
#pragma unroll
  for (int a = 0; a < 4; ++a) acc[a][0] = acc[a][1] = T(0);
  for (int k0 = 0; k0 < k; k0 += SBK) {
    for (int e = threadIdx.x; e < BM * SBK; e += NT) {
      int i, kk;
      if (!TA) { i = e % BM; kk = e / BM; } else { kk = e % SBK; i = e / SBK; }
      const int gi = i0 + i, gk = k0 + kk;
      T v = T(0);
      if (gi < m && gk < k) v = TA ? A[gk + (long long)gi * lda] : A[gi + (long long)gk * lda];
      As[kk][i] = v;
    }
    for (int e = threadIdx.x; e < 32 * SBK; e += NT) {
      int j, kk;
      if (!TB) { kk = e % SBK; j = e / SBK; } else { j = e % 32; kk = e / 32; }
      const int gk = k0 + kk;
      T v = T(0);
      if (j < n && gk < k) v = TB ? B[j + (long long)gk * ldb] : B[gk + (long long)j * ldb];
      Bs[j][kk] = v;
    }
    __syncthreads();
    if (w < n) {
#pragma unroll 4
      for (int kk = 0; kk < SBK; ++kk) {
        const T a0 = As[kk][lane], a1 = As[kk][lane + 32];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int j = w + 8 * q;   // warp-uniform
          if (j < n) {
            const T bv = Bs[j][kk];
            acc[q][0] = fma(a0, bv, acc[q][0]);
            acc[q][1] = fma(a1, bv, acc[q][1]);
          }
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int j = w + 8 * q;
    if (j >= n) continue;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int gi = i0 + lane + 32 * h;
      if (gi >= m) continue;
      T* c = C + gi + (long long)j * ldc;
      *c = BETA ? fma(alpha, acc[q][h], beta * *c) : alpha * acc[q][h];
    }
  }
}

// n <= 4 NQ columns: CTA = 128 rows x 4 NQ columns, 128 threads with a 4 x NQ
// register micro-tile each (rows lane + 32 p, columns warp + 4 q): with NQ = 4,
// 16 FMAs per 8 shared-memory loads, as in the square tile, so the FP64 pipe
// stays fed on the right-hand-side blocks of the solve and the residual matvec.
// NQ = 2 serves blocks of at most 8 columns (a refinement lane's) and NQ = 1
// blocks of at most 4, without the FMAs of zero columns.
template <typename T, bool TA, bool TB, bool BETA, int NQ>
__global__ void __launch_bounds__(128)
gemm_n16_kernel(int m, int n, int k, T alpha, const T* __restrict__ A, int lda, long long sA,
                const T* __restrict__ B, int ldb, long long sB, T beta, T* C, int ldc,
                long long sC) {
  constexpr int TBM = 128, TBK = 16, TNT = 128;
  __shared__ T As[TBK][TBM + 1];
  constexpr int NB = 4 * NQ;
  __shared__ T Bs[TBK][NB + 1];
  const long long bz = blockIdx.z;
  A += bz * sA;
  B += bz * sB;
  C += bz * sC;
  const int i0 = blockIdx.x * TBM;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  T acc[4][NQ];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < NQ; ++b) acc[a][b] = T(0);
  for (int k0 = 0; k0 < k; k0 += TBK) {
#pragma unroll
    for (int e0 = 0; e0 < TBM * TBK; e0 += TNT) {
      const int e = e0 + threadIdx.x;
      int i, kk;
      if (!TA) { i = e % TBM; kk = e / TBM; } else { kk = e % TBK; i = e / TBK; }
      const int gi = i0 + i, gk = k0 + kk;
      T v = T(0);
      if (gi < m && gk < k) v = TA ? A[gk + (long long)gi * lda] : A[gi + (long long)gk * lda];
      As[kk][i] = v;
    }
#pragma unroll
    for (int e0 = 0; e0 < NB * TBK; e0 += TNT) {
      const int e = e0 + threadIdx.x;
      if (NB * TBK % TNT != 0 && e >= NB * TBK) break;   // NQ = 1: half the threads load
      int j, kk;
      if (!TB) { kk = e % TBK; j = e / TBK; } else { j = e % NB; kk = e / NB; }
      const int gk = k0 + kk;
      T v = T(0);
      if (j < n && gk < k) v = TB ? B[j + (long long)gk * ldb] : B[gk + (long long)j * ldb];
      Bs[kk][j] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TBK; ++kk) {
      T a[4], bv[NQ];
#pragma unroll
      for (int t = 0; t < 4; ++t) a[t] = As[kk][lane + 32 * t];
#pragma unroll
      for (int t = 0; t < NQ; ++t) bv[t] = Bs[kk][w + 4 * t];
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < NQ; ++q) acc[p][q] = fma(a[p], bv[q], acc[p][q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int gj = w + 4 * q;
    if (gj >= n) continue;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int gi = i0 + lane + 32 * p;
      if (gi >= m) continue;
      T* c = C + gi + (long long)gj * ldc;
      *c = BETA ? fma(alpha, acc[p][q], beta * *c) : alpha * acc[p][q];
    }
  }
}

// n <= 16 columns, few output tiles: CTA = 32 rows x 16 columns, 64 threads
// with a 2 x 4 micro-tile each (rows lane + 16 p of the half-warp pair,
// columns (warp * 2 + half) + 4 q).  Used when a launch would not fill the
// GPU: a 128-row tile of an FP64 product with k = 256 takes ~0.1 ms on one SM,
// so the top levels of the tree need the rows spread over more SMs.
template <typename T, bool TA, bool TB, bool BETA>
__global__ void __launch_bounds__(64)
gemm_n16_small_kernel(int m, int n, int k, T alpha, const T* __restrict__ A, int lda,
                      long long sA, const T* __restrict__ B, int ldb, long long sB, T beta, T* C,
                      int ldc, long long sC) {
  constexpr int SBM = 32, SBK = 32, SNT = 64;
  __shared__ T As[SBK][SBM + 1];
  __shared__ T Bs[SBK][16 + 1];
  const long long bz = blockIdx.z;
  A += bz * sA;
  B += bz * sB;
  C += bz * sC;
  const int i0 = blockIdx.x * SBM;
  const int tid = threadIdx.x;
  const int rl = tid & 15, cg = tid >> 4;   // row lane 0..15, column group 0..3
  T acc[2][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
  for (int k0 = 0; k0 < k; k0 += SBK) {
    for (int e = tid; e < SBM * SBK; e += SNT) {
      int i, kk;
      if (!TA) { i = e % SBM; kk = e / SBM; } else { kk = e % SBK; i = e / SBK; }
      const int gi = i0 + i, gk = k0 + kk;
      T v = T(0);
      if (gi < m && gk < k) v = TA ? A[gk + (long long)gi * lda] : A[gi + (long long)gk * lda];
      As[kk][i] = v;
    }
    for (int e = tid; e < 16 * SBK; e += SNT) {
      int j, kk;
      if (!TB) { kk = e % SBK; j = e / SBK; } else { j = e % 16; kk = e / 16; }
      const int gk = k0 + kk;
      T v = T(0);
      if (j < n && gk < k) v = TB ? B[j + (long long)gk * ldb] : B[gk + (long long)j * ldb];
      Bs[kk][j] = v;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < SBK; ++kk) {
      const T a0 = As[kk][rl], a1 = As[kk][rl + 16];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const T bv = Bs[kk][cg + 4 * q];
        acc[0][q] = fma(a0, bv, acc[0][q]);
        acc[1][q] = fma(a1, bv, acc[1][q]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int gj = cg + 4 * q;
    if (gj >= n) continue;
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      const int gi = i0 + rl + 16 * p;
      if (gi >= m) continue;
      T* c = C + gi + (long long)gj * ldc;
      *c = BETA ? fma(alpha, acc[p][q], beta * *c) : alpha * acc[p][q];
    }
  }
}

// n <= 16 columns on few nodes: the products at the top of the tree, where a
// launch has only a handful of CTAs and a tile loop leaves each SM's pipe idle
// between dependent steps.  CTA = 32 output rows of one node, lane = row; warp
// w accumulates K slice w of 8 for all n columns (the right-hand block is one
// broadcast read for the 32 rows), and the slices are added in a fixed order.
// TA: op(A) = Aᵀ, each lane walks its own row of Aᵀ (a column of A) through
// L1-resident lines; else the 32 lanes read one column of A, coalesced.
template <typename T, bool TA, bool BETA>
__global__ void __launch_bounds__(256)
gemm_lat_kernel(int m, int n, int k, T alpha, const T* __restrict__ A, int lda, long long sA,
                const T* __restrict__ B, int ldb, long long sB, T beta, T* C, int ldc,
                long long sC) {
  __shared__ T part[8][32][17];
  const long long bz = blockIdx.y;
  A += bz * sA;
  B += bz * sB;
  C += bz * sC;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int i = blockIdx.x * 32 + lane;
  const int kc = (k + 7) / 8, k0 = w * kc, k1 = min(k, k0 + kc);
  T acc[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) acc[j] = T(0);
  if (i < m) {
    for (int kk = k0; kk < k1; ++kk) {
      const T a = TA ? A[kk + (long long)i * lda] : A[i + (long long)kk * lda];
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (j < n) acc[j] = fma(a, B[kk + (long long)j * ldb], acc[j]);
    }
  }
#pragma unroll
  for (int j = 0; j < 16; ++j) part[w][lane][j] = acc[j];
  __syncthreads();
  for (int e = threadIdx.x; e < 32 * n; e += 256) {
    const int rr = e % 32, j = e / 32;
    const int gi = blockIdx.x * 32 + rr;
    if (gi >= m) continue;
    T s = T(0);
#pragma unroll
    for (int q = 0; q < 8; ++q) s += part[q][rr][j];
    T* c = C + gi + (long long)j * ldc;
    *c = BETA ? fma(alpha, s, beta * *c) : alpha * s;
  }
}

// FP32 128 x 128 tile for wide products (the diagonal product of the FP32
// factor): 256 threads with an 8 x 8 micro-tile each, split into four 4 x 4
// quadrants (rows 4 tx and 64 + 4 tx, columns 4 ty and 64 + 4 ty) so that every
// operand fragment is one 128-bit shared load: 4 loads per 64 FMAs.  The next
// K slab is fetched into registers while the current one is multiplied, into
// the other of two shared-memory buffers (one barrier per slab).
constexpr int SBM = 128, SBK8 = 8;

template <bool TA, bool TB, bool BETA>
__global__ void __launch_bounds__(256)
sgemm128_kernel(int m, int n, int k, float alpha, const float* __restrict__ A, int lda,
                long long sA, const float* __restrict__ B, int ldb, long long sB, float beta,
                float* C, int ldc, long long sC) {
  __shared__ __align__(16) float As[2][SBK8][SBM];
  __shared__ __align__(16) float Bs[2][SBK8][SBM];
  const long long bz = blockIdx.z;
  A += bz * sA;
  B += bz * sB;
  C += bz * sC;
  const int i0 = blockIdx.x * SBM, j0 = blockIdx.y * SBM;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  // slab element e = tid + 256 q (q < 4) of the 128 x 8 A slab and the 8 x 128 B slab
  float ra[4], rb[4];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid + 256 * q;
      int i, kk;
      if (!TA) { i = e % SBM; kk = e / SBM; } else { kk = e % SBK8; i = e / SBK8; }
      const int gi = i0 + i, gk = k0 + kk;
      ra[q] = (gi < m && gk < k) ? (TA ? A[gk + (long long)gi * lda] : A[gi + (long long)gk * lda])
                                 : 0.f;
      int j, kb;
      if (!TB) { kb = e % SBK8; j = e / SBK8; } else { j = e % SBM; kb = e / SBM; }
      const int gj = j0 + j, gkb = k0 + kb;
      rb[q] = (gj < n && gkb < k) ? (TB ? B[gj + (long long)gkb * ldb] : B[gkb + (long long)gj * ldb])
                                  : 0.f;
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid + 256 * q;
      int i, kk;
      if (!TA) { i = e % SBM; kk = e / SBM; } else { kk = e % SBK8; i = e / SBK8; }
      As[buf][kk][i] = ra[q];
      int j, kb;
      if (!TB) { kb = e % SBK8; j = e / SBK8; } else { j = e % SBM; kb = e / SBM; }
      Bs[buf][kb][j] = rb[q];
    }
  };
  float acc[8][8];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
  fetch(0);
  store(0);
  __syncthreads();
  int buf = 0;
  for (int k0 = 0; k0 < k; k0 += SBK8) {
    const bool more = k0 + SBK8 < k;
    if (more) fetch(k0 + SBK8);
#pragma unroll
    for (int kk = 0; kk < SBK8; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][4 * tx]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][64 + 4 * tx]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][4 * ty]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][64 + 4 * ty]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int p = 0; p < 8; ++p)
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[p][q] = fmaf(av[p], bv[q], acc[p][q]);
    }
    if (more) {
      store(buf ^ 1);
      __syncthreads();
      buf ^= 1;
    }
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int gj = j0 + (q < 4 ? 4 * ty + q : 64 + 4 * ty + q - 4);
    if (gj >= n) continue;
#pragma unroll
    for (int p = 0; p < 8; ++p) {
      const int gi = i0 + (p < 4 ? 4 * tx + p : 64 + 4 * tx + p - 4);
      if (gi >= m) continue;
      float* c = C + gi + (long long)gj * ldc;
      *c = BETA ? fmaf(alpha, acc[p][q], beta * *c) : alpha * acc[p][q];
    }
  }
}

// the FP32 wide tile where its 128 x 128 tiles still fill the GPU twice over
template <typename T, bool TA, bool TB>
bool launch_sgemm128(int m, int n, int k, T alpha, const T* A, int lda, long long sA, const T* B,
                     int ldb, long long sB, T beta, T* C, int ldc, long long sC, int batch,
                     cudaStream_t st) {
  if constexpr (std::is_same<T, float>::value) {
    const long long tiles = (long long)((m + SBM - 1) / SBM) * ((n + SBM - 1) / SBM) * batch;
    if (n < 64 || m < 64 || tiles < 2 * 152) return false;
    dim3 g((m + SBM - 1) / SBM, (n + SBM - 1) / SBM, batch);
    if (beta != 0.f)
      sgemm128_kernel<TA, TB, true><<<g, 256, 0, st>>>(m, n, k, alpha, A, lda, sA, B, ldb, sB,
                                                       beta, C, ldc, sC);
    else
      sgemm128_kernel<TA, TB, false><<<g, 256, 0, st>>>(m, n, k, alpha, A, lda, sA, B, ldb, sB,
                                                        beta, C, ldc, sC);
    return true;
  } else {
    return false;
  }
}

template <typename T, bool TA, bool TB>
void launch_gemm(int m, int n, int k, T alpha, const T* A, int lda, long long sA, const T* B,
                 int ldb, long long sB, T beta, T* C, int ldc, long long sC, int batch,
                 cudaStream_t st) {
  const bool useb = beta != T(0);
  if (!TB && n <= 16 && (long long)((m + 127) / 128) * batch < 152 && batch <= 65535) {
    // few nodes: the low-latency kernel
    dim3 g((m + 31) / 32, batch);
    if (useb)
      gemm_lat_kernel<T, TA, true><<<g, 256, 0, st>>>(m, n, k, alpha, A, lda, sA, B, ldb, sB, beta,
                                                       C, ldc, sC);
    else
      gemm_lat_kernel<T, TA, false><<<g, 256, 0, st>>>(m, n, k, alpha, A, lda, sA, B, ldb, sB,
                                                        beta, C, ldc, sC);
    return;
  }
  if (n > 4 && n <= 16 && (long long)((m + 127) / 128) * batch < 152) {
    dim3 g((m + 31) / 32, 1, batch);
    if (useb)
      gemm_n16_small_kernel<T, TA, TB, true><<<g, 64, 0, st>>>(m, n, k, alpha, A, lda, sA, B, ldb,
                                                              sB, beta, C, ldc, sC);
    else
      gemm_n16_small_kernel<T, TA, TB, false><<<g, 64, 0, st>>>(m, n, k, alpha, A, lda, sA, B,
                                                               ldb, sB, beta, C, ldc, sC);
    return;
  }
  if (n >= 1 && n <= 16) {
    dim3 g((m + 127) / 128, 1, batch);
#define N16_RUN(B_, NQ_)                                                                     \
  gemm_n16_kernel<T, TA, TB, B_, NQ_><<<g, 128, 0, st>>>(m, n, k, alpha, A, lda, sA, B, ldb, sB, \
                                                        beta, C, ldc, sC)
    if (n <= 4) {   // every thread busy on 4 rows of one column (the skinny kernel would idle
                    // the warps past n)
      if (useb) N16_RUN(true, 1); else N16_RUN(false, 1);
    } else if (n <= 8) {
      if (useb) N16_RUN(true, 2); else N16_RUN(false, 2);
    } else {
      if (useb) N16_RUN(true, 4); else N16_RUN(false, 4);
    }
#undef N16_RUN
    return;
  }
  if (n <= 32) {
    dim3 g((m + BM - 1) / BM, 1, batch);
    if (useb)
      gemm_skinny_kernel<T, TA, TB, true><<<g, NT, 0, st>>>(m, n, k, alpha, A, lda, sA, B, ldb, sB,
                                                           beta, C, ldc, sC);
    else
      gemm_skinny_kernel<T, TA, TB, false><<<g, NT, 0, st>>>(m, n, k, alpha, A, lda, sA, B, ldb,
                                                            sB, beta, C, ldc, sC);
    return;
  }
  if (launch_sgemm128<T, TA, TB>(m, n, k, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, batch,
                                 st))
    return;
  dim3 g((m + BM - 1) / BM, (n + BN - 1) / BN, batch);
  if (useb)
    gemm_tile_kernel<T, TA, TB, true><<<g, NT, 0, st>>>(m, n, k, alpha, A, lda, sA, B, ldb, sB,
                                                       beta, C, ldc, sC);
  else
    gemm_tile_kernel<T, TA, TB, false><<<g, NT, 0, st>>>(m, n, k, alpha, A, lda, sA, B, ldb, sB,
                                                        beta, C, ldc, sC);
}

// lower-triangle tiles only: blockIdx.x enumerates tile pairs (ti >= tj).
// SYRK = true: M = A - P Pᵀ (Q unused); else M = A - (P Qᵀ + Q Pᵀ).
// MERGE (with SYRK): the result of node z is also written, both triangles, into
// diagonal block z & 1 (offset (z & 1) m) of parent block z / 2 of PA (ld ldpa,
// stride sPA): the merge of Alg. 2 as the epilogue of the last Schur update.
template <typename T, bool SYRK = false, bool MERGE = false>
__global__ void __launch_bounds__(NT)
syr2k_lower_kernel(int m, int k, const T* A, int lda, long long sA, const T* __restrict__ P,
                   int ldp, long long sP, const T* __restrict__ Q, int ldq, long long sQ, T* M,
                   int ldm, long long sM, T* PA = nullptr, int ldpa = 0, long long sPA = 0) {
  __shared__ T Pi[BK][BM + 1], Qi[BK][BM + 1], Pj[BK][BN + 1], Qj[BK][BN + 1];
  const long long bz = blockIdx.y;
  A += bz * sA;
  P += bz * sP;
  Q += bz * sQ;
  M += bz * sM;
  // decode tile pair
  int t = blockIdx.x, ti = 0;
  while (t > ti) { t -= ti + 1; ++ti; }
  const int tj = t;
  const int i0 = ti * BM, j0 = tj * BN;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
  for (int k0 = 0; k0 < k; k0 += BK) {
#pragma unroll
    for (int e0 = 0; e0 < BM * BK; e0 += NT) {
      const int e = e0 + threadIdx.x;
      const int i = e % BM, kk = e / BM;
      const int gk = k0 + kk;
      const int gi = i0 + i, gj = j0 + i;
      const bool okk = gk < k;
      Pi[kk][i] = (okk && gi < m) ? P[gi + (long long)gk * ldp] : T(0);
      Pj[kk][i] = (okk && gj < m) ? P[gj + (long long)gk * ldp] : T(0);
      if (!SYRK) {
        Qi[kk][i] = (okk && gi < m) ? Q[gi + (long long)gk * ldq] : T(0);
        Qj[kk][i] = (okk && gj < m) ? Q[gj + (long long)gk * ldq] : T(0);
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T pa[4], qa[4], pb[4], qb[4];
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        pa[s] = Pi[kk][tx + 16 * s];
        pb[s] = Pj[kk][ty + 16 * s];
        if (!SYRK) {
          qa[s] = Qi[kk][tx + 16 * s];
          qb[s] = Qj[kk][ty + 16 * s];
        }
      }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (SYRK) {
            acc[p][q] = fma(pa[p], pb[q], acc[p][q]);
          } else {
            acc[p][q] = fma(pa[p], qb[q], acc[p][q]);
            acc[p][q] = fma(qa[p], pb[q], acc[p][q]);
          }
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int gj = j0 + ty + 16 * q;
    if (gj >= m) continue;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int gi = i0 + tx + 16 * p;
      if (gi >= m || gi < gj) continue;
      const T v = A[gi + (long long)gj * lda] - acc[p][q];
      M[gi + (long long)gj * ldm] = v;
      if (MERGE) {
        T* pa = PA + (bz >> 1) * sPA;
        const int off = (int)(bz & 1) * m;
        pa[(off + gi) + (long long)(off + gj) * ldpa] = v;
        if (gi != gj) pa[(off + gj) + (long long)(off + gi) * ldpa] = v;
      }
    }
  }
}

}  // namespace

template <typename T>
void gemm_batched(bool transA, bool transB, int m, int n, int k, T alpha, const T* A, int lda,
                  long long sA, const T* B, int ldb, long long sB, T beta, T* C, int ldc,
                  long long sC, int batch, cudaStream_t st) {
  if (m <= 0 || n <= 0 || batch <= 0) return;
  if (k <= 0) {
    // C = beta * C: express as a GEMM with a zero operand of depth 1 is not
    // possible without a buffer; callers never pass k = 0 with beta != 1.
    return;
  }
  if (!transA && !transB)
    launch_gemm<T, false, false>(m, n, k, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, batch, st);
  else if (transA && !transB)
    launch_gemm<T, true, false>(m, n, k, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, batch, st);
  else if (!transA && transB)
    launch_gemm<T, false, true>(m, n, k, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, batch, st);
  else
    launch_gemm<T, true, true>(m, n, k, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, batch, st);
}

template <typename T>
void syr2k_lower_batched(int m, int k, const T* A, int lda, long long sA, const T* P, int ldp,
                         long long sP, const T* Q, int ldq, long long sQ, T* M, int ldm,
                         long long sM, int batch, cudaStream_t st) {
  if (m <= 0 || batch <= 0) return;
  const int nt = (m + BM - 1) / BM;
  dim3 g(nt * (nt + 1) / 2, batch);
  syr2k_lower_kernel<T><<<g, NT, 0, st>>>(m, k, A, lda, sA, P, ldp, sP, Q, ldq, sQ, M, ldm, sM);
}

template <typename T>
void syrk_lower_batched(int m, int k, const T* A, int lda, long long sA, const T* P, int ldp,
                        long long sP, T* M, int ldm, long long sM, int batch, cudaStream_t st) {
  if (m <= 0 || batch <= 0) return;
  const int nt = (m + BM - 1) / BM;
  dim3 g(nt * (nt + 1) / 2, batch);
  syr2k_lower_kernel<T, true><<<g, NT, 0, st>>>(m, k, A, lda, sA, P, ldp, sP, P, ldp, sP, M, ldm,
                                                sM);
}

template <typename T>
void syrk_lower_merge_batched(int m, int k, const T* A, int lda, long long sA, const T* P,
                              int ldp, long long sP, T* M, int ldm, long long sM, T* PA, int ldpa,
                              long long sPA, int batch, cudaStream_t st) {
  if (m <= 0 || batch <= 0) return;
  const int nt = (m + BM - 1) / BM;
  dim3 g(nt * (nt + 1) / 2, batch);
  syr2k_lower_kernel<T, true, true><<<g, NT, 0, st>>>(m, k, A, lda, sA, P, ldp, sP, P, ldp, sP, M,
                                                      ldm, sM, PA, ldpa, sPA);
}

template void syrk_lower_merge_batched<double>(int, int, const double*, int, long long,
                                               const double*, int, long long, double*, int,
                                               long long, double*, int, long long, int,
                                               cudaStream_t);
template void syrk_lower_merge_batched<float>(int, int, const float*, int, long long, const float*,
                                              int, long long, float*, int, long long, float*, int,
                                              long long, int, cudaStream_t);
template void syrk_lower_batched<double>(int, int, const double*, int, long long, const double*,
                                         int, long long, double*, int, long long, int,
                                         cudaStream_t);
template void syrk_lower_batched<float>(int, int, const float*, int, long long, const float*, int,
                                        long long, float*, int, long long, int, cudaStream_t);

template void gemm_batched<double>(bool, bool, int, int, int, double, const double*, int, long long,
                                   const double*, int, long long, double, double*, int, long long,
                                   int, cudaStream_t);
template void gemm_batched<float>(bool, bool, int, int, int, float, const float*, int, long long,
                                  const float*, int, long long, float, float*, int, long long, int,
                                  cudaStream_t);
template void syr2k_lower_batched<double>(int, int, const double*, int, long long, const double*,
                                          int, long long, const double*, int, long long, double*,
                                          int, long long, int, cudaStream_t);
template void syr2k_lower_batched<float>(int, int, const float*, int, long long, const float*, int,
                                         long long, const float*, int, long long, float*, int,
                                         long long, int, cudaStream_t);
