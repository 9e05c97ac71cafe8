// Pair-of-FP32 batched GEMM and splitting kernels for the residual of the
// iterative refinement (r = b - A x, the HSS matvec of Sec. 5.1's construction
// error, evaluated with 48-bit significands on the FP32 pipe).
//
// Arithmetic (each step is an error-free transformation except where noted):
//  * product of a = ah + al and b = bh + bl:  p = fl(ah bh) and e = ah bh - p
//    (exact, by one FMA), plus the low part t = ah bl + al bh + e, rounded in
//    FP32 (relative size 2^-24 of p, so its rounding costs ~2^-48 of p); al bl
//    (~2^-48 of p) is dropped;
//  * accumulation into (S, C): two-sum s + err = S + p (Knuth) into S, and
//    C += err + t (rounded); every 4 terms the fast two-sum renormalisation
//    S = fl(S + C), C = C - (S_new - S_old) brings |C| back to <= ulp(S) / 2,
//    so C's own rounding stays near 2^-48 of S per step.
// Every operation is written with the _rn intrinsics, which the compiler never
// contracts into FMAs or reassociates: the transformations rely on the exact
// rounding of each step.
#include <algorithm>

#include "common.cuh"
#include "dfgemm.cuh"

namespace {

constexpr int DT = 128;   // threads: 32 lanes along rows x 4 warps along columns
constexpr int DK = 16;    // k per shared-memory stage

// (S, C) += a b without renormalisation: S takes the two-sum of the leading
// product, C the rounding errors and the low-order products
HSS_DEVINL void df_mac(float& S, float& C, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  const float e = __fmaf_rn(ah, bh, -p);
  const float t = __fmaf_rn(ah, bl, __fmaf_rn(al, bh, e));
  const float s = __fadd_rn(S, p);
  const float v = __fsub_rn(s, S);
  const float err = __fadd_rn(__fsub_rn(S, __fsub_rn(s, v)), __fsub_rn(p, v));
  C = __fadd_rn(C, __fadd_rn(err, t));
  S = s;
}

// fast two-sum renormalisation: |C| <= ulp(S) / 2 afterwards
HSS_DEVINL void df_norm(float& S, float& C) {
  const float s = __fadd_rn(S, C);
  C = __fsub_rn(C, __fsub_rn(s, S));
  S = s;
}

// (S, C) += (h, l)
HSS_DEVINL void df_add(float& S, float& C, float h, float l) {
  const float s = __fadd_rn(S, h);
  const float v = __fsub_rn(s, S);
  const float err = __fadd_rn(__fsub_rn(S, __fsub_rn(s, v)), __fsub_rn(h, v));
  const float c = __fadd_rn(__fadd_rn(C, l), err);
  S = __fadd_rn(s, c);
  C = __fsub_rn(c, __fsub_rn(S, s));
}

// 2^-ilogb(v) (1 for v = 0 or not finite): an exact power-of-two column scale
HSS_DEVINL double pow2_inv_scale(const double* colnorm, int j) {
  if (!colnorm) return 1.0;
  const double v = colnorm[j];
  if (!(v > 0.0) || !isfinite(v)) return 1.0;
  return ldexp(1.0, -ilogb(v));
}

// hi = fl32(a), lo = fl32(a - hi) (lo may be null: the conversion only).  Four
// elements a thread per step with 16-byte loads and stores where the three
// arrays are 16-byte aligned (the arena's sub-buffers are), so that the pass
// runs at the HBM rate; the first elements up to that alignment and the tail
// one at a time.
__global__ void df_split_kernel(const double* __restrict__ a, float* __restrict__ hi,
                                float* __restrict__ lo, long long n, long long head) {
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  auto one = [&](long long i) {
    const double v = a[i];
    const float h = __double2float_rn(v);
    hi[i] = h;
    if (lo) lo[i] = __double2float_rn(v - (double)h);
  };
  for (long long i = tid; i < head; i += stride) one(i);
  const long long nv = (n - head) / 4;
  const double2* a2 = reinterpret_cast<const double2*>(a + head);
  float4* h4 = reinterpret_cast<float4*>(hi + head);
  float4* l4 = lo ? reinterpret_cast<float4*>(lo + head) : nullptr;
  for (long long q = tid; q < nv; q += stride) {
    const double2 u = a2[2 * q], w = a2[2 * q + 1];
    const float4 h = make_float4(__double2float_rn(u.x), __double2float_rn(u.y),
                                 __double2float_rn(w.x), __double2float_rn(w.y));
    h4[q] = h;
    if (l4)
      l4[q] = make_float4(__double2float_rn(u.x - (double)h.x), __double2float_rn(u.y - (double)h.y),
                          __double2float_rn(w.x - (double)h.z), __double2float_rn(w.y - (double)h.w));
  }
  for (long long i = head + 4 * nv + tid; i < n; i += stride) one(i);
}

__global__ void df_split_cols_kernel(const double* __restrict__ a, int lda, int m, int nc,
                                     const double* __restrict__ colnorm, float* __restrict__ hi,
                                     float* __restrict__ lo, int ldo) {
  const int j = blockIdx.y;
  const double s = pow2_inv_scale(colnorm, j);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    const double v = a[i + (long long)j * lda] * s;
    const float h = __double2float_rn(v);
    hi[i + (long long)j * ldo] = h;
    lo[i + (long long)j * ldo] = __double2float_rn(v - (double)h);
  }
}

// One CTA: TBM = 32 RPT rows x 16 columns of one batch entry.  Thread (lane,
// w) accumulates rows lane + 32 p (p < RPT) and columns w + 4 q (q < 4).
template <int RPT, bool TA, bool ACC, bool OUT64>
__global__ void __launch_bounds__(DT)
df_gemm_kernel(int m, int n, int k, const float* __restrict__ Ah, const float* __restrict__ Al,
               int lda, long long sA, const float* __restrict__ Bh, const float* __restrict__ Bl,
               int ldb, long long sB, float* Ch, float* Cl, double* C64, int ldc64,
               const double* __restrict__ colnorm, int ldc, long long sC) {
  constexpr int TBM = 32 * RPT;
  __shared__ float Ash[DK][TBM + 1], Asl[DK][TBM + 1];
  __shared__ float Bsh[DK][17], Bsl[DK][17];
  const long long bz = blockIdx.y;
  Ah += bz * sA;
  Al += bz * sA;
  Bh += bz * sB;
  Bl += bz * sB;
  const int i0 = blockIdx.x * TBM;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  float S[RPT][4], C[RPT][4];
#pragma unroll
  for (int p = 0; p < RPT; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) S[p][q] = C[p][q] = 0.f;
  for (int k0 = 0; k0 < k; k0 += DK) {
#pragma unroll
    for (int e0 = 0; e0 < TBM * DK; e0 += DT) {
      const int e = e0 + tid;
      int i, kk;
      if (!TA) {
        i = e % TBM;
        kk = e / TBM;
      } else {
        kk = e % DK;
        i = e / DK;
      }
      const int gi = i0 + i, gk = k0 + kk;
      float vh = 0.f, vl = 0.f;
      if (gi < m && gk < k) {
        const long long off = TA ? gk + (long long)gi * lda : gi + (long long)gk * lda;
        vh = Ah[off];
        vl = Al[off];
      }
      Ash[kk][i] = vh;
      Asl[kk][i] = vl;
    }
#pragma unroll
    for (int e0 = 0; e0 < 16 * DK; e0 += DT) {
      const int e = e0 + tid;
      const int kk = e % DK, j = e / DK;
      const int gk = k0 + kk;
      float vh = 0.f, vl = 0.f;
      if (j < n && gk < k) {
        vh = Bh[gk + (long long)j * ldb];
        vl = Bl[gk + (long long)j * ldb];
      }
      Bsh[kk][j] = vh;
      Bsl[kk][j] = vl;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < DK; ++kk) {
      float ah[RPT], al[RPT], bh[4], bl[4];
#pragma unroll
      for (int p = 0; p < RPT; ++p) {
        ah[p] = Ash[kk][lane + 32 * p];
        al[p] = Asl[kk][lane + 32 * p];
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        bh[q] = Bsh[kk][w + 4 * q];
        bl[q] = Bsl[kk][w + 4 * q];
      }
#pragma unroll
      for (int p = 0; p < RPT; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) df_mac(S[p][q], C[p][q], ah[p], al[p], bh[q], bl[q]);
      if ((kk & 3) == 3) {   // every 4 terms
#pragma unroll
        for (int p = 0; p < RPT; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) df_norm(S[p][q], C[p][q]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int gj = w + 4 * q;
    if (gj >= n) continue;
    const double unscale = OUT64 ? 1.0 / pow2_inv_scale(colnorm, gj) : 1.0;
#pragma unroll
    for (int p = 0; p < RPT; ++p) {
      const int gi = i0 + lane + 32 * p;
      if (gi >= m) continue;
      const long long off = bz * sC + gi + (long long)gj * ldc;
      float s = S[p][q], c = C[p][q];
      df_norm(s, c);
      if (ACC) df_add(s, c, Ch[off], Cl[off]);
      if (OUT64) {
        C64[bz * sC + gi + (long long)gj * ldc64] = ((double)s + (double)c) * unscale;
      } else {
        Ch[off] = s;
        Cl[off] = c;
      }
    }
  }
}

template <int RPT, bool TA, bool ACC, bool OUT64>
void launch_df(int m, int n, int k, const float* Ah, const float* Al, int lda, long long sA,
               const float* Bh, const float* Bl, int ldb, long long sB, float* Ch, float* Cl,
               double* C64, int ldc64, const double* colnorm, int ldc, long long sC, int batch,
               cudaStream_t st) {
  dim3 g((m + 32 * RPT - 1) / (32 * RPT), batch);
  df_gemm_kernel<RPT, TA, ACC, OUT64><<<g, DT, 0, st>>>(m, n, k, Ah, Al, lda, sA, Bh, Bl, ldb, sB,
                                                        Ch, Cl, C64, ldc64, colnorm, ldc, sC);
}

template <int RPT>
void dispatch_df(bool transA, bool acc, bool out64, int m, int n, int k, const float* Ah,
                 const float* Al, int lda, long long sA, const float* Bh, const float* Bl, int ldb,
                 long long sB, float* Ch, float* Cl, double* C64, int ldc64,
                 const double* colnorm, int ldc, long long sC, int batch, cudaStream_t st) {
#define DF_CASE(TA_, ACC_, O64_)                                                              \
  if (transA == TA_ && acc == ACC_ && out64 == O64_) {                                        \
    launch_df<RPT, TA_, ACC_, O64_>(m, n, k, Ah, Al, lda, sA, Bh, Bl, ldb, sB, Ch, Cl, C64, \
                                    ldc64, colnorm, ldc, sC, batch, st);                      \
    return;                                                                                   \
  }
  DF_CASE(false, false, false)
  DF_CASE(false, true, false)
  DF_CASE(false, true, true)
  DF_CASE(false, false, true)
  DF_CASE(true, false, false)
  DF_CASE(true, true, false)
  DF_CASE(true, true, true)
  DF_CASE(true, false, true)
#undef DF_CASE
}

}  // namespace

cudaError_t launch_df_split(const double* a, float* hi, float* lo, long long n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  // elements before a (and hi, lo) reach 16-byte alignment together; one at a
  // time throughout when they never do
  const uintptr_t pa = reinterpret_cast<uintptr_t>(a), ph = reinterpret_cast<uintptr_t>(hi),
                  pl = reinterpret_cast<uintptr_t>(lo);
  long long head = n;
  for (long long k = 0; k < 4 && k < n; ++k)
    if ((pa + 8 * k) % 16 == 0 && (ph + 4 * k) % 16 == 0 && (!lo || (pl + 4 * k) % 16 == 0)) {
      head = k;
      break;
    }
  const long long blocks = std::min<long long>((n / 4 + 255) / 256 + 1, 152LL * 16);
  df_split_kernel<<<(int)blocks, 256, 0, st>>>(a, hi, lo, n, head);
  return cudaGetLastError();
}

cudaError_t launch_df_split_cols(const double* a, int lda, int m, int nc, const double* colnorm,
                                 float* hi, float* lo, int ldo, cudaStream_t st) {
  if (m <= 0 || nc <= 0) return cudaSuccess;
  dim3 g(std::min((m + 255) / 256, 152 * 4), nc);
  df_split_cols_kernel<<<g, 256, 0, st>>>(a, lda, m, nc, colnorm, hi, lo, ldo);
  return cudaGetLastError();
}

cudaError_t df_gemm(bool transA, int m, int n, int k, const float* Ah, const float* Al, int lda,
                    long long sA, const float* Bh, const float* Bl, int ldb, long long sB,
                    bool accumulate, float* Ch, float* Cl, double* C64, int ldc64,
                    const double* colnorm, int ldc, long long sC, int batch, cudaStream_t st) {
  if (m <= 0 || n <= 0 || batch <= 0) return cudaSuccess;
  if (n > 16 || batch > 65535 || (accumulate && (!Ch || !Cl)) || (!C64 && (!Ch || !Cl)))
    return cudaErrorInvalidValue;
  const bool out64 = C64 != nullptr;
  // 128-row tiles when they fill the GPU twice over, else 32-row tiles
  if ((long long)((m + 127) / 128) * batch >= 2 * 152)
    dispatch_df<4>(transA, accumulate, out64, m, n, k, Ah, Al, lda, sA, Bh, Bl, ldb, sB, Ch, Cl,
                   C64, ldc64, colnorm, ldc, sC, batch, st);
  else
    dispatch_df<1>(transA, accumulate, out64, m, n, k, Ah, Al, lda, sA, Bh, Bl, ldb, sB, Ch, Cl,
                   C64, ldc64, colnorm, ldc, sC, batch, st);
  return cudaGetLastError();
}
