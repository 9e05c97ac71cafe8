// Tensor-core (tcgen05, sm_103a) GEMM for the dense contractions of the
// diagonal product in the mixed-precision factorization (Alg. 2, in the
// compact-WY form): W = A V and the rank-2r update A - Y'Vᵀ - V Y'ᵀ.
//
// One CTA (4 warps) owns a 128 x 128 output tile; the accumulator lives in
// tensor memory (128 lanes x 128 FP32 columns).  The threads stage 128 x 32
// slabs of the FP32 operands into shared memory in the canonical K-major,
// no-swizzle core-matrix layout (8 rows x 16 bytes per core matrix; K-adjacent
// core matrices 128 B apart, 8-row groups 1 KB apart), converting them to the
// MMA input type on the way (TF32 or BF16, optionally split into hi + lo so
// that hi·hi + hi·lo + lo·hi keeps the product close to FP32 accuracy).  One
// thread issues tcgen05.mma; tcgen05.commit arrives on the stage's mbarrier
// when the MMAs that read it are done, which gates the refill of that stage
// (two stages).  The epilogue reads the tile with tcgen05.ld (each warp its 32
// TMEM lanes) and writes alpha·acc + beta·C_in, optionally only on and below
// the diagonal.  Every mbarrier wait is bounded: on expiry the kernel records
// HSS_ERR_TIMEOUT in the status word, stops issuing, waits (bounded) for the
// MMAs already issued, frees its tensor memory and returns.  The pipeline
// waits poll at most `wait_limit` times (set by the caller; 0 polls = give up
// at once); the final wait for issued MMAs always uses the long default, so
// that tensor memory is never released under a pending MMA.
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>

#include "common.cuh"
#include "tc_gemm.cuh"

namespace {

constexpr int TM = 128, TN = 128, TK = 32;   // CTA tile and K slab (elements)
constexpr int TC_THREADS = 128;
constexpr uint32_t kTmemCols = 128;
constexpr long long kWaitLimit = 1LL << 24;   // default polls before a wait gives up

HSS_DEVINL uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor: K-major, no swizzle
HSS_DEVINL uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;   // descriptor version of this architecture
  return d;                  // base offset 0, lbo mode 0, swizzle none
}

// instruction descriptor: D f32, A/B format (0 f16, 1 bf16, 2 tf32), K-major A and B
HSS_DEVINL uint32_t make_idesc(uint32_t ab_format, int m, int n) {
  return (1u << 4) | (ab_format << 7) | (ab_format << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(m >> 4) << 24);
}

HSS_DEVINL bool mbar_wait(uint32_t mbar, uint32_t parity, long long limit) {
  for (long long it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

template <typename E>
struct TcType;
template <>
struct TcType<float> {   // TF32 operands, stored as 32-bit words
  static constexpr uint32_t fmt = 2;
  static constexpr int kpi = 8;   // K per MMA instruction
  HSS_DEVINL static float hi(float x) {
    uint32_t u;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
    return __uint_as_float(u);
  }
  HSS_DEVINL static float conv(float x) { return x; }
};
template <>
struct TcType<__nv_bfloat16> {
  static constexpr uint32_t fmt = 1;
  static constexpr int kpi = 16;
  HSS_DEVINL static float hi(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
  HSS_DEVINL static __nv_bfloat16 conv(float x) { return __float2bfloat16_rn(x); }
};

// byte offset of element (row, k) of a 128 x TK slab in the core-matrix layout
template <typename E>
HSS_DEVINL uint32_t slab_offset(int row, int k) {
  constexpr int epc = 16 / sizeof(E);                  // elements per 16-byte core row
  constexpr uint32_t kcores = TK / epc;                // core matrices along K
  return ((uint32_t)(row >> 3) * kcores + (uint32_t)(k / epc)) * 128u + (uint32_t)(row & 7) * 16u +
         (uint32_t)(k % epc) * (uint32_t)sizeof(E);
}

// Stage rows [r0, r0+128) x k [k0, k0+TK) of an operand into the slab(s).
// mcontig: element (row, k) at X[row + k * ld]; otherwise at X[k + row * ld].
template <typename E, int NPASS>
HSS_DEVINL void stage(const float* X, int ld, bool mcontig, int rows_valid, int r0, int kvalid,
                      int k0, unsigned char* hi_slab, unsigned char* lo_slab) {
  const int tid = threadIdx.x;
  for (int e = tid; e < TM * TK; e += TC_THREADS) {
    int row, k;
    if (mcontig) { row = e % TM; k = e / TM; } else { k = e % TK; row = e / TK; }
    const int gr = r0 + row, gk = k0 + k;
    float v = 0.f;
    if (gr < rows_valid && gk < kvalid) v = mcontig ? X[gr + (long long)gk * ld] : X[gk + (long long)gr * ld];
    const uint32_t off = slab_offset<E>(row, k);
    const float h = TcType<E>::hi(v);
    *reinterpret_cast<E*>(hi_slab + off) = TcType<E>::conv(h);
    if (NPASS == 3) *reinterpret_cast<E*>(lo_slab + off) = TcType<E>::conv(v - h);
  }
}

struct Term {
  const float* A;
  int lda;
  long long sA;
  bool a_mcontig;
  const float* B;
  int ldb;
  long long sB;
  bool b_ncontig;   // element (n, k) of B at B[n + k * ldb] (else at B[k + n * ldb])
  int K;
};

template <typename E, int NPASS>
__global__ void __launch_bounds__(TC_THREADS)
tc_gemm_kernel(int M, int N, Term t1, Term t2, float alpha, float beta, const float* Cin,
               int ldcin, long long sCin, float* C, int ldc, long long sC, int lower_only,
               int tiles_m, int* status, long long wait_limit) {
  constexpr int NSLAB = (NPASS == 3) ? 4 : 2;                  // A hi/lo, B hi/lo
  constexpr uint32_t SLAB = TM * TK * sizeof(E);               // bytes per slab
  constexpr uint32_t STAGE = NSLAB * SLAB;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_base_s;
  __shared__ int abort_s;

  const int tid = threadIdx.x, warp = tid >> 5;
  const long long bz = blockIdx.z;
  // tile coordinates (lower_only: enumerate tile pairs tm >= tn)
  int tm, tn;
  if (lower_only) {
    int t = blockIdx.x, ti = 0;
    while (t > ti) { t -= ti + 1; ++ti; }
    tm = ti;
    tn = t;
  } else {
    tm = blockIdx.x % tiles_m;
    tn = blockIdx.x / tiles_m;
  }
  const int m0 = tm * TM, n0 = tn * TN;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&tmem_base_s)), "r"(kTmemCols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&mbar[0])), "r"(1) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&mbar[1])), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    abort_s = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base_s;

  const int k1s = (t1.K + TK - 1) / TK, k2s = (t2.K + TK - 1) / TK;
  const int nk = k1s + k2s;
  const uint32_t idesc = make_idesc(TcType<E>::fmt, TM, TN);
  int issued = 0;
  for (int kc = 0; kc < nk; ++kc) {
    const int s = kc & 1;
    unsigned char* st = smem + s * STAGE;
    if (kc >= 2) {   // the MMAs that read this stage two slabs ago are done
      if (tid == 0 && !mbar_wait(smem_u32(&mbar[s]), (uint32_t)(((kc >> 1) - 1) & 1), wait_limit))
        abort_s = 1;
      __syncthreads();
      if (abort_s) break;
    }
    const Term& t = (kc < k1s) ? t1 : t2;
    const int k0 = ((kc < k1s) ? kc : kc - k1s) * TK;
    stage<E, NPASS>(t.A + bz * t.sA, t.lda, t.a_mcontig, M, m0, t.K, k0, st,
                    st + 2 * SLAB);
    stage<E, NPASS>(t.B + bz * t.sB, t.ldb, t.b_ncontig, N, n0, t.K, k0, st + SLAB,
                    st + 3 * SLAB);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a_hi = smem_u32(st), b_hi = smem_u32(st + SLAB);
      const uint32_t a_lo = smem_u32(st + 2 * SLAB), b_lo = smem_u32(st + 3 * SLAB);
      constexpr int kpi = TcType<E>::kpi;
      constexpr uint32_t step = (uint32_t)(kpi * sizeof(E) / 16) * 128u;   // bytes per MMA K-step
      constexpr uint32_t sbo = (uint32_t)(TK * sizeof(E) / 16) * 128u;     // 8-row group pitch
      for (int ks = 0; ks < TK / kpi; ++ks) {
        const uint32_t o = ks * step;
        const uint32_t pa[3] = {a_hi, a_hi, a_lo};
        const uint32_t pb[3] = {b_hi, b_lo, b_hi};
        for (int p = 0; p < NPASS; ++p) {
          const uint64_t ad = make_desc(pa[p] + o, 128, sbo);
          const uint64_t bd = make_desc(pb[p] + o, 128, sbo);
          const uint32_t acc = (kc > 0 || ks > 0 || p > 0) ? 1u : 0u;
          if (TcType<E>::fmt == 2)
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                :: "r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(acc) : "memory");
          else
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                :: "r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(acc) : "memory");
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                   :: "r"(smem_u32(&mbar[s])) : "memory");
    }
    issued = kc + 1;
  }
  // wait for every issued MMA (commit tracks all earlier MMAs of the thread)
  if (tid == 0 && issued > 0) {
    const int last = issued - 1;
    if (!mbar_wait(smem_u32(&mbar[last & 1]), (uint32_t)((last >> 1) & 1), kWaitLimit))
      abort_s = 2;
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (abort_s) {
    if (tid == 0) report_failure(status, -6 /*TIMEOUT*/, -1, (int)blockIdx.x, abort_s);
  } else {
    // epilogue: warp w reads TMEM lanes 32w .. 32w+31 (tile rows), 32 columns at a time
    const int row = m0 + warp * 32 + (tid & 31);
    const float* cin = Cin ? Cin + bz * sCin : nullptr;
    float* c = C + bz * sC;
    for (int c0 = 0; c0 < TN; c0 += 32) {
      uint32_t v[32];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
          "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
          "%28, %29, %30, %31}, [%32];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
            "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
            "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
            "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
            "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
            "=r"(v[31])
          : "r"(taddr)
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row < M) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int col = n0 + c0 + j;
          if (col >= N || (lower_only && col > row)) continue;
          float out = alpha * __uint_as_float(v[j]);
          if (cin) out = fmaf(beta, cin[row + (long long)col * ldcin], out);
          c[row + (long long)col * ldc] = out;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kTmemCols)
                 : "memory");
}

template <typename E, int NPASS>
cudaError_t launch(int M, int N, const Term& t1, const Term& t2, float alpha, float beta,
                   const float* Cin, int ldcin, long long sCin, float* C, int ldc, long long sC,
                   bool lower, int batch, int* status, long long wait_limit, cudaStream_t st) {
  constexpr int NSLAB = (NPASS == 3) ? 4 : 2;
  // at least 57 KB so that no more than 4 CTAs (4 x 128 TMEM columns) share an SM
  const size_t smem = std::max<size_t>(2 * (size_t)NSLAB * TM * TK * sizeof(E), 57 * 1024);
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(tc_gemm_kernel<E, NPASS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
      return cudaErrorInvalidConfiguration;
    attr = true;
  }
  const int tiles_m = (M + TM - 1) / TM, tiles_n = (N + TN - 1) / TN;
  const int tiles = lower ? tiles_m * (tiles_m + 1) / 2 : tiles_m * tiles_n;
  dim3 g(tiles, 1, batch);
  tc_gemm_kernel<E, NPASS><<<g, TC_THREADS, smem, st>>>(M, N, t1, t2, alpha, beta, Cin, ldcin, sCin,
                                                       C, ldc, sC, lower ? 1 : 0, tiles_m, status,
                                                       wait_limit);
  return cudaGetLastError();
}

}  // namespace

cudaError_t tc_gemm(TcMode mode, int M, int N, int K, const float* A, int lda, long long sA,
                    const float* B, int ldb, long long sB, bool b_ncontig, float* C, int ldc,
                    long long sC, int batch, int* status, long long wait_budget,
                    cudaStream_t st) {
  const long long wl = wait_budget > 0 ? wait_budget : (wait_budget < 0 ? 0 : kWaitLimit);
  Term t1{A, lda, sA, true, B, ldb, sB, b_ncontig, K};
  Term t2{A, lda, sA, true, B, ldb, sB, b_ncontig, 0};
  switch (mode) {
    case TcMode::TF32: return launch<float, 1>(M, N, t1, t2, 1.f, 0.f, nullptr, 0, 0, C, ldc, sC, false, batch, status, wl, st);
    case TcMode::TF32x3: return launch<float, 3>(M, N, t1, t2, 1.f, 0.f, nullptr, 0, 0, C, ldc, sC, false, batch, status, wl, st);
    case TcMode::BF16: return launch<__nv_bfloat16, 1>(M, N, t1, t2, 1.f, 0.f, nullptr, 0, 0, C, ldc, sC, false, batch, status, wl, st);
    case TcMode::BF16x3: return launch<__nv_bfloat16, 3>(M, N, t1, t2, 1.f, 0.f, nullptr, 0, 0, C, ldc, sC, false, batch, status, wl, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t tc_syr2k_lower(TcMode mode, int m, int k, const float* A, int lda, long long sA,
                           const float* P, int ldp, long long sP, const float* Q, int ldq,
                           long long sQ, float* Mout, int ldm, long long sM, int batch, int* status,
                           long long wait_budget, cudaStream_t st) {
  const long long wl = wait_budget > 0 ? wait_budget : (wait_budget < 0 ? 0 : kWaitLimit);
  // Mout = A - (P Qᵀ + Q Pᵀ) on and below the diagonal: two terms along K,
  // operand A = P then Q (row-contiguous), operand B(n, k) = Q(n, k) then P(n, k)
  Term t1{P, ldp, sP, true, Q, ldq, sQ, true, k};
  Term t2{Q, ldq, sQ, true, P, ldp, sP, true, k};
  switch (mode) {
    case TcMode::TF32: return launch<float, 1>(m, m, t1, t2, -1.f, 1.f, A, lda, sA, Mout, ldm, sM, true, batch, status, wl, st);
    case TcMode::TF32x3: return launch<float, 3>(m, m, t1, t2, -1.f, 1.f, A, lda, sA, Mout, ldm, sM, true, batch, status, wl, st);
    case TcMode::BF16: return launch<__nv_bfloat16, 1>(m, m, t1, t2, -1.f, 1.f, A, lda, sA, Mout, ldm, sM, true, batch, status, wl, st);
    case TcMode::BF16x3: return launch<__nv_bfloat16, 3>(m, m, t1, t2, -1.f, 1.f, A, lda, sA, Mout, ldm, sM, true, batch, status, wl, st);
  }
  return cudaErrorInvalidValue;
}
