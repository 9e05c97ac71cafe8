// Tensor-core (tcgen05, sm_103a) GEMM for the dense contractions of the
// diagonal product in the mixed-precision factorization (Alg. 2, in the
// compact-WY form): W = A V and the rank-2r update A - Y'Vᵀ - V Y'ᵀ.
//
// Operands are packed once per level (tc_pack_kernel) into slabs of 128 rows x
// 32 K elements in the canonical K-major, no-swizzle core-matrix layout of the
// MMA (8 rows x 16 bytes per core matrix; K-adjacent core matrices 128 B apart,
// 8-row groups one K-row of core matrices apart), converted to the MMA input
// type and, in the x3 modes, split into hi + lo parts (hi·hi + hi·lo + lo·hi
// is accumulated).  The GEMM kernel is persistent (one CTA per SM, 6 warps,
// looping over the 128 x 128 output tiles of every node): a producer warp
// streams the slabs through a ring of shared-memory stages with cp.async.bulk
// (the TMA engine, completion counted in bytes on each stage's "full"
// mbarrier); an MMA warp issues tcgen05.mma into one of two FP32 accumulators
// in tensor memory, commits each stage to its "empty" mbarrier (which gates its
// refill) and each finished tile to the epilogue; four epilogue warps read the
// tile with tcgen05.ld (each its 32 TMEM lanes) and write alpha·acc +
// beta·C_in, optionally only on and below the diagonal, while the next tile's
// MMAs run into the other accumulator.
//
// Every wait is bounded.  The pipeline's waits poll at most `wait_limit` times
// (set by the caller; 0 polls = give up at once): on expiry the kernel records
// HSS_ERR_TIMEOUT in the status word, stops issuing, waits with the long
// default for the copies and MMAs it has issued, frees its tensor memory and
// returns without writing the remaining tiles.
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>

#include "common.cuh"
#include "tc_gemm.cuh"

namespace {

constexpr int TM = 128, TN = 128, TK = 32;   // CTA tile and K slab (elements)
constexpr uint32_t kTmemCols = 128;
constexpr long long kWaitLimit = 1LL << 24;   // default polls before a wait gives up
constexpr int kSmemBudget = 200 * 1024;       // dynamic shared memory of the ring

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

HSS_DEVINL void mbar_init(uint32_t mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}

HSS_DEVINL void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes)
               : "memory");
}

// global -> shared bulk copy on the TMA engine; completes `bytes` on mbar
HSS_DEVINL void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(dst),
      "l"(src), "r"(bytes), "r"(mbar)
      : "memory");
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

template <typename E>
constexpr uint32_t slab_bytes() {
  return (uint32_t)(TM * TK * sizeof(E));
}

// Pack rows [rb 128, rb 128 + 128) x K [kb 32, kb 32 + 32) of an operand into
// one slab (and its lo slab right after it), core-matrix order.  The operand's
// element (row, k) is, for k < K1, src1[k + row ld1] (kcontig) or
// src1[row + k ld1], else the same in src2 with k - K1; zero outside rows x K.
// Packed layout per node: [row block][K block][part][slab].  One CTA per slab.
template <typename E, int NPARTS>
__global__ void __launch_bounds__(256)
tc_pack_kernel(const float* __restrict__ s1, int ld1, long long ss1, const float* __restrict__ s2,
               int ld2, long long ss2, int K1, int K, int kcontig, int rows, int nkb,
               unsigned char* __restrict__ out, long long s_out) {
  __shared__ float t[TM][TK + 1];
  const long long node = blockIdx.y;
  const int rb = blockIdx.x / nkb, kb = blockIdx.x % nkb;
  const int r0 = rb * TM, k0 = kb * TK;
  const int tid = threadIdx.x;
  for (int e = tid; e < TM * TK; e += 256) {
    int row, kk;
    if (kcontig) {
      kk = e % TK;
      row = e / TK;
    } else {
      row = e % TM;
      kk = e / TM;
    }
    const int gr = r0 + row, gk = k0 + kk;
    float v = 0.f;
    if (gr < rows && gk < K) {
      const bool first = gk < K1;
      const float* s = first ? s1 + node * ss1 : s2 + node * ss2;
      const int ld = first ? ld1 : ld2;
      const int k = first ? gk : gk - K1;
      v = kcontig ? s[k + (long long)gr * ld] : s[gr + (long long)k * ld];
    }
    t[row][kk] = v;
  }
  __syncthreads();
  constexpr int epc = 16 / sizeof(E);   // elements per 16-byte core row
  constexpr int kcores = TK / epc;      // core matrices along K
  E* hi = reinterpret_cast<E*>(out + node * s_out +
                               (size_t)blockIdx.x * NPARTS * slab_bytes<E>());
  E* lo = hi + TM * TK;
  for (int o = tid; o < TM * TK; o += 256) {
    const int core = o / (8 * epc), within = o % (8 * epc);
    const int row = (core / kcores) * 8 + within / epc;
    const int kk = (core % kcores) * epc + within % epc;
    const float v = t[row][kk];
    const float h = TcType<E>::hi(v);
    hi[o] = TcType<E>::conv(h);
    if (NPARTS == 2) lo[o] = TcType<E>::conv(v - h);
  }
}

}  // namespace

namespace {

// Persistent, warp-specialised GEMM over a list of output tiles: item it of
// the list is tile (it % tiles) of node (it / tiles); CTA x takes items x,
// x + gridDim.x, ...  Warp 0 (one lane) streams the A and B slabs of each item
// into the ring (cp.async.bulk, bytes counted on the stage's "full" barrier;
// a stage is refilled once the MMAs that read it have committed to its "empty"
// barrier).  Warp 1 (one lane) issues the MMAs of item i into tensor-memory
// accumulator i & 1 (two of TN columns each) and commits the item to "accf";
// warps 2..9 (lane quarter warp & 3 of tensor memory, and one half of the
// tile's columns, each) read the accumulator, release it on "acce" and write
// alpha·acc + beta·C_in, while the MMAs of item i + 1 run into the other
// accumulator.  Eight epilogue warps keep twice the global loads and stores in
// flight of four, so the epilogue of a tile is not longer than its MMAs.
//
// Every wait polls at most wait_limit times.  A role whose wait expires records
// HSS_ERR_TIMEOUT and raises the CTA's abort flag; every role leaves its loop
// at its next wait.  Before the CTA exits, the copies it issued have landed
// (the producer waits for the stages the MMA warp did not consume) and the MMAs
// it issued have completed (a final commit waited on with the long default),
// and then its tensor memory is freed.
constexpr int TC_WARPS = 10;

template <typename E, int NPASS>
__global__ void __launch_bounds__(TC_WARPS * 32)
tc_gemm_kernel(int M, int N, int nk, const unsigned char* __restrict__ Ap, long long sAp,
               const unsigned char* __restrict__ Bp, long long sBp, float alpha, float beta,
               const float* Cin, int ldcin, long long sCin, float* C, int ldc, long long sC,
               int lower_only, int tiles_m, int tiles, long long items, int stages, int* status,
               long long wait_limit, int b_krot) {
  constexpr int NPARTS = (NPASS == 3) ? 2 : 1;
  constexpr uint32_t SLAB = slab_bytes<E>();
  constexpr uint32_t OPER = NPARTS * SLAB;    // one operand's slab(s) of a stage
  constexpr uint32_t STAGE = 2 * OPER;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[8], empty[8], accf[2], acce[2], done;
  __shared__ uint32_t tmem_base_s;
  __shared__ volatile int abort_s;
  __shared__ long long consumed_s;   // slabs whose "full" wait the MMA warp passed

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // item -> (node, tm, tn)
  auto item_tile = [&](long long it, long long* node, int* tm, int* tn) {
    *node = it / tiles;
    const int t0 = (int)(it % tiles);
    if (lower_only) {   // tile pairs tm >= tn
      int t = t0, ti = 0;
      while (t > ti) {
        t -= ti + 1;
        ++ti;
      }
      *tm = ti;
      *tn = t;
    } else {
      *tm = t0 % tiles_m;
      *tn = t0 / tiles_m;
    }
  };

  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base_s)),
                 "r"(2 * kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int q = 0; q < stages; ++q) {
      mbar_init(smem_u32(&full[q]), 1);
      mbar_init(smem_u32(&empty[q]), 1);
    }
    for (int q = 0; q < 2; ++q) {
      mbar_init(smem_u32(&accf[q]), 1);
      mbar_init(smem_u32(&acce[q]), TC_WARPS - 2);   // one arrival per epilogue warp
    }
    mbar_init(smem_u32(&done), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    abort_s = 0;
    consumed_s = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base_s;
  const uint32_t sbase = smem_u32(smem);
  long long issued = 0;   // producer: slabs whose copies were issued

  if (warp == 0 && lane == 0) {
    // ---------------------------------------------------------------- producer
    long long g = 0;
    for (long long it = blockIdx.x; it < items && !abort_s; it += gridDim.x) {
      long long node;
      int tm, tn;
      item_tile(it, &node, &tm, &tn);
      const unsigned char* a_src = Ap + node * sAp + (size_t)tm * nk * OPER;
      const unsigned char* b_src = Bp + node * sBp + (size_t)tn * nk * OPER;
      for (int kc = 0; kc < nk; ++kc, ++g) {
        const int q = (int)(g % stages);
        const long long use = g / stages;
        if (use > 0 && !mbar_wait(smem_u32(&empty[q]), (uint32_t)((use - 1) & 1), wait_limit)) {
          report_failure(status, -6 /*TIMEOUT*/, -1, (int)blockIdx.x, 1);
          abort_s = 1;
          break;
        }
        if (abort_s) break;
        const uint32_t dst = sbase + q * STAGE, fb = smem_u32(&full[q]);
        mbar_expect_tx(fb, STAGE);
        bulk_g2s(dst, a_src + (size_t)kc * OPER, OPER, fb);
        // b_krot: B is A's packed buffer with its K slabs rotated (the rank-2r
        // update's right operand [Q P] is the left one [P Q] with halves swapped)
        const int kb = b_krot ? (kc + b_krot) % nk : kc;
        bulk_g2s(dst + OPER, b_src + (size_t)kb * OPER, OPER, fb);
        issued = g + 1;
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------------------------------------------------------- MMA issue
    const uint32_t idesc = make_idesc(TcType<E>::fmt, TM, TN);
    constexpr int kpi = TcType<E>::kpi;
    constexpr uint32_t step = (uint32_t)(kpi * sizeof(E) / 16) * 128u;   // bytes per MMA K-step
    constexpr uint32_t sbo = (uint32_t)(TK * sizeof(E) / 16) * 128u;     // 8-row group pitch
    long long g = 0, i = 0;
    for (long long it = blockIdx.x; it < items && !abort_s; it += gridDim.x, ++i) {
      const int a = (int)(i & 1);
      if (i >= 2 && !mbar_wait(smem_u32(&acce[a]), (uint32_t)(((i >> 1) - 1) & 1), wait_limit)) {
        report_failure(status, -6 /*TIMEOUT*/, -1, (int)blockIdx.x, 2);
        abort_s = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t acc_addr = tmem + (uint32_t)(a * kTmemCols);
      bool ok = true;
      for (int kc = 0; kc < nk; ++kc, ++g) {
        const int q = (int)(g % stages);
        if (!mbar_wait(smem_u32(&full[q]), (uint32_t)((g / stages) & 1), wait_limit) ||
            abort_s) {
          if (!abort_s) report_failure(status, -6 /*TIMEOUT*/, -1, (int)blockIdx.x, 3);
          abort_s = 1;
          ok = false;
          break;
        }
        consumed_s = g + 1;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t a_hi = sbase + q * STAGE, b_hi = a_hi + OPER;
        const uint32_t a_lo = a_hi + SLAB, b_lo = b_hi + SLAB;
#pragma unroll
        for (int ks = 0; ks < TK / kpi; ++ks) {
          const uint32_t o = ks * step;
          const uint32_t pa[3] = {a_hi, a_hi, a_lo};
          const uint32_t pb[3] = {b_hi, b_lo, b_hi};
#pragma unroll
          for (int p = 0; p < NPASS; ++p) {
            const uint64_t ad = make_desc(pa[p] + o, 128, sbo);
            const uint64_t bd = make_desc(pb[p] + o, 128, sbo);
            const uint32_t acc = (kc > 0 || ks > 0 || p > 0) ? 1u : 0u;
            if (TcType<E>::fmt == 2)
              asm volatile(
                  "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                  " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(acc_addr),
                  "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                  : "memory");
            else
              asm volatile(
                  "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                  " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(acc_addr),
                  "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                  : "memory");
          }
        }
        // the stage is free once these MMAs have read it
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&empty[q]))
            : "memory");
      }
      if (!ok) break;
      // the accumulator is complete once every MMA of the item has finished
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_u32(&accf[a]))
          : "memory");
    }
  } else if (warp >= 2) {
    // ---------------------------------------------------------------- epilogue
    const int quarter = warp & 3;   // tensor-memory lanes 32 quarter .. 32 quarter + 31
    const int half = (warp - 2) >> 2;   // columns [64 half, 64 half + 64) of the tile
    long long i = 0;
    for (long long it = blockIdx.x; it < items; it += gridDim.x, ++i) {
      const int a = (int)(i & 1);
      int got = 1;
      if (lane == 0) got = mbar_wait(smem_u32(&accf[a]), (uint32_t)((i >> 1) & 1), wait_limit) &&
                           !abort_s;
      got = __shfl_sync(0xffffffffu, got, 0);
      __syncwarp();
      if (!got) {
        if (lane == 0 && !abort_s) {
          report_failure(status, -6 /*TIMEOUT*/, -1, (int)blockIdx.x, 4);
          abort_s = 1;
        }
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      long long node;
      int tm, tn;
      item_tile(it, &node, &tm, &tn);
      const int row = tm * TM + quarter * 32 + lane, n0 = tn * TN;
      const float* cin = Cin ? Cin + node * sCin : nullptr;
      float* c = C + node * sC;
      const int cb = half * (TN / 2), ce = min(cb + TN / 2, N - n0);
      if (ce <= cb) {   // no columns of this half in the tile: release at once
        __syncwarp();
        if (lane == 0)
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acce[a]))
                       : "memory");
        continue;
      }
      for (int c0 = cb; c0 < ce; c0 += 32) {
        uint32_t v[32];
        const uint32_t taddr =
            tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(a * kTmemCols + c0);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, "
            "%10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, "
            "%27, %28, %29, %30, %31}, [%32];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
              "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
              "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
              "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
              "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
              "=r"(v[31])
            : "r"(taddr)
            : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (c0 + 32 >= ce) {
          // this warp's last read of the accumulator: hand it back
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          __syncwarp();
          if (lane == 0)
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acce[a]))
                         : "memory");
        }
        // a chunk inside N and strictly below the diagonal (or a full matrix)
        // needs no per-element test
        const bool whole = n0 + c0 + 32 <= N && (!lower_only || tm > tn);
        if (whole && row < M) {
          float* cr = c + row + (long long)(n0 + c0) * ldc;
          if (cin) {
            const float* cir = cin + row + (long long)(n0 + c0) * ldcin;
            float ci[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) ci[j] = cir[(long long)j * ldcin];
#pragma unroll
            for (int j = 0; j < 32; ++j)
              cr[(long long)j * ldc] = fmaf(beta, ci[j], alpha * __uint_as_float(v[j]));
          } else {
#pragma unroll
            for (int j = 0; j < 32; ++j) cr[(long long)j * ldc] = alpha * __uint_as_float(v[j]);
          }
        } else if (row < M) {
          // C_in may be C itself: each element is read and written by this
          // thread only, so the 32 reads go out together before any write
          float ci[32];
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int col = n0 + c0 + j;
            const bool ok = cin && col < N && !(lower_only && col > row);
            ci[j] = ok ? cin[row + (long long)col * ldcin] : 0.f;
          }
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int col = n0 + c0 + j;
            if (col >= N || (lower_only && col > row)) continue;
            float out = alpha * __uint_as_float(v[j]);
            if (cin) out = fmaf(beta, ci[j], out);
            c[row + (long long)col * ldc] = out;
          }
        }
      }
    }
  }
  __syncthreads();
  if (abort_s && warp == 0 && lane == 0) {
    // copies still in flight land before the CTA may exit
    for (long long g = consumed_s; g < issued; ++g)
      mbar_wait(smem_u32(&full[g % stages]), (uint32_t)((g / stages) & 1), kWaitLimit);
  }
  if (warp == 1 && lane == 0) {
    // every MMA issued so far completes before the tensor memory is freed
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(&done))
        : "memory");
    if (!mbar_wait(smem_u32(&done), 0u, kWaitLimit))
      report_failure(status, -6 /*TIMEOUT*/, -1, (int)blockIdx.x, 5);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(2 * kTmemCols)
                 : "memory");
}

}  // namespace

namespace {

template <typename E, int NPASS>
size_t packed_bytes(int rows, int K, int batch) {
  constexpr int NPARTS = (NPASS == 3) ? 2 : 1;
  const size_t slabs = (size_t)((rows + TM - 1) / TM) * ((K + TK - 1) / TK);
  return slabs * NPARTS * slab_bytes<E>() * (size_t)batch;
}

template <typename E, int NPASS>
void pack(const TcOperand& x, int rows, int K, int batch, unsigned char* out, cudaStream_t st) {
  constexpr int NPARTS = (NPASS == 3) ? 2 : 1;
  const int nkb = (K + TK - 1) / TK, nrb = (rows + TM - 1) / TM;
  const long long s_out = (long long)nrb * nkb * NPARTS * slab_bytes<E>();
  const float* s2 = x.src2 ? x.src2 : x.src1;
  tc_pack_kernel<E, NPARTS><<<dim3(nrb * nkb, batch), 256, 0, st>>>(
      x.src1, x.ld1, x.s1, s2, x.src2 ? x.ld2 : x.ld1, x.src2 ? x.s2 : x.s1, x.K1 ? x.K1 : K, K,
      x.kcontig ? 1 : 0, rows, nkb, out, s_out);
}

// b_rot_of_a: b is a with its two K halves swapped (K even, each half a whole
// number of K slabs, M = N): B is read from A's packed buffer, K-rotated.
template <typename E, int NPASS>
cudaError_t run(int M, int N, int K, const TcOperand& a, const TcOperand& b, float alpha,
                float beta, const float* Cin, int ldcin, long long sCin, float* C, int ldc,
                long long sC, bool lower, int batch, void* ws, size_t ws_bytes, int* status,
                long long wait_limit, cudaStream_t st, bool b_rot_of_a = false) {
  constexpr int NPARTS = (NPASS == 3) ? 2 : 1;
  constexpr uint32_t STAGE = 2 * NPARTS * slab_bytes<E>();
  const bool rot = b_rot_of_a && M == N && K % (2 * TK) == 0;
  const size_t pa = packed_bytes<E, NPASS>(M, K, batch),
               pb = rot ? 0 : packed_bytes<E, NPASS>(N, K, batch);
  if (M <= 0 || N <= 0 || K <= 0 || batch <= 0) return cudaSuccess;
  if (pa + pb > ws_bytes || batch > 65535) return cudaErrorInvalidValue;
  unsigned char* Ap = static_cast<unsigned char*>(ws);
  unsigned char* Bp = rot ? Ap : Ap + pa;
  pack<E, NPASS>(a, M, K, batch, Ap, st);
  if (!rot) pack<E, NPASS>(b, N, K, batch, Bp, st);
  const int stages = std::min<int>(8, kSmemBudget / STAGE);
  const size_t smem = (size_t)stages * STAGE;
  static size_t attr = 0;
  static int sms = 0, per_sm = 0;
  if (smem > attr) {
    if (cudaFuncSetAttribute(tc_gemm_kernel<E, NPASS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
      return cudaErrorInvalidConfiguration;
    attr = smem;
    per_sm = 0;
  }
  if (!sms) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return cudaErrorInvalidConfiguration;
  }
  if (!per_sm) {
    // resident CTAs per SM: shared memory, and tensor memory (512 columns an SM)
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tc_gemm_kernel<E, NPASS>,
                                                      TC_WARPS * 32, smem) != cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
    per_sm = std::min<int>(per_sm, 512 / (2 * (int)kTmemCols));
  }
  const int nk = (K + TK - 1) / TK;
  const int tiles_m = (M + TM - 1) / TM, tiles_n = (N + TN - 1) / TN;
  const int tiles = lower ? tiles_m * (tiles_m + 1) / 2 : tiles_m * tiles_n;
  const long long items = (long long)tiles * batch;
  const int grid = (int)std::min<long long>(items, (long long)sms * per_sm);
  tc_gemm_kernel<E, NPASS><<<grid, TC_WARPS * 32, smem, st>>>(
      M, N, nk, Ap, (long long)(pa / batch), Bp, (long long)((rot ? pa : pb) / batch), alpha,
      beta, Cin, ldcin, sCin, C, ldc, sC, lower ? 1 : 0, tiles_m, tiles, items, stages, status,
      wait_limit, rot ? nk / 2 : 0);
  return cudaGetLastError();
}

long long wait_limit_of(long long budget) {
  return budget > 0 ? budget : (budget < 0 ? 0 : kWaitLimit);
}

}  // namespace

size_t tc_workspace_bytes(TcMode mode, int M, int N, int K, int batch) {
  switch (mode) {
    case TcMode::TF32: return packed_bytes<float, 1>(M, K, batch) + packed_bytes<float, 1>(N, K, batch);
    case TcMode::TF32x3: return packed_bytes<float, 3>(M, K, batch) + packed_bytes<float, 3>(N, K, batch);
    case TcMode::BF16:
      return packed_bytes<__nv_bfloat16, 1>(M, K, batch) + packed_bytes<__nv_bfloat16, 1>(N, K, batch);
    case TcMode::BF16x3:
      return packed_bytes<__nv_bfloat16, 3>(M, K, batch) + packed_bytes<__nv_bfloat16, 3>(N, K, batch);
  }
  return 0;
}

cudaError_t tc_gemm(TcMode mode, int M, int N, int K, const TcOperand& a, const TcOperand& b,
                    float* C, int ldc, long long sC, int batch, void* ws, size_t ws_bytes,
                    int* status, long long wait_budget, cudaStream_t st) {
  const long long wl = wait_limit_of(wait_budget);
#define TC_RUN(E, NP)                                                                           \
  run<E, NP>(M, N, K, a, b, 1.f, 0.f, nullptr, 0, 0, C, ldc, sC, false, batch, ws, ws_bytes, \
             status, wl, st)
  switch (mode) {
    case TcMode::TF32: return TC_RUN(float, 1);
    case TcMode::TF32x3: return TC_RUN(float, 3);
    case TcMode::BF16: return TC_RUN(__nv_bfloat16, 1);
    case TcMode::BF16x3: return TC_RUN(__nv_bfloat16, 3);
  }
#undef TC_RUN
  return cudaErrorInvalidValue;
}

cudaError_t tc_syr2k_lower(TcMode mode, int m, int k, const float* A, int lda, long long sA,
                           const float* P, int ldp, long long sP, const float* Q, int ldq,
                           long long sQ, float* Mout, int ldm, long long sM, int batch, void* ws,
                           size_t ws_bytes, int* status, long long wait_budget,
                           cudaStream_t st) {
  // Mout = A - [P Q] [Q P]ᵀ on and below the diagonal: K = 2k, the left operand
  // row i = [P(i, :) Q(i, :)], the right one row j = [Q(j, :) P(j, :)]
  const TcOperand a{P, ldp, sP, Q, ldq, sQ, k, false};
  const TcOperand b{Q, ldq, sQ, P, ldp, sP, k, false};
  const long long wl = wait_limit_of(wait_budget);
#define TC_RUN(E, NP)                                                                           \
  run<E, NP>(m, m, 2 * k, a, b, -1.f, 1.f, A, lda, sA, Mout, ldm, sM, true, batch, ws, ws_bytes, \
             status, wl, st, true)
  switch (mode) {
    case TcMode::TF32: return TC_RUN(float, 1);
    case TcMode::TF32x3: return TC_RUN(float, 3);
    case TcMode::BF16: return TC_RUN(__nv_bfloat16, 1);
    case TcMode::BF16x3: return TC_RUN(__nv_bfloat16, 3);
  }
#undef TC_RUN
  return cudaErrorInvalidValue;
}
