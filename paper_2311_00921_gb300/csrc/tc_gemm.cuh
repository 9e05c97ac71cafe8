// Tensor-core (tcgen05) contractions of the mixed-precision diagonal product.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

// MMA input type; the x3 modes split every FP32 operand into hi + lo and sum
// hi·hi + hi·lo + lo·hi (FP32 accumulation throughout).
enum class TcMode { TF32, TF32x3, BF16, BF16x3 };

// One operand of C = op(A) op(B)ᵀ, rows x K, batched: element (row, k) is, for
// k < K1, src1[k + row ld1] (kcontig) or src1[row + k ld1]; for k >= K1 (when
// src2 is given) the same in src2 at k - K1.  K1 = 0 means K1 = K.
struct TcOperand {
  const float* src1;
  int ld1;
  long long s1;   // batch stride
  const float* src2;
  int ld2;
  long long s2;
  int K1;
  bool kcontig;
};

// Bytes of packing workspace that tc_gemm needs for these sizes (tc_syr2k_lower:
// M = N = m, K = 2k).
size_t tc_workspace_bytes(TcMode mode, int M, int N, int K, int batch);

// C (M x N, column-major, ld ldc, batch stride sC) = a · bᵀ with a: M x K and
// b: N x K (see TcOperand).  Packs both operands into ws, then one launch.
// wait_budget: polls of each pipeline wait (0 = default, < 0 = give up at
// once); an expired wait records HSS_ERR_TIMEOUT in status.
cudaError_t tc_gemm(TcMode mode, int M, int N, int K, const TcOperand& a, const TcOperand& b,
                    float* C, int ldc, long long sC, int batch, void* ws, size_t ws_bytes,
                    int* status, long long wait_budget, cudaStream_t st);

// Mout = A - (P Qᵀ + Q Pᵀ) on and below the diagonal (m x m, P and Q m x k,
// column-major).  A may alias Mout.
cudaError_t tc_syr2k_lower(TcMode mode, int m, int k, const float* A, int lda, long long sA,
                           const float* P, int ldp, long long sP, const float* Q, int ldq,
                           long long sQ, float* Mout, int ldm, long long sM, int batch, void* ws,
                           size_t ws_bytes, int* status, long long wait_budget, cudaStream_t st);
