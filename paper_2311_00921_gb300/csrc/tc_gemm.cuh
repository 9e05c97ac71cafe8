// Tensor-core (tcgen05) contractions of the mixed-precision diagonal product.
#pragma once
#include <cuda_runtime.h>

// MMA input type; the x3 modes split every FP32 operand into hi + lo and sum
// hi·hi + hi·lo + lo·hi (FP32 accumulation throughout).
enum class TcMode { TF32, TF32x3, BF16, BF16x3 };

// C (M x N) = A (M x K, column-major) · op(B), batched.  b_ncontig: element
// (n, k) of the right operand at B[n + k ldb] (B is N x K column-major);
// otherwise at B[k + n ldb] (B is K x N column-major, i.e. C = A B).
cudaError_t tc_gemm(TcMode mode, int M, int N, int K, const float* A, int lda, long long sA,
                    const float* B, int ldb, long long sB, bool b_ncontig, float* C, int ldc,
                    long long sC, int batch, int* status, long long wait_budget,
                    cudaStream_t st);

// wait_budget: polls of each pipeline wait (0 = default, < 0 = give up at once);
// an expired wait records HSS_ERR_TIMEOUT in status.
// Mout = A - (P Qᵀ + Q Pᵀ) on and below the diagonal (m x m, P and Q m x k).
// A may alias Mout.
cudaError_t tc_syr2k_lower(TcMode mode, int m, int k, const float* A, int lda, long long sA,
                           const float* P, int ldp, long long sP, const float* Q, int ldq,
                           long long sQ, float* Mout, int ldm, long long sM, int batch, int* status,
                           long long wait_budget, cudaStream_t st);
