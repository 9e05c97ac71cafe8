// Pair-of-FP32 arithmetic for the refinement residual (dfgemm.cu).
//
// A value v is held as two floats (hi, lo) with v = hi + lo and |lo| <= ulp(hi)/2:
// 48 significand bits.  Products use the exact FMA product error, sums the
// exact two-sum, so a length-K dot product carries a relative error of about
// sqrt(K) 2^-48 of the magnitude of its terms: far below the 1e-12 residual the
// refinement stops at, on the FP32 pipe (64x the FP64 rate of the chip).
#pragma once
#include <cuda_runtime.h>

// hi = fl32(a), lo = fl32(a - hi) for n contiguous values (lo may be null: hi only)
cudaError_t launch_df_split(const double* a, float* hi, float* lo, long long n, cudaStream_t st);

// The same for an m x nc column block (ld lda) into ld ldo, each column scaled
// by 2^-e_j, e_j = ilogb(colnorm[j]) (no scaling where colnorm is null or 0),
// so that any column magnitude stays inside the FP32 range.
cudaError_t launch_df_split_cols(const double* a, int lda, int m, int nc, const double* colnorm,
                                 float* hi, float* lo, int ldo, cudaStream_t st);

// Batched C = op(A) B (+ C when accumulate) in pair arithmetic, n <= 16.
// A (m x k, or k x m when transA) and B (k x n) are (hi, lo) pairs with the
// same layout; C (ld ldc, batch stride sC) is written as a pair (Ch, Cl) or,
// when C64 is given, to C64 (ld ldc64, same batch stride) as the double hi + lo
// scaled back by 2^e_j of colnorm (the accumulated input then still comes from
// Ch, Cl).  Errors: cudaErrorInvalidValue for n > 16, batch > 65535 or missing
// outputs.
cudaError_t df_gemm(bool transA, int m, int n, int k, const float* Ah, const float* Al, int lda,
                    long long sA, const float* Bh, const float* Bl, int ldb, long long sB,
                    bool accumulate, float* Ch, float* Cl, double* C64, int ldc64,
                    const double* colnorm, int ldc, long long sC, int batch, cudaStream_t st);
