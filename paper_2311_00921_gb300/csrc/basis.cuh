// Basis completion (Eq. 2-3, Sec. 2) from level-wide products: Cholesky QR
// twice of the reversed basis, then the Householder vectors reconstructed from
// the orthonormal factor (basis.cu).
#pragma once
#include <cuda_runtime.h>

// Per-level scratch of the basis completion chain (n nodes of b x r bases).
template <typename T>
struct BasisScratch {
  T* X = nullptr;    // n x b x r: the orthonormalised reversed basis after one pass
  T* G = nullptr;    // n x r x r: Gram matrices, then S L1⁻ᵀ
  T* R1 = nullptr;   // n x r x r: first Cholesky factor, then P2 U⁻¹
  T* R = nullptr;    // n x r x r: R2 R1
  T* P = nullptr;    // n x r x r: inverse Cholesky factors
  T* U = nullptr;    // n x r x r: R2, then the top block of Q, then the LU's U
  T* Ui = nullptr;   // n x r x r: U⁻¹
  int* fail = nullptr;   // n: nonzero where a Gram Cholesky failed (Householder fallback)
};

// Largest rank the reconstruction path takes (its per-node kernels hold an
// r x r block in shared memory); larger ranks use the Householder kernel.
template <typename T>
int basis_max_rank();

// Kernel classes of the launches (for the tracer): products over the level,
// per-node Cholesky / LU kernels, the reversal and the Householder fallback.
enum BasisLaunchKind { BASIS_GEMM = 0, BASIS_NODE = 1, BASIS_COPY = 2, BASIS_FALLBACK = 3 };

// Called before and after every launch of the chain (kind, algorithmic flops);
// may be null.
struct BasisHook {
  void (*before)(void* ctx, int kind, double flops) = nullptr;
  void (*after)(void* ctx) = nullptr;
  void* ctx = nullptr;
};

// Householder QL completion of the n bases B (b x r, stride sB, leading
// dimension b): on return V (b x r, stride sV), T (r x r upper, stride sT) and
// L_B (r x r lower, stride sL) satisfy Q = I - V T Vᵀ = [Q^R Q^S] orthogonal and
// B = Q [0; L_B], with the signs of LAPACK's dlarfg applied to the reversed
// basis (the convention of ql_basis_kernel).  Requires r <= basis_max_rank<T>().
template <typename T>
cudaError_t launch_basis_completion(const T* B, long long sB, T* V, long long sV, T* Tm,
                                   long long sT, T* LB, long long sL, int b, int r, int n,
                                   const BasisScratch<T>& s, const BasisHook& hook,
                                   cudaStream_t st);
