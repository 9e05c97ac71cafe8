// Shared device helpers for the HSS-ULV kernels (sm_103a).
//
// Storage convention everywhere: column-major blocks, element (i, j) of a
// block with leading dimension ld at [i + j * ld]; blocks of one tree level
// are contiguous in node order with a fixed batch stride.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define HSS_DEVINL __device__ __forceinline__

// status word layout (device int32[8]): [0] error code (0 = ok),
// [1] level, [2] node, [3] column, [4] timeout site
enum { ST_CODE = 0, ST_LEVEL = 1, ST_NODE = 2, ST_COL = 3, ST_SITE = 4 };

// record the first failure only
HSS_DEVINL void report_failure(int* status, int code, int level, int node, int col) {
  if (atomicCAS(status + ST_CODE, 0, code) == 0) {
    status[ST_LEVEL] = level;
    status[ST_NODE] = node;
    status[ST_COL] = col;
  }
}

template <typename T>
HSS_DEVINL T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block-wide sum over blockDim.x threads (multiple of 32); `red` holds >= 32
// elements of shared scratch.  Every thread gets the total.
template <typename T>
HSS_DEVINL T block_sum(T v, T* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  T t = (threadIdx.x < nw) ? red[threadIdx.x] : T(0);
  if (wid == 0) {
    t = warp_sum(t);
    if (lane == 0) red[0] = t;
  }
  __syncthreads();
  T r = red[0];
  return r;
}

// ---------------------------------------------------------------- batched GEMM
// C = alpha * op(A) * op(B) + beta * C for `batch` independent problems.
// op(X) = X or Xᵀ.  Column-major; batch strides in elements.
template <typename T>
void gemm_batched(bool transA, bool transB, int m, int n, int k, T alpha,
                  const T* A, int lda, long long sA, const T* B, int ldb, long long sB,
                  T beta, T* C, int ldc, long long sC, int batch, cudaStream_t st);

// M(i, j) = A(i, j) - sum_k [P(i,k) Q(j,k) + Q(i,k) P(j,k)] on the lower
// triangle (i >= j); P, Q are m x k.  A may alias M.
template <typename T>
void syr2k_lower_batched(int m, int k, const T* A, int lda, long long sA,
                         const T* P, int ldp, long long sP, const T* Q, int ldq, long long sQ,
                         T* M, int ldm, long long sM, int batch, cudaStream_t st);

// As syrk_lower_batched, and the result of node z (both triangles) also goes to
// the diagonal block at offset (z & 1) m of parent block z / 2 of PA (ld ldpa,
// stride sPA): the merge step of Alg. 2 fused into the last Schur update.
template <typename T>
void syrk_lower_merge_batched(int m, int k, const T* A, int lda, long long sA, const T* P,
                              int ldp, long long sP, T* M, int ldm, long long sM, T* PA, int ldpa,
                              long long sPA, int batch, cudaStream_t st);

// M(i, j) = A(i, j) - sum_k P(i,k) P(j,k) on the lower triangle; A may alias M.
template <typename T>
void syrk_lower_batched(int m, int k, const T* A, int lda, long long sA, const T* P, int ldp,
                        long long sP, T* M, int ldm, long long sM, int batch, cudaStream_t st);
