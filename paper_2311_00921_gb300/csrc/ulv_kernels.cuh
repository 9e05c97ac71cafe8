// Launchers of the per-node ULV step kernels (ulv_kernels.cu).
#pragma once
#include <cuda_runtime.h>

// Householder QL basis completion, one CTA per node.  only_if (n flags, may be
// null): complete only the nodes whose flag is nonzero.
// panel: columns per register panel of the blocked QR, 16 or 32 (FP32 only;
// 0 = the default, 32 in FP32 and 16 in FP64).
template <typename T>
cudaError_t launch_ql_basis(const T* Bsrc, int ldb_src, long long sB, T* V, long long sV, T* Tm,
                            long long sT, T* LB, long long sL, int b, int r, int nodes,
                            cudaStream_t st, const int* only_if = nullptr, int panel = 0);

template <typename T>
size_t pchol_smem(int b);

template <typename T>
cudaError_t launch_pchol(T* M, int ldm, long long sM, int b, int c, T* PA, int ldpa, long long sPA,
                  double* logdet_part, int level, int node0, int* status, int nodes,
                  cudaStream_t st);

template <typename T>
cudaError_t launch_trsv_fwd(const T* M, int ldm, long long sM, int b, int c, T* X, int ldx, long long sX,
                     int nrhs, T* Par, int ldpar, long long sPar, int nodes, cudaStream_t st);

template <typename T>
cudaError_t launch_trsv_bwd(const T* M, int ldm, long long sM, int b, int c, T* X, int ldx, long long sX,
                     int nrhs, const T* Par, int ldpar, long long sPar, int nodes,
                     cudaStream_t st);

// One level of the ULV solve per launch, one CTA per node: the forward sweep
// applies Qᵀ = I - V Tᵀ Vᵀ to the node segment and then the triangular forward
// sweep (launch_trsv_fwd); the backward sweep runs the triangular backward sweep
// and then applies Q = I - V T Vᵀ.  V (b x r, batch stride sV) and T (r x r,
// batch stride sT) are the node's compact-WY basis (Eq. 2-3); V = null skips
// the Q application.  nrhs <= 16, r <= min(b, 256).  staging: 0 = the
// largest panel staging shared memory allows, 1 = the staging that needs the
// fewest waves of CTAs over the SMs.
template <typename T>
cudaError_t launch_ulv_fwd(const T* M, int ldm, long long sM, int b, int c, T* X, int ldx,
                           long long sX, int nrhs, T* Par, int ldpar, long long sPar, const T* V,
                           long long sV, const T* Tm, long long sT, int r, int nodes,
                           cudaStream_t st, int staging = 0);
template <typename T>
cudaError_t launch_ulv_bwd(const T* M, int ldm, long long sM, int b, int c, T* X, int ldx,
                           long long sX, int nrhs, const T* Par, int ldpar, long long sPar,
                           const T* V, long long sV, const T* Tm, long long sT, int r, int nodes,
                           cudaStream_t st, int staging = 0);

// Whether a sweep launch with the Q application fused (per-level kernel, or the
// tree kernels at block order b) fits the device's shared memory for nrhs
// columns and rank r; where it does not, the caller applies Q by batched GEMMs
// and runs the per-level sweeps without it.
template <typename T>
bool ulv_fused_fits(int b, int nrhs, int r, bool bwd);
template <typename T>
bool tree_fits(int b, int nrhs, int r);

void launch_logdet_reduce(const double* part, int n, double* out, cudaStream_t st);

// dynamic shared memory of the basis-completion kernel for a b x r basis
template <typename T>
size_t ql_smem(int b, int r, int NBP);

// One panel of a blocked Cholesky, for every node of a batch (stride sM): factor
// the kb x kb diagonal block at the top of each rows x rows matrix M (ld ldm)
// and solve the rows below it, split over `splits` CTAs a node; the trailing
// update is left to the caller.  Writes (or, with accumulate, adds)
// 2 Σ log diag to logdet_part[node].
template <typename T>
cudaError_t launch_chol_panel(T* M, int ldm, long long sM, int rows, int kb, double* logdet_part,
                              int level, int node0, int col0, int* status, int nodes,
                              bool accumulate, cudaStream_t st, int splits = 1);

// The merge step of Alg. 2 as its own pass: Â^SS of node i (lower triangle
// of M[c:, c:], r x r) into block (i & 1) of parent i / 2's diagonal, both triangles.
template <typename T>
cudaError_t launch_scatter_ss(const T* M, int ldm, long long sM, int c, int r, T* PA, int ldpa,
                              long long sPA, int nodes, cudaStream_t st);

// Levels 1 .. lo of the solve as one launch per direction (block order b = 2r
// at every level; index = level): factored blocks M (b x b per node), compact-WY
// V (b x r) and T (r x r), level vectors (node segments of b rows, ld 2^l b;
// vec[0] is the root's vector).
template <typename T>
struct TreeLevels {
  const T* M[24];
  const T* V[24];
  const T* Tm[24];
  T* vec[24];
};

// Forward sweep of levels lo .. 1 (Qᵀ, triangular solve, push to the parent)
// in one launch of 2^lo CTAs with no barrier between levels: the CTA that
// completes the second child of a parent continues with the parent.  cnt: 2^lo
// ints of scratch (cleared here).  nrhs <= 16.
template <typename T>
cudaError_t launch_tree_fwd(const TreeLevels<T>& lv, int lo, int b, int c, int r, int nrhs,
                            int* cnt, cudaStream_t st);

// Backward sweep of levels 1 .. lo in one cooperative launch of 2^lo CTAs:
// each node waits for its parent's flag in ready (2^(lo+1) ints, flag of node
// i of level l at (2^l - 1) + i) to equal epoch, polling at most wait_limit
// times; an expired wait records HSS_ERR_TIMEOUT in status.  Flags are left at
// epoch, so every call passes a new one.
template <typename T>
cudaError_t launch_tree_bwd(const TreeLevels<T>& lv, int lo, int b, int c, int r, int nrhs,
                            int* ready, int epoch, long long wait_limit, int* status,
                            cudaStream_t st);
