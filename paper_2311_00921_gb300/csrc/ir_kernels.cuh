// Launchers of the precision-conversion and refinement kernels (ir_kernels.cu).
#pragma once
#include <cuda_runtime.h>

#include <algorithm>

void launch_f64_to_f32(const double* a, float* b, long long n, cudaStream_t st);
void launch_f32_to_f64(const float* a, double* b, long long n, cudaStream_t st);
void launch_cols_to_f32(const double* src, int ld_src, float* dst, int ld_dst, int m, int nc,
                        const double* scale, cudaStream_t st);
void launch_cols_update(double* x, int ldx, const float* d, int ldd, int m, int nc,
                        const double* scale, int accumulate, cudaStream_t st);
void launch_residual(const double* b, int ldb, double* r, int ldr, int m, int nc, cudaStream_t st);
// 2-norms of nc columns (and their inverses, 0 for a zero column, when inv is
// given) in a fixed summation order; scratch holds 64 doubles per column
void launch_col_norms(const double* v, int ld, int m, int nc, double* norms, double* inv,
                      double* scratch, cudaStream_t st);
void launch_eye(double* a, int n, cudaStream_t st);   // a = I (n x n, column-major)
// a fixed, deterministic n x nc test block (column-major, ld n)
void launch_fill_test(double* x, int n, int nc, cudaStream_t st);
