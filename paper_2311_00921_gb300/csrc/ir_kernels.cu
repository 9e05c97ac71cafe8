// Small element-wise kernels of the mixed-precision path and of iterative
// refinement: precision conversion, residual, per-column norms, update.
#include "common.cuh"
#include "ir_kernels.cuh"

namespace {

constexpr int NT = 256;

__global__ void f64_to_f32_kernel(const double* __restrict__ a, float* __restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < n; i += (long long)gridDim.x * NT)
    b[i] = (float)a[i];
}

__global__ void f32_to_f64_kernel(const float* __restrict__ a, double* __restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < n; i += (long long)gridDim.x * NT)
    b[i] = (double)a[i];
}

// dst (m x nc, ld_dst, float) = src (m x nc, ld_src, double) * scale[j]
__global__ void cols_to_f32_kernel(const double* __restrict__ src, int ld_src, float* dst,
                                   int ld_dst, int m, int nc, const double* __restrict__ scale) {
  const int j = blockIdx.y;
  const double s = scale ? scale[j] : 1.0;
  for (int i = blockIdx.x * NT + threadIdx.x; i < m; i += gridDim.x * NT)
    dst[i + (long long)j * ld_dst] = (float)(src[i + (long long)j * ld_src] * s);
}

// x (double) [+]= d (float) * scale[j]
__global__ void cols_update_kernel(double* x, int ldx, const float* __restrict__ d, int ldd, int m,
                                   int nc, const double* __restrict__ scale, int accumulate) {
  const int j = blockIdx.y;
  const double s = scale ? scale[j] : 1.0;
  for (int i = blockIdx.x * NT + threadIdx.x; i < m; i += gridDim.x * NT) {
    const double v = (double)d[i + (long long)j * ldd] * s;
    double* p = x + i + (long long)j * ldx;
    *p = accumulate ? *p + v : v;
  }
}

// r = b - r (in place on r: r holds A x on entry)
__global__ void residual_kernel(const double* __restrict__ b, int ldb, double* r, int ldr, int m,
                                int nc) {
  const int j = blockIdx.y;
  for (int i = blockIdx.x * NT + threadIdx.x; i < m; i += gridDim.x * NT) {
    double* p = r + i + (long long)j * ldr;
    *p = b[i + (long long)j * ldb] - *p;
  }
}

// norms[j] = ||v(:, j)||_2, fixed-order reduction in one CTA per column;
// inv[j] = 1 / norms[j] (0 when the column is zero)
__global__ void col_norms_kernel(const double* __restrict__ v, int ld, int m, double* norms,
                                 double* inv) {
  __shared__ double red[32];
  const int j = blockIdx.x;
  double s = 0.0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const double a = v[i + (long long)j * ld];
    s = fma(a, a, s);
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) {
    const double nr = sqrt(s);
    norms[j] = nr;
    if (inv) inv[j] = nr > 0.0 ? 1.0 / nr : 0.0;
  }
}

__global__ void eye_kernel(double* a, int n) {
  for (long long e = blockIdx.x * (long long)NT + threadIdx.x; e < (long long)n * n;
       e += (long long)gridDim.x * NT)
    a[e] = (e % n == e / n) ? 1.0 : 0.0;
}

int grid_for(long long n) {
  long long g = (n + NT - 1) / NT;
  return (int)(g < 152 * 16 ? (g < 1 ? 1 : g) : 152 * 16);
}

}  // namespace

void launch_f64_to_f32(const double* a, float* b, long long n, cudaStream_t st) {
  if (n > 0) f64_to_f32_kernel<<<grid_for(n), NT, 0, st>>>(a, b, n);
}

void launch_f32_to_f64(const float* a, double* b, long long n, cudaStream_t st) {
  if (n > 0) f32_to_f64_kernel<<<grid_for(n), NT, 0, st>>>(a, b, n);
}

void launch_cols_to_f32(const double* src, int ld_src, float* dst, int ld_dst, int m, int nc,
                        const double* scale, cudaStream_t st) {
  dim3 g((unsigned)std::min<long long>((m + NT - 1) / NT, 64), nc);
  cols_to_f32_kernel<<<g, NT, 0, st>>>(src, ld_src, dst, ld_dst, m, nc, scale);
}

void launch_cols_update(double* x, int ldx, const float* d, int ldd, int m, int nc,
                        const double* scale, int accumulate, cudaStream_t st) {
  dim3 g((unsigned)std::min<long long>((m + NT - 1) / NT, 64), nc);
  cols_update_kernel<<<g, NT, 0, st>>>(x, ldx, d, ldd, m, nc, scale, accumulate);
}

void launch_residual(const double* b, int ldb, double* r, int ldr, int m, int nc, cudaStream_t st) {
  dim3 g((unsigned)std::min<long long>((m + NT - 1) / NT, 64), nc);
  residual_kernel<<<g, NT, 0, st>>>(b, ldb, r, ldr, m, nc);
}

void launch_col_norms(const double* v, int ld, int m, int nc, double* norms, double* inv,
                      cudaStream_t st) {
  col_norms_kernel<<<nc, 1024, 0, st>>>(v, ld, m, norms, inv);
}

void launch_eye(double* a, int n, cudaStream_t st) {
  eye_kernel<<<grid_for((long long)n * n), NT, 0, st>>>(a, n);
}
