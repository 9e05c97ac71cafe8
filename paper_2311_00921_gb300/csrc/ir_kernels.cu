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
// column norms in two fixed-order passes: kNormParts CTAs per column write
// partial sums of squares, then one warp per column adds them in order
constexpr int kNormParts = 64;

__global__ void col_norms_part_kernel(const double* __restrict__ v, int ld, int m,
                                      double* __restrict__ part) {
  __shared__ double red[32];
  const int j = blockIdx.y, p = blockIdx.x;
  const int chunk = (m + kNormParts - 1) / kNormParts;
  const int i0 = p * chunk, i1 = min(m, i0 + chunk);
  double s = 0.0;
  for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    const double a = v[i + (long long)j * ld];
    s = fma(a, a, s);
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) part[j * kNormParts + p] = s;
}

__global__ void col_norms_final_kernel(const double* __restrict__ part, int nc, double* norms,
                                       double* inv) {
  const int j = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x & 31;
  if (j >= nc) return;
  double s = part[j * kNormParts + lane] + part[j * kNormParts + 32 + lane];
  s = warp_sum(s);
  if (lane == 0) {
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
                      double* scratch, cudaStream_t st) {
  if (nc <= 0) return;
  col_norms_part_kernel<<<dim3(kNormParts, nc), 256, 0, st>>>(v, ld, m, scratch);
  col_norms_final_kernel<<<(nc + 7) / 8, 256, 0, st>>>(scratch, nc, norms, inv);
}

void launch_eye(double* a, int n, cudaStream_t st) {
  eye_kernel<<<grid_for((long long)n * n), NT, 0, st>>>(a, n);
}

__global__ void fill_test_kernel(double* x, int n, int nc) {
  const int j = blockIdx.y;
  for (int i = blockIdx.x * NT + threadIdx.x; i < n; i += gridDim.x * NT)
    x[i + (long long)j * n] = sin(0.37 * i + 1.7 * j) + 0.25 * cos(0.011 * i * (j + 1));
}

void launch_fill_test(double* x, int n, int nc, cudaStream_t st) {
  if (n <= 0 || nc <= 0) return;
  fill_test_kernel<<<dim3(grid_for(n), nc), NT, 0, st>>>(x, n, nc);
}
