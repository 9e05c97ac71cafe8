// Uneven trees in the uniform kernels.  A tree whose leaves have orders b_i <=
// leaf (ranks r_i = min(rank, b_i), and min(rank, r_c1 + r_c2) above) is
// embedded in the uniform (leaf, rank) tree:
//   D_i -> [[D_i, 0], [0, I]]                       (leaf x leaf)
//   U_i -> [[U_i, 0], [0, J]]                       (leaf x rank)
//   E_p -> real rows/columns in place, the padded columns on padded rows
//   S   -> [[S, 0], [0, 0]]                          (rank x rank)
// where J and the padded columns of E_p are columns of the identity placed on
// padded rows.  Every real column of a nested basis is then the real basis on
// the real rows (zero on padded rows), the couplings touch real columns only,
// so the padded matrix is A on the real rows, I on the padded ones and zero
// between them: A ⊕ I up to a row permutation.  Its solution restricted to the
// real rows is A⁻¹ b and its log det that of A.  The padded basis directions
// keep every basis of full column rank.
#include <algorithm>

#include "uneven.cuh"

namespace {

// column-major block of rows x cols at dst (ld), src packed column-major
void put_block(double* dst, int ld, const double* src, int rows, int cols) {
  for (int j = 0; j < cols; ++j)
    for (int i = 0; i < rows; ++i) dst[i + (long long)j * ld] = src[i + (long long)j * rows];
}

__global__ void pad_rows_kernel(const double* __restrict__ V, int ldv, double* __restrict__ P,
                                int ldp, const int* __restrict__ pmap, int npad, int nc,
                                int to_pad) {
  const int j = blockIdx.y;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npad; p += gridDim.x * blockDim.x) {
    const int q = pmap[p];
    if (to_pad)
      P[p + (long long)j * ldp] = q >= 0 ? V[q + (long long)j * ldv] : 0.0;
    else if (q >= 0)
      const_cast<double*>(V)[q + (long long)j * ldv] = P[p + (long long)j * ldp];
  }
}

}  // namespace

int pad_uneven(const hss_shape& s, const double* D, const double* U, const double* E,
               const double* S, UnevenPad* out) {
  const int L = s.levels, leaf = s.leaf, R = s.rank;
  if (!s.node_sizes || L < 1 || L > 24 || leaf < 1 || R < 1 || R > leaf) return HSS_ERR_INVALID_ARG;
  const long long nl = 1LL << L;
  long long total = 0;
  for (long long i = 0; i < nl; ++i) {
    const int b = s.node_sizes[i];
    if (b < 1 || b > leaf) return HSS_ERR_INVALID_ARG;
    total += b;
  }
  if (total != s.n) return HSS_ERR_INVALID_ARG;
  // ranks per level
  std::vector<std::vector<int>> rk(L + 1);
  rk[L].resize(nl);
  for (long long i = 0; i < nl; ++i) rk[L][i] = std::min(R, s.node_sizes[i]);
  for (int l = L - 1; l >= 1; --l) {
    rk[l].resize(1LL << l);
    for (long long i = 0; i < (1LL << l); ++i)
      rk[l][i] = std::min(R, rk[l + 1][2 * i] + rk[l + 1][2 * i + 1]);
  }
  UnevenPad& o = *out;
  o.npad = nl * leaf;
  const long long rr = (long long)R * R;
  o.D.assign(nl * leaf * leaf, 0.0);
  o.U.assign(nl * leaf * R, 0.0);
  long long esz = 0, ssz = 0;
  for (int l = 1; l <= L - 1; ++l) esz += (1LL << l) * 2 * rr;
  for (int l = 1; l <= L; ++l) ssz += (1LL << (l - 1)) * rr;
  o.E.assign(std::max<long long>(esz, 1), 0.0);
  o.S.assign(ssz, 0.0);
  o.pmap.assign(o.npad, -1);
  // leaves
  const double *dp = D, *up = U;
  long long row = 0;
  for (long long i = 0; i < nl; ++i) {
    const int b = s.node_sizes[i], r = rk[L][i];
    double* Dd = o.D.data() + i * leaf * leaf;
    put_block(Dd, leaf, dp, b, b);
    for (int q = b; q < leaf; ++q) Dd[q + (long long)q * leaf] = 1.0;
    double* Ud = o.U.data() + i * leaf * R;
    put_block(Ud, leaf, up, b, r);
    for (int j = r; j < R; ++j) Ud[(b + (j - r)) + (long long)j * leaf] = 1.0;
    dp += (long long)b * b;
    up += (long long)b * r;
    for (int q = 0; q < b; ++q) o.pmap[i * leaf + q] = (int)(row + q);
    row += b;
  }
  // transfer matrices: children's real rows at 0 .. r1-1 and R .. R+r2-1
  const double* ep = E;
  long long eo = 0;
  for (int l = 1; l <= L - 1; ++l) {
    for (long long i = 0; i < (1LL << l); ++i) {
      const int r1 = rk[l + 1][2 * i], r2 = rk[l + 1][2 * i + 1], rp = rk[l][i];
      double* Ed = o.E.data() + eo + i * 2 * rr;
      for (int j = 0; j < rp; ++j) {
        for (int q = 0; q < r1; ++q) Ed[q + (long long)j * 2 * R] = ep[q + (long long)j * (r1 + r2)];
        for (int q = 0; q < r2; ++q)
          Ed[(R + q) + (long long)j * 2 * R] = ep[(r1 + q) + (long long)j * (r1 + r2)];
      }
      // padded columns on padded rows: first the first child's, then the second's
      int t = 0;
      for (int j = rp; j < R; ++j, ++t) {
        const int prow = t < R - r1 ? r1 + t : R + r2 + (t - (R - r1));
        Ed[prow + (long long)j * 2 * R] = 1.0;
      }
      ep += (long long)(r1 + r2) * rp;
    }
    eo += (1LL << l) * 2 * rr;
  }
  // couplings
  const double* sp = S;
  long long so = 0;
  for (int l = 1; l <= L; ++l) {
    for (long long k = 0; k < (1LL << (l - 1)); ++k) {
      const int r1 = rk[l][2 * k], r2 = rk[l][2 * k + 1];
      put_block(o.S.data() + so + k * rr, R, sp, r2, r1);
      sp += (long long)r2 * r1;
    }
    so += (1LL << (l - 1)) * rr;
  }
  return HSS_OK;
}

void launch_pad_rows(const double* V, int ldv, double* P, int ldp, const int* pmap, int npad,
                     int nc, int to_pad, cudaStream_t st) {
  if (npad <= 0 || nc <= 0) return;
  const int blocks = std::min((npad + 255) / 256, 1024);
  pad_rows_kernel<<<dim3(blocks, nc), 256, 0, st>>>(V, ldv, P, ldp, pmap, npad, nc, to_pad);
}
