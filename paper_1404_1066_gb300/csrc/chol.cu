// FP64 Cholesky factorisation H = L L^T and the two triangular solves of
// the Newton system of Section 4's reoptimisation.  Blocked right-looking
// factorisation with 64 x 64 blocks: diagonal block in shared memory, panel
// triangular solve, trailing symmetric update.
#include "internal.h"

namespace spsvm {

namespace {

constexpr int NB = 64;

__global__ void __launch_bounds__(256) potrf_diag(double* __restrict__ H, int64_t ldh, int64_t m,
                                                  int64_t k0, int32_t* __restrict__ info) {
  __shared__ double A[NB][NB + 1];
  __shared__ int fail;
  if (*info != 0) return;
  const int nb = (int)min64(NB, m - k0);
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int r = e / NB, c = e % NB;
    A[r][c] = (r < nb && c <= r) ? H[(k0 + r) * ldh + k0 + c] : 0.0;
  }
  if (threadIdx.x == 0) fail = 0;
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    if (threadIdx.x == 0) {
      const double d = A[j][j];
      if (!(d > 0.0)) {
        fail = j + 1;
      } else {
        A[j][j] = sqrt(d);
      }
    }
    __syncthreads();
    if (fail) break;
    const double inv = 1.0 / A[j][j];
    for (int i = j + 1 + threadIdx.x; i < nb; i += blockDim.x) A[i][j] *= inv;
    __syncthreads();
    // trailing update of the lower triangle: rows i > j, columns j < l <= i
    const int w = nb - j - 1;
    for (int e = threadIdx.x; e < w * w; e += blockDim.x) {
      const int i = j + 1 + e / w, l = j + 1 + e % w;
      if (l <= i) A[i][l] -= A[i][j] * A[l][j];
    }
    __syncthreads();
  }
  if (fail) {
    if (threadIdx.x == 0) *info = (int32_t)(k0 + fail);
    return;
  }
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int r = e / NB, c = e % NB;
    if (r < nb && c <= r) H[(k0 + r) * ldh + k0 + c] = A[r][c];
  }
}

// Rows r >= k0 + NB: L[r][k0:k0+nb] = H[r][k0:k0+nb] L_kk^{-T}.
__global__ void __launch_bounds__(128) trsm_panel(double* __restrict__ H, int64_t ldh, int64_t m,
                                                  int64_t k0, const int32_t* __restrict__ info) {
  __shared__ double L[NB][NB + 1];
  if (*info != 0) return;
  const int nb = (int)min64(NB, m - k0);
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int r = e / NB, c = e % NB;
    double v = 0.0;
    if (r < nb && c <= r) v = H[(k0 + r) * ldh + k0 + c];
    else if (r == c) v = 1.0;   // identity padding of a partial block
    L[r][c] = v;
  }
  __syncthreads();
  const int64_t r = k0 + NB + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= m) return;
  double* row = H + r * ldh + k0;
  double x[NB];
#pragma unroll
  for (int j = 0; j < NB; ++j) x[j] = (j < nb) ? row[j] : 0.0;
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    double s = x[j];
#pragma unroll
    for (int l = 0; l < j; ++l) s -= x[l] * L[j][l];
    x[j] = s / L[j][j];
  }
#pragma unroll
  for (int j = 0; j < NB; ++j)
    if (j < nb) row[j] = x[j];
}

// Trailing update A[r][c] -= sum_l L[r][k0+l] L[c][k0+l] for r >= c >= k0 + NB.
__global__ void __launch_bounds__(256) syrk_trailing(double* __restrict__ H, int64_t ldh,
                                                     int64_t m, int64_t k0,
                                                     const int32_t* __restrict__ info) {
  __shared__ double Ar[16][64 + 1];
  __shared__ double Ac[16][64 + 1];
  if (*info != 0) return;
  const int nb = (int)min64(NB, m - k0);
  const int64_t base = k0 + NB;
  const int64_t T = ceil_div(m - base, (int64_t)64);
  // lower tile (ti >= tj) from the linear block index
  int64_t t = blockIdx.x, ti = 0;
  while (t > ti) { t -= ti + 1; ++ti; }
  const int64_t tj = t;
  if (ti >= T) return;
  const int64_t r0 = base + ti * 64, c0 = base + tj * 64;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  for (int l0 = 0; l0 < nb; l0 += 16) {
    for (int e = threadIdx.x; e < 16 * 64; e += blockDim.x) {
      const int rr = e / 16, ll = e % 16;
      const int64_t gr = r0 + rr, gc = c0 + rr;
      const bool okl = l0 + ll < nb;
      Ar[ll][rr] = (okl && gr < m) ? H[gr * ldh + k0 + l0 + ll] : 0.0;
      Ac[ll][rr] = (okl && gc < m) ? H[gc * ldh + k0 + l0 + ll] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int ll = 0; ll < 16; ++ll) {
      double av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = Ar[ll][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Ac[ll][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int64_t r = r0 + ty + 16 * a;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int64_t c = c0 + tx + 16 * b;
      if (r < m && c <= r) H[r * ldh + c] -= acc[a][b];
    }
  }
}

// Inverse of each lower-triangular diagonal block L_kk, stored transposed in
// the (otherwise unused) strict upper triangle of the block: element (i, j),
// i > j, of inv(L_kk) at H[(k0 + j) * ldh + k0 + i].  The diagonal of the
// inverse is 1 / L_ii and is not stored.
__global__ void __launch_bounds__(64) diag_inverse(double* __restrict__ H, int64_t ldh, int64_t m) {
  __shared__ double Ls[NB][NB + 1];
  const int64_t k0 = (int64_t)blockIdx.x * NB;
  const int nb = (int)min64(NB, m - k0);
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int r = e / NB, c = e % NB;
    Ls[r][c] = (r < nb && c <= r) ? H[(k0 + r) * ldh + k0 + c] : (r == c ? 1.0 : 0.0);
  }
  __syncthreads();
  // thread j solves L x = e_j (column j of the inverse) for rows i > j and
  // keeps x_i in its own row of the upper triangle, Ls[j][i]; it reads only
  // the lower triangle (Ls[i][l], l < i) and its own row.
  const int j = threadIdx.x;
  if (j < nb) {
    const double xj = 1.0 / Ls[j][j];
    for (int i = j + 1; i < nb; ++i) {
      double acc = Ls[i][j] * xj;
      for (int l = j + 1; l < i; ++l) acc += Ls[i][l] * Ls[j][l];
      Ls[j][i] = -acc / Ls[i][i];
    }
    for (int i = j + 1; i < nb; ++i) H[(k0 + j) * ldh + k0 + i] = Ls[j][i];
  }
}

// inv(L_kk)[i][j] for i >= j from the stored block inverse.
__device__ __forceinline__ double inv_at(const double* __restrict__ L, int64_t ldh, int64_t k0,
                                         int i, int j) {
  return (i == j) ? 1.0 / L[(k0 + i) * ldh + k0 + i] : L[(k0 + j) * ldh + k0 + i];
}

constexpr int SV_T = 256;
constexpr int SV_ROWS = 64;   // rows updated per block (8 warps x 8 rows)

// Forward step for block k: z_k = inv(L_kk) b_k (into z), b_r -= L[r][k] z_k
// for the rows r below the block handled by this CTA.
__global__ void __launch_bounds__(SV_T) trsv_fwd_step(const double* __restrict__ L, int64_t ldh,
                                                      int64_t m, int64_t k0,
                                                      double* __restrict__ b,
                                                      double* __restrict__ z) {
  __shared__ double zs[NB];
  __shared__ double bs[NB];
  const int nb = (int)min64(NB, m - k0);
  if (threadIdx.x < NB) bs[threadIdx.x] = threadIdx.x < nb ? b[k0 + threadIdx.x] : 0.0;
  __syncthreads();
  {
    // 4 threads per row of the block
    const int i = threadIdx.x >> 2, q = threadIdx.x & 3;
    double acc = 0.0;
    if (i < nb)
      for (int j = q; j <= i; j += 4) acc += inv_at(L, ldh, k0, i, j) * bs[j];
    acc += __shfl_xor_sync(0xffffffffu, acc, 1);
    acc += __shfl_xor_sync(0xffffffffu, acc, 2);
    if (q == 0 && i < NB) zs[i] = (i < nb) ? acc : 0.0;
  }
  __syncthreads();
  if (blockIdx.x == 0 && threadIdx.x < nb) z[k0 + threadIdx.x] = zs[threadIdx.x];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t r0 = k0 + nb + (int64_t)blockIdx.x * SV_ROWS;
  for (int rr = warp; rr < SV_ROWS; rr += SV_T / 32) {
    const int64_t r = r0 + rr;
    if (r >= m) break;
    double s = 0.0;
    for (int l = lane; l < nb; l += 32) s += L[r * ldh + k0 + l] * zs[l];
    s = warp_sum(s);
    if (lane == 0) b[r] -= s;
  }
}

// Backward step for block k: x_k = inv(L_kk)^T z_k (into x), z_r -= sum_l
// L[k0+l][r] x_l for the rows r < k0 handled by this CTA.
__global__ void __launch_bounds__(SV_T) trsv_bwd_step(const double* __restrict__ L, int64_t ldh,
                                                      int64_t m, int64_t k0,
                                                      double* __restrict__ z,
                                                      double* __restrict__ x) {
  __shared__ double xs[NB];
  __shared__ double zsh[NB];
  const int nb = (int)min64(NB, m - k0);
  if (threadIdx.x < NB) zsh[threadIdx.x] = threadIdx.x < nb ? z[k0 + threadIdx.x] : 0.0;
  __syncthreads();
  {
    const int j = threadIdx.x >> 2, q = threadIdx.x & 3;
    double acc = 0.0;
    if (j < nb)
      for (int i = j + q; i < nb; i += 4) acc += inv_at(L, ldh, k0, i, j) * zsh[i];
    acc += __shfl_xor_sync(0xffffffffu, acc, 1);
    acc += __shfl_xor_sync(0xffffffffu, acc, 2);
    if (q == 0 && j < NB) xs[j] = (j < nb) ? acc : 0.0;
  }
  __syncthreads();
  if (blockIdx.x == 0 && threadIdx.x < nb) x[k0 + threadIdx.x] = xs[threadIdx.x];
  const int64_t r = (int64_t)blockIdx.x * SV_T + threadIdx.x;
  if (r >= k0) return;
  double s = 0.0;
  for (int l = 0; l < nb; ++l) s += L[(k0 + l) * ldh + r] * xs[l];
  z[r] -= s;
}

}  // namespace
}  // namespace spsvm

using namespace spsvm;

extern "C" int spsvm_cholesky(double* H, int64_t m, int64_t ldh, int32_t* info, void* stream) {
  if (!H || !info || m < 0 || ldh < m) return set_error(SPSVM_ERR_ARG, "cholesky: bad arguments");
  cudaStream_t s = as_stream(stream);
  ProfScope prof(PROF_CHOLESKY, s, (double)m * m * m / 3.0);
  SPSVM_CUDA_TRY(cudaMemsetAsync(info, 0, sizeof(int32_t), s));
  for (int64_t k0 = 0; k0 < m; k0 += NB) {
    potrf_diag<<<1, 256, 0, s>>>(H, ldh, m, k0, info);
    SPSVM_LAUNCH_CHECK();
    const int64_t below = m - (k0 + NB);
    if (below <= 0) break;
    trsm_panel<<<(unsigned)ceil_div(below, 128), 128, 0, s>>>(H, ldh, m, k0, info);
    SPSVM_LAUNCH_CHECK();
    const int64_t T = ceil_div(below, (int64_t)64);
    syrk_trailing<<<(unsigned)(T * (T + 1) / 2), 256, 0, s>>>(H, ldh, m, k0, info);
    SPSVM_LAUNCH_CHECK();
  }
  if (m > 0) {
    diag_inverse<<<(unsigned)ceil_div(m, (int64_t)NB), 64, 0, s>>>(H, ldh, m);
    SPSVM_LAUNCH_CHECK();
  }
  return SPSVM_OK;
}

extern "C" int spsvm_cholesky_solve(const double* L, int64_t m, int64_t ldh, double* b,
                                    double* work, void* stream) {
  if (!L || !b || !work || m < 0 || ldh < m)
    return set_error(SPSVM_ERR_ARG, "cholesky_solve: bad arguments");
  if (m == 0) return SPSVM_OK;
  cudaStream_t s = as_stream(stream);
  ProfScope prof(PROF_SOLVE, s, 8.0 * (double)m * m);
  // forward: rows below each block are updated in b, z_k goes to work
  for (int64_t k0 = 0; k0 < m; k0 += NB) {
    const int64_t below = m - min64(m, k0 + NB);
    const unsigned grid = (unsigned)(below > 0 ? ceil_div(below, (int64_t)SV_ROWS) : 1);
    trsv_fwd_step<<<grid, SV_T, 0, s>>>(L, ldh, m, k0, b, work);
    SPSVM_LAUNCH_CHECK();
  }
  // backward: rows above each block are updated in work, x_k goes to b
  for (int64_t k0 = ((m - 1) / NB) * NB; k0 >= 0; k0 -= NB) {
    const unsigned grid = (unsigned)(k0 > 0 ? ceil_div(k0, (int64_t)SV_T) : 1);
    trsv_bwd_step<<<grid, SV_T, 0, s>>>(L, ldh, m, k0, work, b);
    SPSVM_LAUNCH_CHECK();
  }
  return SPSVM_OK;
}
