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

// L L^T x = b in place, one block of 1024 threads.
__global__ void __launch_bounds__(1024) chol_solve_kernel(const double* __restrict__ L,
                                                          int64_t ldh, int64_t m,
                                                          double* __restrict__ b) {
  __shared__ double xs[NB];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  // forward: L z = b
  for (int64_t k0 = 0; k0 < m; k0 += NB) {
    const int nb = (int)min64(NB, m - k0);
    if (warp == 0) {
      for (int j = 0; j < nb; ++j) {
        double s = 0.0;
        for (int l = lane; l < j; l += 32) s += L[(k0 + j) * ldh + k0 + l] * xs[l];
        s = warp_sum(s);
        if (lane == 0) xs[j] = (b[k0 + j] - s) / L[(k0 + j) * ldh + k0 + j];
        __syncwarp();
      }
    }
    __syncthreads();
    if (threadIdx.x < nb) b[k0 + threadIdx.x] = xs[threadIdx.x];
    // update the rows below: b_r -= L[r][k0:k0+nb] . z_k
    for (int64_t r = k0 + nb + warp; r < m; r += nw) {
      double s = 0.0;
      for (int l = lane; l < nb; l += 32) s += L[r * ldh + k0 + l] * xs[l];
      s = warp_sum(s);
      if (lane == 0) b[r] -= s;
    }
    __syncthreads();
  }
  // backward: L^T x = z
  const int64_t nblk = ceil_div(m, (int64_t)NB);
  for (int64_t kb = nblk - 1; kb >= 0; --kb) {
    const int64_t k0 = kb * NB;
    const int nb = (int)min64(NB, m - k0);
    if (warp == 0) {
      for (int j = nb - 1; j >= 0; --j) {
        double s = 0.0;
        for (int l = j + 1 + lane; l < nb; l += 32) s += L[(k0 + l) * ldh + k0 + j] * xs[l];
        s = warp_sum(s);
        if (lane == 0) xs[j] = (b[k0 + j] - s) / L[(k0 + j) * ldh + k0 + j];
        __syncwarp();
      }
    }
    __syncthreads();
    if (threadIdx.x < nb) b[k0 + threadIdx.x] = xs[threadIdx.x];
    // z_r -= sum_{l in block} L[l][r] x_l for r < k0
    for (int64_t r = threadIdx.x; r < k0; r += blockDim.x) {
      double s = 0.0;
      for (int l = 0; l < nb; ++l) s += L[(k0 + l) * ldh + r] * xs[l];
      b[r] -= s;
    }
    __syncthreads();
  }
}

}  // namespace
}  // namespace spsvm

using namespace spsvm;

extern "C" int spsvm_cholesky(double* H, int64_t m, int64_t ldh, int32_t* info, void* stream) {
  if (!H || !info || m < 0 || ldh < m) return set_error(SPSVM_ERR_ARG, "cholesky: bad arguments");
  cudaStream_t s = as_stream(stream);
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
  return SPSVM_OK;
}

extern "C" int spsvm_cholesky_solve(const double* L, int64_t m, int64_t ldh, double* b,
                                    void* stream) {
  if (!L || !b || m < 0 || ldh < m) return set_error(SPSVM_ERR_ARG, "cholesky_solve: bad arguments");
  if (m == 0) return SPSVM_OK;
  chol_solve_kernel<<<1, 1024, 0, as_stream(stream)>>>(L, ldh, m, b);
  SPSVM_LAUNCH_CHECK();
  return SPSVM_OK;
}
