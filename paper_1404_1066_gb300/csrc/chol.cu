// FP64 Cholesky factorisation H = L L^T and the two triangular solves of
// the Newton system of Section 4's reoptimisation.  Blocked right-looking
// factorisation with 64 x 64 blocks: diagonal block in shared memory, panel
// triangular solve, trailing symmetric update.
#include "internal.h"

namespace spsvm {

namespace {

constexpr int NB = 64;   // diagonal blocks of the triangular solve
constexpr int PB = 32;   // panel width of the factorisation

// 1 / sqrt(d) in FP64 without the long-latency FP64 sqrt and division: the
// FP32 estimate refined by two Newton steps y <- y (3 - d y^2) / 2, each of
// which doubles the number of correct bits (about 23 -> 46 -> full FP64).
__device__ __forceinline__ double rsqrt_fp64(double d) {
  double y = (double)rsqrtf((float)d);
  y = y * fma(-0.5 * d, y * y, 1.5);
  y = y * fma(-0.5 * d, y * y, 1.5);
  return y;
}

__device__ __forceinline__ double shfl_d(double v, int src) {
  return __shfl_sync(0xffffffffu, v, src);
}

// Factors the PB x PB diagonal block at k0 in place with one warp: lane i
// holds row i of the block in registers; pivots and column entries are
// broadcast with warp shuffles.
__global__ void __launch_bounds__(32) potrf_diag(double* __restrict__ H, int64_t ldh, int64_t m,
                                                 int64_t k0, int32_t* __restrict__ info) {
  if (*info != 0) return;
  const int nb = (int)min64(PB, m - k0);
  const int i = threadIdx.x;
  double a[PB];
#pragma unroll
  for (int c = 0; c < PB; ++c)
    a[c] = (i < nb && c <= i) ? H[(k0 + i) * ldh + k0 + c] : (c == i ? 1.0 : 0.0);
  int fail = 0;
#pragma unroll
  for (int j = 0; j < PB; ++j) {
    if (j < nb && fail == 0) {
      const double djj = shfl_d(a[j], j);   // A[j][j], updated by the previous columns
      if (!(djj > 0.0) || !(djj < 1e300)) {
        fail = j + 1;
      } else {
        const double y = rsqrt_fp64(djj);
        if (i == j) a[j] = djj * y;          // L_jj = sqrt(d)
        else if (i > j) a[j] *= y;           // L[i][j]
#pragma unroll
        for (int l = j + 1; l < PB; ++l) {
          const double llj = shfl_d(a[j], l);  // L[l][j]
          if (i >= l) a[l] = fma(-a[j], llj, a[l]);
        }
      }
    }
  }
  if (fail) {
    if (i == 0) *info = (int32_t)(k0 + fail);
    return;
  }
  if (i < nb) {
#pragma unroll
    for (int c = 0; c < PB; ++c)
      if (c <= i) H[(k0 + i) * ldh + k0 + c] = a[c];
  }
}

// Rows r >= k0 + PB: L[r][k0:k0+PB] = H[r][k0:k0+PB] L_kk^{-T}, one thread per
// row, column-oriented substitution: x_j = b_j / L_jj, then b_l -= x_j L_lj
// for the remaining l (independent updates, so the dependent chain is two
// operations per column).
__global__ void __launch_bounds__(32) trsm_panel(double* __restrict__ H, int64_t ldh, int64_t m,
                                                 int64_t k0, const int32_t* __restrict__ info) {
  __shared__ double L[PB][PB + 1];
  __shared__ double rd[PB];
  if (*info != 0) return;
  for (int e = threadIdx.x; e < PB * PB; e += blockDim.x) {
    const int r = e / PB, c = e % PB;
    L[r][c] = (c <= r) ? H[(k0 + r) * ldh + k0 + c] : 0.0;
  }
  __syncthreads();
  if (threadIdx.x < PB) rd[threadIdx.x] = 1.0 / L[threadIdx.x][threadIdx.x];
  __syncthreads();
  const int64_t r = k0 + PB + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= m) return;
  double* row = H + r * ldh + k0;
  double x[PB];
#pragma unroll
  for (int j = 0; j < PB; ++j) x[j] = row[j];
#pragma unroll
  for (int j = 0; j < PB; ++j) {
    x[j] *= rd[j];
#pragma unroll
    for (int l = j + 1; l < PB; ++l) x[l] = fma(-x[j], L[l][j], x[l]);
  }
#pragma unroll
  for (int j = 0; j < PB; ++j) row[j] = x[j];
}

// Trailing update A[r][c] -= sum_l L[r][k0+l] L[c][k0+l] for r >= c >= k0 + PB,
// 64 x 64 lower tiles.
__global__ void __launch_bounds__(256) syrk_trailing(double* __restrict__ H, int64_t ldh,
                                                     int64_t m, int64_t k0,
                                                     const int32_t* __restrict__ info) {
  __shared__ double Ar[16][64 + 1];
  __shared__ double Ac[16][64 + 1];
  if (*info != 0) return;
  const int64_t base = k0 + PB;
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
#pragma unroll
  for (int l0 = 0; l0 < PB; l0 += 16) {
    for (int e = threadIdx.x; e < 16 * 64; e += blockDim.x) {
      const int rr = e / 16, ll = e % 16;
      const int64_t gr = r0 + rr, gc = c0 + rr;
      Ar[ll][rr] = (gr < m) ? H[gr * ldh + k0 + l0 + ll] : 0.0;
      Ac[ll][rr] = (gc < m) ? H[gc * ldh + k0 + l0 + ll] : 0.0;
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

constexpr int SV_T = 256;      // threads of the block-inverse product
constexpr int SV_ROWS = 64;    // rows updated per CTA

// Loads inv(L_kk) (lower, 64 x 64, zero above the diagonal) of block k0.
__device__ __forceinline__ void load_block_inverse(const double* __restrict__ L, int64_t ldh,
                                                   int64_t k0, int nb, double (*Li)[NB + 1]) {
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int j = e / NB, i = e % NB;   // i fastest: row k0+j of the stored inverse
    double v = 0.0;
    if (i < nb && j < nb) {
      if (i == j) v = 1.0 / L[(k0 + i) * ldh + k0 + i];
      else if (j < i) v = L[(k0 + j) * ldh + k0 + i];
    }
    Li[i][j] = v;
  }
}

// Forward step for block k: z_k = inv(L_kk) b_k (into z), then b_r -= L[r][k] z_k
// for the rows below the block, one thread per row.
__global__ void __launch_bounds__(SV_T) trsv_fwd_step(const double* __restrict__ L, int64_t ldh,
                                                      int64_t m, int64_t k0,
                                                      double* __restrict__ b,
                                                      double* __restrict__ z) {
  __shared__ double Li[NB][NB + 1];
  __shared__ double zs[NB];
  __shared__ double bs[NB];
  const int nb = (int)min64(NB, m - k0);
  load_block_inverse(L, ldh, k0, nb, Li);
  if (threadIdx.x < NB) bs[threadIdx.x] = threadIdx.x < nb ? b[k0 + threadIdx.x] : 0.0;
  __syncthreads();
  {
    const int i = threadIdx.x >> 2, q = threadIdx.x & 3;
    double acc = 0.0;
#pragma unroll
    for (int j = q; j < NB; j += 4) acc += Li[i][j] * bs[j];
    acc += __shfl_xor_sync(0xffffffffu, acc, 1);
    acc += __shfl_xor_sync(0xffffffffu, acc, 2);
    if (q == 0) zs[i] = acc;
  }
  __syncthreads();
  if (blockIdx.x == 0 && threadIdx.x < nb) z[k0 + threadIdx.x] = zs[threadIdx.x];
  if (threadIdx.x >= SV_ROWS) return;
  const int64_t r = k0 + nb + (int64_t)blockIdx.x * SV_ROWS + threadIdx.x;
  if (r >= m) return;
  const double2* row = reinterpret_cast<const double2*>(L + r * ldh + k0);
  double s = 0.0;
  if (nb == NB && ((reinterpret_cast<uintptr_t>(row) & 15) == 0)) {
#pragma unroll
    for (int l = 0; l < NB / 2; ++l) {
      const double2 v = row[l];
      s += v.x * zs[2 * l] + v.y * zs[2 * l + 1];
    }
  } else {
    for (int l = 0; l < nb; ++l) s += L[r * ldh + k0 + l] * zs[l];
  }
  b[r] -= s;
}

// Backward step for block k: x_k = inv(L_kk)^T z_k (into x), then z_r -=
// sum_l L[k0+l][r] x_l for the rows r < k0, one thread per row.
__global__ void __launch_bounds__(SV_T) trsv_bwd_step(const double* __restrict__ L, int64_t ldh,
                                                      int64_t m, int64_t k0,
                                                      double* __restrict__ z,
                                                      double* __restrict__ x) {
  __shared__ double Li[NB][NB + 1];
  __shared__ double xs[NB];
  __shared__ double zsh[NB];
  const int nb = (int)min64(NB, m - k0);
  load_block_inverse(L, ldh, k0, nb, Li);
  if (threadIdx.x < NB) zsh[threadIdx.x] = threadIdx.x < nb ? z[k0 + threadIdx.x] : 0.0;
  __syncthreads();
  {
    const int j = threadIdx.x >> 2, q = threadIdx.x & 3;
    double acc = 0.0;
#pragma unroll
    for (int i = q; i < NB; i += 4) acc += Li[i][j] * zsh[i];
    acc += __shfl_xor_sync(0xffffffffu, acc, 1);
    acc += __shfl_xor_sync(0xffffffffu, acc, 2);
    if (q == 0) xs[j] = acc;
  }
  __syncthreads();
  if (blockIdx.x == 0 && threadIdx.x < nb) x[k0 + threadIdx.x] = xs[threadIdx.x];
  if (threadIdx.x >= SV_ROWS) return;
  const int64_t r = (int64_t)blockIdx.x * SV_ROWS + threadIdx.x;
  if (r >= k0) return;
  double s = 0.0;
#pragma unroll 16
  for (int l = 0; l < NB; ++l)
    if (l < nb) s += L[(k0 + l) * ldh + r] * xs[l];
  z[r] -= s;
}

}  // namespace
}  // namespace spsvm

using namespace spsvm;

namespace spsvm {
size_t chol_tc_work_bytes(int64_t m);
int chol_tc_panel_update(double* H, int64_t ldh, int64_t m, int64_t k0, const int32_t* info,
                         cudaStream_t s);
int chol_tc_trailing(double* H, int64_t ldh, int64_t m, int64_t k0, const int32_t* info,
                     void* work, cudaStream_t s);
}  // namespace spsvm

extern "C" size_t spsvm_cholesky_work_bytes(int64_t m) {
  return m > 0 ? chol_tc_work_bytes(m) : 0;
}

extern "C" int spsvm_cholesky(double* H, int64_t m, int64_t ldh, int32_t* info, void* work,
                              size_t work_bytes, void* stream) {
  if (!H || !info || m < 0 || ldh < m) return set_error(SPSVM_ERR_ARG, "cholesky: bad arguments");
  cudaStream_t s = as_stream(stream);
  ProfScope prof(PROF_CHOLESKY, s, (double)m * m * m / 3.0);
  SPSVM_CUDA_TRY(cudaMemsetAsync(info, 0, sizeof(int32_t), s));
  int64_t k0 = 0;
  if (work && work_bytes >= chol_tc_work_bytes(m)) {
    // 64-column steps with the trailing update on the tensor cores while the
    // trailing matrix is large; the last few hundred columns run natively
    for (; m - (k0 + 64) >= 256; k0 += 64) {
      potrf_diag<<<1, 32, 0, s>>>(H, ldh, m, k0, info);
      SPSVM_LAUNCH_CHECK();
      trsm_panel<<<(unsigned)ceil_div(m - (k0 + PB), 32), 32, 0, s>>>(H, ldh, m, k0, info);
      SPSVM_LAUNCH_CHECK();
      SPSVM_TRY(chol_tc_panel_update(H, ldh, m, k0, info, s));
      potrf_diag<<<1, 32, 0, s>>>(H, ldh, m, k0 + PB, info);
      SPSVM_LAUNCH_CHECK();
      trsm_panel<<<(unsigned)ceil_div(m - (k0 + 2 * PB), 32), 32, 0, s>>>(H, ldh, m, k0 + PB, info);
      SPSVM_LAUNCH_CHECK();
      SPSVM_TRY(chol_tc_trailing(H, ldh, m, k0, info, work, s));
    }
  }
  for (; k0 < m; k0 += PB) {
    potrf_diag<<<1, 32, 0, s>>>(H, ldh, m, k0, info);
    SPSVM_LAUNCH_CHECK();
    const int64_t below = m - (k0 + PB);
    if (below <= 0) break;
    trsm_panel<<<(unsigned)ceil_div(below, 32), 32, 0, s>>>(H, ldh, m, k0, info);
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
    const unsigned grid = (unsigned)(k0 > 0 ? ceil_div(k0, (int64_t)SV_ROWS) : 1);
    trsv_bwd_step<<<grid, SV_T, 0, s>>>(L, ldh, m, k0, work, b);
    SPSVM_LAUNCH_CHECK();
  }
  return SPSVM_OK;
}
