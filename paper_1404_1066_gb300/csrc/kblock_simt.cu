// Kernel block and candidate scores in plain FP32 SIMT arithmetic (the
// SPSVM_FP32 form).  RBF kernel of Section 2 through the distance expansion
// ||x - z||^2 = ||x||^2 + ||z||^2 - 2 x^T z; the basis-vector score of
// Section 4 ("Basis vector selection") fused into the same tile loop.
#include <algorithm>

#include "internal.h"

namespace spsvm {

namespace {

constexpr int TM = 128;   // points per tile
constexpr int TN = 64;    // basis / candidate columns per tile
constexpr int TK = 16;    // feature chunk
constexpr int NT = 256;   // threads: 32 (points) x 8 (columns)

// Accumulates the 128 x 64 tile of x_i^T z_c for points i0.. and columns
// idx[c0..] into acc[a][b] for point tx + 32a, column ty + 8b.
__device__ __forceinline__ void dot_tile(const float* __restrict__ X, int64_t n, int64_t d,
                                         int64_t ldx, const int64_t* __restrict__ zrow,
                                         int64_t i0, int m_here, float (*Xs)[TM + 4],
                                         float (*Zs)[TN + 4], float acc[4][8]) {
  const int t = threadIdx.x, tx = t & 31, ty = t >> 5;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
  for (int64_t k0 = 0; k0 < d; k0 += TK) {
    // X tile: 128 rows x 16 features
#pragma unroll
    for (int r = 0; r < (TM * TK) / NT; ++r) {
      const int e = t + NT * r;
      const int row = e / TK, col = e % TK;
      const int64_t i = i0 + row, k = k0 + col;
      Xs[col][row] = (i < n && k < d) ? X[i * ldx + k] : 0.f;
    }
#pragma unroll
    for (int r = 0; r < (TN * TK) / NT; ++r) {
      const int e = t + NT * r;
      const int row = e / TK, col = e % TK;
      const int64_t k = k0 + col;
      Zs[col][row] = (row < m_here && k < d) ? X[zrow[row] * ldx + k] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      float av[4], bv[8];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = Xs[kk][tx + 32 * a];
#pragma unroll
      for (int b = 0; b < 8; ++b) bv[b] = Zs[kk][ty + 8 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(NT) kernel_block_simt(
    const float* __restrict__ X, int64_t n, int64_t d, int64_t ldx,
    const float* __restrict__ norms, const int64_t* __restrict__ idx, int32_t m,
    float gamma, void* out, int32_t format, int64_t ld, int64_t plane, int64_t row0) {
  __shared__ float Xs[TK][TM + 4];
  __shared__ float Zs[TK][TN + 4];
  __shared__ int64_t zrow[TN];
  __shared__ float zn[TN];
  const int64_t i0 = (int64_t)blockIdx.x * TM;
  const int c0 = blockIdx.y * TN;
  const int m_here = min(TN, m - c0);
  if (threadIdx.x < TN) {
    const int c = threadIdx.x;
    const int64_t r = (c < m_here) ? idx[c0 + c] : 0;
    zrow[c] = r;
    zn[c] = (c < m_here) ? norms[r] : 0.f;
  }
  __syncthreads();
  float acc[4][8];
  dot_tile(X, n, d, ldx, zrow, i0, m_here, Xs, Zs, acc);
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int64_t i = i0 + tx + 32 * a;
    if (i >= n) continue;
    const float xn = norms[i];
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int c = ty + 8 * b;
      if (c >= m_here) continue;
      const float v = rbf_from_dot(xn, zn[c], acc[a][b], gamma);
      kstore(out, format, plane, (row0 + c0 + c) * ld + i, v);
    }
  }
}

// Per tile of 128 points: partial sums over i in S of (o_i - y_i) K_ic and
// K_ic^2 for the tile's 64 candidates, written to part[tile][c] (FP64).
__global__ void __launch_bounds__(NT) score_partials_simt(
    const float* __restrict__ X, int64_t n, int64_t d, int64_t ldx,
    const float* __restrict__ norms, const float* __restrict__ y,
    const float* __restrict__ o, const int64_t* __restrict__ idx, int32_t kappa,
    float gamma, double2* __restrict__ part) {
  __shared__ float Xs[TK][TM + 4];
  __shared__ float Zs[TK][TN + 4];
  __shared__ int64_t zrow[TN];
  __shared__ float zn[TN];
  __shared__ double2 red[8][TN];
  const int64_t i0 = (int64_t)blockIdx.x * TM;
  const int c0 = blockIdx.y * TN;
  const int m_here = min(TN, kappa - c0);
  if (threadIdx.x < TN) {
    const int c = threadIdx.x;
    const int64_t r = (c < m_here) ? idx[c0 + c] : 0;
    zrow[c] = r;
    zn[c] = (c < m_here) ? norms[r] : 0.f;
  }
  __syncthreads();
  float acc[4][8];
  dot_tile(X, n, d, ldx, zrow, i0, m_here, Xs, Zs, acc);
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  float res[4], act[4], xn[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int64_t i = i0 + tx + 32 * a;
    if (i < n) {
      const float oi = o[i], yi = y[i];
      const bool s = yi * oi < 1.0f;
      res[a] = s ? (oi - yi) : 0.f;
      act[a] = s ? 1.f : 0.f;
      xn[a] = norms[i];
    } else {
      res[a] = 0.f; act[a] = 0.f; xn[a] = 0.f;
    }
  }
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    const int c = ty + 8 * b;
    float gs = 0.f, hs = 0.f;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const float v = rbf_from_dot(xn[a], zn[c], acc[a][b], gamma);
      gs = fmaf(res[a], v, gs);
      hs = fmaf(act[a] * v, v, hs);
    }
    double gd = warp_sum((double)gs), hd = warp_sum((double)hs);
    if (tx == 0) red[ty][c] = make_double2(gd, hd);
  }
  __syncthreads();
  if (threadIdx.x < TN && threadIdx.x < m_here) {
    const int c = threadIdx.x;
    // each column c was written by exactly one warp (ty = c % 8)
    part[(int64_t)blockIdx.x * kappa + c0 + c] = red[c % 8][c];
  }
}

// g_k = lambda o[c] + sum_tiles G, h_k = lambda + sum_tiles H, delta = g^2/(2h).
__global__ void score_finish(const double2* __restrict__ part, int64_t tiles, int32_t kappa,
                             const float* __restrict__ o, const int64_t* __restrict__ idx,
                             double lambda, double* g, double* h, double* delta) {
  const int k = blockIdx.x;
  __shared__ double sh[32];
  double gs = 0.0, hs = 0.0;
  for (int64_t t = threadIdx.x; t < tiles; t += blockDim.x) {
    const double2 p = part[t * kappa + k];
    gs += p.x;
    hs += p.y;
  }
  gs = block_sum(gs, sh);
  __syncthreads();
  hs = block_sum(hs, sh);
  if (threadIdx.x == 0) {
    const double gg = lambda * (double)o[idx[k]] + gs;
    const double hh = lambda + hs;
    g[k] = gg;
    h[k] = hh;
    delta[k] = gg * gg / (2.0 * hh);
  }
}

}  // namespace

int launch_kernel_block_simt(const spsvm_points* p, const int64_t* idx, int32_t m,
                             float gamma, spsvm_kmat* out, int64_t row0, cudaStream_t s) {
  if (m == 0 || p->n == 0) return SPSVM_OK;
  dim3 grid((unsigned)ceil_div(p->n, TM), (unsigned)ceil_div(m, TN));
  kernel_block_simt<<<grid, NT, 0, s>>>(p->X, p->n, p->d, p->ldx, p->norms, idx, m, gamma,
                                        out->data, out->format, out->ld, out->plane, row0);
  SPSVM_LAUNCH_CHECK();
  return SPSVM_OK;
}

}  // namespace spsvm

using namespace spsvm;

extern "C" size_t spsvm_kernel_block_scratch_bytes(int64_t m, int64_t d, int32_t precision) {
  if (m < 0 || d < 1 || precision != SPSVM_BF16SPLIT) return 0;
  return kernel_block_tc_scratch(m, round_up(d, 64));
}

extern "C" int spsvm_kernel_block(const spsvm_points* p, const int64_t* idx, int32_t m,
                                  float gamma, int32_t precision, spsvm_kmat* out,
                                  int64_t row0, void* scratch, size_t scratch_bytes,
                                  void* stream) {
  if (!p || !p->X || !p->norms || !idx) return set_error(SPSVM_ERR_ARG, "kernel_block: NULL pointer");
  SPSVM_TRY(check_kmat(out, "kernel_block"));
  if (m < 0 || row0 < 0 || row0 + m > out->rows || out->n != p->n || !(gamma > 0.f))
    return set_error(SPSVM_ERR_ARG, "kernel_block: m=%d row0=%lld rows=%lld n=%lld/%lld gamma=%g",
                     m, (long long)row0, (long long)out->rows, (long long)out->n,
                     (long long)p->n, (double)gamma);
  // algorithmic work: 2 n m d multiply-adds, times the six products of the split form
  ProfScope prof(PROF_KERNEL_BLOCK, as_stream(stream),
                 (precision == SPSVM_BF16SPLIT ? 12.0 : 2.0) * (double)p->n * m * (double)p->d);
  if (precision == SPSVM_BF16SPLIT) {
    if (!p->hi || !p->mid || !p->lo)
      return set_error(SPSVM_ERR_ARG, "kernel_block: BF16SPLIT needs the split planes of the points");
    return launch_kernel_block_tc(p, idx, m, gamma, out, row0, scratch, scratch_bytes,
                                  as_stream(stream));
  }
  if (precision != SPSVM_FP32) return set_error(SPSVM_ERR_ARG, "kernel_block: bad precision");
  return launch_kernel_block_simt(p, idx, m, gamma, out, row0, as_stream(stream));
}

namespace spsvm {
int launch_score_tc(const spsvm_points* p, const float* y, const float* o, const int64_t* idx,
                    int32_t kappa, float gamma, double2* part, int64_t tiles, void* zbuf,
                    size_t zbytes, cudaStream_t s);
int64_t score_tc_tiles(int64_t n);
namespace {
// per-tile partial sums (tiles of 128 points in both forms), then room for
// the gathered candidate rows of the tensor-core form
size_t score_part_bytes(int64_t n, int32_t kappa) {
  // the larger of the two forms' tile counts (both tile 128 points today)
  const int64_t tiles = std::max<int64_t>(ceil_div(n, TM), score_tc_tiles(n));
  return (size_t)round_up(tiles * (int64_t)kappa * (int64_t)sizeof(double2), 256);
}
}  // namespace
}  // namespace spsvm

extern "C" size_t spsvm_score_scratch_bytes(int64_t n, int64_t d, int32_t kappa) {
  if (n < 0 || kappa < 0 || d < 1) return 0;
  return score_part_bytes(n, kappa) + kernel_block_tc_scratch(kappa, round_up(d, 64));
}

extern "C" int spsvm_score_candidates(const spsvm_points* p, const float* y, const float* o,
                                      const int64_t* idx, int32_t kappa, float gamma,
                                      double lambda, int32_t precision, double* g, double* h,
                                      double* delta, void* scratch, size_t scratch_bytes,
                                      void* stream) {
  if (!p || !p->X || !p->norms || !y || !o || !idx || !g || !h || !delta)
    return set_error(SPSVM_ERR_ARG, "score_candidates: NULL pointer");
  if (kappa < 0 || p->n < 1 || !(gamma > 0.f) || !(lambda > 0.0))
    return set_error(SPSVM_ERR_ARG, "score_candidates: bad arguments");
  if (kappa == 0) return SPSVM_OK;
  const size_t need = spsvm_score_scratch_bytes(p->n, p->d, kappa);
  if (scratch_bytes < need || !scratch)
    return set_error(SPSVM_ERR_OOM, "score_candidates: scratch %zu < %zu", scratch_bytes, need);
  cudaStream_t s = as_stream(stream);
  ProfScope prof(PROF_SCORE, s, (precision == SPSVM_BF16SPLIT ? 12.0 : 2.0) * (double)p->n * kappa * (double)p->d);
  double2* part = static_cast<double2*>(scratch);
  int64_t tiles = ceil_div(p->n, TM);
  if (precision == SPSVM_BF16SPLIT) {
    if (!p->hi || !p->mid || !p->lo)
      return set_error(SPSVM_ERR_ARG, "score_candidates: BF16SPLIT needs split planes");
    tiles = score_tc_tiles(p->n);
    const size_t pb = score_part_bytes(p->n, kappa);
    SPSVM_TRY(launch_score_tc(p, y, o, idx, kappa, gamma, part, tiles,
                              static_cast<char*>(scratch) + pb, scratch_bytes - pb, s));
  } else if (precision == SPSVM_FP32) {
    dim3 grid((unsigned)tiles, (unsigned)ceil_div(kappa, TN));
    score_partials_simt<<<grid, NT, 0, s>>>(p->X, p->n, p->d, p->ldx, p->norms, y, o, idx,
                                            kappa, gamma, part);
    SPSVM_LAUNCH_CHECK();
  } else {
    return set_error(SPSVM_ERR_ARG, "score_candidates: bad precision");
  }
  score_finish<<<kappa, 256, 0, s>>>(part, tiles, kappa, o, idx, lambda, g, h, delta);
  SPSVM_LAUNCH_CHECK();
  return SPSVM_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free candidate scoring.  Some callers must not allocate device
// memory at all: a serving loop that has handed the whole HBM budget to a
// pool it does not own, a host framework whose allocator owns every device
// byte, or code running where cudaMalloc would synchronise the device at a
// moment it must not.  For them the score's per-tile partial sums live in a
// fixed array in this library's device memory instead of caller scratch.
// ---------------------------------------------------------------------------
#include <cuda.h>

#include <mutex>

namespace spsvm {
namespace {
// 16 MiB: enough for n = 500,000 points and 256 candidates in either form
// (16.2 MB of per-tile partial sums and gathered candidate rows).
constexpr size_t kScoreScratchMax = size_t(16) << 20;
// Held by every GPU that loads this library until the process exits.
__device__ __align__(256) unsigned char g_score_scratch[kScoreScratchMax];
std::mutex g_score_scratch_mu;
// the array's device address per device, with the context it was looked up
// in (a context torn down and made again, e.g. by cudaDeviceReset, may load
// the module at another address: the set-up then runs again)
void* g_score_scratch_ptr[64] = {};
CUcontext g_score_scratch_ctx[64] = {};

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
CtxGetCurrentFn ctx_get_current() {
  static const CtxGetCurrentFn fn = []() {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<CtxGetCurrentFn>(f);
    cudaGetLastError();
    return (CtxGetCurrentFn) nullptr;
  }();
  return fn;
}
}  // namespace
}  // namespace spsvm

extern "C" int spsvm_score_candidates_noalloc(const spsvm_points* p, const float* y,
                                              const float* o, const int64_t* idx, int32_t kappa,
                                              float gamma, double lambda, int32_t precision,
                                              double* g, double* h, double* delta, void* stream) {
  if (!p || kappa < 0 || p->n < 1)
    return set_error(SPSVM_ERR_ARG, "score_candidates_noalloc: bad arguments");
  const size_t need = spsvm_score_scratch_bytes(p->n, p->d, kappa);
  if (need > kScoreScratchMax)
    return set_error(SPSVM_ERR_ARG,
                     "score_candidates_noalloc: n=%lld, d=%lld, kappa=%d need %zu bytes of "
                     "scratch, more than the fixed %zu-byte array; use spsvm_score_candidates",
                     (long long)p->n, (long long)p->d, kappa, need, kScoreScratchMax);
  int dev = 0;
  SPSVM_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return set_error(SPSVM_ERR_ARG, "score_candidates_noalloc: device %d", dev);
  void* ptr = nullptr;
  {
    // set-up on the first call on this device (current), and again when the
    // device's context is not the one of the last set-up: look up the
    // array's device address
    CUcontext ctx = nullptr;
    if (auto fn = ctx_get_current()) fn(&ctx);
    std::lock_guard<std::mutex> lk(g_score_scratch_mu);
    if (!g_score_scratch_ptr[dev] || g_score_scratch_ctx[dev] != ctx) {
      void* a = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&a, g_score_scratch);
      if (e != cudaSuccess || !a)
        return set_error(SPSVM_ERR_CUDA, "score_candidates_noalloc: cudaGetSymbolAddress: %s",
                         cudaGetErrorString(e));
      g_score_scratch_ptr[dev] = a;
      g_score_scratch_ctx[dev] = ctx;
    }
    ptr = g_score_scratch_ptr[dev];
  }
  return spsvm_score_candidates(p, y, o, idx, kappa, gamma, lambda, precision, g, h, delta, ptr,
                                kScoreScratchMax, stream);
}
