// FP64 Cholesky factorisation H = L L^T and the two triangular solves of
// the Newton system of Section 4's reoptimisation.  Blocked right-looking
// factorisation with 64 x 64 blocks: diagonal block in shared memory, panel
// triangular solve, trailing symmetric update.
#include <atomic>
#include <mutex>
#include <vector>

#include "internal.h"

namespace spsvm {

namespace {

constexpr int NB = 64;   // diagonal blocks of the triangular solve
constexpr int PB = 32;   // panel width of the factorisation

// 1 / sqrt(d) in FP64 without the long-latency FP64 sqrt and division: the
// FP32 estimate refined by two Newton steps y <- y (3 - d y^2) / 2, each of
// which doubles the number of correct bits (about 23 -> 46 -> full FP64).
__device__ __forceinline__ double rsqrt_t(double d) {
  double y = (double)rsqrtf((float)d);
  y = y * fma(-0.5 * d, y * y, 1.5);
  y = y * fma(-0.5 * d, y * y, 1.5);
  return y;
}

// FP32: the hardware estimate and one Newton step.
__device__ __forceinline__ float rsqrt_t(float d) {
  const float y = rsqrtf(d);
  return y * fmaf(-0.5f * d, y * y, 1.5f);
}

// GB300 issues FP64 at about half an operation per clock per SM
// sub-partition, so a warp-wide FP64 instruction occupies its pipe for ~64
// clocks: the panel kernels below spread their FP64 work over four warps (all
// four sub-partitions) and give each thread columns interleaved with stride
// 4, so that a triangular loop wastes at most one predicated slot per step.
constexpr int PT = 128;   // threads of the panel kernels

// Factors the PB x PB diagonal block at k0 in place, left-looking: for
// column j, every row r >= j first subtracts sum_{k<j} L[r][k] L[j][k] (four
// threads per row, each over k = q mod 4, two accumulators, reduced by
// shuffle), then warp 0 alone takes the pivot: L_jj = sqrt(d), L[r][j] /= L_jj.
// Only one warp spends FP64 issue slots on the reciprocal square root, and
// no rank-1 update sits between two pivots.
template <typename T>
__global__ void __launch_bounds__(PT) potrf_diag(T* __restrict__ H, int64_t ldh, int64_t m,
                                                 int64_t k0, int32_t* __restrict__ info) {
  __shared__ T A[PB][PB + 1];
  __shared__ int fail_s;
  if (*info != 0) return;
  const int nb = (int)min64(PB, m - k0);
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  for (int e = t; e < PB * PB; e += PT) {
    const int r = e / PB, c = e % PB;
    A[r][c] = (r < nb && c <= r) ? H[(k0 + r) * ldh + k0 + c] : (r == c ? 1.0 : 0.0);
  }
  if (t == 0) fail_s = 0;
  __syncthreads();
  const int r = t >> 2, q = t & 3;
  for (int j = 0; j < nb; ++j) {
    const bool act = r >= j && r < nb;
    T s0 = 0.0, s1 = 0.0;
    if (act) {
      for (int k = q; k < j; k += 8) {
        s0 = fma(A[r][k], A[j][k], s0);
        if (k + 4 < j) s1 = fma(A[r][k + 4], A[j][k + 4], s1);
      }
    }
    T sum = s0 + s1;
    sum += __shfl_xor_sync(0xffffffffu, sum, 1);
    sum += __shfl_xor_sync(0xffffffffu, sum, 2);
    if (act && q == 0) A[r][j] -= sum;
    __syncthreads();
    if (warp == 0) {
      const T d = A[j][j];
      if (!(d > 0.0) || !(d < 1e300)) {
        if (lane == 0) fail_s = j + 1;
      } else {
        const T y = rsqrt_t(d);
        if (lane > j && lane < nb) A[lane][j] *= y;   // L[lane][j]
        __syncwarp();
        if (lane == 0) A[j][j] = d * y;               // L_jj = sqrt(d)
      }
    }
    __syncthreads();
    if (fail_s) break;   // the same value in every thread
  }
  if (fail_s) {
    if (t == 0) *info = (int32_t)(k0 + fail_s);
    return;
  }
  for (int e = t; e < PB * PB; e += PT) {
    const int rr = e / PB, cc = e % PB;
    if (rr < nb && cc <= rr) H[(k0 + rr) * ldh + k0 + cc] = A[rr][cc];
  }
}

// Rows r >= k0 + PB: L[r][k0:k0+PB] = H[r][k0:k0+PB] L_kk^{-T} by
// column-oriented substitution, x_j = b_j / L_jj then b_l -= x_j L_lj for
// l > j.  Four threads per row (32 rows per CTA); thread q of a row holds
// columns q + 4 i and x_j travels by shuffle from the thread that owns it.
template <typename T>
__global__ void __launch_bounds__(PT) trsm_panel(T* __restrict__ H, int64_t ldh, int64_t m,
                                                 int64_t k0, const int32_t* __restrict__ info) {
  __shared__ T L[PB][PB + 1];
  __shared__ T rd[PB];
  if (*info != 0) return;
  for (int e = threadIdx.x; e < PB * PB; e += PT) {
    const int r = e / PB, c = e % PB;
    L[r][c] = (c <= r) ? H[(k0 + r) * ldh + k0 + c] : 0.0;
  }
  __syncthreads();
  if (threadIdx.x < PB) rd[threadIdx.x] = T(1) / L[threadIdx.x][threadIdx.x];
  __syncthreads();
  const int t = threadIdx.x, lane = t & 31, q = t & 3;
  const int64_t r = k0 + PB + (int64_t)blockIdx.x * (PT / 4) + (t >> 2);
  const bool ok = r < m;
  T* row = H + (ok ? r : k0) * ldh + k0;
  T x[PB / 4];
#pragma unroll
  for (int i = 0; i < PB / 4; ++i) x[i] = ok ? row[q + 4 * i] : 0.0;
#pragma unroll
  for (int j = 0; j < PB; ++j) {
    const int owner = j & 3, ji = j >> 2;
    if (q == owner) x[ji] *= rd[j];
    const T xj = __shfl_sync(0xffffffffu, x[ji], (lane & ~3) | owner);
#pragma unroll
    for (int i = ji; i < PB / 4; ++i)
      if (q + 4 * i > j) x[i] = fma(-xj, L[q + 4 * i][j], x[i]);
  }
  if (ok) {
#pragma unroll
    for (int i = 0; i < PB / 4; ++i) row[q + 4 * i] = x[i];
  }
}

// Trailing update A[r][c] -= sum_l L[r][k0+l] L[c][k0+l] for r >= c >= k0 + PB
// over 32 x 32 lower tiles (small tiles spread the FP64 work over more SMs);
// thread t: row t / 4 of the tile, columns t % 4 + 4 i.
template <typename T>
__global__ void __launch_bounds__(PT) syrk_trailing(T* __restrict__ H, int64_t ldh,
                                                    int64_t m, int64_t k0,
                                                    const int32_t* __restrict__ info) {
  __shared__ T Ar[PB][PB + 1];   // Ar[rr][l] = L[r0 + rr][k0 + l]
  __shared__ T Ac[PB][PB + 1];   // Ac[l][cc] = L[c0 + cc][k0 + l]
  if (*info != 0) return;
  const int64_t base = k0 + PB;
  const int64_t ntile = ceil_div(m - base, (int64_t)PB);
  // lower tile (ti >= tj) from the linear block index
  int64_t tt = blockIdx.x, ti = 0;
  while (tt > ti) {
    tt -= ti + 1;
    ++ti;
  }
  const int64_t tj = tt;
  if (ti >= ntile) return;
  const int64_t r0 = base + ti * PB, c0 = base + tj * PB;
  for (int e = threadIdx.x; e < PB * PB; e += PT) {
    const int rr = e / PB, ll = e % PB;
    const int64_t gr = r0 + rr, gc = c0 + rr;
    Ar[rr][ll] = (gr < m) ? H[gr * ldh + k0 + ll] : 0.0;
    Ac[ll][rr] = (gc < m) ? H[gc * ldh + k0 + ll] : 0.0;
  }
  __syncthreads();
  const int rr = threadIdx.x >> 2, q = threadIdx.x & 3;
  T acc[PB / 4];
#pragma unroll
  for (int i = 0; i < PB / 4; ++i) acc[i] = 0.0;
#pragma unroll 8
  for (int l = 0; l < PB; ++l) {
    const T a = Ar[rr][l];
#pragma unroll
    for (int i = 0; i < PB / 4; ++i) acc[i] = fma(a, Ac[l][q + 4 * i], acc[i]);
  }
  const int64_t r = r0 + rr;
  if (r < m) {
#pragma unroll
    for (int i = 0; i < PB / 4; ++i) {
      const int64_t c = c0 + q + 4 * i;
      if (c <= r) H[r * ldh + c] -= acc[i];
    }
  }
}

// Inverse of each lower-triangular diagonal block L_kk, stored transposed in
// the (otherwise unused) strict upper triangle of the block: element (i, j),
// i > j, of inv(L_kk) at H[(k0 + j) * ldh + k0 + i].  The diagonal of the
// inverse is 1 / L_ii and is not stored.  With L_kk = [[A, 0], [B, C]] in
// 32 x 32 blocks, inv = [[inv A, 0], [-inv C B inv A, inv C]]: the two
// half inverses are formed at once (128 threads each, row by row, four
// threads per column with a shuffle reduction), then the off-diagonal block
// by two 32 x 32 products (256 threads, four outputs each).
constexpr int DI_T = 256;
template <typename T>
__global__ void __launch_bounds__(DI_T) diag_inverse(T* __restrict__ H, int64_t ldh, int64_t m) {
  __shared__ T Ls[NB][NB + 1];   // lower: L; strict upper of each half: that half's inverse
  __shared__ T Xs[NB / 2][NB / 2 + 1];   // inv C B inv A (lower-left block), then negated
  __shared__ T rd[NB];
  const int64_t k0 = (int64_t)blockIdx.x * NB;
  const int nb = (int)min64(NB, m - k0);
  const int t = threadIdx.x;
  for (int e = t; e < NB * NB; e += DI_T) {
    const int r = e / NB, c = e % NB;
    Ls[r][c] = (r < nb && c <= r) ? H[(k0 + r) * ldh + k0 + c] : (r == c ? 1.0 : 0.0);
  }
  __syncthreads();
  if (t < NB) rd[t] = T(1) / Ls[t][t];
  __syncthreads();
  // half h (0: rows/cols 0-31, 1: 32-63); X = inv(L_hh) kept as X[i][c] at Ls[o + c][o + i]
  // (strict upper of the half), i > c; X[c][c] = rd.
  {
    const int h = t >> 7, o = 32 * h;
    const int c = (t & 127) >> 2, q = t & 3;
    for (int i = 1; i < 32; ++i) {
      // X[i][c] = -(sum_{k=c}^{i-1} L[i][k] X[k][c]) / L[i][i], c < i
      T s = 0.0;
      if (c < i) {
        for (int k = c + q; k < i; k += 4) {
          const T xkc = (k == c) ? rd[o + c] : Ls[o + c][o + k];
          s = fma(Ls[o + i][o + k], xkc, s);
        }
      }
      s += __shfl_xor_sync(0xffffffffu, s, 1);
      s += __shfl_xor_sync(0xffffffffu, s, 2);
      if (c < i && q == 0) Ls[o + c][o + i] = -s * rd[o + i];
      __syncthreads();
    }
  }
  // T = B inv A (B = L[32..63][0..31]), then X21 = -inv C T; thread: row rr, columns cc + 8 v
  {
    const int rr = t >> 3, c0 = t & 7;
    T acc[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int cc = c0 + 8 * v;
      T sum = 0.0;
      for (int k = cc; k < 32; ++k) {
        const T aik = (k == cc) ? rd[cc] : Ls[cc][k];   // inv A [k][cc]
        sum = fma(Ls[32 + rr][k], aik, sum);
      }
      acc[v] = sum;
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) Xs[rr][c0 + 8 * v] = acc[v];
    __syncthreads();
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int cc = c0 + 8 * v;
      T sum = 0.0;
      for (int k = 0; k <= rr; ++k) {
        const T cik = (k == rr) ? rd[32 + rr] : Ls[32 + k][32 + rr];   // inv C [rr][k]
        sum = fma(cik, Xs[k][cc], sum);
      }
      acc[v] = -sum;
    }
    __syncthreads();
#pragma unroll
    for (int v = 0; v < 4; ++v) Xs[rr][c0 + 8 * v] = acc[v];
  }
  __syncthreads();
  // store: element (i, j), i > j, of the inverse at H[(k0 + j) * ldh + k0 + i]
  for (int e = t; e < NB * NB; e += DI_T) {
    const int j = e / NB, i = e % NB;
    if (i <= j || i >= nb) continue;
    T v;
    if (i < 32) v = Ls[j][i];                       // inv A
    else if (j >= 32) v = Ls[j][i];                 // inv C (its strict upper, same layout)
    else v = Xs[i - 32][j];                         // lower-left block
    H[(k0 + j) * ldh + k0 + i] = v;
  }
}

// ---------------------------------------------------------------------------
// Triangular solves in one launch each.  One CTA per 64-row block row; the
// block row is taken from an atomic ticket, so every block a CTA waits for
// belongs to a CTA that started earlier and is running or done (no
// dependence on the order in which the hardware dispatches CTAs).  A CTA
// reads its off-diagonal blocks of L and the inverse of its diagonal block
// while it waits, applies each published block of the solution as it
// arrives, and publishes its own block with a release flag.  Flag values:
// 0 pending, 1 published, 2 abandoned (a wait gave up; dependants give up
// at once and the status word holds the site).
// ---------------------------------------------------------------------------
constexpr int SV_THREADS = 256;

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// One thread waits for a flag to leave 0, giving up after the wait limit
// (by default 2^23 polls, roughly a second) with the stream's status set.
__device__ unsigned wait_flag(const unsigned* f, int code, const WaitCtx& w) {
  const uint32_t lim = wait_limit(w, 1u << 23);
  for (uint32_t it = 0; it < lim; ++it) {
    const unsigned v = ld_acquire_u32(f);
    if (v != 0u) return v;
    if (it >= 16) __nanosleep(64);
  }
  wait_gave_up(w, code);
  return 2u;
}

// Inverse of the 64 x 64 diagonal block at r0 (lower), Li[i][j], from the
// transposed copy diag_inverse leaves in the upper triangle; zero-padded
// past nb.
// All of a thread's loads are issued before its first store (the block is
// read at the start of every solve CTA, the first one's on the critical path).
template <typename T>
__device__ __forceinline__ void load_diag_inverse(const T* __restrict__ L, int64_t ldh,
                                                  int64_t r0, int nb, T (*Li)[NB + 1]) {
  if (blockDim.x == SV_THREADS) {
    constexpr int PER = NB * NB / SV_THREADS;
    T v[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int e = threadIdx.x + SV_THREADS * u;
      const int j = e / NB, i = e % NB;   // stored at (row r0 + j, column r0 + i)
      v[u] = T(0);
      if (i < nb && j < nb && j <= i) v[u] = L[(r0 + j) * ldh + r0 + i];
    }
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int e = threadIdx.x + SV_THREADS * u;
      const int j = e / NB, i = e % NB;
      Li[i][j] = (i == j && i < nb) ? T(1) / v[u] : v[u];
    }
    return;
  }
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int j = e / NB, i = e % NB;   // stored at (row r0 + j, column r0 + i)
    T v = 0.0;
    if (i < nb && j < nb) {
      if (i == j) v = T(1) / L[(r0 + i) * ldh + r0 + i];
      else if (j < i) v = L[(r0 + j) * ldh + r0 + i];
    }
    Li[i][j] = v;
  }
}

// z = L^{-1} b.  Thread t: row t / 4 of the block row, columns 16 (t % 4) ..
// + 15 of each 64-column block.
template <typename T>
__global__ void __launch_bounds__(SV_THREADS) trsv_fwd_onepass(
    const T* __restrict__ L, int64_t ldh, int64_t m, const T* __restrict__ b,
    T* __restrict__ z, unsigned* __restrict__ flags, unsigned* __restrict__ ticket, WaitCtx wc) {
  __shared__ T Li[NB][NB + 1];
  __shared__ T xs[2][NB];
  __shared__ T v[NB];
  __shared__ unsigned k_s, state_s;
  const int t = threadIdx.x;
  if (t == 0) k_s = atomicAdd(ticket, 1u);
  __syncthreads();
  const int64_t k = k_s;
  const int64_t r0 = k * NB;
  const int nb = (int)min64(NB, m - r0);
  load_diag_inverse(L, ldh, r0, nb, Li);
  const int r = t >> 2, q = t & 3;
  const bool row_ok = r < nb;
  const T* __restrict__ Lrow = L + (r0 + (row_ok ? r : 0)) * ldh + 16 * q;
  T acc = 0.0;
  bool ok = true;
  for (int64_t j = 0; j < k; ++j) {
    T a[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) a[c] = row_ok ? __ldg(Lrow + j * NB + c) : 0.0;
    if (t == 0) state_s = wait_flag(&flags[j], 221, wc);
    __syncthreads();
    if (state_s != 1u) {
      ok = false;
      break;
    }
    T* xb = xs[j & 1];
    if (t < NB) xb[t] = __ldcg(z + j * NB + t);   // blocks before the last are full
    __syncthreads();
#pragma unroll
    for (int c = 0; c < 16; ++c) acc = fma(a[c], xb[16 * q + c], acc);
  }
  if (!ok) {
    if (t == 0) st_release_u32(&flags[k], 2u);
    return;
  }
  acc += __shfl_xor_sync(0xffffffffu, acc, 1);
  acc += __shfl_xor_sync(0xffffffffu, acc, 2);
  if (q == 0) v[r] = row_ok ? b[r0 + r] - acc : 0.0;
  __syncthreads();
  T sres = 0.0;
#pragma unroll
  for (int c = 0; c < 16; ++c) sres = fma(Li[r][16 * q + c], v[16 * q + c], sres);
  sres += __shfl_xor_sync(0xffffffffu, sres, 1);
  sres += __shfl_xor_sync(0xffffffffu, sres, 2);
  if (q == 0 && row_ok) __stcg(z + r0 + r, sres);
  __threadfence();
  __syncthreads();
  if (t == 0) st_release_u32(&flags[k], 1u);
}

// x = L^{-T} z.  Block rows from the last; thread t: column t % 64 of the
// block, rows 16 (t / 64) .. + 15 of each later 64-row block.
template <typename T>
__global__ void __launch_bounds__(SV_THREADS) trsv_bwd_onepass(
    const T* __restrict__ L, int64_t ldh, int64_t m, const T* __restrict__ z,
    T* __restrict__ x, unsigned* __restrict__ flags, unsigned* __restrict__ ticket, WaitCtx wc) {
  __shared__ T Li[NB][NB + 1];
  __shared__ T xs[2][NB];
  __shared__ T part[4][NB];
  __shared__ T v[NB];
  __shared__ unsigned k_s, state_s;
  const int t = threadIdx.x;
  const int64_t B = ceil_div(m, (int64_t)NB);
  if (t == 0) k_s = atomicAdd(ticket, 1u);
  __syncthreads();
  const int64_t k = B - 1 - (int64_t)k_s;
  const int64_t r0 = k * NB;
  const int nb = (int)min64(NB, m - r0);
  load_diag_inverse(L, ldh, r0, nb, Li);
  const int c = t & (NB - 1), g = t >> 6;
  T acc = 0.0;
  bool ok = true;
  for (int64_t j = B - 1; j > k; --j) {
    T a[16];
    const int64_t rb = j * NB + 16 * g;
#pragma unroll
    for (int rr = 0; rr < 16; ++rr)
      a[rr] = (c < nb && rb + rr < m) ? __ldg(L + (rb + rr) * ldh + r0 + c) : 0.0;
    if (t == 0) state_s = wait_flag(&flags[j], 222, wc);
    __syncthreads();
    if (state_s != 1u) {
      ok = false;
      break;
    }
    T* xb = xs[j & 1];
    if (t < NB) xb[t] = (j * NB + t < m) ? __ldcg(x + j * NB + t) : 0.0;
    __syncthreads();
#pragma unroll
    for (int rr = 0; rr < 16; ++rr) acc = fma(a[rr], xb[16 * g + rr], acc);
  }
  if (!ok) {
    if (t == 0) st_release_u32(&flags[k], 2u);
    return;
  }
  part[g][c] = acc;
  __syncthreads();
  if (t < NB) v[t] = (t < nb) ? z[r0 + t] - (part[0][t] + part[1][t] + part[2][t] + part[3][t]) : 0.0;
  __syncthreads();
  // x_k = Li^T v, the 64 rows of the sum split over the four thread groups
  T sres = 0.0;
#pragma unroll
  for (int i = 0; i < 16; ++i) sres = fma(Li[16 * g + i][c], v[16 * g + i], sres);
  part[g][c] = sres;
  __syncthreads();
  if (t < nb) __stcg(x + r0 + t, part[0][t] + part[1][t] + part[2][t] + part[3][t]);
  __threadfence();
  __syncthreads();
  if (t == 0) st_release_u32(&flags[k], 1u);
}

// FP32 one-pass triangular solves whose results travel as self-validating
// 64-bit words (tag << 32 | float bits; a 64-bit store is single-copy
// atomic), so a block's result needs no flag, fence or second load.  In each
// CTA warp 0 alone polls (two words per lane cover a 64-value block), takes
// up to SV_BATCH published blocks at once into shared memory, and one
// barrier hands them to the CTA.  A block that gives up publishes with the
// tag's top bit set; its dependants give up at once.
constexpr int SV_BATCH = 8;

// A refinement step's kernels return at once when the solve's stop word is
// set (the backward error was reached, or the refinement failed): the host
// enqueues several steps ahead and checks once.
__device__ __forceinline__ bool refine_stopped(const int* stop) {
  return stop && *reinterpret_cast<const volatile int*>(stop) != 0;
}


__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Warp 0: stages the published blocks blk[0], blk[1], ... (up to want, in
// that order; rows at or past m count as published zeros) into xs until the
// first one not yet published, waiting (bounded) while not even blk[0] is.
// Returns the number staged, or -1 when a block is abandoned or the wait
// runs out.
__device__ int grab_blocks(const unsigned long long* __restrict__ wt, int64_t m, int64_t first,
                           int step, int want, unsigned tag, float (*xs)[NB], int code,
                           const WaitCtx& w) {
  const uint32_t lim = wait_limit(w, 1u << 20);
  const int lane = threadIdx.x & 31;
  const unsigned abt = tag | 0x80000000u;
  for (uint32_t it = 0;; ++it) {
    unsigned long long w0[SV_BATCH], w1[SV_BATCH];
#pragma unroll
    for (int u = 0; u < SV_BATCH; ++u) {
      const int64_t base = (first + (int64_t)step * u) * NB;
      w0[u] = w1[u] = (unsigned long long)tag << 32;
      if (u < want) {
        if (base + lane < m) w0[u] = ld_relaxed_u64(wt + base + lane);
        if (base + 32 + lane < m) w1[u] = ld_relaxed_u64(wt + base + 32 + lane);
      }
    }
    int got = 0;
    bool ab = false;
#pragma unroll
    for (int u = 0; u < SV_BATCH; ++u) {
      if (u < want && got == u && !ab) {
        const unsigned h0 = (unsigned)(w0[u] >> 32), h1 = (unsigned)(w1[u] >> 32);
        ab = __any_sync(0xffffffffu, h0 == abt || h1 == abt);
        if (!ab && __all_sync(0xffffffffu, h0 == tag && h1 == tag)) {
          xs[u][lane] = __uint_as_float((unsigned)w0[u]);
          xs[u][32 + lane] = __uint_as_float((unsigned)w1[u]);
          ++got;
        }
      }
    }
    if (ab) return -1;
    if (got > 0) return got;
    if (it >= lim) {
      if (lane == 0) wait_gave_up(w, code);
      return -1;
    }
    if (it >= 8) __nanosleep(32);
  }
}

// z = L^{-1} b (FP32).  Thread t: row t / 4 of the block row, columns
// 16 (t % 4) .. + 15 of each earlier 64-column block.
__global__ void __launch_bounds__(SV_THREADS) trsv32_fwd(const float* __restrict__ L, int64_t ldh,
                                                        int64_t m, const float* __restrict__ b,
                                                        unsigned long long* __restrict__ zt,
                                                        float* __restrict__ z,
                                                        unsigned* __restrict__ ticket, unsigned tag,
                                                        WaitCtx wc, const int* stop) {
  if (refine_stopped(stop)) return;
  __shared__ float Li[NB][NB + 1];
  __shared__ float xs[SV_BATCH][NB];
  __shared__ float v[NB];
  __shared__ unsigned k_s;
  __shared__ int n_s;
  const int t = threadIdx.x;
  if (t == 0) k_s = atomicAdd(ticket, 1u);
  __syncthreads();
  const int64_t k = k_s;
  const int64_t r0 = k * NB;
  const int nb = (int)min64(NB, m - r0);
  load_diag_inverse(L, ldh, r0, nb, Li);
  const int r = t >> 2, q = t & 3;
  const bool row_ok = r < nb;
  const float* __restrict__ Lrow = L + (r0 + (row_ok ? r : 0)) * ldh + 16 * q;
  float acc = 0.0f;
  bool ok = true;
  // the row's values against block jj (zeros past k); blocks j (a) and
  // j + 1 (nxt) are loaded a step ahead of their use
  auto ld = [&](float (&v)[16], int64_t jj) {
    const bool in = row_ok && jj < k;
#pragma unroll
    for (int c = 0; c < 16; ++c) v[c] = in ? __ldg(Lrow + jj * NB + c) : 0.0f;
  };
  float a[16], nxt[16];
  ld(a, 0);
  ld(nxt, 1);
  for (int64_t j = 0; j < k;) {
    if (t < 32) {
      const int g = grab_blocks(zt, m, j, 1, (int)min64(SV_BATCH, k - j), tag, xs, 221, wc);
      if (t == 0) n_s = g;
    }
    __syncthreads();
    const int got = n_s;
    if (got < 0) {
      ok = false;
      break;
    }
#pragma unroll
    for (int c = 0; c < 16; ++c) acc = fmaf(a[c], xs[0][16 * q + c], acc);
    if (got > 1) {
#pragma unroll
      for (int c = 0; c < 16; ++c) acc = fmaf(nxt[c], xs[1][16 * q + c], acc);
    }
    for (int u = 2; u < got; ++u) {
#pragma unroll
      for (int c = 0; c < 16; ++c)
        acc = fmaf(row_ok ? __ldg(Lrow + (j + u) * NB + c) : 0.0f, xs[u][16 * q + c], acc);
    }
    __syncthreads();   // xs free again
    j += got;
    if (got == 1) {
#pragma unroll
      for (int c = 0; c < 16; ++c) a[c] = nxt[c];
    } else {
      ld(a, j);
    }
    ld(nxt, j + 1);
  }
  acc += __shfl_xor_sync(0xffffffffu, acc, 1);
  acc += __shfl_xor_sync(0xffffffffu, acc, 2);
  if (q == 0) v[r] = row_ok ? b[r0 + r] - acc : 0.0f;
  __syncthreads();
  float sres = 0.0f;
#pragma unroll
  for (int c = 0; c < 16; ++c) sres = fmaf(Li[r][16 * q + c], v[16 * q + c], sres);
  sres += __shfl_xor_sync(0xffffffffu, sres, 1);
  sres += __shfl_xor_sync(0xffffffffu, sres, 2);
  if (q == 0 && row_ok) {
    z[r0 + r] = sres;
    st_relaxed_u64(zt + r0 + r, ((unsigned long long)(ok ? tag : (tag | 0x80000000u)) << 32) |
                                    __float_as_uint(sres));
  }
}

// x = L^{-T} z (FP32).  Block rows from the last; thread t: column t % 64 of
// the block, rows 16 (t / 64) .. + 15 of each later 64-row block.
__global__ void __launch_bounds__(SV_THREADS) trsv32_bwd(const float* __restrict__ L, int64_t ldh,
                                                        int64_t m, const float* __restrict__ z,
                                                        unsigned long long* __restrict__ xt,
                                                        double* __restrict__ xacc,
                                                        double* __restrict__ xmax,
                                                        unsigned* __restrict__ ticket, unsigned tag,
                                                        WaitCtx wc, const int* stop) {
  if (refine_stopped(stop)) return;
  __shared__ float Li[NB][NB + 1];
  __shared__ float xs[SV_BATCH][NB];
  __shared__ float part[4][NB];
  __shared__ float v[NB];
  __shared__ double xm[2];
  __shared__ unsigned k_s;
  __shared__ int n_s;
  const int t = threadIdx.x;
  const int64_t B = ceil_div(m, (int64_t)NB);
  if (t == 0) k_s = atomicAdd(ticket, 1u);
  __syncthreads();
  const int64_t k = B - 1 - (int64_t)k_s;
  const int64_t r0 = k * NB;
  const int nb = (int)min64(NB, m - r0);
  load_diag_inverse(L, ldh, r0, nb, Li);
  const int c = t & (NB - 1), g = t >> 6;
  const bool col_ok = c < nb;
  float acc = 0.0f;
  bool ok = true;
  // block jj's rows against this block's column (zeros at or before k);
  // blocks j (a) and j - 1 (nxt) are loaded a step ahead of their use
  auto ld = [&](float (&v)[16], int64_t jj) {
    const int64_t rb = jj * NB + 16 * g;
    const bool live = col_ok && jj > k;
#pragma unroll
    for (int rr = 0; rr < 16; ++rr)
      v[rr] = (live && rb + rr < m) ? __ldg(L + (rb + rr) * ldh + r0 + c) : 0.0f;
  };
  float a[16], nxt[16];
  ld(a, B - 1);
  ld(nxt, B - 2);
  for (int64_t j = B - 1; j > k;) {   // later blocks, last first
    if (t < 32) {
      const int gb = grab_blocks(xt, m, j, -1, (int)min64(SV_BATCH, j - k), tag, xs, 222, wc);
      if (t == 0) n_s = gb;
    }
    __syncthreads();
    const int got = n_s;
    if (got < 0) {
      ok = false;
      break;
    }
#pragma unroll
    for (int rr = 0; rr < 16; ++rr) acc = fmaf(a[rr], xs[0][16 * g + rr], acc);
    if (got > 1) {
#pragma unroll
      for (int rr = 0; rr < 16; ++rr) acc = fmaf(nxt[rr], xs[1][16 * g + rr], acc);
    }
    for (int u = 2; u < got; ++u) {
      const int64_t rbu = (j - u) * NB + 16 * g;   // a full block (only the last is partial)
#pragma unroll
      for (int rr = 0; rr < 16; ++rr)
        acc = fmaf(col_ok ? __ldg(L + (rbu + rr) * ldh + r0 + c) : 0.0f, xs[u][16 * g + rr], acc);
    }
    __syncthreads();
    j -= got;
    if (got == 1) {
#pragma unroll
      for (int rr = 0; rr < 16; ++rr) a[rr] = nxt[rr];
    } else {
      ld(a, j);
    }
    ld(nxt, j - 1);
  }
  part[g][c] = acc;
  __syncthreads();
  if (t < NB) v[t] = (t < nb) ? z[r0 + t] - (part[0][t] + part[1][t] + part[2][t] + part[3][t]) : 0.0f;
  __syncthreads();
  float sres = 0.0f;
#pragma unroll
  for (int i = 0; i < 16; ++i) sres = fmaf(Li[16 * g + i][c], v[16 * g + i], sres);
  part[g][c] = sres;
  __syncthreads();
  // publish the block (the chain), then x += the correction in FP64 and
  // the block's maximum of |x|
  double am = 0.0;
  if (t < nb) {
    const float xv = part[0][t] + part[1][t] + part[2][t] + part[3][t];
    st_relaxed_u64(xt + r0 + t, ((unsigned long long)(ok ? tag : (tag | 0x80000000u)) << 32) |
                                    __float_as_uint(xv));
    const double xn = xacc[r0 + t] + (double)xv;
    xacc[r0 + t] = xn;
    am = fabs(xn);
  }
  if (t < NB) {   // warps 0 and 1
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) am = fmax(am, __shfl_xor_sync(0xffffffffu, am, o));
    if ((t & 31) == 0) xm[t >> 5] = am;
  }
  __syncthreads();
  if (t == 0) xmax[k] = fmax(xm[0], xm[1]);
}

// ---------------------------------------------------------------------------
// Mixed precision: FP32 factor of H + shift I, FP64 iterative refinement.
// ---------------------------------------------------------------------------
constexpr int MX_T = 256;

// FP64 -> FP32 with round to nearest even, from the IEEE-754 encodings with
// integer operations only (GB300 issues the FP64 conversion instruction at
// its FP64 rate).  Results below the FP32 normal range flush to signed zero
// and results above it become infinity (an FP32 factor then breaks down and
// the caller falls back to FP64).
__device__ __forceinline__ float f64_to_f32_rn(double v) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  const unsigned sign = (unsigned)(u >> 32) & 0x80000000u;
  const int e = (int)((u >> 52) & 0x7ff) - 1023 + 127;
  const unsigned long long man = u & 0xfffffffffffffull;
  if ((int)((u >> 52) & 0x7ff) == 0x7ff)   // inf / nan
    return __uint_as_float(sign | 0x7f800000u | (man ? 0x400000u : 0u));
  if (e <= 0) return __uint_as_float(sign);
  if (e >= 255) return __uint_as_float(sign | 0x7f800000u);
  const unsigned m23 = (unsigned)(man >> 29);
  const unsigned rem = (unsigned)(man & 0x1fffffffu);
  const unsigned up = (rem > 0x10000000u) || (rem == 0x10000000u && (m23 & 1u));
  unsigned bits = ((unsigned)e << 23) + m23 + up;   // a carry moves into the exponent
  if (bits >= 0x7f800000u) bits = 0x7f800000u;
  return __uint_as_float(sign | bits);
}

// L (FP32, lower triangle) = H + shift I, one block per row (the row's
// loads all in flight at once); rowsum[r] = sum_c |H_rc + shift [c = r]|,
// accumulated in FP32 (a norm estimate for the backward error; GB300's FP64
// rate would make an FP64 add per element the bound of this pass).  The
// infinity norm is the maximum of rowsum (order-independent).
__global__ void __launch_bounds__(MX_T) to_f32_shift(const double* __restrict__ H, int64_t ldh,
                                                     int64_t m, double shift, float* __restrict__ L,
                                                     int64_t ldl, double* __restrict__ rowsum) {
  __shared__ float ws[MX_T / 32];
  const int64_t r = blockIdx.x;
  const double* __restrict__ Hr = H + r * ldh;
  float* __restrict__ Lr = L + r * ldl;
  float rs = 0.0f;
#pragma unroll 4
  for (int64_t c = threadIdx.x; c < m; c += MX_T) {
    float v = (c == r) ? f64_to_f32_rn(Hr[c] + shift) : f64_to_f32_rn(Hr[c]);
    rs += fabsf(v);
    if (c <= r) Lr[c] = v;
  }
  rs = warp_sum(rs);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = rs;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int k = 0; k < MX_T / 32; ++k) t += ws[k];
    rowsum[r] = (double)t;
  }
}

// ---------------------------------------------------------------------------
// FP32 factor in one persistent launch over 64 x 64 tiles, left-looking.
// Tile (i, j), i >= j, is C_ij - sum_{k<j} L_ik L_jk^T, then the factor of
// the diagonal tile (i == j) or the solve X L_jj^T = C (i > j).  One CTA
// runs the chain of diagonal and sub-diagonal tiles; the others take the
// rest by ticket, so columns overlap without a launch boundary between
// them.  A finished tile publishes its flag (1 done, 2 abandoned, 3 the
// partial a helper leaves for the chain); waits are bounded, and an
// abandoned or timed-out dependency abandons the tile.
// ---------------------------------------------------------------------------
// Upper bound on the tile factorisation's grid (0: one CTA per SM).
std::atomic<uint32_t> g_factor_ctas{0};

constexpr int DT = 64;          // tile
constexpr int DP = DT + 4;      // staging rows, 16-byte aligned
constexpr int DAG_T = 256;
// two stages of (A, B), and the chain's last diagonal tile
constexpr size_t DAG_SMEM = (size_t)5 * DT * DP * sizeof(float);

// Rows r0 .. r0+63 (zeros past m), columns c0 .. c0+63 of L as 16-byte
// vectors; a warp covers 8 rows x 64 contiguous bytes per vector.
__device__ __forceinline__ void dag_load(float4 (&v)[4], const float* __restrict__ L, int64_t ldl,
                                         int64_t m, int64_t r0, int64_t c0) {
  const int t = threadIdx.x, lane = t & 31;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int w = (t >> 5) + 8 * u;
    const int row = 8 * (w & 7) + (lane & 7), c4 = 4 * (w >> 3) + (lane >> 3);
    const int64_t gr = r0 + row;
    v[u] = gr < m ? __ldcg(reinterpret_cast<const float4*>(L + gr * ldl + c0) + c4)
                  : make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// S[l][r] = tile[r][l] (transposed, so the update reads 16-byte vectors).
__device__ __forceinline__ void dag_stage(float (*S)[DP], const float4 (&v)[4]) {
  const int t = threadIdx.x, lane = t & 31;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int w = (t >> 5) + 8 * u;
    const int row = 8 * (w & 7) + (lane & 7), c4 = 4 * (w >> 3) + (lane >> 3);
    S[4 * c4 + 0][row] = v[u].x;
    S[4 * c4 + 1][row] = v[u].y;
    S[4 * c4 + 2][row] = v[u].z;
    S[4 * c4 + 3][row] = v[u].w;
  }
}

// acc[a][b] -= sum_l A^T[l][4 ty + a] B^T[l][4 tx + b]
__device__ __forceinline__ void dag_update(float (&acc)[4][4], const float (*A)[DP],
                                           const float (*B)[DP]) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll 8
  for (int l = 0; l < DT; ++l) {
    const float4 av = *reinterpret_cast<const float4*>(&A[l][4 * ty]);
    const float4 bv = *reinterpret_cast<const float4*>(&B[l][4 * tx]);
    const float ar[4] = {av.x, av.y, av.z, av.w};
    const float br[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(-ar[a], br[b], acc[a][b]);
  }
}

__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Warp 0: the first k in [k0, j) whose flags (i, k) or (j, k) are not yet
// done (j if all are), by relaxed loads 32 at a time, followed by an acquire
// fence for the flags seen done; -1 if that first flag is abandoned.  Waits,
// bounded, while the flag at k0 itself is not done.
__device__ int64_t dag_scan(const unsigned* __restrict__ fi, const unsigned* __restrict__ fj,
                            int64_t k0, int64_t j, int code, const WaitCtx& w) {
  const int lane = threadIdx.x & 31;
  const uint32_t lim = wait_limit(w, 1u << 22);
  for (uint32_t it = 0; it < lim; ++it) {
    int64_t r = j;
    for (int64_t base = k0; base < j; base += 32) {
      const int64_t k = base + lane;
      unsigned a = 1u, b = 1u;
      if (k < j) {
        a = ld_relaxed_u32(fi + k);
        b = ld_relaxed_u32(fj + k);
      }
      const unsigned notdone = __ballot_sync(0xffffffffu, !(a == 1u && b == 1u));
      if (notdone) {
        const int first = __ffs(notdone) - 1;
        const unsigned bad = __ballot_sync(0xffffffffu, a == 2u || b == 2u);
        r = (bad >> first) & 1u ? -1 : base + first;
        break;
      }
    }
    if (r != k0) {
      asm volatile("fence.acq_rel.gpu;" ::: "memory");
      return r;
    }
    if (it >= 16) __nanosleep(64);
  }
  if (lane == 0) wait_gave_up(w, code);
  return -1;
}

// Tiles (i, j) of the factor, i >= j, left-looking: C_ij - sum_{k<j} L_ik
// L_jk^T, then the factor of a diagonal tile or the solve X L_jj^T = C of an
// off-diagonal one.  The chain of the factorisation runs through each
// diagonal tile and the tile just below it, and one CTA (the one that
// draws ticket 0) runs that chain alone: for s = 1, 2, ... it takes the partials of (s, s-1) and
// (s, s) (both accumulated over k < s-1 by helper CTAs and left in place,
// flag 3), solves (s, s-1) against (s-1, s-1), which it factored itself and
// keeps in shared memory, applies it to (s, s) and factors (s, s) -- no
// hand-off between CTAs on the chain.  The other tickets are, for s = 1,
// 2, ...: P(s) (the partial of (s, s-1)), D(s) (the partial of (s, s)),
// then the tiles (s+1 .., s-1).  With the chain's step s placed right after
// D(s), every piece of work waits only for pieces before it.  While the
// chain waits for P(s) and D(s) it takes any ticket up to D(s) that no CTA
// holds yet and does that work itself, so the schedule progresses whatever
// the number of resident CTAs, down to the chain's own (launches on other
// streams may hold the rest of the GPU).  A helper publishes its partial
// (flag 3) only over flag 0, so an abandoned chain step (flag 2) stays
// abandoned.

// Ticket tk -> work: kind 0 the chain, kind 2 the tile (i, j), kind 3 the
// helper P(s) (i = s, j = s - 1), kind 4 the helper D(s) (i = j = s); -1
// past the end.
__device__ __forceinline__ int dag_decode(int64_t tk, int64_t T, int64_t* i, int64_t* j) {
  *i = 0;
  *j = 0;
  if (tk <= 0) return tk == 0 ? 0 : -1;
  tk -= 1;
  // block s (s >= 1) = P(s), D(s), then rows s+1 .. T-1 of column s-1:
  // T - s + 1 tickets
  int64_t s = 1, start = 0;
  while (s < T && start + (T - s + 1) <= tk) {
    start += T - s + 1;
    ++s;
  }
  if (s >= T) return -1;
  const int64_t e = tk - start;
  if (e == 0) {
    *i = s;
    *j = s - 1;
    return 3;
  }
  if (e == 1) {
    *i = s;
    *j = s;
    return 4;
  }
  *i = s + e - 1;
  *j = s - 1;
  return 2;
}

// The ticket of D(s): 1 + the tickets of blocks 1 .. s-1, + 1.
__device__ __forceinline__ int64_t dag_ticket_of_D(int64_t s, int64_t T) {
  return 1 + (s - 1) * (T + 1) - (s - 1) * s / 2 + 1;
}

// Waits (bounded) for a factored diagonal tile: 1 when done, 2 when
// abandoned or the wait gave up (flag 3, the helper's partial, still waits).
__device__ unsigned dag_wait_final(const unsigned* f, const WaitCtx& w) {
  const uint32_t lim = wait_limit(w, 1u << 23);
  for (uint32_t it = 0; it < lim; ++it) {
    const unsigned v = ld_acquire_u32(f);
    if (v == 1u || v == 2u) return v;
    if (it >= 16) __nanosleep(64);
  }
  wait_gave_up(w, 224);
  return 2u;
}

// acc1 -= sum_{k<kend} L_ik L_jk^T (L_ik L_ik^T when same) as the tiles of
// columns k come in, and with TWO also acc2 -= sum_{k<kend} L_ik L_ik^T.
// All threads; false when a dependency was abandoned or a wait gave up.
template <bool TWO>
__device__ bool dag_accumulate(float (&acc1)[4][4], float (&acc2)[4][4],
                               const float* __restrict__ L, int64_t ldl, int64_t m, int64_t i,
                               int64_t j, int64_t kend, bool same,
                               const unsigned* __restrict__ flags, int64_t T,
                               float (*As)[DT][DP], float (*Bs)[DT][DP], int64_t* rdy_s,
                               const WaitCtx& wc) {
  const int t = threadIdx.x;
  bool ok = true;
  if (kend > 0) {
    // rdy: the first k whose tiles are not known to be done
    const unsigned* fi = flags + i * T;
    const unsigned* fj = flags + j * T;
    if (t < 32) {
      const int64_t r = dag_scan(fi, fj, 0, kend, 223, wc);
      if (t == 0) *rdy_s = r;
    }
    __syncthreads();
    int64_t rdy = *rdy_s;
    ok = rdy > 0;
    float4 pa[4], pb[4];
    if (ok) {
      dag_load(pa, L, ldl, m, i * DT, 0);
      if (!same) dag_load(pb, L, ldl, m, j * DT, 0);
    }
    for (int64_t k = 0; ok && k < kend; ++k) {
      const int sb = (int)(k & 1);
      dag_stage(As[sb], pa);
      if (!same) dag_stage(Bs[sb], pb);
      __syncthreads();
      const bool pre = k + 1 < rdy;
      if (pre) {   // next tiles known done: their loads overlap this update
        dag_load(pa, L, ldl, m, i * DT, (k + 1) * DT);
        if (!same) dag_load(pb, L, ldl, m, j * DT, (k + 1) * DT);
      }
      dag_update(acc1, As[sb], same ? As[sb] : Bs[sb]);
      if (TWO) dag_update(acc2, As[sb], As[sb]);
      if (k + 1 < kend && !pre) {
        if (t < 32) {
          const int64_t r = dag_scan(fi, fj, k + 1, kend, 223, wc);
          if (t == 0) *rdy_s = r;
        }
        __syncthreads();
        rdy = *rdy_s;
        if (rdy < 0) {
          ok = false;
        } else {
          dag_load(pa, L, ldl, m, i * DT, (k + 1) * DT);
          if (!same) dag_load(pb, L, ldl, m, j * DT, (k + 1) * DT);
        }
      }
    }
  }
  __syncthreads();   // staging buffers free
  return ok;
}

// Factor of a diagonal tile held transposed in shared memory (AT[c][r] =
// A[r][c], lower part; the rest is ignored), in place: AT[c][r] = L[r][c],
// rd the reciprocals of L's diagonal.  By blocks of 16 columns: one warp
// factors the 16 x 16 diagonal block (lane i holds row i; the two entries
// of row c + 2 that the next pivots need travel by shuffle ahead of the
// column update, so the chain per column is one reciprocal square root and
// two FMAs), then one thread per row solves the panel below against it, then
// the CTA applies the panel to the later column blocks.  All threads;
// returns 0, or 1 + the tile column of the first non-positive pivot.
__device__ int dag_factor_blk(float (*AT)[DP], float* __restrict__ rd, int* fail_s) {
  const int t = threadIdx.x;
  if (t == 0) *fail_s = 0;
#pragma unroll 1
  for (int q = 0; q < DT / 16; ++q) {
    const int b = 16 * q;
    if (t < 32) {
      const int i = t & 15;   // lanes 16..31 repeat lanes 0..15
      float g[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) g[j] = AT[b + j][b + i];
      // pivot d, and row c + 1's entries (c + 1, c + 1), (c + 1, c)
      float d = __shfl_sync(0xffffffffu, g[0], 0);
      float An = __shfl_sync(0xffffffffu, g[1], 1), Bn = __shfl_sync(0xffffffffu, g[0], 1);
      int fail = 0;
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        fail = (fail == 0 && !(d > 0.0f && d < 3.0e38f)) ? c + 1 : fail;
        const float y = rsqrt_t(d);
        const float l = g[c] * y;    // L[i][c] (meaningful for i > c)
        const float lb = Bn * y;     // L[c + 1][c]
        const float dn = fmaf(-lb, lb, An);
        float An2 = 0.0f, Bn2 = 0.0f;
        if (c + 2 < 16) {
          An2 = __shfl_sync(0xffffffffu, fmaf(-l, l, g[c + 2]), c + 2);
          Bn2 = __shfl_sync(0xffffffffu, fmaf(-l, lb, g[c + 1]), c + 2);
        }
        g[c] = (i == c) ? d * y : l;
        if (c + 1 < 16) g[c + 1] = fmaf(-l, lb, g[c + 1]);
#pragma unroll
        for (int j = c + 2; j < 16; ++j) g[j] = fmaf(-l, __shfl_sync(0xffffffffu, l, j), g[j]);
        if (t == 0) rd[b + c] = y;
        d = dn;
        An = An2;
        Bn = Bn2;
      }
      if (t < 16) {
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (j <= i) AT[b + j][b + i] = g[j];
      }
      if (t == 0 && fail) *fail_s = b + fail;
    }
    __syncthreads();
    if (*fail_s) return *fail_s;
    if (q + 1 == DT / 16) break;
    // the panel below, one thread per row: X L_bb^T = A[rows][b .. b + 15]
    if (t >= b + 16 && t < DT) {
      float x[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) x[k] = AT[b + k][t];
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        x[k] *= rd[b + k];
        const float* lr = &AT[b + k][b];   // lr[k2] = L[b + k2][b + k]
#pragma unroll
        for (int k2 = k + 1; k2 < 16; ++k2) x[k2] = fmaf(-x[k], lr[k2], x[k2]);
      }
#pragma unroll
      for (int k = 0; k < 16; ++k) AT[b + k][t] = x[k];
    }
    __syncthreads();
    // the later column blocks: A[r][cb] -= sum_k L[r][b + k] L[cb][b + k],
    // rows 4 r4 .. +3 at or below each block
    {
      const int r4 = t >> 4, c = t & 15;
      if (4 * r4 >= b + 16) {
        float xv[16][4];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const float4 v = *reinterpret_cast<const float4*>(&AT[b + k][4 * r4]);
          xv[k][0] = v.x; xv[k][1] = v.y; xv[k][2] = v.z; xv[k][3] = v.w;
        }
        for (int qb = q + 1; qb < DT / 16 && 16 * qb <= 4 * r4; ++qb) {
          const float4 o = *reinterpret_cast<const float4*>(&AT[16 * qb + c][4 * r4]);
          float ov[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            const float lv = AT[b + k][16 * qb + c];
#pragma unroll
            for (int e = 0; e < 4; ++e) ov[e] = fmaf(-xv[k][e], lv, ov[e]);
          }
          *reinterpret_cast<float4*>(&AT[16 * qb + c][4 * r4]) = make_float4(ov[0], ov[1], ov[2], ov[3]);
        }
      }
    }
    __syncthreads();
  }
  return 0;
}

// Lower part of a factored diagonal tile held transposed (AT[c][r] =
// L[r][c]) to L, rows below m only.
__device__ __forceinline__ void dag_store_diag_T(const float (*AT)[DP], float* __restrict__ L,
                                                 int64_t ldl, int64_t m, int64_t r0, int64_t c0) {
  const int t = threadIdx.x, r = t & (DT - 1), g = t >> 6;
  const int64_t gr = r0 + r;
  if (gr >= m || 16 * g > r) return;
  float* dst = L + gr * ldl + c0 + 16 * g;
  if (16 * g + 15 <= r) {
#pragma unroll
    for (int k4 = 0; k4 < 4; ++k4)
      __stcg(reinterpret_cast<float4*>(dst) + k4,
             make_float4(AT[16 * g + 4 * k4][r], AT[16 * g + 4 * k4 + 1][r], AT[16 * g + 4 * k4 + 2][r],
                         AT[16 * g + 4 * k4 + 3][r]));
  } else {
#pragma unroll
    for (int k = 0; k < 16; ++k)
      if (16 * g + k <= r) __stcg(dst + k, AT[16 * g + k][r]);
  }
}

// Lower part of a factored diagonal tile to L (rows below m only).
__device__ __forceinline__ void dag_store_diag(const float (&acc)[4][4], float* __restrict__ L,
                                               int64_t ldl, int64_t m, int64_t r0, int64_t c0) {
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  if (ty < tx) return;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int64_t gr = r0 + 4 * ty + a;
    if (gr >= m) continue;
    float* dst = L + gr * ldl + c0 + 4 * tx;
    if (ty > tx) {
      __stcg(reinterpret_cast<float4*>(dst), make_float4(acc[a][0], acc[a][1], acc[a][2], acc[a][3]));
    } else {
#pragma unroll
      for (int b = 0; b <= a; ++b) __stcg(dst + b, acc[a][b]);
    }
  }
}

// X L_jj^T = C for an off-diagonal tile held transposed in shared memory
// (XT[c][r] = X[r][c], C on entry), with S[c][r] = L_jj[r][c] and rd the
// reciprocals of its diagonal, by blocks of 16 columns: threads 0..63 each
// solve one row of the block against its 16 x 16 diagonal part, then every
// thread applies the block to the later ones.  The rows are independent, so
// the chain per column is one multiply and one FMA in one thread, and the
// bulk of the work is the block updates across the CTA.  All threads; ends
// with a barrier.
__device__ __forceinline__ void dag_solve_blk(float (*XT)[DP], const float (*S)[DP],
                                              const float* __restrict__ rd) {
  const int t = threadIdx.x;
#pragma unroll 1
  for (int q = 0; q < DT / 16; ++q) {
    if (t < DT) {
      float x[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) x[k] = XT[16 * q + k][t];
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        x[k] *= rd[16 * q + k];
        const float* lr = &S[16 * q + k][16 * q];   // L_jj[16 q + k2][16 q + k]
#pragma unroll
        for (int k2 = k + 1; k2 < 16; ++k2) x[k2] = fmaf(-x[k], lr[k2], x[k2]);
      }
#pragma unroll
      for (int k = 0; k < 16; ++k) XT[16 * q + k][t] = x[k];
    }
    __syncthreads();
    if (q + 1 < DT / 16) {
      // rows 4 r4 .. +3 of the later blocks' column c: C -= X_q L_jj[., q]^T
      const int r4 = t >> 4, c = t & 15;
      float xv[16][4];
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const float4 v = *reinterpret_cast<const float4*>(&XT[16 * q + k][4 * r4]);
        xv[k][0] = v.x; xv[k][1] = v.y; xv[k][2] = v.z; xv[k][3] = v.w;
      }
      for (int qb = q + 1; qb < DT / 16; ++qb) {
        const float4 o = *reinterpret_cast<const float4*>(&XT[16 * qb + c][4 * r4]);
        float ov[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const float l = S[16 * q + k][16 * qb + c];
#pragma unroll
          for (int e = 0; e < 4; ++e) ov[e] = fmaf(-xv[k][e], l, ov[e]);
        }
        *reinterpret_cast<float4*>(&XT[16 * qb + c][4 * r4]) = make_float4(ov[0], ov[1], ov[2], ov[3]);
      }
    }
    __syncthreads();
  }
}

// XT[c][r] = L[r0 + r][c0 + c] (zeros past m): thread (r, 16-column group).
__device__ __forceinline__ void dag_load_T(float (*XT)[DP], const float* __restrict__ L, int64_t ldl,
                                           int64_t m, int64_t r0, int64_t c0) {
  const int t = threadIdx.x, r = t & (DT - 1), g = t >> 6;
  const int64_t gr = r0 + r;
#pragma unroll
  for (int k4 = 0; k4 < 4; ++k4) {
    const float4 v = gr < m ? __ldcg(reinterpret_cast<const float4*>(L + gr * ldl + c0 + 16 * g) + k4)
                            : make_float4(0.f, 0.f, 0.f, 0.f);
    XT[16 * g + 4 * k4 + 0][r] = v.x;
    XT[16 * g + 4 * k4 + 1][r] = v.y;
    XT[16 * g + 4 * k4 + 2][r] = v.z;
    XT[16 * g + 4 * k4 + 3][r] = v.w;
  }
}

// L[r0 + r][c0 + c] = XT[c][r] for rows below m.
__device__ __forceinline__ void dag_store_T(const float (*XT)[DP], float* __restrict__ L, int64_t ldl,
                                            int64_t m, int64_t r0, int64_t c0) {
  const int t = threadIdx.x, r = t & (DT - 1), g = t >> 6;
  const int64_t gr = r0 + r;
  if (gr >= m) return;
#pragma unroll
  for (int k4 = 0; k4 < 4; ++k4)
    __stcg(reinterpret_cast<float4*>(L + gr * ldl + c0 + 16 * g) + k4,
           make_float4(XT[16 * g + 4 * k4][r], XT[16 * g + 4 * k4 + 1][r], XT[16 * g + 4 * k4 + 2][r],
                       XT[16 * g + 4 * k4 + 3][r]));
}

// Waits for the factored diagonal tile (j, j), stages it transposed into S
// with the reciprocals of its diagonal in rd, and solves the off-diagonal
// tile held transposed in XT against it.  All threads; false when the tile
// was abandoned or the wait gave up.
__device__ bool dag_sub_from_diag(float (*XT)[DP], const float* __restrict__ L, int64_t ldl,
                                  int64_t m, int64_t j, const unsigned* __restrict__ flags,
                                  int64_t T, float (*S)[DP], float* __restrict__ rd,
                                  unsigned* st_s, const WaitCtx& wc) {
  const int t = threadIdx.x;
  if (t == 0) *st_s = dag_wait_final(&flags[j * T + j], wc);
  __syncthreads();
  if (*st_s != 1u) return false;
  float4 pd[4];
  dag_load(pd, L, ldl, m, j * DT, j * DT);   // j < T - 1: a full tile
  dag_stage(S, pd);                          // S[c][r] = L_jj[r][c]
  __syncthreads();
  if (t < DT) rd[t] = 1.0f / S[t][t];
  __syncthreads();
  dag_solve_blk(XT, S, rd);
  return true;
}

__device__ __forceinline__ void dag_store_full(const float (&acc)[4][4], float* __restrict__ L,
                                               int64_t ldl, int64_t m, int64_t r0, int64_t c0) {
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int64_t gr = r0 + 4 * ty + a;
    if (gr < m)
      __stcg(reinterpret_cast<float4*>(L + gr * ldl + c0 + 4 * tx),
             make_float4(acc[a][0], acc[a][1], acc[a][2], acc[a][3]));
  }
}

// The tile (i, j) of H + shift I already converted into L: full, or the
// lower part of a diagonal tile with the identity past m.
__device__ __forceinline__ void dag_load_tile(float (&acc)[4][4], const float* __restrict__ L,
                                              int64_t ldl, int64_t m, int64_t r0, int64_t c0,
                                              bool diag) {
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int r = 4 * ty + a;
    const int64_t gr = r0 + r;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int c = 4 * tx + b;
      const int64_t gc = c0 + c;
      float v = 0.0f;
      if (gr < m && gc < m && (!diag || c <= r)) v = __ldcg(L + gr * ldl + gc);
      if (diag && r == c && gr >= m) v = 1.0f;   // identity past m in the last diagonal tile
      acc[a][b] = v;
    }
  }
}

__device__ __forceinline__ void dag_publish(unsigned* flags, int64_t idx, bool ok,
                                            unsigned done = 1u) {
  __syncthreads();   // the tile's stores, then one release (cumulative over the CTA)
  if (threadIdx.x == 0) {
    __threadfence();
    st_release_u32(&flags[idx], ok ? done : 2u);
  }
}

// Stages a register tile transposed into S (S[c][r] = tile[r][c]).
__device__ __forceinline__ void dag_stage_regs(float (*S)[DP], const float (&acc)[4][4]) {
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) S[4 * tx + b][4 * ty + a] = acc[a][b];
}

// One ticket's work (all threads): a helper's partial (kinds 3 and 4) or a
// tile below the chain (kind 2).  Uses As, Bs, rd and acc; ends with the
// tile's publish.
__device__ __forceinline__ void dag_ticket_work(int kind, int64_t i, int64_t j, float* __restrict__ L,
                                                int64_t ldl, int64_t m, int64_t T,
                                                unsigned* __restrict__ flags, float (*As)[DT][DP],
                                                float (*Bs)[DT][DP], float* __restrict__ rd,
                                                int64_t* rdy_s, unsigned* st_s, const WaitCtx& wc) {
  const int t = threadIdx.x;
  float acc[4][4];
  if (kind == 3 || kind == 4) {
    // a helper: (s, s-1) or (s, s) accumulated over k < s-1, left in place
    const bool diag = kind == 4;
    const int64_t kend = i - 1;
    dag_load_tile(acc, L, ldl, m, i * DT, j * DT, diag);
    const bool ok = dag_accumulate<false>(acc, acc, L, ldl, m, i, diag ? i : j, kend, diag, flags, T,
                                          As, Bs, rdy_s, wc);
    if (ok) {
      if (diag) dag_store_diag(acc, L, ldl, m, i * DT, j * DT);
      else dag_store_full(acc, L, ldl, m, i * DT, j * DT);
    }
    __syncthreads();   // the partial's stores, then one release over flag 0 only
    if (t == 0) {
      __threadfence();
      atomicCAS(&flags[i * T + j], 0u, ok ? 3u : 2u);
    }
    return;
  }
  // an off-diagonal tile below the chain: accumulate, then solve against its
  // column's diagonal tile
  dag_load_tile(acc, L, ldl, m, i * DT, j * DT, false);
  bool ok = dag_accumulate<false>(acc, acc, L, ldl, m, i, j, j, false, flags, T, As, Bs, rdy_s, wc);
  if (ok) {
    dag_stage_regs(As[1], acc);   // transposed, for the solve
    ok = dag_sub_from_diag(As[1], L, ldl, m, j, flags, T, As[0], rd, st_s, wc);
  }
  if (ok) dag_store_T(As[1], L, ldl, m, i * DT, j * DT);
  dag_publish(flags, i * T + j, ok);
}

__global__ void __launch_bounds__(DAG_T, 1) chol32_dag(float* __restrict__ L, int64_t ldl, int64_t m,
                                                      int64_t T, unsigned* __restrict__ flags,
                                                      unsigned* __restrict__ ticket,
                                                      int32_t* __restrict__ info, WaitCtx wc) {
  extern __shared__ __align__(16) float dag_smem[];
  float (*As)[DT][DP] = reinterpret_cast<float (*)[DT][DP]>(dag_smem);
  float (*Bs)[DT][DP] = reinterpret_cast<float (*)[DT][DP]>(dag_smem + 2 * DT * DP);
  float (*Cs)[DP] = reinterpret_cast<float (*)[DP]>(dag_smem + 4 * DT * DP);
  __shared__ int64_t tile_s[2], rdy_s, took_s;
  __shared__ int kind_s, chs_s;
  __shared__ unsigned st_s;
  __shared__ float rd[DT], rdc[DT];
  __shared__ int fail_s;
  const int t = threadIdx.x;
  if (t == 0) {
    const int64_t tk = (int64_t)atomicAdd(ticket, 1u);
    int64_t i = 0, j = 0;
    kind_s = dag_decode(tk, T, &i, &j);
    tile_s[0] = i;
    tile_s[1] = j;
  }
  __syncthreads();
  if (kind_s == 0) {
    // ---- the chain: (0, 0), then for s = 1, 2, ... (s, s-1) and (s, s).
    // Cs keeps the last factored diagonal tile transposed (with rdc the
    // reciprocals of its diagonal); As[1] holds the sub-diagonal tile
    // transposed, for its solve and for the update of (s, s).
    int64_t s = 0;
    bool ok = true;
    {
      float acc[4][4];
      dag_load_tile(acc, L, ldl, m, 0, 0, true);
      dag_stage_regs(Cs, acc);
    }
    __syncthreads();
    {
      const int f = dag_factor_blk(Cs, rdc, &fail_s);
      if (f) {
        if (t == 0) atomicCAS(info, 0, (int32_t)f);
        ok = false;
      } else {
        dag_store_diag_T(Cs, L, ldl, m, 0, 0);
      }
    }
    dag_publish(flags, 0, ok);
    const uint32_t lim = wait_limit(wc, 1u << 23);
    for (s = 1; ok && s < T; ++s) {
      // the helpers' partials of (s, s-1) and (s, s); meanwhile this CTA
      // takes any ticket up to D(s) that nobody holds yet
      const int64_t tkD = dag_ticket_of_D(s, T);
      for (uint32_t idle = 0;;) {
        if (t == 0) {
          const unsigned fp = ld_acquire_u32(&flags[s * T + s - 1]);
          const unsigned fd = ld_acquire_u32(&flags[s * T + s]);
          int st = 0;   // 0 pending, 1 both ready, 2 abandoned
          if (fp == 3u && fd == 3u) st = 1;
          else if ((fp != 0u && fp != 3u) || (fd != 0u && fd != 3u)) st = 2;
          int64_t took = -1;
          if (st == 0) {
            const unsigned cur = ld_relaxed_u32(ticket);
            if ((int64_t)cur <= tkD && atomicCAS(ticket, cur, cur + 1u) == cur) took = cur;
          }
          chs_s = st;
          took_s = took;
        }
        __syncthreads();
        const int st = chs_s;
        const int64_t took = took_s;
        __syncthreads();   // read before thread 0 writes them again
        if (st == 1) break;
        if (st == 2) {
          ok = false;
          break;
        }
        if (took >= 0) {
          int64_t i = 0, j = 0;
          const int kind = dag_decode(took, T, &i, &j);
          dag_ticket_work(kind, i, j, L, ldl, m, T, flags, As, Bs, rd, &rdy_s, &st_s, wc);
          idle = 0;
          continue;
        }
        if (++idle >= lim) {
          if (t == 0) wait_gave_up(wc, 225);
          ok = false;
          break;
        }
        if (idle >= 16) __nanosleep(64);
      }
      if (!ok) break;
      float accd[4][4];
      dag_load_T(As[1], L, ldl, m, s * DT, (s - 1) * DT);
      dag_load_tile(accd, L, ldl, m, s * DT, s * DT, true);
      __syncthreads();
      dag_solve_blk(As[1], Cs, rdc);
      dag_store_T(As[1], L, ldl, m, s * DT, (s - 1) * DT);
      dag_publish(flags, s * T + s - 1, true);
      // (s, s) -= L_s,s-1 L_s,s-1^T (As[1] holds it transposed), then its factor
      dag_update(accd, As[1], As[1]);
      dag_stage_regs(Cs, accd);   // the solve above was the last reader of L_{s-1,s-1}
      __syncthreads();
      const int f = dag_factor_blk(Cs, rdc, &fail_s);
      if (f) {
        if (t == 0) atomicCAS(info, 0, (int32_t)(s * DT + f));
        ok = false;
      } else {
        dag_store_diag_T(Cs, L, ldl, m, s * DT, s * DT);
      }
      dag_publish(flags, s * T + s, ok);
      __syncthreads();   // As[1] is rewritten at the top of the next step
    }
    if (!ok) {
      // the rest of the chain is abandoned: its waiters give up at once
      __syncthreads();
      if (t == 0) {
        __threadfence();
        for (int64_t r = s; r < T; ++r) {
          if (r > 0) st_release_u32(&flags[r * T + r - 1], 2u);
          st_release_u32(&flags[r * T + r], 2u);
        }
      }
    }
    return;
  }
  // ---- helpers and the other tiles, by ticket
  for (bool first = true;; first = false) {
    if (!first) {
      __syncthreads();   // every thread has read the last ticket's kind_s, tile_s
      if (t == 0) {
        const int64_t tk = (int64_t)atomicAdd(ticket, 1u);
        int64_t i = 0, j = 0;
        kind_s = dag_decode(tk, T, &i, &j);
        tile_s[0] = i;
        tile_s[1] = j;
      }
      __syncthreads();
    }
    const int kind = kind_s;
    const int64_t i = tile_s[0], j = tile_s[1];
    if (kind < 0) return;
    dag_ticket_work(kind, i, j, L, ldl, m, T, flags, As, Bs, rd, &rdy_s, &st_s, wc);
  }
}

// r = b - (H + shift I) x (H full and symmetric, FP64), one warp per row,
// 16-byte loads four deep per lane when H's rows and x are 16-byte aligned;
// z = (float) r, the next refinement step's right-hand side; block maxima
// of |r|.
template <bool VEC>
__global__ void __launch_bounds__(MX_T) residual_f64(const double* __restrict__ H, int64_t ldh,
                                                     int64_t m, double shift,
                                                     const double* __restrict__ b,
                                                     const double* __restrict__ x,
                                                     double* __restrict__ r,
                                                     float* __restrict__ z,
                                                     double* __restrict__ rmax, const int* stop) {
  if (refine_stopped(stop)) return;
  __shared__ double wm[MX_T / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t i = (int64_t)blockIdx.x * (MX_T / 32) + w;
  double a = 0.0;
  if (i < m) {
    const double* __restrict__ Hi = H + i * ldh;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    if (VEC) {
      const double2* __restrict__ H2 = reinterpret_cast<const double2*>(Hi);
      const double2* __restrict__ x2 = reinterpret_cast<const double2*>(x);
      const int64_t half = m >> 1;
      for (int64_t c = lane; c < half; c += 128) {
        double2 h0 = make_double2(0, 0), h1 = h0, h2 = h0, h3 = h0;
        double2 x0 = h0, x1 = h0, y2 = h0, x3 = h0;
        if (c < half) { h0 = H2[c]; x0 = x2[c]; }
        if (c + 32 < half) { h1 = H2[c + 32]; x1 = x2[c + 32]; }
        if (c + 64 < half) { h2 = H2[c + 64]; y2 = x2[c + 64]; }
        if (c + 96 < half) { h3 = H2[c + 96]; x3 = x2[c + 96]; }
        s0 = fma(h0.y, x0.y, fma(h0.x, x0.x, s0));
        s1 = fma(h1.y, x1.y, fma(h1.x, x1.x, s1));
        s2 = fma(h2.y, y2.y, fma(h2.x, y2.x, s2));
        s3 = fma(h3.y, x3.y, fma(h3.x, x3.x, s3));
      }
      if ((m & 1) && lane == 0) s0 = fma(Hi[m - 1], x[m - 1], s0);
    } else {
      for (int64_t c = lane; c < m; c += 128) {
        s0 = fma(Hi[c], x[c], s0);
        if (c + 32 < m) s1 = fma(Hi[c + 32], x[c + 32], s1);
        if (c + 64 < m) s2 = fma(Hi[c + 64], x[c + 64], s2);
        if (c + 96 < m) s3 = fma(Hi[c + 96], x[c + 96], s3);
      }
    }
    const double s = warp_sum((s0 + s1) + (s2 + s3));
    if (lane == 0) {
      const double ri = b[i] - s - shift * x[i];
      r[i] = ri;
      z[i] = f64_to_f32_rn(ri);
      a = fabs(ri);
    }
  }
  if (lane == 0) wm[w] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double mx = 0.0;
    for (int k = 0; k < MX_T / 32; ++k) mx = fmax(mx, wm[k]);
    rmax[blockIdx.x] = mx;
  }
}

// Block maxima of |v|, and z = (float) v.
__global__ void __launch_bounds__(MX_T) absmax_blocks(const double* __restrict__ v, int64_t m,
                                                      double* __restrict__ out, float* __restrict__ z) {
  __shared__ double wm[MX_T / 32];
  const int64_t i = (int64_t)blockIdx.x * MX_T + threadIdx.x;
  double a = 0.0;
  if (i < m) {
    a = fabs(v[i]);
    z[i] = f64_to_f32_rn(v[i]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double mx = 0.0;
    for (int k = 0; k < MX_T / 32; ++k) mx = fmax(mx, wm[k]);
    out[blockIdx.x] = mx;
  }
}

// ---------------------------------------------------------------------------
// Low-rank correction of the FP32 factor.  Between Newton steps of Section
// 4's reoptimisation the active set changes by a few points, and with it the
// Newton matrix by a rank-k term: H = H_a + W^T Sigma W, W (k x m) the kernel
// rows of the points that entered (Sigma = +1) or left (-1) S since the
// factored matrix H_a = L L^T.  With V = L^{-1} W^T (m x k) and the k x k
// capacitance C = Sigma + V^T V, the Sherman-Morrison-Woodbury identity gives
//   H^{-1} = L^{-T} (I - V C^{-1} V^T) L^{-1},
// which the refinement loop applies as its preconditioner (the residual is
// still taken with the freshly built FP64 H, so the result reaches the same
// FP64 backward error).
// ---------------------------------------------------------------------------
constexpr int LR_G = 16;     // columns of a V tile
constexpr int LR_T = 256;    // threads of the tile solve

// Tile (block row i, column group g) of V = L^{-1} W^T, left-looking:
// V_ig = L_ii^{-1} (W_ig - sum_{j<i} L_ij V_jg).  Tiles are taken by ticket
// in (i, g) order, so each waits only for tiles of CTAs that started before
// it.  Thread t: row t / 4, columns 4 (t % 4) .. + 3 of the tile.  Flags:
// 0 pending, 1 published, 2 abandoned (a wait gave up).
__global__ void __launch_bounds__(LR_T) lr_trsm_fwd(const float* __restrict__ L, int64_t ldl,
                                                   int64_t m, const float* __restrict__ Wt,
                                                   int64_t ldw_in, int32_t k,
                                                   float* __restrict__ V, int64_t ldv, int32_t G,
                                                   unsigned* __restrict__ flags,
                                                   unsigned* __restrict__ ticket, WaitCtx wc) {
  __shared__ float Li[NB][NB + 1];
  __shared__ float Ls[NB][NB + 1];
  __shared__ float Vs[NB][LR_G];
  __shared__ unsigned k_s;
  __shared__ unsigned st_s;
  const int t = threadIdx.x;
  if (t == 0) k_s = atomicAdd(ticket, 1u);
  __syncthreads();
  const int64_t i = k_s / G;
  const int g = (int)(k_s % G);
  const int64_t r0 = i * NB;
  const int nb = (int)min64(NB, m - r0);
  const int r = t >> 2, c0 = 4 * (t & 3);
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  bool ok = true;
  // the diagonal block's inverse does not depend on V: read it first, off
  // the chain of tiles
  load_diag_inverse(L, ldl, r0, nb, Li);
  for (int64_t j = 0; j < i && ok; ++j) {
    // (the previous pass's reads of Ls / Vs end at this barrier)
    if (t == 0) st_s = wait_flag(&flags[j * G + g], 231, wc);
    __syncthreads();
    if (st_s != 1u) {
      ok = false;
      break;
    }
    for (int e = t; e < NB * NB; e += LR_T) {
      const int rr = e / NB, cc = e % NB;
      Ls[rr][cc] = rr < nb ? L[(r0 + rr) * ldl + j * NB + cc] : 0.f;
    }
    for (int e = t; e < NB * LR_G; e += LR_T) {
      const int rr = e / LR_G, cc = e % LR_G;
      Vs[rr][cc] = __ldcg(V + (j * NB + rr) * ldv + g * LR_G + cc);
    }
    __syncthreads();
#pragma unroll 8
    for (int q = 0; q < NB; ++q) {
      const float a = Ls[r][q];
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[c] = fmaf(a, Vs[q][c0 + c], acc[c]);
    }
  }
  __syncthreads();
  // right-hand side minus the updates, then the diagonal-block inverse
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int col = g * LR_G + c0 + c;   // columns past k are zero
    Vs[r][c0 + c] = (r < nb && col < k) ? Wt[(r0 + r) * ldw_in + col] - acc[c] : 0.f;
  }
  __syncthreads();
  float out[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 8
  for (int q = 0; q < NB; ++q) {
    const float a = Li[r][q];
#pragma unroll
    for (int c = 0; c < 4; ++c) out[c] = fmaf(a, Vs[q][c0 + c], out[c]);
  }
  if (r < nb)
#pragma unroll
    for (int c = 0; c < 4; ++c) __stcg(V + (r0 + r) * ldv + g * LR_G + c0 + c, out[c]);
  __threadfence();
  __syncthreads();
  if (t == 0) st_release_u32(&flags[i * G + g], ok ? 1u : 2u);
}

// Partial sums of V^T V over slices of LR_ROWS rows of V (FP32 products,
// FP64 sums): part[z][a][b] for slice z.  One block per 16 x 16 tile of the
// k x k result and slice; thread t: entry (t / 16, t % 16).
constexpr int LR_ROWS = 256;
__global__ void __launch_bounds__(256) lr_capacitance(const float* __restrict__ V, int64_t ldv,
                                                     int64_t m, int64_t ldp,
                                                     double* __restrict__ part) {
  __shared__ float A[64][LR_G + 1], B[64][LR_G + 1];
  const int a = threadIdx.x >> 4, b = threadIdx.x & 15;
  const int ga = blockIdx.x * LR_G, gb = blockIdx.y * LR_G;
  const int64_t lo = (int64_t)blockIdx.z * LR_ROWS, hi = min64(m, lo + LR_ROWS);
  double acc = 0.0;
  for (int64_t i0 = lo; i0 < hi; i0 += 64) {
    for (int e = threadIdx.x; e < 64 * LR_G; e += 256) {
      const int rr = e / LR_G, cc = e % LR_G;
      const bool in = i0 + rr < hi;
      A[rr][cc] = in ? V[(i0 + rr) * ldv + ga + cc] : 0.f;
      B[rr][cc] = in ? V[(i0 + rr) * ldv + gb + cc] : 0.f;
    }
    __syncthreads();
    float f = 0.f;
#pragma unroll 8
    for (int q = 0; q < 64; ++q) f = fmaf(A[q][a], B[q][b], f);
    acc += (double)f;
    __syncthreads();
  }
  part[(int64_t)blockIdx.z * ldp * ldp + (int64_t)(ga + a) * ldp + gb + b] = acc;
}

// C = Sigma + sum_z part[z] (slices in order), stored FP32 with row pitch ldc.
__global__ void lr_capacitance_sum(const double* __restrict__ part, int64_t slices, int64_t ldp,
                                   const float* __restrict__ sign, int32_t k, float* __restrict__ C,
                                   int64_t ldc) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)k * k) return;
  const int64_t a = e / k, b = e % k;
  double v = a == b ? (double)sign[a] : 0.0;
  for (int64_t z = 0; z < slices; ++z) v += part[z * ldp * ldp + a * ldp + b];
  C[a * ldc + b] = (float)v;
}

// In-place Gauss-Jordan inversion of the k x k capacitance with partial
// pivoting (one CTA; C in shared memory): C <- C^{-1}.  info: 0, or p + 1
// when pivot p is below kLrPivotTol of the largest entry of C (C too
// ill-conditioned for an FP32 inverse: the caller refactors instead).
constexpr int LR_INV_T = 1024;
// a pivot below this fraction of max |C| rejects the correction: an FP32
// inverse of a worse-conditioned capacitance slows the refinement down more
// than a fresh factorisation costs
constexpr float kLrPivotTol = 1e-3f;
__global__ void __launch_bounds__(LR_INV_T) lr_invert(float* __restrict__ C, int64_t ldc, int32_t k,
                                                      int32_t* __restrict__ info) {
  extern __shared__ float sh[];
  float* A = sh;                              // k x (k + 1)
  int* perm = reinterpret_cast<int*>(A + k * (k + 1));
  __shared__ int piv_s;
  __shared__ float cmax_s;
  __shared__ float wmax[32];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int ld = k + 1;
  float lmax = 0.f;
  for (int e = t; e < k * k; e += LR_INV_T) {
    const float v = C[(e / k) * ldc + e % k];
    A[(e / k) * ld + e % k] = v;
    lmax = fmaxf(lmax, fabsf(v));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
  if (lane == 0) wmax[w] = lmax;
  __syncthreads();
  if (t == 0) {
    float mx = 0.f;
    for (int q = 0; q < LR_INV_T / 32; ++q) mx = fmaxf(mx, wmax[q]);
    cmax_s = mx;
  }
  __syncthreads();
  const float tiny = kLrPivotTol * cmax_s;
  for (int p = 0; p < k; ++p) {
    // pivot: the largest |A[r][p]|, r >= p (ties to the smaller row)
    if (w == 0) {
      float best = -1.f;
      int bi = p;
      for (int rr = p + lane; rr < k; rr += 32) {
        const float v = fabsf(A[rr * ld + p]);
        if (v > best) { best = v; bi = rr; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (lane == 0) {
        piv_s = (best > tiny) ? bi : -1;
        perm[p] = bi;
      }
    }
    __syncthreads();
    const int pr = piv_s;
    if (pr < 0) {
      if (t == 0) *info = p + 1;
      return;
    }
    if (pr != p)
      for (int c = t; c < k; c += LR_INV_T) {
        const float a = A[p * ld + c];
        A[p * ld + c] = A[pr * ld + c];
        A[pr * ld + c] = a;
      }
    __syncthreads();
    const float inv = 1.0f / A[p * ld + p];
    __syncthreads();
    for (int c = t; c < k; c += LR_INV_T) A[p * ld + c] = (c == p ? 1.0f : A[p * ld + c]) * inv;
    __syncthreads();
    // eliminate column p from every other row (the pivot column becomes the
    // inverse's column: A[i][p] <- -A[i][p] / pivot)
    for (int e = t; e < k * k; e += LR_INV_T) {
      const int ii = e / k, c = e % k;
      if (ii == p) continue;
      const float f = A[ii * ld + p];
      if (c == p) continue;
      A[ii * ld + c] = fmaf(-f, A[p * ld + c], A[ii * ld + c]);
    }
    __syncthreads();
    for (int ii = t; ii < k; ii += LR_INV_T)
      if (ii != p) A[ii * ld + p] = -A[ii * ld + p] * inv;
    __syncthreads();
  }
  // undo the row interchanges as column interchanges, last first
  for (int p = k - 1; p >= 0; --p) {
    const int pr = perm[p];
    if (pr != p)
      for (int rr = t; rr < k; rr += LR_INV_T) {
        const float a = A[rr * ld + p];
        A[rr * ld + p] = A[rr * ld + pr];
        A[rr * ld + pr] = a;
      }
    __syncthreads();
  }
  for (int e = t; e < k * k; e += LR_INV_T) C[(e / k) * ldc + e % k] = A[(e / k) * ld + e % k];
  if (t == 0) *info = 0;
}

// Partial dot products s_z[a] = sum_{i in slice z} V[i][a] z[i] over slices
// of LR_ROWS rows (FP32 products and sums): one block per slice and 16
// columns; thread t: column t % 16, rows t / 16 + 16 q of the slice.
__global__ void __launch_bounds__(256) lr_dots(const float* __restrict__ V, int64_t ldv, int64_t m,
                                              const float* __restrict__ z, int64_t ldp,
                                              float* __restrict__ sp, const int* stop) {
  if (refine_stopped(stop)) return;
  __shared__ float part[16][LR_G + 1];
  const int c = threadIdx.x & 15, rr = threadIdx.x >> 4;
  const int a = blockIdx.x * LR_G + c;
  const int64_t lo = (int64_t)blockIdx.y * LR_ROWS, hi = min64(m, lo + LR_ROWS);
  float f = 0.f;
  for (int64_t i = lo + rr; i < hi; i += 16) f = fmaf(V[i * ldv + a], z[i], f);
  part[rr][c] = f;
  __syncthreads();
  if (rr == 0) {
    float v = 0.f;
    for (int q = 0; q < 16; ++q) v += part[q][c];
    sp[(int64_t)blockIdx.y * ldp + a] = v;
  }
}

// z[i] -= sum_a V[i][a] w[a], w = C^{-1} s with s the sum of the slices'
// partial dot products (fixed order), computed by every block (k^2
// multiply-adds, cheap next to a launch).  Sixteen rows per block pass; lane
// c of a row covers columns c, c + 16, ...
__global__ void __launch_bounds__(256) lr_update(const float* __restrict__ V, int64_t ldv, int64_t m,
                                                const float* __restrict__ Ci, int64_t ldc,
                                                const float* __restrict__ sp, int64_t slices,
                                                int64_t ldp, int32_t k, float* __restrict__ z,
                                                const int* stop) {
  if (refine_stopped(stop)) return;
  __shared__ float ws[SPSVM_LOWRANK_KMAX];
  __shared__ float ss[SPSVM_LOWRANK_KMAX];
  for (int a = threadIdx.x; a < k; a += 256) {
    double v = 0.0;
    for (int64_t q = 0; q < slices; ++q) v += (double)sp[q * ldp + a];
    ss[a] = (float)v;
  }
  __syncthreads();
  for (int a = threadIdx.x; a < k; a += 256) {
    float v = 0.f;
    for (int b = 0; b < k; ++b) v = fmaf(Ci[a * ldc + b], ss[b], v);
    ws[a] = v;
  }
  __syncthreads();
  const int c = threadIdx.x & 15, rr = threadIdx.x >> 4;
  for (int64_t i0 = (int64_t)blockIdx.x * 16; i0 < m; i0 += (int64_t)gridDim.x * 16) {
    const int64_t i = i0 + rr;
    float v = 0.f;
    if (i < m)
      for (int a = c; a < k; a += 16) v = fmaf(V[i * ldv + a], ws[a], v);
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, 16);
    if (c == 0 && i < m) z[i] -= v;
  }
}

// The refinement's state on the device: stop word (0 running, 1 backward
// error reached, 2 stagnation, 3 not finite, 4 the FP32 factorisation broke
// down), steps taken, the last backward error and residual norm.
struct RefineState {
  int32_t stop, iters;
  double be, rprev;
};

// Maximum of v[0..n) over the block (result in thread 0).
__device__ double block_max(const double* __restrict__ v, int64_t n, double* sh) {
  double a = 0.0;
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) a = fmax(a, v[e]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = a;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r = fmax(r, sh[k]);
  return r;
}

// After refinement step `it` (one block of MX_T threads): the norms from the
// block maxima (at the first step also ||H + shift I|| and ||b||), the
// normwise backward error ||r|| / (||H + shift I|| ||x|| + ||b||), and the
// stop word.  Stagnation (the residual norm not halved) counts from the
// third step, the first two being the FP32 solve and its first correction.
__global__ void __launch_bounds__(MX_T) refine_decide(
    const double* __restrict__ xmax, int64_t nx, const double* __restrict__ rmax, int64_t nr,
    const double* __restrict__ rowmax, int64_t nh, const double* __restrict__ bmax, int64_t nbm,
    double* __restrict__ norms, const int32_t* __restrict__ finfo, int it, double tol, void* state) {
  __shared__ double sh[MX_T / 32];
  __shared__ int stop_s;
  RefineState* st = static_cast<RefineState*>(state);
  if (threadIdx.x == 0) stop_s = *reinterpret_cast<const volatile int32_t*>(&st->stop);
  __syncthreads();
  if (stop_s) return;
  if (it == 0) {
    const double h = block_max(rowmax, nh, sh);
    const double bb = block_max(bmax, nbm, sh);
    if (threadIdx.x == 0) {
      norms[0] = h;
      norms[1] = bb;
    }
  }
  const double xn = block_max(xmax, nx, sh);
  const double rn = block_max(rmax, nr, sh);
  if (threadIdx.x != 0) return;
  if (finfo && *finfo != 0) {
    st->stop = 4;
    return;
  }
  const double hn = norms[0], bn = norms[1];
  const double denom = hn * xn + bn;
  const double be = denom > 0.0 ? rn / denom : 0.0;
  st->iters = it + 1;
  st->be = be;
  if (!(be == be)) st->stop = 3;
  else if (be <= tol) st->stop = 1;
  else if (it >= 2 && rn > 0.5 * st->rprev) st->stop = 2;
  st->rprev = rn;
}

}  // namespace
}  // namespace spsvm

using namespace spsvm;

namespace spsvm {
size_t chol_tc_work_bytes(int64_t m);
int chol_tc_panel_update(double* H, int64_t ldh, int64_t m, int64_t k0, const int32_t* info,
                         cudaStream_t s);
int chol_tc_slice(const double* H, int64_t ldh, int64_t m, int64_t k0, const int32_t* info,
                  void* work, int buf, cudaStream_t s);
int chol_tc_update(double* H, int64_t ldh, int64_t m, int64_t cbase, int64_t cend,
                   const int32_t* info, void* work, int buf, cudaStream_t s);
int chol_tc_carveout();

namespace {

// A second stream (highest priority) and two events for the look-ahead of
// the factorisation, taken from a per-device pool for the duration of one
// call.
struct SideStream {
  int dev = -1;
  cudaStream_t s = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
};

std::mutex g_side_mu;
std::vector<SideStream> g_side_pool;

int side_acquire(SideStream* out) {
  int dev = 0;
  SPSVM_CUDA_TRY(cudaGetDevice(&dev));
  {
    std::lock_guard<std::mutex> lk(g_side_mu);
    for (size_t k = 0; k < g_side_pool.size(); ++k) {
      if (g_side_pool[k].dev == dev) {
        *out = g_side_pool[k];
        g_side_pool.erase(g_side_pool.begin() + (std::ptrdiff_t)k);
        return SPSVM_OK;
      }
    }
  }
  SideStream ss;
  ss.dev = dev;
  int least = 0, greatest = 0;
  SPSVM_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&least, &greatest));
  SPSVM_CUDA_TRY(cudaStreamCreateWithPriority(&ss.s, cudaStreamNonBlocking, greatest));
  SPSVM_CUDA_TRY(cudaEventCreateWithFlags(&ss.a, cudaEventDisableTiming));
  SPSVM_CUDA_TRY(cudaEventCreateWithFlags(&ss.b, cudaEventDisableTiming));
  *out = ss;
  return SPSVM_OK;
}

void side_release(const SideStream& ss) {
  std::lock_guard<std::mutex> lk(g_side_mu);
  g_side_pool.push_back(ss);
}

struct SideGuard {
  SideStream ss;
  bool held = false;
  ~SideGuard() {
    if (held) side_release(ss);
  }
};

}  // namespace
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
  if (work && work_bytes >= chol_tc_work_bytes(m) && m - 64 >= 256) {
    // 64-column steps with the trailing update on the tensor cores while the
    // trailing matrix is large; the last few hundred columns run natively.
    // Look-ahead: the panel chain and the update of the next panel's 64
    // columns run on a high-priority stream p; the rest of the trailing
    // update runs on s while p factors the next panel (with equal
    // priorities the update's pending tiles would hold the SMs and the panel
    // kernels would wait for the whole grid).
    // the panel kernels run beside the tensor-core update, which takes the
    // largest shared-memory carveout; an SM holds CTAs of one carveout only
    SPSVM_TRY(chol_tc_carveout());
    SPSVM_CUDA_TRY(cudaFuncSetAttribute(potrf_diag<double>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                        (int)cudaSharedmemCarveoutMaxShared));
    SPSVM_CUDA_TRY(cudaFuncSetAttribute(trsm_panel<double>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                        (int)cudaSharedmemCarveoutMaxShared));
    SideGuard side;
    SPSVM_TRY(side_acquire(&side.ss));
    side.held = true;
    cudaStream_t p = side.ss.s;
    SPSVM_CUDA_TRY(cudaEventRecord(side.ss.b, s));   // H as the caller left it
    SPSVM_CUDA_TRY(cudaStreamWaitEvent(p, side.ss.b, 0));
    int buf = 0;
    for (; m - (k0 + 64) >= 256; k0 += 64, buf ^= 1) {
      potrf_diag<double><<<1, PT, 0, p>>>(H, ldh, m, k0, info);
      SPSVM_LAUNCH_CHECK();
      trsm_panel<double><<<(unsigned)ceil_div(m - (k0 + PB), PT / 4), PT, 0, p>>>(H, ldh, m, k0, info);
      SPSVM_LAUNCH_CHECK();
      SPSVM_TRY(chol_tc_panel_update(H, ldh, m, k0, info, p));
      potrf_diag<double><<<1, PT, 0, p>>>(H, ldh, m, k0 + PB, info);
      SPSVM_LAUNCH_CHECK();
      trsm_panel<double><<<(unsigned)ceil_div(m - (k0 + 2 * PB), PT / 4), PT, 0, p>>>(H, ldh, m, k0 + PB,
                                                                             info);
      SPSVM_LAUNCH_CHECK();
      // slices of this panel (the buffer was last read by the update on s
      // two panels ago, which p waited for one panel ago)
      SPSVM_TRY(chol_tc_slice(H, ldh, m, k0, info, work, buf, p));
      // the update on s of the previous panel touches the columns updated next
      SPSVM_CUDA_TRY(cudaStreamWaitEvent(p, side.ss.b, 0));
      SPSVM_TRY(chol_tc_update(H, ldh, m, k0 + 64, k0 + 128, info, work, buf, p));
      SPSVM_CUDA_TRY(cudaEventRecord(side.ss.a, p));
      SPSVM_CUDA_TRY(cudaStreamWaitEvent(s, side.ss.a, 0));
      SPSVM_TRY(chol_tc_update(H, ldh, m, k0 + 128, m, info, work, buf, s));
      SPSVM_CUDA_TRY(cudaEventRecord(side.ss.b, s));
    }
    // s has waited for everything p did (the last record of a)
  }
  for (; k0 < m; k0 += PB) {
    potrf_diag<double><<<1, PT, 0, s>>>(H, ldh, m, k0, info);
    SPSVM_LAUNCH_CHECK();
    const int64_t below = m - (k0 + PB);
    if (below <= 0) break;
    trsm_panel<double><<<(unsigned)ceil_div(below, PT / 4), PT, 0, s>>>(H, ldh, m, k0, info);
    SPSVM_LAUNCH_CHECK();
    const int64_t T = ceil_div(below, (int64_t)PB);
    syrk_trailing<double><<<(unsigned)(T * (T + 1) / 2), PT, 0, s>>>(H, ldh, m, k0, info);
    SPSVM_LAUNCH_CHECK();
  }
  if (m > 0) {
    diag_inverse<double><<<(unsigned)ceil_div(m, (int64_t)NB), DI_T, 0, s>>>(H, ldh, m);
    SPSVM_LAUNCH_CHECK();
  }
  return SPSVM_OK;
}

static int64_t solve_flags_offset(int64_t m) { return round_up(m * 8, (int64_t)256); }

extern "C" size_t spsvm_cholesky_solve_work_bytes(int64_t m) {
  if (m <= 0) return 0;
  const int64_t B = ceil_div(m, (int64_t)NB);
  return (size_t)(solve_flags_offset(m) + round_up((2 * B + 2) * 4, (int64_t)256));
}

extern "C" int spsvm_cholesky_solve(const double* L, int64_t m, int64_t ldh, double* b,
                                    void* work, size_t work_bytes, void* stream) {
  if (!L || !b || m < 0 || ldh < m) return set_error(SPSVM_ERR_ARG, "cholesky_solve: bad arguments");
  if (m == 0) return SPSVM_OK;
  if (!work || work_bytes < spsvm_cholesky_solve_work_bytes(m) ||
      (reinterpret_cast<uintptr_t>(work) & 15) != 0)
    return set_error(SPSVM_ERR_OOM, "cholesky_solve: work too small or misaligned");
  cudaStream_t s = as_stream(stream);
  ProfScope prof(PROF_SOLVE, s, 8.0 * (double)m * m);
  const int64_t B = ceil_div(m, (int64_t)NB);
  double* z = static_cast<double*>(work);
  unsigned* flags = reinterpret_cast<unsigned*>(static_cast<char*>(work) + solve_flags_offset(m));
  SPSVM_CUDA_TRY(cudaMemsetAsync(flags, 0, (size_t)(2 * B + 2) * 4, s));
  WaitCtx wc;
  SPSVM_TRY(wait_ctx(s, &wc));
  trsv_fwd_onepass<double><<<(unsigned)B, SV_THREADS, 0, s>>>(L, ldh, m, b, z, flags, flags + 2 * B, wc);
  SPSVM_LAUNCH_CHECK();
  trsv_bwd_onepass<double><<<(unsigned)B, SV_THREADS, 0, s>>>(L, ldh, m, z, b, flags + B, flags + 2 * B + 1,
                                                              wc);
  SPSVM_LAUNCH_CHECK();
  return SPSVM_OK;
}

// ---------------------------------------------------------------------------
// Mixed-precision Newton solve (host side)
// ---------------------------------------------------------------------------
namespace {

constexpr int kTicketSteps = 64;   // refinement steps between ticket resets

struct MixedLayout {
  int64_t ldl, B, nrow_blocks, nvec_blocks;
  size_t L, sw, sw_bytes, z32, r, rowmax, xmax, rmax, bmax, norms, state, dag, total;
  int64_t tiles;   // tile rows of the factor
};

MixedLayout mixed_layout(int64_t m) {
  MixedLayout ly{};
  auto al = [](size_t b) { return (size_t)round_up((int64_t)b, (int64_t)256); };
  ly.ldl = round_up(m, (int64_t)4);
  ly.B = ceil_div(m, (int64_t)NB);
  ly.nrow_blocks = ceil_div(m, (int64_t)(MX_T / 32));
  ly.nvec_blocks = ceil_div(m, (int64_t)MX_T);
  size_t off = 0;
  ly.L = off;      off += al((size_t)m * ly.ldl * 4);
  // solve scratch: the forward result (FP32), the tagged words of both
  // solves, and per-step tickets of the two launches (zeroed once per call)
  ly.sw = off;     ly.sw_bytes = al((size_t)m * 4) + al((size_t)m * 16) + al((size_t)2 * kTicketSteps * 4);
  off += ly.sw_bytes;
  ly.z32 = off;    off += al((size_t)m * 4);
  ly.r = off;      off += al((size_t)m * 8);
  ly.rowmax = off; off += al((size_t)m * 8);
  ly.xmax = off;   off += al((size_t)ly.B * 8);   // per 64-row block of the backward solve
  ly.rmax = off;   off += al((size_t)ly.nrow_blocks * 8);
  ly.bmax = off;   off += al((size_t)ly.nvec_blocks * 8);
  ly.norms = off;  off += al(8 * 8);
  ly.state = off;  off += al(sizeof(RefineState));
  ly.tiles = ceil_div(m, (int64_t)DT);
  ly.dag = off;    off += al((size_t)(ly.tiles * ly.tiles + 1) * 4);   // tile flags, ticket
  ly.total = off;
  return ly;
}

}  // namespace

extern "C" size_t spsvm_mixed_work_bytes(int64_t m) { return m > 0 ? mixed_layout(m).total : 0; }

extern "C" int spsvm_cholesky_mixed(const double* H, int64_t m, int64_t ldh, double shift,
                                    int32_t* info, void* work, size_t work_bytes, void* stream) {
  if (!H || !info || m < 0 || ldh < m || !(shift >= 0.0))
    return set_error(SPSVM_ERR_ARG, "cholesky_mixed: bad arguments");
  cudaStream_t s = as_stream(stream);
  SPSVM_CUDA_TRY(cudaMemsetAsync(info, 0, sizeof(int32_t), s));
  if (m == 0) return SPSVM_OK;
  const MixedLayout ly = mixed_layout(m);
  if (!work || work_bytes < ly.total || (reinterpret_cast<uintptr_t>(work) & 255) != 0)
    return set_error(SPSVM_ERR_OOM, "cholesky_mixed: work too small or misaligned");
  ProfScope prof(PROF_CHOLESKY, s, (double)m * m * m / 3.0);
  char* w = static_cast<char*>(work);
  float* L = reinterpret_cast<float*>(w + ly.L);
  unsigned* dflags = reinterpret_cast<unsigned*>(w + ly.dag);
  // block 0 runs the chain; the others take T (T + 1) / 2 - 1 tickets
  const int64_t T = ly.tiles, ntiles = T * (T + 1) / 2;
  SPSVM_CUDA_TRY(cudaMemsetAsync(dflags, 0, (size_t)(T * T + 1) * 4, s));
  to_f32_shift<<<(unsigned)m, MX_T, 0, s>>>(H, ldh, m, shift, L, ly.ldl,
                                            reinterpret_cast<double*>(w + ly.rowmax));
  SPSVM_LAUNCH_CHECK();
  SPSVM_CUDA_TRY(cudaFuncSetAttribute(chol32_dag, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)DAG_SMEM));
  WaitCtx wc;
  SPSVM_TRY(wait_ctx(s, &wc));
  int64_t grid = min64(ntiles, (int64_t)sm_count());
  const uint32_t cap = g_factor_ctas.load(std::memory_order_relaxed);
  if (cap > 0) grid = min64(grid, (int64_t)cap);
  chol32_dag<<<(unsigned)grid, DAG_T, DAG_SMEM, s>>>(
      L, ly.ldl, m, T, dflags, dflags + T * T, info, wc);
  SPSVM_LAUNCH_CHECK();
  diag_inverse<float><<<(unsigned)ly.B, DI_T, 0, s>>>(L, ly.ldl, m);
  SPSVM_LAUNCH_CHECK();
  return SPSVM_OK;
}

namespace {

// The low-rank correction's state inside its work buffer (sizes from k).
struct LowRankLayout {
  int64_t ldv, G, slices;
  size_t V, Ci, s, cpart, flags, total;
};

LowRankLayout lowrank_layout(int64_t m, int32_t k) {
  auto al = [](size_t b) { return (size_t)round_up((int64_t)b, (int64_t)256); };
  LowRankLayout ly{};
  ly.G = ceil_div((int64_t)k, (int64_t)LR_G);
  ly.ldv = ly.G * LR_G;
  ly.slices = ceil_div(m, (int64_t)LR_ROWS);
  const int64_t B = ceil_div(m, (int64_t)NB);
  size_t off = 0;
  ly.V = off;      off += al((size_t)B * NB * ly.ldv * 4);
  ly.Ci = off;     off += al((size_t)k * ly.ldv * 4);
  ly.s = off;      off += al((size_t)ly.slices * ly.ldv * 4);              // partial dots
  ly.cpart = off;  off += al((size_t)ly.slices * ly.ldv * ly.ldv * 8);     // partial V^T V
  ly.flags = off;  off += al((size_t)(B * ly.G + 1) * 4);
  ly.total = off;
  return ly;
}

struct LowRankView {
  const float* V;
  const float* Ci;
  float* s;
  int64_t ldv, slices;
  int32_t k, G;
};

}  // namespace

// Refinement steps queued before the first host check.
constexpr int kRefineAhead = 3;

static int solve_mixed_impl(const double* H, int64_t m, int64_t ldh, double shift,
                            const double* b, double* x, int32_t max_iter, double tol,
                            int32_t* iters, double* backward_error, void* work,
                            size_t work_bytes, const LowRankView* lr, const int32_t* factor_info,
                            void* stream) {
  if (!H || !b || !x || m < 0 || ldh < m || max_iter < 1 || !(tol > 0.0) || !(shift >= 0.0))
    return set_error(SPSVM_ERR_ARG, "solve_mixed: bad arguments");
  if (iters) *iters = 0;
  if (backward_error) *backward_error = 0.0;
  if (m == 0) return SPSVM_OK;
  const MixedLayout ly = mixed_layout(m);
  if (!work || work_bytes < ly.total || (reinterpret_cast<uintptr_t>(work) & 255) != 0)
    return set_error(SPSVM_ERR_OOM, "solve_mixed: work too small or misaligned");
  cudaStream_t s = as_stream(stream);
  ProfScope prof(PROF_SOLVE, s, 8.0 * (double)m * m);
  char* w = static_cast<char*>(work);
  const float* L = reinterpret_cast<const float*>(w + ly.L);
  float* zw = reinterpret_cast<float*>(w + ly.sw);
  char* tagged_region = w + ly.sw + round_up(m * 4, (int64_t)256);
  unsigned long long* zt = reinterpret_cast<unsigned long long*>(tagged_region);
  unsigned long long* xt = zt + m;
  unsigned* tickets = reinterpret_cast<unsigned*>(tagged_region + round_up(m * 16, (int64_t)256));
  const size_t tagged_bytes = (size_t)round_up(m * 16, (int64_t)256) + (size_t)2 * kTicketSteps * 4;
  float* z32 = reinterpret_cast<float*>(w + ly.z32);
  double* r = reinterpret_cast<double*>(w + ly.r);
  double* rowmax = reinterpret_cast<double*>(w + ly.rowmax);
  double* xmax = reinterpret_cast<double*>(w + ly.xmax);
  double* rmax = reinterpret_cast<double*>(w + ly.rmax);
  double* bmax = reinterpret_cast<double*>(w + ly.bmax);
  double* norms = reinterpret_cast<double*>(w + ly.norms);
  const unsigned vb = (unsigned)ly.nvec_blocks, rb = (unsigned)ly.nrow_blocks;
  const bool vec = (ldh % 2) == 0 && (reinterpret_cast<uintptr_t>(H) & 15) == 0 &&
                   (reinterpret_cast<uintptr_t>(x) & 15) == 0;
  RefineState* state = reinterpret_cast<RefineState*>(w + ly.state);
  const int* stop = &state->stop;
  WaitCtx wc;
  SPSVM_TRY(wait_ctx(s, &wc));
  SPSVM_CUDA_TRY(cudaMemsetAsync(x, 0, (size_t)m * 8, s));
  SPSVM_CUDA_TRY(cudaMemsetAsync(tagged_region, 0, tagged_bytes, s));
  SPSVM_CUDA_TRY(cudaMemsetAsync(state, 0, sizeof(RefineState), s));
  // block maxima of |b| (||b||_inf) and the first right-hand side z = (float) b
  absmax_blocks<<<vb, MX_T, 0, s>>>(b, m, bmax, z32);
  SPSVM_LAUNCH_CHECK();
  // One refinement step: z = (L L^T)^{-1} r in FP32, x += z (with the
  // backward solve), r = b - (H + shift I) x in FP64 and the next z =
  // (float) r, then the norms and the stop word.  Every kernel of a step
  // returns at once once the stop word is set.
  auto step = [&](int it) -> int {
    // tags 1, 2, ... (the tagged words start zeroed); tickets per step
    const unsigned tag = (unsigned)(it + 1);
    if (it > 0 && it % kTicketSteps == 0)
      SPSVM_CUDA_TRY(cudaMemsetAsync(tickets, 0, (size_t)2 * kTicketSteps * 4, s));
    unsigned* tk = tickets + 2 * (it % kTicketSteps);
    trsv32_fwd<<<(unsigned)ly.B, SV_THREADS, 0, s>>>(L, ly.ldl, m, z32, zt, zw, tk, tag, wc, stop);
    SPSVM_LAUNCH_CHECK();
    if (lr) {   // z <- (I - V C^{-1} V^T) z
      lr_dots<<<dim3((unsigned)lr->G, (unsigned)lr->slices), 256, 0, s>>>(lr->V, lr->ldv, m, zw,
                                                                          lr->ldv, lr->s, stop);
      SPSVM_LAUNCH_CHECK();
      lr_update<<<(unsigned)min64(ceil_div(m, (int64_t)16), 2 * (int64_t)sm_count()), 256, 0, s>>>(
          lr->V, lr->ldv, m, lr->Ci, lr->ldv, lr->s, lr->slices, lr->ldv, lr->k, zw, stop);
      SPSVM_LAUNCH_CHECK();
    }
    trsv32_bwd<<<(unsigned)ly.B, SV_THREADS, 0, s>>>(L, ly.ldl, m, zw, xt, x, xmax, tk + 1, tag, wc,
                                                     stop);
    SPSVM_LAUNCH_CHECK();
    if (vec)
      residual_f64<true><<<rb, MX_T, 0, s>>>(H, ldh, m, shift, b, x, r, z32, rmax, stop);
    else
      residual_f64<false><<<rb, MX_T, 0, s>>>(H, ldh, m, shift, b, x, r, z32, rmax, stop);
    SPSVM_LAUNCH_CHECK();
    refine_decide<<<1, MX_T, 0, s>>>(xmax, ly.B, rmax, ly.nrow_blocks, rowmax, m, bmax,
                                     ly.nvec_blocks, norms, it <= 1 ? factor_info : nullptr, it, tol,
                                     state);
    SPSVM_LAUNCH_CHECK();
    return SPSVM_OK;
  };
  // an FP32 factor reaches FP64 backward error in about three steps: they
  // are queued before the first host check, later ones one at a time
  int it = 0;
  for (; it < max_iter && it < kRefineAhead; ++it) SPSVM_TRY(step(it));
  for (;;) {
    RefineState h{};
    const ReadChunk c{&h, state, sizeof(h)};
    SPSVM_TRY(read_back(s, &c, 1));
    if (iters) *iters = h.iters;
    if (backward_error) *backward_error = h.be;
    switch (h.stop) {
      case 1:
        return SPSVM_OK;
      case 2:
        return set_error(SPSVM_ERR_NO_CONVERGE, "solve_mixed: refinement stagnates (backward error %.3g)",
                         h.be);
      case 3:
        return set_error(SPSVM_ERR_NO_CONVERGE, "solve_mixed: not finite");
      case 4: {
        int32_t fi = 0;
        const ReadChunk cf{&fi, factor_info, sizeof(fi)};
        SPSVM_TRY(read_back(s, &cf, 1));
        return set_error(SPSVM_ERR_NOT_PD, "solve_mixed: the FP32 factorisation broke down at pivot %d",
                         fi - 1);
      }
      default:
        break;
    }
    if (it >= max_iter)
      return set_error(SPSVM_ERR_NO_CONVERGE, "solve_mixed: %d iterations not enough", max_iter);
    SPSVM_TRY(step(it));
    ++it;
  }
}

extern "C" int spsvm_solve_mixed(const double* H, int64_t m, int64_t ldh, double shift,
                                 const double* b, double* x, int32_t max_iter, double tol,
                                 int32_t* iters, double* backward_error, void* work,
                                 size_t work_bytes, void* stream) {
  return solve_mixed_impl(H, m, ldh, shift, b, x, max_iter, tol, iters, backward_error, work,
                          work_bytes, nullptr, nullptr, stream);
}

// spsvm_solve_mixed right after spsvm_cholesky_mixed, without a host read of
// the factorisation's info in between: the first refinement check reads it
// and returns SPSVM_ERR_NOT_PD when the FP32 factorisation broke down (the
// refinement's results are then discarded).
int spsvm::solve_mixed_after_factor(const double* H, int64_t m, int64_t ldh, double shift,
                                    const double* b, double* x, int32_t max_iter, double tol,
                                    void* work, size_t work_bytes, const int32_t* factor_info,
                                    void* stream) {
  return solve_mixed_impl(H, m, ldh, shift, b, x, max_iter, tol, nullptr, nullptr, work,
                          work_bytes, nullptr, factor_info, stream);
}

extern "C" size_t spsvm_lowrank_work_bytes(int64_t m, int32_t kmax) {
  if (m < 1 || kmax < 1 || kmax > SPSVM_LOWRANK_KMAX) return 0;
  return lowrank_layout(m, kmax).total;
}

extern "C" int spsvm_lowrank_factor(void* mixed_work, size_t mixed_bytes, int64_t m, const float* Wt,
                                    int64_t ldw, const float* sign, int32_t k, void* lr_work,
                                    size_t lr_bytes, int32_t* info, void* stream) {
  if (!mixed_work || !Wt || !sign || !lr_work || !info || m < 1 || k < 1 ||
      k > SPSVM_LOWRANK_KMAX || ldw < k)
    return set_error(SPSVM_ERR_ARG, "lowrank_factor: bad arguments (m=%lld k=%d)", (long long)m, k);
  const MixedLayout ml = mixed_layout(m);
  const LowRankLayout ly = lowrank_layout(m, k);
  if (mixed_bytes < ml.total || lr_bytes < ly.total || (reinterpret_cast<uintptr_t>(lr_work) & 255) != 0)
    return set_error(SPSVM_ERR_OOM, "lowrank_factor: work too small or misaligned");
  cudaStream_t s = as_stream(stream);
  ProfScope prof(PROF_LOWRANK, s, (double)m * m * k + 2.0 * (double)m * k * k + (double)k * k * k);
  char* w = static_cast<char*>(lr_work);
  const float* L = reinterpret_cast<const float*>(static_cast<char*>(mixed_work) + ml.L);
  float* V = reinterpret_cast<float*>(w + ly.V);
  float* Ci = reinterpret_cast<float*>(w + ly.Ci);
  unsigned* flags = reinterpret_cast<unsigned*>(w + ly.flags);
  const int64_t B = ceil_div(m, (int64_t)NB);
  SPSVM_CUDA_TRY(cudaMemsetAsync(info, 0, sizeof(int32_t), s));
  SPSVM_CUDA_TRY(cudaMemsetAsync(flags, 0, (size_t)(B * ly.G + 1) * 4, s));
  WaitCtx wc;
  SPSVM_TRY(wait_ctx(s, &wc));
  lr_trsm_fwd<<<(unsigned)(B * ly.G), LR_T, 0, s>>>(L, ml.ldl, m, Wt, ldw, k, V, ly.ldv, (int32_t)ly.G,
                                                    flags, flags + B * ly.G, wc);
  SPSVM_LAUNCH_CHECK();
  double* cpart = reinterpret_cast<double*>(w + ly.cpart);
  lr_capacitance<<<dim3((unsigned)ly.G, (unsigned)ly.G, (unsigned)ly.slices), 256, 0, s>>>(
      V, ly.ldv, m, ly.ldv, cpart);
  SPSVM_LAUNCH_CHECK();
  lr_capacitance_sum<<<(unsigned)ceil_div((int64_t)k * k, (int64_t)256), 256, 0, s>>>(
      cpart, ly.slices, ly.ldv, sign, k, Ci, ly.ldv);
  SPSVM_LAUNCH_CHECK();
  const size_t smem = (size_t)k * (k + 1) * 4 + (size_t)k * 4;
  SPSVM_CUDA_TRY(cudaFuncSetAttribute(lr_invert, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  lr_invert<<<1, LR_INV_T, smem, s>>>(Ci, ly.ldv, k, info);
  SPSVM_LAUNCH_CHECK();
  return SPSVM_OK;
}

extern "C" int spsvm_solve_lowrank(const double* H, int64_t m, int64_t ldh, const double* b, double* x,
                                   int32_t max_iter, double tol, int32_t* iters,
                                   double* backward_error, void* mixed_work, size_t mixed_bytes,
                                   void* lr_work, size_t lr_bytes, int32_t k, void* stream) {
  if (!lr_work || k < 1 || k > SPSVM_LOWRANK_KMAX || m < 1)
    return set_error(SPSVM_ERR_ARG, "solve_lowrank: bad arguments");
  const LowRankLayout ly = lowrank_layout(m, k);
  if (lr_bytes < ly.total) return set_error(SPSVM_ERR_OOM, "solve_lowrank: work too small");
  char* w = static_cast<char*>(lr_work);
  LowRankView v{reinterpret_cast<const float*>(w + ly.V), reinterpret_cast<const float*>(w + ly.Ci),
                reinterpret_cast<float*>(w + ly.s), ly.ldv, ly.slices, k, (int32_t)ly.G};
  return solve_mixed_impl(H, m, ldh, 0.0, b, x, max_iter, tol, iters, backward_error, mixed_work,
                          mixed_bytes, &v, nullptr, stream);
}

extern "C" void spsvm_set_factor_ctas(uint32_t ctas) {
  spsvm::g_factor_ctas.store(ctas, std::memory_order_relaxed);
}
