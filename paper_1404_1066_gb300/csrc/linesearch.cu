// Exact line search along the Newton direction d (Section 4's Newton
// reoptimisation of Eq. 4; f is convex and piecewise quadratic along a
// line).  phi'(t) = a0 + a1 t - sum_i v_i max(0, m_i - t v_i) is piecewise
// linear and nondecreasing; each pass evaluates it on a 33-point grid over
// the current bracket and counts the breakpoints m_i / v_i inside each of
// the 32 cells, so that the root is solved exactly on a cell free of
// breakpoints.  The whole search is one cooperative launch: all CTAs make a
// pass and write their partial sums; after a grid barrier, 65 CTAs each
// reduce one of the pass's values over the CTAs (a fixed order); after a
// second barrier every CTA reads the 65 totals and takes the same decision
// on the next bracket -- no host round trip per pass.
#include <cmath>
#include <mutex>
#include <vector>

#include "internal.h"

namespace spsvm {

namespace {

constexpr int LP = 33;          // grid points per pass
constexpr int LC = LP - 1;      // cells
constexpr int LT = 256;
constexpr int kMaxPasses = 64;  // the search needs at most 1 + 12 + 9

// Result of the search (CTA 0 writes it) and the barrier's error word.
struct LsState {
  double lo, hi, t;
  int32_t done, err;
};

// Scratch after the state and the barrier words: the pass totals (phi' sums
// at the grid points, breakpoint counts per cell, and a0, a1), then the
// CTAs' partials transposed (value-major, so one CTA reads one value's
// partials contiguously).
struct LsTotals {
  double F[LP];
  double a[2];
  int32_t C[LC];
};
constexpr size_t kLsHead = 256;                       // state, barrier
constexpr size_t kLsTotals = 1024;                    // LsTotals, padded
constexpr size_t kLsPartOff = kLsHead + kLsTotals;
static_assert(sizeof(LsTotals) <= kLsTotals, "line search totals");

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Barrier of all CTAs of a cooperative launch (counter + generation; the
// last arrival resets the counter and advances the generation).  Gives up
// after about a second and returns true.
__device__ bool grid_barrier(unsigned* bar, unsigned nblocks) {
  __shared__ int to_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned* count = bar;
    unsigned* gen = bar + 1;
    const unsigned g = ld_acquire_u32(gen);
    __threadfence();
    int to = 0;
    if (atomicAdd(count, 1u) == nblocks - 1) {
      atomicExch(count, 0u);
      st_release_u32(gen, g + 1);
    } else {
      for (uint32_t it = 0; ld_acquire_u32(gen) == g; ++it) {
        if (it >= (1u << 22)) {
          to = 1;
          break;
        }
        if (it >= 32) __nanosleep(64);
      }
    }
    to_s = to;
  }
  __syncthreads();
  return to_s != 0;
}

// One pass of this CTA over its points for the bracket [lo, hi].
__device__ void ls_pass(const float* __restrict__ o, const float* __restrict__ u,
                        const float* __restrict__ y, int64_t n, double lo, double hi,
                        double* __restrict__ PF, int32_t* __restrict__ PC, double (*red)[LP],
                        int32_t* cnt) {
  if (threadIdx.x < LC) cnt[threadIdx.x] = 0;
  __syncthreads();
  const double h = (hi - lo) / (double)LC;
  const float flo = (float)(lo - 1e-4 * fabs(lo)) - 1e-30f;
  const float fhi = (float)(hi + 1e-4 * fabs(hi)) + 1e-30f;
  float tk[LP];
#pragma unroll
  for (int k = 0; k < LP; ++k) tk[k] = (float)(lo + h * (double)k);
  float F[LP];
#pragma unroll
  for (int k = 0; k < LP; ++k) F[k] = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * LT + threadIdx.x; i < n; i += (int64_t)gridDim.x * LT) {
    const float yi = y[i];
    const float m = 1.0f - yi * o[i];
    const float v = yi * u[i];
    if (v == 0.0f) continue;
#pragma unroll
    for (int k = 0; k < LP; ++k) F[k] = fmaf(v, fmaxf(0.0f, fmaf(-tk[k], v, m)), F[k]);
    // the exact breakpoint (FP64 division, slow on GB300) only where a
    // fast FP32 estimate (error a few ulp) puts it near the bracket
    const float bf = __fdividef(m, v);
    if (!(bf > flo && bf < fhi)) continue;
    const double b = (double)m / (double)v;
    if (b > lo && b < hi) {
      int c = (int)((b - lo) / h);
      c = c < 0 ? 0 : (c >= LC ? LC - 1 : c);
      // strictly inside the cell (a breakpoint on a grid point splits nothing)
      const double left = lo + h * (double)c, right = lo + h * (double)(c + 1);
      if (b > left && b < right) atomicAdd(&cnt[c], 1);
    }
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  // warp sums: grid points 0..31 by the column-sum exchange (lane k ends
  // with point k), point 32 by a plain reduction
  float v32[32];
#pragma unroll
  for (int k = 0; k < 32; ++k) v32[k] = F[k];
  const float fk = warp_column_sums(v32, lane);
  const float f32 = warp_sum(F[LP - 1]);
  red[w][lane] = (double)fk;
  if (lane == 0) red[w][LP - 1] = (double)f32;
  __syncthreads();
  const unsigned G = gridDim.x;
  if (threadIdx.x < LP) {
    double s = 0.0;
    for (int q = 0; q < LT / 32; ++q) s += red[q][threadIdx.x];
    PF[(size_t)threadIdx.x * G + blockIdx.x] = s;
  }
  if (threadIdx.x < LC) PC[(size_t)threadIdx.x * G + blockIdx.x] = cnt[threadIdx.x];
}

__global__ void __launch_bounds__(LT) ls_search(const float* __restrict__ o,
                                                const float* __restrict__ u,
                                                const float* __restrict__ y, int64_t n,
                                                const double* __restrict__ d,
                                                const int64_t* __restrict__ J, int32_t m,
                                                double lambda, char* __restrict__ work,
                                                LsState* __restrict__ st, unsigned* __restrict__ bar,
                                                const double* __restrict__ b0) {
  __shared__ double red[LT / 32][LP];
  __shared__ int32_t cnt[LC];
  __shared__ double Fs[LP], sh[32];
  __shared__ int32_t Cs[LC];
  __shared__ double a_s[2];
  __shared__ double lo_s, hi_s;
  __shared__ int done_s;
  const int t = threadIdx.x;
  const unsigned nb = gridDim.x;
  LsTotals* tot = reinterpret_cast<LsTotals*>(work + kLsHead);
  double* PF = reinterpret_cast<double*>(work + kLsPartOff);
  int32_t* PC = reinterpret_cast<int32_t*>(PF + (size_t)LP * nb);
  // thread 0 of every CTA carries the search state across passes (all CTAs
  // see the same totals and take the same decisions)
  double a0 = 0.0, a1 = 0.0, d0 = 0.0;
  int phase = 0, grow = 0, depth = 0;
  if (t == 0) {
    lo_s = 0.0;
    hi_s = 2.0;
    done_s = 0;
  }
  __syncthreads();
  for (int pass = 0; pass < kMaxPasses; ++pass) {
    const double lo = lo_s, hi = hi_s;
    ls_pass(o, u, y, n, lo, hi, PF, PC, red, cnt);
    if (pass == 0 && blockIdx.x == nb - 1) {
      // a0 = lambda d^T K_JJ beta, a1 = lambda d^T K_JJ d: (K_JJ beta)_k = o
      // at basis point k (minus the bias b0 = beta_0 when slot 0, point
      // index -1, holds it; that slot has no regulariser row)
      const double bb = b0 ? *b0 : 0.0, db = b0 ? d[0] : 0.0;
      double s0 = 0.0, s1 = 0.0;
      for (int k = t; k < m; k += LT) {
        const int64_t j = J[k];
        if (j < 0) continue;
        s0 += d[k] * ((double)o[j] - bb);
        s1 += d[k] * ((double)u[j] - db);
      }
      s0 = block_sum(s0, sh);
      __syncthreads();
      s1 = block_sum(s1, sh);
      if (t == 0) {
        tot->a[0] = lambda * s0;
        tot->a[1] = lambda * s1;
      }
    }
    if (grid_barrier(bar, nb)) {
      if (t == 0) atomicExch(&st->err, 1);
      return;
    }
    // CTA v < LP + LC: the total of value v over the CTAs, in a fixed order
    for (unsigned v = blockIdx.x; v < (unsigned)(LP + LC); v += nb) {
      if (v < (unsigned)LP) {
        double sv = 0.0;
        for (unsigned b = t; b < nb; b += LT) sv += __ldcg(&PF[(size_t)v * nb + b]);
        sv = block_sum(sv, sh);
        if (t == 0) tot->F[v] = sv;
      } else {
        int sv = 0;
        for (unsigned b = t; b < nb; b += LT) sv += __ldcg(&PC[(size_t)(v - LP) * nb + b]);
        sv = block_sum(sv, reinterpret_cast<int*>(sh));
        if (t == 0) tot->C[v - LP] = sv;
      }
      __syncthreads();
    }
    if (grid_barrier(bar, nb)) {
      if (t == 0) atomicExch(&st->err, 1);
      return;
    }
    if (t < LP) Fs[t] = __ldcg(&tot->F[t]);
    if (t < LC) Cs[t] = __ldcg(&tot->C[t]);
    if (pass == 0 && t < 2) a_s[t] = __ldcg(&tot->a[t]);
    __syncthreads();
    if (t == 0) {
      if (pass == 0) {
        a0 = a_s[0];
        a1 = a_s[1];
      }
      auto dphi = [&](int k) {
        const double tk = lo + (hi - lo) / (double)LC * (double)k;
        return a0 + a1 * tk - Fs[k];
      };
      double tt = 0.0, nlo = lo, nhi = hi;
      int done = 0;
      bool next = false;
      if (phase == 0) {
        d0 = dphi(0);
        if (!(d0 < 0.0)) {
          tt = 0.0;
          done = 1;
        } else if (fabs(dphi(LC / 2)) <= 1e-6 * fabs(d0)) {
          tt = 1.0;
          done = 1;
        } else {
          phase = 1;
        }
      }
      if (!done && phase == 1) {   // grow the bracket until phi' >= 0 at its right end
        if (dphi(LC) < 0.0 && grow < 12) {
          nlo = hi;
          nhi = hi * 8.0;
          ++grow;
          next = true;
        } else if (dphi(LC) < 0.0) {
          tt = hi;   // phi still decreasing: take the far end (bounded)
          done = 1;
        } else {
          phase = 2;
        }
      }
      if (!done && !next) {   // the cell holding the root
        int k = 0;
        while (k < LC && dphi(k + 1) < 0.0) ++k;
        if (k >= LC) k = LC - 1;
        const double hstep = (hi - lo) / (double)LC;
        const double tl = lo + hstep * k, tr = lo + hstep * (k + 1);
        const double fl = dphi(k), fr = dphi(k + 1);
        if (Cs[k] == 0 || depth >= 8 || !(fr > fl)) {
          tt = (fr > fl) ? tl - fl * (tr - tl) / (fr - fl) : tl;
          if (tt < tl) tt = tl;
          if (tt > tr) tt = tr;
          done = 1;
        } else {
          nlo = tl;
          nhi = tr;
          ++depth;
        }
      }
      if (pass == kMaxPasses - 1 && !done) {
        tt = lo;
        done = 1;
      }
      lo_s = nlo;
      hi_s = nhi;
      done_s = done;
      if (blockIdx.x == 0) {
        st->lo = nlo;
        st->hi = nhi;
        st->t = tt;
        st->done = done;
      }
    }
    __syncthreads();
    if (done_s) break;
  }
}

// The search's result for the caller's stream-ordered use: t and the
// grid-barrier error word.
__global__ void ls_export(const LsState* __restrict__ st, double* __restrict__ t_dev,
                          int32_t* __restrict__ err_dev) {
  *t_dev = st->err ? 0.0 : st->t;
  *err_dev = st->err;
}

int ls_grid() {
  static std::mutex mu;
  static int per_sm[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return -1;
  std::lock_guard<std::mutex> g(mu);
  if (per_sm[dev] == 0) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, ls_search, LT, 0) != cudaSuccess || b < 1)
      return -1;
    per_sm[dev] = b < 2 ? b : 2;
  }
  return per_sm[dev] * sm_count();
}

}  // namespace
}  // namespace spsvm

using namespace spsvm;

extern "C" size_t spsvm_line_scratch_bytes(int64_t n) {
  (void)n;
  return kLsPartOff + (size_t)(2 * sm_count()) * (LP * sizeof(double) + LC * sizeof(int32_t));
}

extern "C" int spsvm_line_search(const float* o, const float* u, const float* y, int64_t n,
                                 const double* d, const int64_t* J, int32_t m, double lambda,
                                 double* t_host, double* t_dev, void* scratch,
                                 size_t scratch_bytes, void* stream) {
  return spsvm::line_search_impl(o, u, y, n, d, J, m, lambda, t_host, t_dev, scratch, scratch_bytes,
                                 stream, nullptr);
}

int spsvm::line_search_impl(const float* o, const float* u, const float* y, int64_t n,
                            const double* d, const int64_t* J, int32_t m, double lambda,
                            double* t_host, double* t_dev, void* scratch, size_t scratch_bytes,
                            void* stream, const double* b0) {
  if (!o || !u || !y || !d || !J || !t_host || n < 0 || m < 0)
    return set_error(SPSVM_ERR_ARG, "line_search: bad arguments");
  if (!scratch || scratch_bytes < spsvm_line_scratch_bytes(n))
    return set_error(SPSVM_ERR_OOM, "line_search: scratch too small");
  cudaStream_t s = as_stream(stream);
  ProfScope prof(PROF_LINE, s, 12.0 * (double)n);
  const int grid = ls_grid();
  if (grid < 1) return set_error(SPSVM_ERR_CUDA, "line_search: occupancy query failed");
  LsState* st = static_cast<LsState*>(scratch);
  unsigned* bar = reinterpret_cast<unsigned*>(static_cast<char*>(scratch) + 128);
  char* work = static_cast<char*>(scratch);
  SPSVM_CUDA_TRY(cudaMemsetAsync(scratch, 0, kLsHead, s));
  void* args[] = {(void*)&o, (void*)&u, (void*)&y, (void*)&n, (void*)&d, (void*)&J,
                  (void*)&m, (void*)&lambda, (void*)&work, (void*)&st, (void*)&bar, (void*)&b0};
  SPSVM_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)ls_search, dim3(grid), dim3(LT), args, 0, s));
  SPSVM_LAUNCH_CHECK();
  LsState h{};
  SPSVM_CUDA_TRY(cudaMemcpyAsync(&h, st, sizeof(LsState), cudaMemcpyDeviceToHost, s));
  SPSVM_CUDA_TRY(cudaStreamSynchronize(s));
  if (h.err) return set_error(SPSVM_ERR_TIMEOUT, "line_search: grid barrier timed out");
  *t_host = h.t;
  if (t_dev) SPSVM_CUDA_TRY(cudaMemcpyAsync(t_dev, t_host, sizeof(double), cudaMemcpyHostToDevice, s));
  return SPSVM_OK;
}

int spsvm::line_search_async(const float* o, const float* u, const float* y, int64_t n,
                             const double* d, const int64_t* J, int32_t m, double lambda,
                             double* t_dev, int32_t* err_dev, void* scratch, size_t scratch_bytes,
                             void* stream, const double* b0) {
  if (!o || !u || !y || !d || !J || !t_dev || !err_dev || n < 0 || m < 0)
    return set_error(SPSVM_ERR_ARG, "line_search: bad arguments");
  if (!scratch || scratch_bytes < spsvm_line_scratch_bytes(n))
    return set_error(SPSVM_ERR_OOM, "line_search: scratch too small");
  cudaStream_t s = as_stream(stream);
  ProfScope prof(PROF_LINE, s, 12.0 * (double)n);
  const int grid = ls_grid();
  if (grid < 1) return set_error(SPSVM_ERR_CUDA, "line_search: occupancy query failed");
  LsState* st = static_cast<LsState*>(scratch);
  unsigned* bar = reinterpret_cast<unsigned*>(static_cast<char*>(scratch) + 128);
  char* work = static_cast<char*>(scratch);
  SPSVM_CUDA_TRY(cudaMemsetAsync(scratch, 0, kLsHead, s));
  void* args[] = {(void*)&o, (void*)&u, (void*)&y, (void*)&n, (void*)&d, (void*)&J,
                  (void*)&m, (void*)&lambda, (void*)&work, (void*)&st, (void*)&bar, (void*)&b0};
  SPSVM_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)ls_search, dim3(grid), dim3(LT), args, 0, s));
  SPSVM_LAUNCH_CHECK();
  ls_export<<<1, 1, 0, s>>>(st, t_dev, err_dev);
  SPSVM_LAUNCH_CHECK();
  return SPSVM_OK;
}
