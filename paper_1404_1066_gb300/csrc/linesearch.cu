// Exact line search along the Newton direction d (Section 4's Newton
// reoptimisation of Eq. 4; f is convex and piecewise quadratic along a
// line).  phi'(t) = a0 + a1 t - sum_i v_i max(0, m_i - t v_i) is piecewise
// linear and nondecreasing; each pass evaluates it on a 33-point grid over
// the current bracket and counts the breakpoints m_i / v_i inside each of
// the 32 cells, so that the root is solved exactly on a cell free of
// breakpoints.
#include <cmath>
#include <vector>

#include "internal.h"

namespace spsvm {

namespace {

constexpr int LP = 33;          // grid points per pass
constexpr int LC = LP - 1;      // cells
constexpr int LT = 256;

struct LsPart {
  double F[LP];
  int32_t cnt[LC];
};

__global__ void ls_coeffs(const float* __restrict__ o, const float* __restrict__ u,
                          const double* __restrict__ d, const int64_t* __restrict__ J, int32_t m,
                          double lambda, double* __restrict__ out) {
  __shared__ double sh[32];
  double s0 = 0.0, s1 = 0.0;
  for (int k = threadIdx.x; k < m; k += blockDim.x) {
    const int64_t j = J[k];
    s0 += d[k] * (double)o[j];
    s1 += d[k] * (double)u[j];
  }
  s0 = block_sum(s0, sh);
  __syncthreads();
  s1 = block_sum(s1, sh);
  if (threadIdx.x == 0) {
    out[0] = lambda * s0;
    out[1] = lambda * s1;
  }
}

__global__ void __launch_bounds__(LT) ls_pass(const float* __restrict__ o, const float* __restrict__ u,
                                              const float* __restrict__ y, int64_t n, double lo,
                                              double hi, LsPart* __restrict__ part) {
  __shared__ double red[LT / 32][LP];
  __shared__ int32_t cnt[LC];
  if (threadIdx.x < LC) cnt[threadIdx.x] = 0;
  __syncthreads();
  const double h = (hi - lo) / (double)LC;
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
#pragma unroll
  for (int k = 0; k < LP; ++k) {
    const double s = warp_sum((double)F[k]);
    if (lane == 0) red[w][k] = s;
  }
  __syncthreads();
  if (threadIdx.x < LP) {
    double s = 0.0;
    for (int q = 0; q < LT / 32; ++q) s += red[q][threadIdx.x];
    part[blockIdx.x].F[threadIdx.x] = s;
  }
  if (threadIdx.x < LC) part[blockIdx.x].cnt[threadIdx.x] = cnt[threadIdx.x];
}

__global__ void ls_reduce(const LsPart* __restrict__ part, int nblocks, LsPart* __restrict__ out) {
  const int k = threadIdx.x;
  if (k < LP) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += part[b].F[k];
    out->F[k] = s;
  }
  if (k < LC) {
    int32_t c = 0;
    for (int b = 0; b < nblocks; ++b) c += part[b].cnt[k];
    out->cnt[k] = c;
  }
}

int ls_blocks() { return 2 * sm_count(); }

}  // namespace
}  // namespace spsvm

using namespace spsvm;

extern "C" size_t spsvm_line_scratch_bytes(int64_t n) {
  (void)n;
  return (size_t)(ls_blocks() + 1) * sizeof(LsPart) + 256;
}

extern "C" int spsvm_line_search(const float* o, const float* u, const float* y, int64_t n,
                                 const double* d, const int64_t* J, int32_t m, double lambda,
                                 double* t_host, double* t_dev, void* scratch,
                                 size_t scratch_bytes, void* stream) {
  if (!o || !u || !y || !d || !J || !t_host || n < 0 || m < 0)
    return set_error(SPSVM_ERR_ARG, "line_search: bad arguments");
  if (!scratch || scratch_bytes < spsvm_line_scratch_bytes(n))
    return set_error(SPSVM_ERR_OOM, "line_search: scratch too small");
  cudaStream_t s = as_stream(stream);
  ProfScope prof(PROF_LINE, s, 12.0 * (double)n);
  const int nb = ls_blocks();
  double* coef = static_cast<double*>(scratch);
  LsPart* part = reinterpret_cast<LsPart*>(static_cast<char*>(scratch) + 256);
  LsPart* res = part + nb;
  ls_coeffs<<<1, 256, 0, s>>>(o, u, d, J, m, lambda, coef);
  SPSVM_LAUNCH_CHECK();
  double a[2];
  SPSVM_CUDA_TRY(cudaMemcpyAsync(a, coef, sizeof(a), cudaMemcpyDeviceToHost, s));
  LsPart h;
  auto run = [&](double lo, double hi) -> int {
    ls_pass<<<nb, LT, 0, s>>>(o, u, y, n, lo, hi, part);
    SPSVM_LAUNCH_CHECK();
    ls_reduce<<<1, 64, 0, s>>>(part, nb, res);
    SPSVM_LAUNCH_CHECK();
    SPSVM_CUDA_TRY(cudaMemcpyAsync(&h, res, sizeof(LsPart), cudaMemcpyDeviceToHost, s));
    SPSVM_CUDA_TRY(cudaStreamSynchronize(s));
    return SPSVM_OK;
  };
  double lo = 0.0, hi = 2.0;
  SPSVM_TRY(run(lo, hi));
  auto dphi = [&](int k, double l, double r) {
    const double tk = l + (r - l) / (double)LC * (double)k;
    return a[0] + a[1] * tk - h.F[k];
  };
  double t = 0.0;
  const double d0 = dphi(0, lo, hi);
  if (!(d0 < 0.0)) {
    t = 0.0;
  } else if (std::fabs(dphi(LC / 2, lo, hi)) <= 1e-6 * std::fabs(d0)) {
    t = 1.0;
  } else {
    // grow the bracket until phi' >= 0 at its right end
    int grow = 0;
    while (dphi(LC, lo, hi) < 0.0 && grow < 12) {
      lo = hi;
      hi = hi * 8.0;
      SPSVM_TRY(run(lo, hi));
      ++grow;
    }
    if (dphi(LC, lo, hi) < 0.0) {
      t = hi;   // phi still decreasing: take the far end (bounded)
    } else {
      for (int depth = 0;; ++depth) {
        int k = 0;
        while (k < LC && dphi(k + 1, lo, hi) < 0.0) ++k;
        if (k >= LC) k = LC - 1;
        const double hstep = (hi - lo) / (double)LC;
        const double tl = lo + hstep * k, tr = lo + hstep * (k + 1);
        const double fl = dphi(k, lo, hi), fr = dphi(k + 1, lo, hi);
        if (h.cnt[k] == 0 || depth >= 8 || !(fr > fl)) {
          t = (fr > fl) ? tl - fl * (tr - tl) / (fr - fl) : tl;
          if (t < tl) t = tl;
          if (t > tr) t = tr;
          break;
        }
        lo = tl;
        hi = tr;
        SPSVM_TRY(run(lo, hi));
      }
    }
  }
  *t_host = t;
  if (t_dev) SPSVM_CUDA_TRY(cudaMemcpyAsync(t_dev, t_host, sizeof(double), cudaMemcpyHostToDevice, s));
  return SPSVM_OK;
}
