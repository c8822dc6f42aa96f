// Exact one-dimensional variant of the basis-selection score (Section 4's
// selection estimates the loss reduction of each sampled point): f
// restricted to a new coefficient beta_c is convex and piecewise quadratic,
//   phi_c'(t) = a0 + a1 t - sum_i v_i max(0, m_i - t v_i),
//   a0 = s lambda o_c, a1 = lambda K_cc, m_i = 1 - y_i o_i, v_i = s y_i K_ic,
// along the direction s = -sign(phi_c'(0)).  Each candidate's root is found
// exactly as in the line search (33-point grid passes counting the
// breakpoints in each cell, until the root's cell holds none), all
// candidates in lockstep inside one cooperative launch; a last pass sums
// the change of the loss terms at the root, and
//   delta_c = -(a0 t + a1 t^2 / 2 + 1/2 sum_i [max(0, m_i - t v_i)^2 - max(0, m_i)^2]).
#include <cmath>
#include <mutex>

#include "internal.h"

namespace spsvm {
namespace {

constexpr int XP = 33;          // grid points per pass
constexpr int XC = XP - 1;      // cells
constexpr int XT = 256;
constexpr int kMaxPasses = 48;  // sign pass + 24 growth + 9 refinement, with room

struct ExPart {
  double F[XP];
  int32_t cnt[XC];
  double q;
};

struct ExState {
  double lo, hi, t, a0, sgn;
  int32_t phase, grow, depth, done;
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Barrier of all CTAs of the cooperative launch (bounded; true on timeout).
__device__ bool xgrid_barrier(unsigned* bar, unsigned nblocks) {
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

// CTA (candidate k = blockIdx.x / cpc, part = blockIdx.x % cpc): points
// [part n / cpc, (part + 1) n / cpc) of candidate row k of Kc.
__global__ void __launch_bounds__(XT) exact_score_kernel(
    KView Kc, int64_t n, const float* __restrict__ y, const float* __restrict__ o,
    const int64_t* __restrict__ idx, int32_t kappa, int32_t cpc, double lambda,
    const double* __restrict__ bias, ExPart* __restrict__ part, ExState* __restrict__ st,
    unsigned* __restrict__ ctl, double* __restrict__ delta, double* __restrict__ t_out) {
  __shared__ double red[XT / 32][XP];
  __shared__ int32_t cnt[XC];
  __shared__ double qred[XT / 32];
  __shared__ double lo_s, hi_s, sgn_s, t_s;
  __shared__ int done_s, all_s;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int32_t k = (int32_t)(blockIdx.x / cpc), pidx = (int32_t)(blockIdx.x % cpc);
  const int64_t i0 = n * pidx / cpc, i1 = n * (pidx + 1) / cpc;
  unsigned* bar = ctl;
  unsigned* ndone = ctl + 2;
  const unsigned nb = gridDim.x;
  const double a1 = lambda;   // lambda K_cc, K_cc = 1 for the RBF kernel
  ExState* S = st + k;
  if (pidx == 0 && t == 0) {
    S->lo = 0.0;
    S->hi = 2.0;
    S->t = 0.0;
    S->a0 = lambda * ((double)o[idx[k]] - (bias ? *bias : 0.0));   // lambda k_cJ beta
    S->sgn = 1.0;
    S->phase = 0;
    S->grow = 0;
    S->depth = 0;
    S->done = 0;
  }
  if (xgrid_barrier(bar, nb)) {
    if (t == 0) atomicExch(ctl + 3, 1u);
    return;
  }
  for (int pass = 0; pass < kMaxPasses; ++pass) {
    if (t == 0) {
      lo_s = __ldcg(&S->lo);
      hi_s = __ldcg(&S->hi);
      sgn_s = __ldcg(&S->sgn);
      done_s = __ldcg(&S->done);
    }
    if (t < XC) cnt[t] = 0;
    __syncthreads();
    const double lo = lo_s, hi = hi_s;
    const float sg = (float)sgn_s;
    if (!done_s) {
      const double h = (hi - lo) / (double)XC;
      const float flo = (float)(lo - 1e-4 * fabs(lo)) - 1e-30f;
      const float fhi = (float)(hi + 1e-4 * fabs(hi)) + 1e-30f;
      float tk[XP], F[XP];
#pragma unroll
      for (int q = 0; q < XP; ++q) {
        tk[q] = (float)(lo + h * (double)q);
        F[q] = 0.f;
      }
      for (int64_t i = i0 + t; i < i1; i += XT) {
        const float yi = y[i];
        const float m = 1.0f - yi * o[i];
        const float v = sg * yi * Kc.at(k, i);
        if (v == 0.0f) continue;
#pragma unroll
        for (int q = 0; q < XP; ++q) F[q] = fmaf(v, fmaxf(0.0f, fmaf(-tk[q], v, m)), F[q]);
        const float bf = __fdividef(m, v);
        if (!(bf > flo && bf < fhi)) continue;
        const double b = (double)m / (double)v;
        if (b > lo && b < hi) {
          int c = (int)((b - lo) / h);
          c = c < 0 ? 0 : (c >= XC ? XC - 1 : c);
          const double left = lo + h * (double)c, right = lo + h * (double)(c + 1);
          if (b > left && b < right) atomicAdd(&cnt[c], 1);
        }
      }
#pragma unroll
      for (int q = 0; q < XP; ++q) {
        const double sv = warp_sum((double)F[q]);
        if (lane == 0) red[w][q] = sv;
      }
      __syncthreads();
      if (t < XP) {
        double sv = 0.0;
        for (int ww = 0; ww < XT / 32; ++ww) sv += red[ww][t];
        part[blockIdx.x].F[t] = sv;
      }
      if (t < XC) part[blockIdx.x].cnt[t] = cnt[t];
    }
    if (xgrid_barrier(bar, nb)) {
      if (t == 0) atomicExch(ctl + 3, 1u);
      return;
    }
    if (pidx == 0 && t == 0 && !done_s) {
      double Fs[XP];
      int32_t Cs[XC];
      for (int q = 0; q < XP; ++q) {
        double sv = 0.0;
        for (int p2 = 0; p2 < cpc; ++p2) sv += __ldcg(&part[blockIdx.x + p2].F[q]);
        Fs[q] = sv;
      }
      for (int q = 0; q < XC; ++q) {
        int32_t sv = 0;
        for (int p2 = 0; p2 < cpc; ++p2) sv += __ldcg(&part[blockIdx.x + p2].cnt[q]);
        Cs[q] = sv;
      }
      const double a0 = S->sgn * S->a0;
      auto dphi = [&](int q) { return a0 + a1 * (lo + (hi - lo) / (double)XC * (double)q) - Fs[q]; };
      int phase = S->phase, done = 0;
      double tt = 0.0, nlo = lo, nhi = hi;
      bool next = false;
      if (phase == 0) {   // phi'(0) in the + direction fixes the sign
        const double g0 = dphi(0);
        if (g0 == 0.0) {
          done = 1;
        } else if (g0 > 0.0) {
          S->sgn = -1.0;   // descend along -e_c: one more pass on [0, 2]
          phase = 1;
          next = true;
        } else {
          phase = 1;
        }
      }
      if (!done && !next && phase == 1) {
        if (dphi(XC) < 0.0 && S->grow < 24) {
          nlo = hi;
          nhi = hi * 8.0;
          ++S->grow;
          next = true;
        } else if (dphi(XC) < 0.0) {
          tt = hi;
          done = 1;
        } else {
          phase = 2;
        }
      }
      if (!done && !next) {
        int q = 0;
        while (q < XC && dphi(q + 1) < 0.0) ++q;
        if (q >= XC) q = XC - 1;
        const double hstep = (hi - lo) / (double)XC;
        const double tl = lo + hstep * q, tr = lo + hstep * (q + 1);
        const double fl = dphi(q), fr = dphi(q + 1);
        if (Cs[q] == 0 || S->depth >= 8 || !(fr > fl)) {
          tt = (fr > fl) ? tl - fl * (tr - tl) / (fr - fl) : tl;
          if (tt < tl) tt = tl;
          if (tt > tr) tt = tr;
          done = 1;
        } else {
          nlo = tl;
          nhi = tr;
          ++S->depth;
        }
      }
      if (pass == kMaxPasses - 2 && !done) {
        tt = lo;
        done = 1;
      }
      S->phase = phase;
      S->lo = nlo;
      S->hi = nhi;
      S->t = tt;
      if (done) {
        S->done = 1;
        atomicAdd(ndone, 1u);
      }
    }
    if (xgrid_barrier(bar, nb)) {
      if (t == 0) atomicExch(ctl + 3, 1u);
      return;
    }
    if (t == 0) all_s = (int)(ld_acquire_u32(ndone) >= (unsigned)kappa);
    __syncthreads();
    if (all_s) break;
  }
  // change of the loss terms at the root: 1/2 sum [max(0, m - t v)^2 - max(0, m)^2]
  if (t == 0) {
    t_s = __ldcg(&S->t);
    sgn_s = __ldcg(&S->sgn);
  }
  __syncthreads();
  const float tf = (float)t_s, sg = (float)sgn_s;
  double q = 0.0;
  float qf = 0.0f;
  int cntq = 0;
  for (int64_t i = i0 + t; i < i1; i += XT) {
    const float yi = y[i];
    const float m = 1.0f - yi * o[i];
    const float v = sg * yi * Kc.at(k, i);
    const float ma = m - tf * v;
    float d = 0.0f;
    if (m > 0.0f && ma > 0.0f) d = -tf * v * (2.0f * m - tf * v);
    else if (m > 0.0f) d = -m * m;
    else if (ma > 0.0f) d = ma * ma;
    qf += d;
    if (++cntq == 32) {
      q += (double)qf;
      qf = 0.0f;
      cntq = 0;
    }
  }
  q += (double)qf;
  q = warp_sum(q);
  if (lane == 0) qred[w] = q;
  __syncthreads();
  if (t == 0) {
    double sv = 0.0;
    for (int ww = 0; ww < XT / 32; ++ww) sv += qred[ww];
    part[blockIdx.x].q = sv;
  }
  if (xgrid_barrier(bar, nb)) {
    if (t == 0) atomicExch(ctl + 3, 1u);
    return;
  }
  if (pidx == 0 && t == 0) {
    double qs = 0.0;
    for (int p2 = 0; p2 < cpc; ++p2) qs += __ldcg(&part[blockIdx.x + p2].q);
    const double tt = S->t, a0 = S->sgn * S->a0;
    delta[k] = -(a0 * tt + 0.5 * a1 * tt * tt + 0.5 * qs);
    if (t_out) t_out[k] = S->sgn * tt;
  }
}

int max_coresident() {
  static std::mutex mu;
  static int per_sm[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return -1;
  std::lock_guard<std::mutex> g(mu);
  if (per_sm[dev] == 0) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, exact_score_kernel, XT, 0) != cudaSuccess ||
        b < 1)
      return -1;
    per_sm[dev] = b < 4 ? b : 4;
  }
  return per_sm[dev] * sm_count();
}

struct ExLayout {
  size_t state, ctl, part, kb, kc, total;
  int64_t ld;
};

ExLayout ex_layout(int64_t n, int64_t d, int32_t kappa, int32_t precision) {
  auto al = [](size_t b) { return (size_t)round_up((int64_t)b, (int64_t)256); };
  ExLayout L{};
  L.ld = round_up(n > 0 ? n : 1, 128);
  size_t off = 0;
  L.state = off;  off += al((size_t)kappa * sizeof(ExState));
  L.ctl = off;    off += al(16);
  L.part = off;   off += al((size_t)4 * 2048 * sizeof(ExPart));   // up to 4 CTAs per SM x 512 SMs
  L.kb = off;     off += al(spsvm_kernel_block_scratch_bytes(kappa, d, precision));
  L.kc = off;     off += al((size_t)kappa * L.ld * 4);               // FP32
  L.total = off;
  return L;
}

}  // namespace
}  // namespace spsvm

using namespace spsvm;

extern "C" size_t spsvm_score_exact_scratch_bytes(int64_t n, int64_t d, int32_t kappa,
                                                  int32_t precision) {
  if (n < 0 || d < 0 || kappa < 0) return 0;
  return ex_layout(n, d, kappa, precision).total;
}

extern "C" int spsvm_score_candidates_exact(const spsvm_points* p, const float* y, const float* o,
                                            const int64_t* idx, int32_t kappa, float gamma,
                                            double lambda, int32_t precision, const double* bias,
                                            double* delta, double* t, void* scratch,
                                            size_t scratch_bytes, void* stream) {
  if (!p || !y || !o || !idx || !delta || kappa < 0 || !(gamma > 0.0f) || !(lambda > 0.0))
    return set_error(SPSVM_ERR_ARG, "score_exact: bad arguments");
  if (kappa == 0 || p->n == 0) return SPSVM_OK;
  const ExLayout ly = ex_layout(p->n, p->d, kappa, precision);
  if (!scratch || scratch_bytes < ly.total || (reinterpret_cast<uintptr_t>(scratch) & 255) != 0)
    return set_error(SPSVM_ERR_OOM, "score_exact: scratch too small or misaligned");
  cudaStream_t s = as_stream(stream);
  char* w = static_cast<char*>(scratch);
  // the candidates' kernel rows, computed once in the given precision and
  // stored in FP32
  spsvm_kmat kc{};
  kc.data = w + ly.kc;
  kc.format = SPSVM_FP32;
  kc.n = p->n;
  kc.rows = kappa;
  kc.ld = ly.ld;
  kc.plane = 0;
  SPSVM_TRY(spsvm_kernel_block(p, idx, kappa, gamma, precision, &kc, 0, w + ly.kb,
                               spsvm_kernel_block_scratch_bytes(kappa, p->d, precision), stream));
  const int slots = max_coresident();
  if (slots < 1) return set_error(SPSVM_ERR_CUDA, "score_exact: occupancy query failed");
  // candidates in groups that fit one cooperative launch
  for (int32_t k0 = 0; k0 < kappa; k0 += slots) {
    const int32_t kk = (int32_t)min64(slots, kappa - k0);
    const int32_t cpc = (int32_t)min64(8, slots / kk);
    SPSVM_CUDA_TRY(cudaMemsetAsync(w + ly.ctl, 0, 16, s));
    KView kv = view(&kc);
    kv.data = static_cast<const char*>(kc.data) + (size_t)k0 * ly.ld * 4;
    const int64_t* ix = idx + k0;
    double* dl = delta + k0;
    double* tt = t ? t + k0 : nullptr;
    ExPart* part = reinterpret_cast<ExPart*>(w + ly.part);
    ExState* st = reinterpret_cast<ExState*>(w + ly.state);
    unsigned* ctl = reinterpret_cast<unsigned*>(w + ly.ctl);
    int64_t n = p->n;
    void* args[] = {(void*)&kv, (void*)&n, (void*)&y, (void*)&o, (void*)&ix, (void*)&kk,
                    (void*)&cpc, (void*)&lambda, (void*)&bias, (void*)&part, (void*)&st,
                    (void*)&ctl, (void*)&dl, (void*)&tt};
    SPSVM_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)exact_score_kernel, dim3((unsigned)(kk * cpc)),
                                               dim3(XT), args, 0, s));
    SPSVM_LAUNCH_CHECK();
    unsigned err = 0;
    SPSVM_CUDA_TRY(cudaMemcpyAsync(&err, ctl + 3, 4, cudaMemcpyDeviceToHost, s));
    SPSVM_CUDA_TRY(cudaStreamSynchronize(s));
    if (err) return set_error(SPSVM_ERR_TIMEOUT, "score_exact: grid barrier timed out");
  }
  return SPSVM_OK;
}
