// SP-SVM fit orchestration (Section 4, "Sparse primal optimization"): the
// cycle of basis-vector selection and reoptimisation of Eq. 4, built from
// the step-level entry points; the model object and prediction.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "internal.h"
#include "gram.h"

struct spsvm_model {
  int64_t n = 0, d = 0;
  float gamma = 0.f;
  double lambda = 0.0;
  int32_t precision = SPSVM_FP32;
  std::vector<int64_t> J;
  std::vector<double> beta;
  std::vector<spsvm_step> history;
  std::vector<std::vector<int64_t>> cand_rounds, chosen_rounds;
  std::vector<float> o;
  double objective = 0.0;
  int32_t status = SPSVM_OK;
  int32_t rounds = 0;
  int device = 0;
  double bias = 0.0;             // Eq. 4's b (0 unless fitted)
  float* basis_dev = nullptr;    // |J| x d, row-major
  double* beta_dev = nullptr;
  void* scratch_dev = nullptr;   // decision scratch
  size_t scratch_bytes = 0;
};

namespace spsvm {

namespace {

constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;

uint64_t splitmix_at(uint64_t seed, uint64_t counter) {
  uint64_t z = seed + (counter + 1) * kGolden;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// ---- small device kernels used by the orchestration ---------------------
__global__ void sub_kernel(const float* __restrict__ a, const float* __restrict__ b, int64_t n,
                           float* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = a[i] - b[i];
}

// (K_JJ w)_k from outputs v = K_nJ w read at the basis points: the bias slot
// (J_k < 0) has no regulariser row, and a bias w_0 (b0) carried by every
// output is taken off.
__device__ __forceinline__ double reg_at(const float* __restrict__ v, const int64_t* __restrict__ J,
                                         int k, const double* __restrict__ b0) {
  const int64_t j = J[k];
  if (j < 0) return 0.0;
  return (double)v[j] - (b0 ? *b0 : 0.0);
}

// g_k = lambda (K_JJ beta)_k + gs_k ; rhs_k = -g_k
__global__ void grad_finish(const float* __restrict__ o, const int64_t* __restrict__ J,
                            const double* __restrict__ gs, int32_t m, double lambda,
                            double* __restrict__ g, double* __restrict__ rhs,
                            const double* __restrict__ b0) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= m) return;
  const double v = lambda * reg_at(o, J, k, b0) + gs[k];
  g[k] = v;
  rhs[k] = -v;
}

// rho_k = -g_k - lambda u[J_k] - ws_k   (residual of H d = -g, H applied exactly)
__global__ void refine_resid(const double* __restrict__ g, const float* __restrict__ u,
                             const int64_t* __restrict__ J, const double* __restrict__ ws,
                             int32_t m, double lambda, double* __restrict__ rho) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= m) return;
  rho[k] = -g[k] - lambda * (double)u[J[k]] - ws[k];
}

__global__ void axpy_d(double* __restrict__ y, const double* __restrict__ x, double a, int32_t m) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < m) y[k] += a * x[k];
}

// beta += t d and o += t u with t read on the device (the line search's
// result, 0 when it found no descent)
__global__ void axpy_t(double* __restrict__ y, const double* __restrict__ x,
                       const double* __restrict__ t, int32_t m) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const double a = *t;
  if (k < m && a != 0.0) y[k] += a * x[k];
}

__global__ void update_o_t(float* __restrict__ o, const float* __restrict__ u,
                           const double* __restrict__ t, int64_t n) {
  const double a = *t;
  if (a == 0.0) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    o[i] = (float)((double)o[i] + a * (double)u[i]);
}

__global__ void count_diff(const uint8_t* __restrict__ a, const uint8_t* __restrict__ b, int64_t n,
                           unsigned long long* __restrict__ out) {
  __shared__ int sh[32];
  int c = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    c += (a[i] != b[i]);
  c = block_sum(c, sh);
  if (threadIdx.x == 0 && c) atomicAdd(out, (unsigned long long)c);
}

// out[0] = beta^T K_JJ beta ; out[1] = sum g_k^2 ; out[2] = sum r_k^2
__global__ void small_dots(const double* __restrict__ beta, const float* __restrict__ o,
                           const int64_t* __restrict__ J, const double* __restrict__ g,
                           const double* __restrict__ r, int32_t m, double* __restrict__ out,
                           const double* __restrict__ b0) {
  __shared__ double sh[32];
  double a = 0.0, b = 0.0, c = 0.0;
  for (int k = threadIdx.x; k < m; k += blockDim.x) {
    a += beta[k] * reg_at(o, J, k, b0);
    b += g[k] * g[k];
    c += r[k] * r[k];
  }
  a = block_sum(a, sh);
  __syncthreads();
  b = block_sum(b, sh);
  __syncthreads();
  c = block_sum(c, sh);
  if (threadIdx.x == 0) {
    out[0] = a;
    out[1] = b;
    out[2] = c;
  }
}

// out[0] = ||d||^2, out[1] = ||beta||^2
__global__ void step_norms(const double* __restrict__ d, const double* __restrict__ beta, int32_t m,
                           double* __restrict__ out) {
  __shared__ double sh[32];
  double a = 0.0, b = 0.0;
  for (int k = threadIdx.x; k < m; k += blockDim.x) {
    a += d[k] * d[k];
    b += beta[k] * beta[k];
  }
  a = block_sum(a, sh);
  __syncthreads();
  b = block_sum(b, sh);
  if (threadIdx.x == 0) {
    out[0] = a;
    out[1] = b;
  }
}

// With the bias the heuristic score's lambda o_c term carries b: take it off
// (h_c does not depend on it).
__global__ void score_bias_fix(double* __restrict__ g, const double* __restrict__ h,
                               double* __restrict__ delta, int32_t kappa, double lambda,
                               const double* __restrict__ b0) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= kappa) return;
  const double gg = g[k] - lambda * (*b0);
  g[k] = gg;
  delta[k] = gg * gg / (2.0 * h[k]);
}

// Row 0 of the kernel matrix as the bias's column of ones (zero past n).
__global__ void fill_bias_row(void* __restrict__ data, int32_t format, int64_t n, int64_t ld,
                              int64_t plane) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ld;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (format == SPSVM_FP32) {
      static_cast<float*>(data)[i] = i < n ? 1.0f : 0.0f;
    } else {
      __nv_bfloat16* h = static_cast<__nv_bfloat16*>(data);
      h[i] = __float2bfloat16_rn(i < n ? 1.0f : 0.0f);
      h[plane + i] = __float2bfloat16_rn(0.0f);
    }
  }
}

__global__ void add_const(float* __restrict__ v, int64_t n, float c) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    v[i] += c;
}

__global__ void add_diag(double* __restrict__ H, int64_t ldh, int32_t m, double shift) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < m) H[(int64_t)k * ldh + k] += shift;
}

__global__ void diag_sum(const double* __restrict__ H, int64_t ldh, int32_t m, double* out) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int k = threadIdx.x; k < m; k += blockDim.x) s += H[(int64_t)k * ldh + k];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) *out = s;
}

__global__ void gather_rows(const float* __restrict__ X, int64_t ldx, int64_t d,
                            const int64_t* __restrict__ J, int32_t m, float* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)m * d) return;
  const int64_t r = e / d, k = e % d;
  out[e] = X[J[r] * ldx + k];
}

int grid_for(int64_t n, int threads) {
  int64_t b = ceil_div(n, threads);
  const int64_t cap = 8 * (int64_t)sm_count();
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

// smallest |J| at which a changed active set corrects the factor in hand by
// a low-rank term instead of factoring afresh (below it the factorisation
// is as cheap as the correction)
constexpr int64_t kLowRankMinBasis = 512;
// largest rank of the correction the fit uses (the correction's cost grows
// with it, and past it a fresh factorisation costs about the same)
constexpr int64_t kLowRankMax = 64;

// ---- workspace layout ------------------------------------------------------
struct Layout {
  int64_t n, d, ldn, ldh, jcap, kappa, q;
  size_t off_norms, off_xhi, off_xmid, off_xlo, off_K, off_Kc, off_o, off_u, off_res, off_act0, off_act1,
      off_pos, off_H, off_beta, off_dir, off_g, off_r, off_rhs, off_tmp, off_tmp2, off_ws, off_sv, off_J,
      off_cand,
      off_cg, off_ch, off_cd, off_small, off_scratch, off_chw, off_mix, off_kjj, off_anchor, off_Wt,
      off_sign, off_lr, total;
  size_t scratch_bytes;
  size_t kbytes;
  size_t chw_bytes, sv_bytes, mix_bytes, lr_bytes;
};

size_t al(size_t x) { return (x + 255) & ~size_t(255); }

Layout make_layout(int64_t n, int64_t d, int32_t budget, int32_t precision, int32_t kappa,
                   int32_t q, int32_t solver, int32_t score, int32_t bias, int32_t lowrank) {
  Layout L{};
  L.n = n;
  L.d = d;
  L.ldn = round_up(n > 0 ? n : 1, 128);
  L.ldh = round_up(d, 64);
  L.jcap = round_up(budget + (bias ? 1 : 0), 64);   // slot 0 holds the bias
  L.kappa = kappa;
  L.q = q;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += al(bytes);
    return o;
  };
  L.off_norms = take(n * 4);
  const bool bf = precision == SPSVM_BF16SPLIT;
  L.off_xhi = take(bf ? (size_t)n * L.ldh * 2 : 0);
  L.off_xmid = take(bf ? (size_t)n * L.ldh * 2 : 0);
  L.off_xlo = take(bf ? (size_t)n * L.ldh * 2 : 0);
  L.kbytes = (size_t)L.jcap * L.ldn * 4;   // FP32, or two BF16 planes
  L.off_K = take(L.kbytes);
  L.off_Kc = take(L.kbytes);
  L.off_o = take(n * 4);
  L.off_u = take(n * 4);
  L.off_res = take(n * 4);
  L.off_act0 = take(n);
  L.off_act1 = take(n);
  L.off_pos = take(n * 4);
  L.off_H = take((size_t)L.jcap * L.jcap * 8);
  L.off_beta = take(L.jcap * 8);
  L.off_dir = take(L.jcap * 8);
  L.off_g = take(L.jcap * 8);
  L.off_r = take(L.jcap * 8);
  L.off_rhs = take(L.jcap * 8);
  L.off_tmp = take(L.jcap * 8);
  L.off_tmp2 = take(L.jcap * 8);
  L.off_ws = take(L.jcap * 8);
  L.sv_bytes = spsvm_cholesky_solve_work_bytes(L.jcap);
  L.off_sv = take(L.sv_bytes);
  L.off_J = take(L.jcap * 8);
  L.off_cand = take(kappa * 8);
  L.off_cg = take(kappa * 8);
  L.off_ch = take(kappa * 8);
  L.off_cd = take(kappa * 8);
  L.off_small = take(256);
  size_t sc = spsvm_score_scratch_bytes(n, d, kappa);
  sc = std::max(sc, spsvm_kernel_block_scratch_bytes(L.jcap, d, precision));
  sc = std::max(sc, spsvm_reduce_scratch_bytes(n));
  sc = std::max(sc, spsvm_compact_scratch_bytes(n, L.jcap));
  // the Gram split count depends on |J|: cover every size the fit can reach
  for (int64_t mm = 1; mm <= L.jcap; ++mm) sc = std::max(sc, gram_part_bytes(mm, n));
  sc = std::max(sc, spsvm_line_scratch_bytes(n));
  if (score == SPSVM_SCORE_EXACT) sc = std::max(sc, spsvm_score_exact_scratch_bytes(n, d, kappa, precision));
  L.scratch_bytes = al(sc);
  L.off_scratch = take(L.scratch_bytes);
  L.chw_bytes = spsvm_cholesky_work_bytes(L.jcap);
  L.off_chw = take(L.chw_bytes);
  // FP32 factor and refinement vectors of the mixed Newton solve
  L.mix_bytes = solver == SPSVM_SOLVE_MIXED ? spsvm_mixed_work_bytes(L.jcap) : 0;
  L.off_mix = take(L.mix_bytes);
  // symmetric K_JJ (FP64), extended as the basis grows; read by the Gram finish
  L.off_kjj = take((size_t)L.jcap * L.jcap * 8);
  // low-rank correction of the mixed solve: active flags of the factored
  // matrix, kernel rows and signs of the changed points, the correction
  const bool lr = lowrank && solver == SPSVM_SOLVE_MIXED && L.jcap >= kLowRankMinBasis;
  L.off_anchor = take(lr ? (size_t)n : 0);
  L.off_Wt = take(lr ? (size_t)L.jcap * SPSVM_LOWRANK_KMAX * 4 : 0);
  L.off_sign = take(lr ? (size_t)SPSVM_LOWRANK_KMAX * 4 : 0);
  L.lr_bytes = lr ? spsvm_lowrank_work_bytes(L.jcap, SPSVM_LOWRANK_KMAX) : 0;
  L.off_lr = take(L.lr_bytes);
  L.total = off;
  return L;
}

struct Opts {
  int32_t kappa, q, max_newton, precision, refine, record, solver, score, bias, lowrank;
  double growth_tol, rel_tol;
  uint64_t seed;
  bool fixed;
  cudaStream_t stream;
};

Opts resolve(const spsvm_options* o) {
  Opts r{};
  r.kappa = (o && o->candidates > 0) ? o->candidates : 256;
  r.q = (o && o->add_per_round > 0) ? o->add_per_round : 64;
  r.max_newton = (o && o->max_newton > 0) ? o->max_newton : 50;
  r.precision = o ? o->precision : SPSVM_FP32;
  r.refine = (o && o->refine > 0) ? o->refine : 0;
  r.record = o ? o->record : 0;
  r.growth_tol = o ? o->growth_tol : 0.0;
  r.rel_tol = (o && o->rel_tol > 0) ? o->rel_tol : 1e-6;
  r.seed = o ? o->seed : 0;
  r.fixed = o && o->fixed_basis;
  r.stream = o ? as_stream(o->stream) : nullptr;
  r.solver = (o && o->newton_solver == SPSVM_SOLVE_FP64) ? SPSVM_SOLVE_FP64 : SPSVM_SOLVE_MIXED;
  r.score = (o && o->score == SPSVM_SCORE_EXACT) ? SPSVM_SCORE_EXACT : SPSVM_SCORE_HEURISTIC;
  r.bias = (o && o->bias) ? 1 : 0;
  r.lowrank = (o && o->lowrank) ? 1 : 0;
  return r;
}

constexpr int32_t kJitterMaxLevel = 8;   // largest jitter 1e-2 tr(H)/|J|
// kinds of the Newton-system factor in hand
enum { FAC_MIXED = 0, FAC_LOWRANK = 1, FAC_FP64 = 2 };
// Newton stop once the gradient is small (||grad|| <= rel_tol ||r||): the
// next Newton step is below this fraction of ||beta|| (and is not taken)
constexpr double kStepTol = 1e-5;
// rounding-level stop only below this gradient level (relative to ||r||)
constexpr double kFloorGuard = 1e-3;
// gradient level (relative to ||r||) that ends the iteration of a fit that
// runs with a diagonal jitter
constexpr double kJitterRelTol = 5e-6;
// mixed Newton solve: refinement steps and the normwise backward error it
// must reach (else the FP64 factorisation is used).  1e-11 is about 1e5 units
// of FP64 rounding: the direction's relative error stays below cond(H) 1e-11,
// far under what the Newton stop (on the exact gradient) can see, and the
// fit's steps and minimiser are those of an FP64 solve.
constexpr int32_t kMixedIters = 30;
constexpr double kMixedTol = 1e-11;

struct Fit {
  const float* X;
  const float* y;
  int64_t n, d, ldx;
  float gamma;
  double lambda, tol;
  int32_t budget;
  Opts op;
  Layout L;
  char* ws;
  cudaStream_t s;
  spsvm_points pts;
  spsvm_model* model;
  std::vector<int64_t> J;     // host copy of the basis
  int32_t m = 0;              // current |J|
  int32_t act_cur = 0;        // which active buffer holds the current flags
  int32_t jitter = -1;        // jitter level that factorised the last Newton matrix
  int64_t anchor_m = -1;      // |J| of the unshifted FP32 factor in hand (its active set
                              // in the anchor flags), or -1
  int32_t lr_k = 0;           // rank of the low-rank correction in hand

  template <typename T>
  T* at(size_t off) { return reinterpret_cast<T*>(ws + off); }

  // K_nJ is stored in FP32 in both forms; the compact copy K_SJ, the Gram
  // matrix's operand, is FP32 for the FP32 form and the hi / lo BF16 planes
  // of the tensor-core Gram matrix for BF16SPLIT (same 4 bytes per element)
  spsvm_kmat kmat() {
    spsvm_kmat K{};
    K.data = ws + L.off_K;
    K.format = SPSVM_FP32;
    K.n = n;
    K.rows = m;
    K.ld = L.ldn;
    K.plane = 0;
    return K;
  }
  spsvm_kmat kcmat() {
    spsvm_kmat K = kmat();
    K.data = ws + L.off_Kc;
    K.n = L.ldn;
    K.format = op.precision == SPSVM_BF16SPLIT ? SPSVM_BF16SPLIT : SPSVM_FP32;
    K.plane = (int64_t)L.jcap * L.ldn;
    return K;
  }

  // Waits for the fit's stream and checks the bounded waits of the
  // tensor-core kernels (kernel block, Gram and the Cholesky update, which
  // runs in both precisions).
  int sync() {
    int32_t code = 0;
    return device_status_on(s, &code);
  }

  // bytes from device memory to the host after the work queued on the
  // stream, with the bounded-wait check, through one synchronisation
  int read(void* dst, const void* src, size_t bytes) {
    const ReadChunk c{dst, src, bytes};
    return read_back(s, &c, 1);
  }

  // Refresh active flags and stats from the current o into buffer `which`.
  int flags(int which, double stats_host[3]) {
    spsvm_kmat K = kmat();
    uint8_t* act = at<uint8_t>(which ? L.off_act1 : L.off_act0);
    double* st = at<double>(L.off_small);
    SPSVM_TRY(spsvm_outputs(&K, nullptr, y, at<float>(L.off_o), act, st, ws + L.off_scratch,
                            L.scratch_bytes, s));
    return read(stats_host, st, 3 * sizeof(double));
  }

  int newton() {
    spsvm_kmat K = kmat();
    spsvm_kmat Kc = kcmat();
    const int tpb = 256;
    const int mb = (int)ceil_div(m, tpb);
    double* beta = at<double>(L.off_beta);
    double* dir = at<double>(L.off_dir);
    double* g = at<double>(L.off_g);
    double* r = at<double>(L.off_r);
    double* rhs = at<double>(L.off_rhs);
    double* tmp = at<double>(L.off_tmp);
    double* wsum = at<double>(L.off_ws);
    double* H = at<double>(L.off_H);
    float* o = at<float>(L.off_o);
    float* u = at<float>(L.off_u);
    float* res = at<float>(L.off_res);
    int64_t* Jd = at<int64_t>(L.off_J);
    char* small = ws + L.off_small;
    int64_t* n_active = reinterpret_cast<int64_t*>(small + 64);
    int32_t* info = reinterpret_cast<int32_t*>(small + 80);
    unsigned long long* ndiff = reinterpret_cast<unsigned long long*>(small + 96);
    double* dots = reinterpret_cast<double*>(small + 128);
    void* scratch = ws + L.off_scratch;
    const size_t sb = L.scratch_bytes;
    const int64_t ldH = L.jcap;

    // exact outputs at the start of the reoptimisation
    double st[3];
    SPSVM_TRY(spsvm_outputs(&K, beta, y, o, at<uint8_t>(act_cur ? L.off_act1 : L.off_act0),
                            at<double>(L.off_small), scratch, sb, s));
    SPSVM_TRY(read(st, at<double>(L.off_small), sizeof(st)));
    int32_t status = SPSVM_ERR_NO_CONVERGE;
    double* tmp2 = at<double>(L.off_tmp2);
    void* mixw = ws + L.off_mix;
    void* lrw = ws + L.off_lr;
    float* Wt = at<float>(L.off_Wt);
    float* sgn = at<float>(L.off_sign);
    int32_t* kdev = reinterpret_cast<int32_t*>(small + 184);
    uint8_t* anchor = at<uint8_t>(L.off_anchor);
    // (H + shift I)^{-1} b with the factor in hand: the FP32 one with FP64
    // refinement (H kept), the same plus the low-rank correction for the
    // points that changed since it was formed, or the FP64 one in H
    auto solve_with = [&](int kind, double sh, const double* b, double* x, double btol) -> int {
      if (kind == FAC_MIXED)
        return spsvm_solve_mixed(H, m, ldH, sh, b, x, kMixedIters, btol, nullptr, nullptr, mixw,
                                 L.mix_bytes, s);
      if (kind == FAC_LOWRANK)
        return spsvm_solve_lowrank(H, m, ldH, b, x, kMixedIters, btol, nullptr, nullptr, mixw,
                                   L.mix_bytes, lrw, L.lr_bytes, lr_k, s);
      if (x != b) SPSVM_CUDA_TRY(cudaMemcpyAsync(x, b, m * sizeof(double), cudaMemcpyDeviceToDevice, s));
      return spsvm_cholesky_solve(H, m, ldH, x, ws + L.off_sv, L.sv_bytes, s);
    };
    // u = K_nJ d, then the optional refinement sweeps against the exactly
    // applied H (two more passes over K each)
    auto finish_direction = [&](const uint8_t* act, int kind, double sh) -> int {
      SPSVM_TRY(spsvm_gemv(&K, dir, u, 0, s));
      for (int k = 0; k < op.refine; ++k) {
        SPSVM_TRY(spsvm_compact_active(&K, act, u, nullptr, wsum, nullptr, nullptr, n_active,
                                       at<int32_t>(L.off_pos), scratch, sb, s));
        refine_resid<<<mb, tpb, 0, s>>>(g, u, Jd, wsum, m, lambda, tmp);
        SPSVM_LAUNCH_CHECK();
        // a correction of ~1e-5 relative size: 1e-6 backward error suffices
        const int rc = solve_with(kind, sh, tmp, tmp2, 1e-6);
        if (rc != SPSVM_OK && rc != SPSVM_ERR_NO_CONVERGE) return rc;
        axpy_d<<<mb, tpb, 0, s>>>(dir, tmp2, 1.0, m);
        SPSVM_LAUNCH_CHECK();
        SPSVM_TRY(spsvm_gemv(&K, tmp2, u, 1, s));
      }
      return SPSVM_OK;
    };
    // the factor in hand (valid while the active set does not change)
    bool reuse = false;
    int fac_kind = FAC_MIXED;
    double fac_shift = 0.0;
    // ||d|| <= kStepTol ||beta|| for the direction just solved
    auto step_small = [&](bool* small) -> int {
      step_norms<<<1, 256, 0, s>>>(dir, beta, m, dots + 4);
      SPSVM_LAUNCH_CHECK();
      double v[2];
      SPSVM_TRY(read(v, dots + 4, sizeof(v)));
      *small = std::sqrt(v[0]) <= kStepTol * std::sqrt(v[1]);
      return SPSVM_OK;
    };
    // gradient norm before the previous step, and whether that step kept the
    // active set
    double gprev = INFINITY;
    bool kept_prev = false;
    // Gradient pass on the flags `act`: residuals o - y, compaction with the
    // masked transposed products (w = K_SJ^T (o_S - y_S), r = K_SJ^T y_S;
    // the copy K_SJ is rewritten unless *kc_cond is zero, i.e. unless the
    // active set is unchanged), gradient and the dots of the stopping test.
    auto grad_pass = [&](uint8_t* act_f, const unsigned long long* kc_cond) -> int {
      sub_kernel<<<grid_for(n, tpb), tpb, 0, s>>>(o, y, n, res);
      SPSVM_LAUNCH_CHECK();
      SPSVM_TRY(compact_active_impl(&K, act_f, res, y, wsum, r, &Kc, kc_cond, n_active,
                                    at<int32_t>(L.off_pos), scratch, sb, s));
      grad_finish<<<mb, tpb, 0, s>>>(o, Jd, wsum, m, op_lambda(), g, rhs, b0());
      SPSVM_LAUNCH_CHECK();
      small_dots<<<1, 256, 0, s>>>(beta, o, Jd, g, r, m, dots, b0());
      SPSVM_LAUNCH_CHECK();
      return SPSVM_OK;
    };
    // the small area's layout, read back in one copy after each step:
    // [0, 24) loss / errors / |S|, [96, 104) changed flags, [128, 152) dots,
    // [200, 208) the line search's t, [208, 212) its error word
    constexpr size_t kSmallRead = 216;
    double* t_dev = reinterpret_cast<double*>(small + 200);
    int32_t* ls_err = reinterpret_cast<int32_t*>(small + 208);
    double dh[3] = {0.0, 0.0, 0.0};
    double st_next[3] = {0.0, 0.0, 0.0}, dh_next[3] = {0.0, 0.0, 0.0};
    unsigned long long nd_next = 0;
    // The line search along dir and, in the same stream order, the step it
    // gives with its consequences -- beta += t dir, o += t u, the new flags
    // and stats, the count of changed flags and the next gradient pass --
    // then one read of all their scalars.  With t = 0 (no descent) the step
    // leaves beta and o as they were and the rest recomputes the same values.
    auto search_and_step = [&](double* t_out) -> int {
      SPSVM_TRY(line_search_async(o, u, y, n, dir, Jd, m, lambda, t_dev, ls_err, scratch, sb, s, b0()));
      axpy_t<<<mb, tpb, 0, s>>>(beta, dir, t_dev, m);
      SPSVM_LAUNCH_CHECK();
      update_o_t<<<grid_for(n, tpb), tpb, 0, s>>>(o, u, t_dev, n);
      SPSVM_LAUNCH_CHECK();
      const int nxt = act_cur ^ 1;
      {
        spsvm_kmat Kf = kmat();
        SPSVM_TRY(spsvm_outputs(&Kf, nullptr, y, o, at<uint8_t>(nxt ? L.off_act1 : L.off_act0),
                                at<double>(L.off_small), scratch, sb, s));
      }
      SPSVM_CUDA_TRY(cudaMemsetAsync(ndiff, 0, sizeof(*ndiff), s));
      count_diff<<<grid_for(n, tpb), tpb, 0, s>>>(at<uint8_t>(L.off_act0), at<uint8_t>(L.off_act1),
                                                  n, ndiff);
      SPSVM_LAUNCH_CHECK();
      SPSVM_TRY(grad_pass(at<uint8_t>(nxt ? L.off_act1 : L.off_act0), ndiff));
      alignas(8) unsigned char sm_h[kSmallRead];
      SPSVM_TRY(read(sm_h, small, kSmallRead));
      int32_t err = 0;
      std::memcpy(&err, sm_h + 208, sizeof(err));
      if (err) return set_error(SPSVM_ERR_TIMEOUT, "line_search: grid barrier timed out");
      std::memcpy(st_next, sm_h, sizeof(st_next));
      std::memcpy(&nd_next, sm_h + 96, sizeof(nd_next));
      std::memcpy(dh_next, sm_h + 128, sizeof(dh_next));
      std::memcpy(t_out, sm_h + 200, sizeof(double));
      return SPSVM_OK;
    };
    SPSVM_TRY(grad_pass(at<uint8_t>(act_cur ? L.off_act1 : L.off_act0), nullptr));
    SPSVM_TRY(read(dh, dots, sizeof(dh)));
    for (int it = 0; it < op.max_newton; ++it) {
      uint8_t* act = at<uint8_t>(act_cur ? L.off_act1 : L.off_act0);
      const double gnorm = std::sqrt(dh[1]), rnorm = std::sqrt(dh[2]);
      model->objective = 0.5 * lambda * dh[0] + st[0];
      // Newton stop (the paper gives none):
      //  * ||grad|| <= tol;
      //  * rounding level: a near-full step that kept the active set did not
      //    halve ||grad|| (on a fixed active set the Newton step is exact up
      //    to the rounding of H), with ||grad|| <= kFloorGuard ||r||, where
      //    r = K_SJ^T y_S;
      //  * with a diagonal jitter in use, ||grad|| <= max(rel_tol,
      //    kJitterRelTol) ||r||: H is at rounding level in its smallest
      //    directions, where beta is not determined;
      //  * otherwise, once ||grad|| <= rel_tol ||r||: the next Newton step
      //    is below kStepTol ||beta|| (checked below, once the step is
      //    solved; it is then not taken), or a step finds no descent.
      const bool gsmall = gnorm <= op.rel_tol * rnorm;
      // with a jitter the damped steps converge slowly in the directions
      // where H is at rounding level, which the objective hardly sees
      const bool gsmall_jit = gnorm <= std::max(op.rel_tol, kJitterRelTol) * rnorm;
      auto converged = [&]() {
        spsvm_step rec{m, (int32_t)st[2], gnorm, 0.0, st[0], (int32_t)st[1], jitter, 0,
                       SPSVM_NEWTON_NONE};
        model->history.push_back(rec);
        status = SPSVM_OK;
      };
      if (gnorm <= tol || (gsmall_jit && jitter >= 0) || (gsmall && kept_prev && gnorm > 0.5 * gprev) ||
          (kept_prev && gnorm > 0.5 * gprev && gnorm <= kFloorGuard * rnorm)) {
        converged();
        break;
      }
      gprev = gnorm;
      bool done = false;
      // Newton system on the active set.  Factorise H + 10^(l-10) tr(H)/|J| I
      // for l = jitter, jitter + 1, ... (l = -1: H itself): a computed H of a
      // smooth kernel can be indefinite at rounding level.  The direction is
      // d = -(H + shift I)^{-1} grad f; when the line search finds no descent
      // along it (t = 0: the computed H is too far from the exact one in its
      // smallest directions) the level goes up and d is recomputed.  The
      // level never goes down within a fit.
      double t = 0.0;
      bool stepped = false;
      bool h_fresh = false;   // H holds the unfactorised, unshifted matrix
      int how = SPSVM_NEWTON_FACTOR;
      // A direction from the factor in hand (kind, shift), then u = K_nJ d
      // and the line search; false when the solve does not reach FP64
      // backward error or the line search finds no descent (the caller then
      // factors afresh).
      bool searched = false;   // try_direction ran the line search
      auto try_direction = [&](int kind, double sh, bool* ok) -> int {
        *ok = false;
        searched = false;
        const int rc = solve_with(kind, sh, rhs, dir, kMixedTol);
        if (rc == SPSVM_ERR_NO_CONVERGE) return SPSVM_OK;
        SPSVM_TRY(rc);
        if (gsmall) SPSVM_TRY(step_small(&done));
        if (done) return SPSVM_OK;
        SPSVM_TRY(finish_direction(act, kind, sh));
        SPSVM_TRY(search_and_step(&t));
        searched = true;
        *ok = t > 0.0;
        return SPSVM_OK;
      };
      if (reuse) {
        // the active set has not changed since the factor in hand (and its
        // low-rank correction) was formed, so H has not either: only the
        // right-hand side is new
        SPSVM_TRY(try_direction(fac_kind, fac_shift, &stepped));
        how = SPSVM_NEWTON_REUSE;
        if (!stepped && searched && gsmall && !done) {   // no descent at rounding level
          converged();
          break;
        }
      } else if (op.lowrank && anchor_m == m && jitter < 0 && m >= kLowRankMinBasis) {
        // the active set moved by k points since the unshifted FP32 factor in
        // hand was formed: correct that factor by the rank-k term instead of
        // factoring afresh (H itself is rebuilt for the refinement residuals)
        const int32_t kmax = (int32_t)std::min<int64_t>(kLowRankMax, m / 8);
        SPSVM_TRY(spsvm_active_diff(&K, act, anchor, kmax, Wt, SPSVM_LOWRANK_KMAX, sgn, kdev, scratch,
                                    sb, s));
        int32_t kk = 0;
        SPSVM_TRY(read(&kk, kdev, sizeof(kk)));
        if (kk >= 1 && kk <= kmax) {
          SPSVM_TRY(gram_impl(&Kc, n_active, n, &K, Jd, lambda, op.precision, H, ldH, scratch, sb, s,
                              st[2], at<double>(L.off_kjj), L.jcap));
          h_fresh = true;
          int32_t* lr_info = reinterpret_cast<int32_t*>(small + 188);
          SPSVM_TRY(spsvm_lowrank_factor(mixw, L.mix_bytes, m, Wt, SPSVM_LOWRANK_KMAX, sgn, kk, lrw,
                                         L.lr_bytes, lr_info, s));
          int32_t li = 1;
          SPSVM_TRY(read(&li, lr_info, sizeof(li)));
          if (li == 0) {
            lr_k = kk;
            SPSVM_TRY(try_direction(FAC_LOWRANK, 0.0, &stepped));
            if (stepped || done) {
              fac_kind = FAC_LOWRANK;
              fac_shift = 0.0;
              how = SPSVM_NEWTON_LOWRANK;
            }
          }
        }
      }
      if (done) {
        converged();
        break;
      }
      if (!stepped) how = SPSVM_NEWTON_FACTOR;
      bool mixed = false;     // the factor in use is the FP32 one (H kept intact)
      double tr = -1.0, shift = 0.0;
      for (; !stepped;) {
        for (int32_t lv = jitter;; ++lv) {
          if (lv > kJitterMaxLevel)
            return set_error(SPSVM_ERR_NOT_PD,
                             "Newton matrix not positive definite up to jitter 1e-2 tr(H)/|J| (|J|=%d)", m);
          if (!h_fresh) {
            SPSVM_TRY(gram_impl(&Kc, n_active, n, &K, Jd, lambda, op.precision, H, ldH, scratch, sb,
                                s, st[2], at<double>(L.off_kjj), L.jcap));
            h_fresh = true;
          }
          if (lv >= 0 && tr < 0.0) {
            diag_sum<<<1, 256, 0, s>>>(H, ldH, m, dots + 3);
            SPSVM_LAUNCH_CHECK();
            SPSVM_TRY(read(&tr, dots + 3, sizeof(tr)));
          }
          shift = lv >= 0 ? std::pow(10.0, lv - 10) * tr / m : 0.0;
          int32_t info_h = 0;
          // FP32 factor of H + shift I and FP64 refinement to FP64 backward
          // error; H is kept, so a failure costs no Gram rebuild
          mixed = false;
          if (op.solver == SPSVM_SOLVE_MIXED) {
            // the factorisation's info is read at the refinement's first check
            SPSVM_TRY(spsvm_cholesky_mixed(H, m, ldH, shift, info, mixw, L.mix_bytes, s));
            const int rc = solve_mixed_after_factor(H, m, ldH, shift, rhs, dir, kMixedIters,
                                                    kMixedTol, mixw, L.mix_bytes, info, s);
            if (rc == SPSVM_OK) mixed = true;
            else if (rc != SPSVM_ERR_NO_CONVERGE && rc != SPSVM_ERR_NOT_PD) return rc;
            // the factor in the mixed work is now that of this matrix: an
            // anchor for low-rank corrections when unshifted and refined
            anchor_m = (op.lowrank && mixed && shift == 0.0 && m >= kLowRankMinBasis) ? m : -1;
            if (anchor_m == m)
              SPSVM_CUDA_TRY(cudaMemcpyAsync(anchor, act, n, cudaMemcpyDeviceToDevice, s));
          }
          if (mixed) {
            jitter = lv;
            break;
          }
          // FP64 factorisation in place (H is overwritten by its factor)
          if (lv >= 0) {
            add_diag<<<mb, tpb, 0, s>>>(H, ldH, m, shift);
            SPSVM_LAUNCH_CHECK();
          }
          h_fresh = false;
          SPSVM_TRY(spsvm_cholesky(H, m, ldH, info, ws + L.off_chw, L.chw_bytes, s));
          SPSVM_TRY(read(&info_h, info, sizeof(info_h)));
          if (info_h == 0) {
            jitter = lv;
            SPSVM_CUDA_TRY(cudaMemcpyAsync(dir, rhs, m * sizeof(double), cudaMemcpyDeviceToDevice, s));
            SPSVM_TRY(spsvm_cholesky_solve(H, m, ldH, dir, ws + L.off_sv, L.sv_bytes, s));
            break;
          }
        }
        fac_kind = mixed ? FAC_MIXED : FAC_FP64;
        fac_shift = shift;
        if (gsmall) SPSVM_TRY(step_small(&done));
        if (done) break;
        // d = -(H + shift I)^{-1} g (computed above), u = K_nJ d
        SPSVM_TRY(finish_direction(act, fac_kind, shift));
        t = 0.0;
        SPSVM_TRY(search_and_step(&t));
        // with a small gradient, no descent means rounding level: no jitter
        if (t > 0.0 || gsmall || jitter >= kJitterMaxLevel) break;
        ++jitter;
      }
      if (done) {
        converged();
        break;
      }
      if (!(t > 0.0)) {
        // no descent even at the largest jitter (or with a small gradient):
        // rounding level reached
        spsvm_step rec{m, (int32_t)st[2], gnorm, 0.0, st[0], (int32_t)st[1], jitter, 0,
                       SPSVM_NEWTON_NONE};
        model->history.push_back(rec);
        if (gsmall) status = SPSVM_OK;
        break;
      }
      // the step and its consequences ran with the line search
      const int nxt = act_cur ^ 1;
      double st2[3];
      const unsigned long long nd = nd_next;
      std::memcpy(st2, st_next, sizeof(st2));
      std::memcpy(dh, dh_next, sizeof(dh));
      spsvm_step rec{m, (int32_t)st[2], gnorm, t, st2[0], (int32_t)st2[1], jitter, (int32_t)nd, how};
      model->history.push_back(rec);
      act_cur = nxt;
      std::memcpy(st, st2, sizeof(st));
      // a full Newton step that keeps the active set lands on the minimiser of
      // f when the direction is exact (unshifted, refined against the exactly
      // applied H); otherwise the next step's gradient test decides, and that
      // step reuses the factor (the active set, hence H, is unchanged)
      if (t == 1.0 && nd == 0 && jitter < 0 && op.refine > 0) {
        status = SPSVM_OK;
        break;
      }
      reuse = nd == 0;
      kept_prev = nd == 0 && t >= 0.5;
    }
    model->status = status;
    return SPSVM_OK;
  }

  double op_lambda() const { return lambda; }
  // the bias b = beta_0 on the device when fitted, else NULL
  const double* b0() const { return op.bias ? reinterpret_cast<const double*>(ws + L.off_beta) : nullptr; }

  int run() {
    s = op.stream;
    ProfScope prof(PROF_FIT, s, 1.0);
    std::memset(&pts, 0, sizeof(pts));
    pts.X = X;
    pts.n = n;
    pts.d = d;
    pts.ldx = ldx;
    pts.norms = at<float>(L.off_norms);
    pts.ldh = L.ldh;
    if (op.precision == SPSVM_BF16SPLIT) {
      pts.hi = at<uint16_t>(L.off_xhi);
      pts.mid = at<uint16_t>(L.off_xmid);
      pts.lo = at<uint16_t>(L.off_xlo);
    }
    SPSVM_TRY(spsvm_prepare_points(&pts, op.precision, s));
    SPSVM_CUDA_TRY(cudaMemsetAsync(ws + L.off_beta, 0, L.jcap * 8, s));
    SPSVM_CUDA_TRY(cudaMemsetAsync(ws + L.off_o, 0, n * 4, s));
    int64_t* Jd = at<int64_t>(L.off_J);
    // Eq. 4's bias: slot 0 of the basis, point index -1, a row of ones in K
    const int32_t nb0 = op.bias ? 1 : 0;
    if (op.bias) J.insert(J.begin(), -1);
    if (!J.empty()) {
      m = (int32_t)J.size();
      SPSVM_CUDA_TRY(cudaMemcpyAsync(Jd, J.data(), m * 8, cudaMemcpyHostToDevice, s));
      spsvm_kmat K = kmat();
      if (op.bias) {
        fill_bias_row<<<grid_for(K.ld, 256), 256, 0, s>>>(K.data, K.format, n, K.ld, K.plane);
        SPSVM_LAUNCH_CHECK();
      }
      if (m > nb0)
        SPSVM_TRY(spsvm_kernel_block(&pts, Jd + nb0, m - nb0, gamma, op.precision, &K, nb0,
                                     ws + L.off_scratch, L.scratch_bytes, s));
      SPSVM_TRY(kjj_fill(&K, Jd, m, 0, at<double>(L.off_kjj), L.jcap, s));
      SPSVM_TRY(newton());
    }
    double st[3];
    SPSVM_TRY(flags(act_cur, st));
    double E_prev = st[1] / (double)n;
    uint32_t round = 0;
    std::vector<int64_t> cand(op.kappa);
    std::vector<double> delta(op.kappa);
    while (!op.fixed && m - nb0 < budget) {
      const int32_t nc = spsvm_draw_candidates(n, J.data(), m, op.kappa, op.seed, round, cand.data());
      if (nc <= 0) break;
      int64_t* cd = at<int64_t>(L.off_cand);
      SPSVM_CUDA_TRY(cudaMemcpyAsync(cd, cand.data(), nc * 8, cudaMemcpyHostToDevice, s));
      if (op.score == SPSVM_SCORE_EXACT) {
        SPSVM_TRY(spsvm_score_candidates_exact(&pts, y, at<float>(L.off_o), cd, nc, gamma, lambda,
                                               op.precision, b0(), at<double>(L.off_cd),
                                               at<double>(L.off_cg), ws + L.off_scratch,
                                               L.scratch_bytes, s));
      } else {
        SPSVM_TRY(spsvm_score_candidates(&pts, y, at<float>(L.off_o), cd, nc, gamma, lambda,
                                         op.precision, at<double>(L.off_cg), at<double>(L.off_ch),
                                         at<double>(L.off_cd), ws + L.off_scratch, L.scratch_bytes, s));
        if (op.bias) {
          score_bias_fix<<<(unsigned)ceil_div((int64_t)nc, (int64_t)256), 256, 0, s>>>(
              at<double>(L.off_cg), at<double>(L.off_ch), at<double>(L.off_cd), nc, lambda, b0());
          SPSVM_LAUNCH_CHECK();
        }
      }
      SPSVM_TRY(read(delta.data(), at<double>(L.off_cd), nc * 8));
      const int32_t qq = std::min<int32_t>(std::min(op.q, budget - (m - nb0)), nc);
      std::vector<int32_t> order(nc);
      std::iota(order.begin(), order.end(), 0);
      std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
        if (delta[a] != delta[b]) return delta[a] > delta[b];
        return cand[a] < cand[b];
      });
      std::vector<int64_t> chosen(qq);
      for (int k = 0; k < qq; ++k) chosen[k] = cand[order[k]];
      if (op.record) {
        model->cand_rounds.emplace_back(cand.begin(), cand.begin() + nc);
        model->chosen_rounds.push_back(chosen);
      }
      SPSVM_CUDA_TRY(cudaMemcpyAsync(Jd + m, chosen.data(), qq * 8, cudaMemcpyHostToDevice, s));
      for (auto c : chosen) J.push_back(c);
      const int32_t m0 = m;
      m += qq;
      spsvm_kmat K = kmat();
      SPSVM_TRY(spsvm_kernel_block(&pts, Jd + m0, qq, gamma, op.precision, &K, m0,
                                   ws + L.off_scratch, L.scratch_bytes, s));
      SPSVM_TRY(kjj_fill(&K, Jd, m, m0, at<double>(L.off_kjj), L.jcap, s));
      SPSVM_TRY(newton());
      ++round;
      SPSVM_TRY(flags(act_cur, st));
      const double E = st[1] / (double)n;
      if (op.growth_tol > 0 && (E_prev - E) / qq < op.growth_tol) break;
      E_prev = E;
    }
    model->rounds = (int32_t)round;
    return finish();
  }

  int finish() {
    // the bias slot (0, when fitted) is kept apart from the basis
    const int32_t nb0 = op.bias ? 1 : 0;
    std::vector<double> bh(m, 0.0);
    if (m > 0)
      SPSVM_CUDA_TRY(cudaMemcpyAsync(bh.data(), ws + L.off_beta, m * 8, cudaMemcpyDeviceToHost, s));
    model->o.assign(n, 0.f);
    SPSVM_CUDA_TRY(cudaMemcpyAsync(model->o.data(), ws + L.off_o, n * 4, cudaMemcpyDeviceToHost, s));
    SPSVM_TRY(sync());
    model->bias = (op.bias && m > 0) ? bh[0] : 0.0;
    model->J.assign(J.begin() + std::min<int32_t>(nb0, m), J.end());
    model->beta.assign(bh.begin() + std::min<int32_t>(nb0, m), bh.end());
    const int32_t mr = (int32_t)model->J.size();
    if (mr > 0) {
      SPSVM_CUDA_TRY(cudaMalloc(&model->basis_dev, (size_t)mr * d * 4));
      SPSVM_CUDA_TRY(cudaMalloc(&model->beta_dev, (size_t)mr * 8));
      gather_rows<<<(unsigned)ceil_div((int64_t)mr * d, 256), 256, 0, s>>>(
          X, ldx, d, at<int64_t>(L.off_J) + nb0, mr, model->basis_dev);
      SPSVM_LAUNCH_CHECK();
      SPSVM_CUDA_TRY(cudaMemcpyAsync(model->beta_dev, model->beta.data(), mr * 8,
                                     cudaMemcpyHostToDevice, s));
    }
    // the SIMT form's basis norms (the split form's decision work is per call)
    model->scratch_bytes = spsvm_decision_scratch_bytes(0, mr, d, SPSVM_FP32);
    SPSVM_CUDA_TRY(cudaMalloc(&model->scratch_dev, model->scratch_bytes));
    return sync();
  }
};

}  // namespace
}  // namespace spsvm

using namespace spsvm;

extern "C" int32_t spsvm_draw_candidates(int64_t n, const int64_t* J, int32_t nJ, int32_t kappa,
                                         uint64_t seed, uint32_t round, int64_t* out) {
  if (n < 0 || nJ < 0 || kappa < 0 || (nJ > 0 && !J) || (kappa > 0 && !out)) return -1;
  std::vector<char> inJ((size_t)n, 0);
  for (int32_t k = 0; k < nJ; ++k)
    if (J[k] >= 0 && J[k] < n) inJ[(size_t)J[k]] = 1;
  std::vector<int64_t> pool;
  pool.reserve((size_t)n);
  for (int64_t i = 0; i < n; ++i)
    if (!inJ[(size_t)i]) pool.push_back(i);
  const int64_t mm = (int64_t)pool.size();
  const int32_t kk = (int32_t)std::min<int64_t>(kappa, mm);
  for (int32_t k = 0; k < kk; ++k) {
    const uint64_t r = splitmix_at(seed, ((uint64_t)round << 32) | (uint64_t)(uint32_t)k);
    const int64_t j = k + (int64_t)(r % (uint64_t)(mm - k));
    std::swap(pool[k], pool[j]);
  }
  for (int32_t k = 0; k < kk; ++k) out[k] = pool[k];
  return kk;
}

extern "C" size_t spsvm_fit_workspace_bytes(int64_t n, int64_t d, int32_t basis_budget,
                                            const spsvm_options* opt) {
  if (n < 1 || d < 1 || basis_budget < 1) return 0;
  const Opts op = resolve(opt);
  return make_layout(n, d, basis_budget, op.precision, op.kappa, op.q, op.solver, op.score, op.bias,
                     op.lowrank).total;
}

extern "C" int spsvm_fit(const float* X, int64_t n, int64_t d, int64_t ldx, const float* y,
                         float gamma, double lambda, int32_t basis_budget, double tol,
                         const spsvm_options* opt, void* workspace, size_t workspace_bytes,
                         spsvm_model** out) {
  if (!out) return set_error(SPSVM_ERR_ARG, "fit: NULL out");
  *out = nullptr;
  if (!X || !y || n < 1 || d < 1 || ldx < d)
    return set_error(SPSVM_ERR_ARG, "fit: bad data arguments (n=%lld d=%lld ldx=%lld)",
                     (long long)n, (long long)d, (long long)ldx);
  if (!(gamma > 0.f) || !(lambda > 0.0) || basis_budget < 1 || basis_budget > n || tol < 0)
    return set_error(SPSVM_ERR_ARG, "fit: need gamma > 0, lambda > 0, 1 <= budget <= n, tol >= 0");
  if (n > (int64_t)INT32_MAX) return set_error(SPSVM_ERR_ARG, "fit: n too large");
  Opts op = resolve(opt);
  if (op.precision != SPSVM_FP32 && op.precision != SPSVM_BF16SPLIT)
    return set_error(SPSVM_ERR_ARG, "fit: bad precision %d", op.precision);
  if (op.bias && op.refine > 0)
    return set_error(SPSVM_ERR_ARG, "fit: refinement sweeps are not available with the bias");
  std::vector<int64_t> J0;
  if (opt && opt->n_initial > 0) {
    if (!opt->initial_basis) return set_error(SPSVM_ERR_ARG, "fit: NULL initial_basis");
    std::vector<char> seen((size_t)n, 0);
    for (int32_t k = 0; k < opt->n_initial; ++k) {
      const int64_t j = opt->initial_basis[k];
      if (j < 0 || j >= n || seen[(size_t)j])
        return set_error(SPSVM_ERR_ARG, "fit: initial basis index %lld invalid or repeated",
                         (long long)j);
      seen[(size_t)j] = 1;
      J0.push_back(j);
    }
    if ((int32_t)J0.size() > basis_budget) basis_budget = (int32_t)J0.size();
  }
  if (op.fixed && J0.empty()) return set_error(SPSVM_ERR_ARG, "fit: fixed_basis needs an initial basis");
  Layout L = make_layout(n, d, basis_budget, op.precision, op.kappa, op.q, op.solver, op.score, op.bias,
                     op.lowrank);
  bool own = false;
  if (!workspace) {
    cudaError_t e = cudaMalloc(&workspace, L.total);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return set_error(SPSVM_ERR_OOM, "fit: cannot allocate %zu bytes", L.total);
    }
    own = true;
  } else if (workspace_bytes < L.total) {
    return set_error(SPSVM_ERR_OOM, "fit: workspace %zu < %zu bytes", workspace_bytes, L.total);
  }
  if ((reinterpret_cast<uintptr_t>(workspace) & 255) != 0) {
    if (own) cudaFree(workspace);
    return set_error(SPSVM_ERR_ARG, "fit: workspace must be 256-byte aligned");
  }
  spsvm_model* model = new spsvm_model();
  model->n = n;
  model->d = d;
  model->gamma = gamma;
  model->lambda = lambda;
  model->precision = op.precision;
  cudaGetDevice(&model->device);
  Fit f;
  f.X = X;
  f.y = y;
  f.n = n;
  f.d = d;
  f.ldx = ldx;
  f.gamma = gamma;
  f.lambda = lambda;
  f.tol = tol;
  f.budget = basis_budget;
  f.op = op;
  f.L = L;
  f.ws = static_cast<char*>(workspace);
  f.model = model;
  f.J = J0;
  int rc = f.run();
  if (own) {
    cudaStreamSynchronize(f.s);
    cudaFree(workspace);
  }
  if (rc != SPSVM_OK) {
    spsvm_free(model);
    return rc;
  }
  *out = model;
  return model->status == SPSVM_ERR_NO_CONVERGE ? SPSVM_ERR_NO_CONVERGE : SPSVM_OK;
}

extern "C" size_t spsvm_predict_work_bytes(const spsvm_model* model, int64_t nq) {
  if (!model || nq < 1 || model->J.empty() || model->precision != SPSVM_BF16SPLIT) return 0;
  return spsvm_decision_scratch_bytes(nq, (int64_t)model->J.size(), model->d, SPSVM_BF16SPLIT);
}

extern "C" int spsvm_predict_ws(const spsvm_model* model, const float* Xq, int64_t nq, int64_t ldq,
                                float* decision, void* work, size_t work_bytes, void* stream) {
  if (!model || !Xq || !decision || nq < 0 || ldq < model->d)
    return set_error(SPSVM_ERR_ARG, "predict: bad arguments");
  if (nq == 0) return SPSVM_OK;
  cudaStream_t s = as_stream(stream);
  if (model->J.empty()) {
    SPSVM_CUDA_TRY(cudaMemsetAsync(decision, 0, nq * 4, s));
  } else if (model->precision == SPSVM_BF16SPLIT) {
    const size_t need = spsvm_predict_work_bytes(model, nq);
    if (!work || work_bytes < need)
      return set_error(SPSVM_ERR_OOM, "predict: work %zu < %zu bytes", work_bytes, need);
    SPSVM_TRY(spsvm_decision(model->basis_dev, (int64_t)model->J.size(), model->d, model->beta_dev,
                             Xq, nq, ldq, model->d, model->gamma, SPSVM_BF16SPLIT, decision, work,
                             work_bytes, stream));
  } else {
    SPSVM_TRY(spsvm_decision(model->basis_dev, (int64_t)model->J.size(), model->d, model->beta_dev,
                             Xq, nq, ldq, model->d, model->gamma, SPSVM_FP32, decision,
                             model->scratch_dev, model->scratch_bytes, stream));
  }
  if (model->bias != 0.0) {   // f(x) + b
    add_const<<<grid_for(nq, 256), 256, 0, s>>>(decision, nq, (float)model->bias);
    SPSVM_LAUNCH_CHECK();
  }
  return SPSVM_OK;
}

extern "C" int spsvm_predict(const spsvm_model* model, const float* Xq, int64_t nq, int64_t ldq,
                             float* decision, void* stream) {
  if (!model) return set_error(SPSVM_ERR_ARG, "predict: NULL model");
  const size_t need = spsvm_predict_work_bytes(model, nq);
  if (need == 0) return spsvm_predict_ws(model, Xq, nq, ldq, decision, nullptr, 0, stream);
  // stream-ordered work memory: no device synchronisation, and every
  // concurrent call on the same model has its own
  cudaStream_t s = as_stream(stream);
  void* w = nullptr;
  SPSVM_CUDA_TRY(cudaMallocAsync(&w, need, s));
  const int rc = spsvm_predict_ws(model, Xq, nq, ldq, decision, w, need, stream);
  const cudaError_t e = cudaFreeAsync(w, s);
  if (rc != SPSVM_OK) return rc;
  if (e != cudaSuccess)
    return set_error(SPSVM_ERR_CUDA, "predict: cudaFreeAsync: %s", cudaGetErrorString(e));
  return SPSVM_OK;
}

extern "C" size_t spsvm_model_device_bytes(const spsvm_model* m) {
  if (!m) return 0;
  const size_t mr = m->J.size();
  return (m->basis_dev ? mr * (size_t)m->d * 4 : 0) + (m->beta_dev ? mr * 8 : 0) +
         (m->scratch_dev ? m->scratch_bytes : 0);
}

extern "C" int spsvm_model_bias(const spsvm_model* m, double* b) {
  if (!m || !b) return set_error(SPSVM_ERR_ARG, "model_bias: NULL argument");
  *b = m->bias;
  return SPSVM_OK;
}

extern "C" int spsvm_model_info(const spsvm_model* m, int32_t* n_basis, int64_t* d, float* gamma,
                                double* lambda, double* objective, int32_t* newton_steps,
                                int32_t* rounds, int32_t* status) {
  if (!m) return set_error(SPSVM_ERR_ARG, "model_info: NULL model");
  if (n_basis) *n_basis = (int32_t)m->J.size();
  if (d) *d = m->d;
  if (gamma) *gamma = m->gamma;
  if (lambda) *lambda = m->lambda;
  if (objective) *objective = m->objective;
  if (newton_steps) {
    int32_t c = 0;
    for (const auto& h : m->history) c += (h.t != 0.0);
    *newton_steps = c;
  }
  if (rounds) *rounds = m->rounds;
  if (status) *status = m->status;
  return SPSVM_OK;
}

extern "C" int spsvm_model_get(const spsvm_model* m, int64_t* basis_idx, double* beta) {
  if (!m) return set_error(SPSVM_ERR_ARG, "model_get: NULL model");
  if (basis_idx) std::copy(m->J.begin(), m->J.end(), basis_idx);
  if (beta) std::copy(m->beta.begin(), m->beta.end(), beta);
  return SPSVM_OK;
}

extern "C" int spsvm_model_history(const spsvm_model* m, spsvm_step* out, int32_t cap,
                                   int32_t* count) {
  if (!m) return set_error(SPSVM_ERR_ARG, "model_history: NULL model");
  if (count) *count = (int32_t)m->history.size();
  if (out && cap > 0) {
    const size_t k = std::min<size_t>(cap, m->history.size());
    std::copy(m->history.begin(), m->history.begin() + k, out);
  }
  return SPSVM_OK;
}

extern "C" int spsvm_model_round(const spsvm_model* m, int32_t r, int64_t* candidates,
                                 int32_t* n_candidates, int64_t* chosen, int32_t* n_chosen) {
  if (!m) return set_error(SPSVM_ERR_ARG, "model_round: NULL model");
  if (r < 0 || r >= (int32_t)m->cand_rounds.size())
    return set_error(SPSVM_ERR_ARG, "model_round: round %d not recorded", r);
  const auto& c = m->cand_rounds[r];
  const auto& h = m->chosen_rounds[r];
  if (n_candidates) *n_candidates = (int32_t)c.size();
  if (n_chosen) *n_chosen = (int32_t)h.size();
  if (candidates) std::copy(c.begin(), c.end(), candidates);
  if (chosen) std::copy(h.begin(), h.end(), chosen);
  return SPSVM_OK;
}

extern "C" int spsvm_model_outputs(const spsvm_model* m, float* o, int64_t n) {
  if (!m || !o || n != m->n) return set_error(SPSVM_ERR_ARG, "model_outputs: bad arguments");
  std::copy(m->o.begin(), m->o.end(), o);
  return SPSVM_OK;
}

extern "C" void spsvm_free(spsvm_model* m) {
  if (!m) return;
  if (m->basis_dev) cudaFree(m->basis_dev);
  if (m->beta_dev) cudaFree(m->beta_dev);
  if (m->scratch_dev) cudaFree(m->scratch_dev);
  delete m;
}
