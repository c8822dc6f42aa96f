// FP64 Cholesky factorisation H = L L^T and the two triangular solves of
// the Newton system of Section 4's reoptimisation.  Blocked right-looking
// factorisation with 64 x 64 blocks: diagonal block in shared memory, panel
// triangular solve, trailing symmetric update.
#include <mutex>
#include <vector>

#include "internal.h"

namespace spsvm {

// Status word of the triangular solves' bounded waits (site codes 21, 22).
__device__ int g_sv_status = 0;

int sv_status_address(void** p) {
  SPSVM_CUDA_TRY(cudaGetSymbolAddress(p, g_sv_status));
  return SPSVM_OK;
}

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

// GB300 issues FP64 at about half an operation per clock per SM
// sub-partition, so a warp-wide FP64 instruction occupies its pipe for ~64
// clocks: the panel kernels below spread their FP64 work over four warps (all
// four sub-partitions) and give each thread columns interleaved with stride
// 4, so that a triangular loop wastes at most one predicated slot per step.
constexpr int PT = 128;   // threads of the panel kernels

// Factors the PB x PB diagonal block at k0 in place, column by column in
// shared memory: pivot, column scaling, rank-1 update of the trailing lower
// triangle.  Thread t updates row t / 4, columns t % 4 + 4 i.
__global__ void __launch_bounds__(PT) potrf_diag(double* __restrict__ H, int64_t ldh, int64_t m,
                                                 int64_t k0, int32_t* __restrict__ info) {
  __shared__ double A[PB][PB + 1];
  __shared__ double piv[PB];
  if (*info != 0) return;
  const int nb = (int)min64(PB, m - k0);
  const int t = threadIdx.x;
  for (int e = t; e < PB * PB; e += PT) {
    const int r = e / PB, c = e % PB;
    A[r][c] = (r < nb && c <= r) ? H[(k0 + r) * ldh + k0 + c] : (r == c ? 1.0 : 0.0);
  }
  __syncthreads();
  const int r = t >> 2, q = t & 3;
  int fail = 0;
  for (int j = 0; j < nb; ++j) {
    const double d = A[j][j];   // updated by the previous columns; not written in this one
    if (!(d > 0.0) || !(d < 1e300)) {
      fail = j + 1;             // the same value in every thread
      break;
    }
    const double y = rsqrt_fp64(d);
    if (t == 0) piv[j] = d * y;               // L_jj = sqrt(d)
    if (t > j && t < nb) A[t][j] *= y;         // L[t][j]
    __syncthreads();
    if (r > j) {
      const double lr = A[r][j];
#pragma unroll
      for (int i = 0; i < PB / 4; ++i) {
        const int c = q + 4 * i;
        if (c > j && c <= r) A[r][c] = fma(-lr, A[c][j], A[r][c]);
      }
    }
    __syncthreads();
  }
  if (fail) {
    if (t == 0) *info = (int32_t)(k0 + fail);
    return;
  }
  for (int e = t; e < PB * PB; e += PT) {
    const int rr = e / PB, cc = e % PB;
    if (rr < nb && cc <= rr) H[(k0 + rr) * ldh + k0 + cc] = (rr == cc) ? piv[rr] : A[rr][cc];
  }
}

// Rows r >= k0 + PB: L[r][k0:k0+PB] = H[r][k0:k0+PB] L_kk^{-T} by
// column-oriented substitution, x_j = b_j / L_jj then b_l -= x_j L_lj for
// l > j.  Four threads per row (32 rows per CTA); thread q of a row holds
// columns q + 4 i and x_j travels by shuffle from the thread that owns it.
__global__ void __launch_bounds__(PT) trsm_panel(double* __restrict__ H, int64_t ldh, int64_t m,
                                                 int64_t k0, const int32_t* __restrict__ info) {
  __shared__ double L[PB][PB + 1];
  __shared__ double rd[PB];
  if (*info != 0) return;
  for (int e = threadIdx.x; e < PB * PB; e += PT) {
    const int r = e / PB, c = e % PB;
    L[r][c] = (c <= r) ? H[(k0 + r) * ldh + k0 + c] : 0.0;
  }
  __syncthreads();
  if (threadIdx.x < PB) rd[threadIdx.x] = 1.0 / L[threadIdx.x][threadIdx.x];
  __syncthreads();
  const int t = threadIdx.x, lane = t & 31, q = t & 3;
  const int64_t r = k0 + PB + (int64_t)blockIdx.x * (PT / 4) + (t >> 2);
  const bool ok = r < m;
  double* row = H + (ok ? r : k0) * ldh + k0;
  double x[PB / 4];
#pragma unroll
  for (int i = 0; i < PB / 4; ++i) x[i] = ok ? row[q + 4 * i] : 0.0;
#pragma unroll
  for (int j = 0; j < PB; ++j) {
    const int owner = j & 3, ji = j >> 2;
    if (q == owner) x[ji] *= rd[j];
    const double xj = __shfl_sync(0xffffffffu, x[ji], (lane & ~3) | owner);
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
__global__ void __launch_bounds__(PT) syrk_trailing(double* __restrict__ H, int64_t ldh,
                                                    int64_t m, int64_t k0,
                                                    const int32_t* __restrict__ info) {
  __shared__ double Ar[PB][PB + 1];   // Ar[rr][l] = L[r0 + rr][k0 + l]
  __shared__ double Ac[PB][PB + 1];   // Ac[l][cc] = L[c0 + cc][k0 + l]
  if (*info != 0) return;
  const int64_t base = k0 + PB;
  const int64_t T = ceil_div(m - base, (int64_t)PB);
  // lower tile (ti >= tj) from the linear block index
  int64_t tt = blockIdx.x, ti = 0;
  while (tt > ti) {
    tt -= ti + 1;
    ++ti;
  }
  const int64_t tj = tt;
  if (ti >= T) return;
  const int64_t r0 = base + ti * PB, c0 = base + tj * PB;
  for (int e = threadIdx.x; e < PB * PB; e += PT) {
    const int rr = e / PB, ll = e % PB;
    const int64_t gr = r0 + rr, gc = c0 + rr;
    Ar[rr][ll] = (gr < m) ? H[gr * ldh + k0 + ll] : 0.0;
    Ac[ll][rr] = (gc < m) ? H[gc * ldh + k0 + ll] : 0.0;
  }
  __syncthreads();
  const int rr = threadIdx.x >> 2, q = threadIdx.x & 3;
  double acc[PB / 4];
#pragma unroll
  for (int i = 0; i < PB / 4; ++i) acc[i] = 0.0;
#pragma unroll 8
  for (int l = 0; l < PB; ++l) {
    const double a = Ar[rr][l];
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

// One thread waits for a flag to leave 0, giving up after roughly a second.
__device__ unsigned wait_flag(const unsigned* f, int code) {
  for (uint32_t it = 0; it < (1u << 23); ++it) {
    const unsigned v = ld_acquire_u32(f);
    if (v != 0u) return v;
    if (it >= 16) __nanosleep(64);
  }
  atomicCAS(&g_sv_status, 0, code);
  return 2u;
}

// Inverse of the 64 x 64 diagonal block at r0 (lower), Li[i][j], from the
// transposed copy diag_inverse leaves in the upper triangle; zero-padded
// past nb.
__device__ __forceinline__ void load_diag_inverse(const double* __restrict__ L, int64_t ldh,
                                                  int64_t r0, int nb, double (*Li)[NB + 1]) {
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int j = e / NB, i = e % NB;   // stored at (row r0 + j, column r0 + i)
    double v = 0.0;
    if (i < nb && j < nb) {
      if (i == j) v = 1.0 / L[(r0 + i) * ldh + r0 + i];
      else if (j < i) v = L[(r0 + j) * ldh + r0 + i];
    }
    Li[i][j] = v;
  }
}

// z = L^{-1} b.  Thread t: row t / 4 of the block row, columns 16 (t % 4) ..
// + 15 of each 64-column block.
__global__ void __launch_bounds__(SV_THREADS) trsv_fwd_onepass(
    const double* __restrict__ L, int64_t ldh, int64_t m, const double* __restrict__ b,
    double* __restrict__ z, unsigned* __restrict__ flags, unsigned* __restrict__ ticket) {
  __shared__ double Li[NB][NB + 1];
  __shared__ double xs[2][NB];
  __shared__ double v[NB];
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
  const double* __restrict__ Lrow = L + (r0 + (row_ok ? r : 0)) * ldh + 16 * q;
  double acc = 0.0;
  bool ok = true;
  for (int64_t j = 0; j < k; ++j) {
    double a[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) a[c] = row_ok ? __ldg(Lrow + j * NB + c) : 0.0;
    if (t == 0) state_s = wait_flag(&flags[j], 21);
    __syncthreads();
    if (state_s != 1u) {
      ok = false;
      break;
    }
    double* xb = xs[j & 1];
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
  double sres = 0.0;
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
__global__ void __launch_bounds__(SV_THREADS) trsv_bwd_onepass(
    const double* __restrict__ L, int64_t ldh, int64_t m, const double* __restrict__ z,
    double* __restrict__ x, unsigned* __restrict__ flags, unsigned* __restrict__ ticket) {
  __shared__ double Li[NB][NB + 1];
  __shared__ double xs[2][NB];
  __shared__ double part[4][NB];
  __shared__ double v[NB];
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
  double acc = 0.0;
  bool ok = true;
  for (int64_t j = B - 1; j > k; --j) {
    double a[16];
    const int64_t rb = j * NB + 16 * g;
#pragma unroll
    for (int rr = 0; rr < 16; ++rr)
      a[rr] = (c < nb && rb + rr < m) ? __ldg(L + (rb + rr) * ldh + r0 + c) : 0.0;
    if (t == 0) state_s = wait_flag(&flags[j], 22);
    __syncthreads();
    if (state_s != 1u) {
      ok = false;
      break;
    }
    double* xb = xs[j & 1];
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
  double sres = 0.0;
#pragma unroll
  for (int i = 0; i < 16; ++i) sres = fma(Li[16 * g + i][c], v[16 * g + i], sres);
  part[g][c] = sres;
  __syncthreads();
  if (t < nb) __stcg(x + r0 + t, part[0][t] + part[1][t] + part[2][t] + part[3][t]);
  __threadfence();
  __syncthreads();
  if (t == 0) st_release_u32(&flags[k], 1u);
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
    SPSVM_CUDA_TRY(cudaFuncSetAttribute(potrf_diag, cudaFuncAttributePreferredSharedMemoryCarveout,
                                        (int)cudaSharedmemCarveoutMaxShared));
    SPSVM_CUDA_TRY(cudaFuncSetAttribute(trsm_panel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                        (int)cudaSharedmemCarveoutMaxShared));
    SideGuard side;
    SPSVM_TRY(side_acquire(&side.ss));
    side.held = true;
    cudaStream_t p = side.ss.s;
    SPSVM_CUDA_TRY(cudaEventRecord(side.ss.b, s));   // H as the caller left it
    SPSVM_CUDA_TRY(cudaStreamWaitEvent(p, side.ss.b, 0));
    int buf = 0;
    for (; m - (k0 + 64) >= 256; k0 += 64, buf ^= 1) {
      potrf_diag<<<1, PT, 0, p>>>(H, ldh, m, k0, info);
      SPSVM_LAUNCH_CHECK();
      trsm_panel<<<(unsigned)ceil_div(m - (k0 + PB), PT / 4), PT, 0, p>>>(H, ldh, m, k0, info);
      SPSVM_LAUNCH_CHECK();
      SPSVM_TRY(chol_tc_panel_update(H, ldh, m, k0, info, p));
      potrf_diag<<<1, PT, 0, p>>>(H, ldh, m, k0 + PB, info);
      SPSVM_LAUNCH_CHECK();
      trsm_panel<<<(unsigned)ceil_div(m - (k0 + 2 * PB), PT / 4), PT, 0, p>>>(H, ldh, m, k0 + PB,
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
    potrf_diag<<<1, PT, 0, s>>>(H, ldh, m, k0, info);
    SPSVM_LAUNCH_CHECK();
    const int64_t below = m - (k0 + PB);
    if (below <= 0) break;
    trsm_panel<<<(unsigned)ceil_div(below, PT / 4), PT, 0, s>>>(H, ldh, m, k0, info);
    SPSVM_LAUNCH_CHECK();
    const int64_t T = ceil_div(below, (int64_t)PB);
    syrk_trailing<<<(unsigned)(T * (T + 1) / 2), PT, 0, s>>>(H, ldh, m, k0, info);
    SPSVM_LAUNCH_CHECK();
  }
  if (m > 0) {
    diag_inverse<<<(unsigned)ceil_div(m, (int64_t)NB), 64, 0, s>>>(H, ldh, m);
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
  trsv_fwd_onepass<<<(unsigned)B, SV_THREADS, 0, s>>>(L, ldh, m, b, z, flags, flags + 2 * B);
  SPSVM_LAUNCH_CHECK();
  trsv_bwd_onepass<<<(unsigned)B, SV_THREADS, 0, s>>>(L, ldh, m, z, b, flags + B, flags + 2 * B + 1);
  SPSVM_LAUNCH_CHECK();
  return SPSVM_OK;
}
