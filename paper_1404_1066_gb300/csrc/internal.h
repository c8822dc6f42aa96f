// Internal helpers shared by the CUDA translation units of libspsvm.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <stddef.h>

#include "spsvm.h"

namespace spsvm {

// Records a message for spsvm_last_error() and returns `code`.
int set_error(int code, const char* fmt, ...);

#define SPSVM_CUDA_TRY(expr)                                                 \
  do {                                                                       \
    cudaError_t e_ = (expr);                                                 \
    if (e_ != cudaSuccess)                                                   \
      return ::spsvm::set_error(SPSVM_ERR_CUDA, "%s:%d %s: %s", __FILE__,    \
                                __LINE__, #expr, cudaGetErrorString(e_));    \
  } while (0)

void count_launch();

#define SPSVM_LAUNCH_CHECK()                                                 \
  do {                                                                       \
    ::spsvm::count_launch();                                                 \
    cudaError_t e_ = cudaGetLastError();                                     \
    if (e_ != cudaSuccess)                                                   \
      return ::spsvm::set_error(SPSVM_ERR_CUDA, "%s:%d launch: %s", __FILE__, \
                                __LINE__, cudaGetErrorString(e_));           \
  } while (0)

#define SPSVM_TRY(expr)                                                      \
  do {                                                                       \
    int s_ = (expr);                                                         \
    if (s_ != SPSVM_OK) return s_;                                           \
  } while (0)

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

__host__ __device__ inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }
__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
__host__ __device__ inline int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }
__host__ __device__ inline int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }

// Number of SMs of the current device (cached per device).
int sm_count();

// Checks a stored-kernel-matrix descriptor.
int check_kmat(const spsvm_kmat* K, const char* what);

// Element (row j, column i) of a stored kernel matrix as FP32.
struct KView {
  const void* data;
  int32_t format;
  int64_t ld, plane;
  __device__ __forceinline__ float at(int64_t j, int64_t i) const {
    if (format == SPSVM_FP32) return static_cast<const float*>(data)[j * ld + i];
    const __nv_bfloat16* h = static_cast<const __nv_bfloat16*>(data);
    return __bfloat162float(h[j * ld + i]) + __bfloat162float(h[plane + j * ld + i]);
  }
};

inline KView view(const spsvm_kmat* K) {
  return KView{K->data, K->format, K->ld, K->plane};
}

// Splits an FP32 value into BF16 hi + lo (hi = round(x), lo = round(x - hi)).
__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(x);
  lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// Stores an FP32 kernel value into a kernel matrix (FP32 or hi/lo planes).
__device__ __forceinline__ void kstore(void* data, int32_t format, int64_t plane,
                                       int64_t off, float v) {
  if (format == SPSVM_FP32) {
    static_cast<float*>(data)[off] = v;
  } else {
    __nv_bfloat16 h, l;
    split_bf16(v, h, l);
    __nv_bfloat16* p = static_cast<__nv_bfloat16*>(data);
    p[off] = h;
    p[plane + off] = l;
  }
}

// RBF value from the distance expansion; clamps rounding below zero.
__device__ __forceinline__ float rbf_from_dot(float xn, float zn, float dot, float gamma) {
  float d2 = fmaxf(xn + zn - 2.0f * dot, 0.0f);
  return expf(-gamma * d2);
}

// Warp sum of a double.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ int warp_sum(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Column sums of a warp's 32 x 32 block (lane = row, v[j] = column j): after
// five exchange steps, each halving the columns a lane holds and summing
// the pair, lane l holds the sum of column l (31 shuffles in all).
__device__ __forceinline__ float warp_column_sums(float (&v)[32], int lane) {
#pragma unroll
  for (int h = 16; h >= 1; h >>= 1) {
    const bool upper = (lane & h) != 0;
#pragma unroll
    for (int k = 0; k < h; ++k) {
      const float give = upper ? v[k] : v[k + h];
      const float keep = upper ? v[k + h] : v[k];
      v[k] = keep + __shfl_xor_sync(0xffffffffu, give, h);
    }
  }
  return v[0];
}

// Block sum (blockDim.x multiple of 32, <= 1024); result valid in thread 0.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* sh /* >= 32 entries */) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  const int nw = blockDim.x >> 5;
  T r = (threadIdx.x < nw) ? sh[threadIdx.x] : T(0);
  if (w == 0) r = warp_sum(r);
  return r;
}

// Kernel timing slots (CUDA events on the launching stream, when enabled).
enum ProfSlot {
  PROF_KERNEL_BLOCK = 0, PROF_SCORE, PROF_OUTPUTS, PROF_GEMV, PROF_COMPACT, PROF_GRAM,
  PROF_CHOLESKY, PROF_SOLVE, PROF_LINE, PROF_DECISION, PROF_FIT, PROF_LOWRANK, PROF_SLOTS
};
struct ProfScope {
  int slot;
  cudaStream_t s;
  double work;
  void* e0;
  ProfScope(int slot, cudaStream_t s, double work);
  ~ProfScope();
};

// Host-side launchers implemented in the .cu files (used by the fit).
int launch_kernel_block_simt(const spsvm_points* p, const int64_t* idx, int32_t m,
                             float gamma, spsvm_kmat* out, int64_t row0, cudaStream_t s);
int launch_kernel_block_tc(const spsvm_points* p, const int64_t* idx, int32_t m,
                           float gamma, spsvm_kmat* out, int64_t row0, void* scratch,
                           size_t scratch_bytes, cudaStream_t s);
size_t kernel_block_tc_scratch(int64_t m, int64_t ldh);
bool tc_available();

// Bounded device waits.  Every kernel that waits on the device gets the
// wait context of the stream it runs on: the stream's status word (the site
// code of the first wait that gave up, 0 while none did; a word of its own
// per stream, so that concurrent fits never see each other's codes) and the
// iteration limit of each wait (0: the site's default, about a second;
// spsvm_set_wait_limit sets it).
struct WaitCtx {
  int* st;
  uint32_t lim;
};
// The wait context for launches on stream s.
int wait_ctx(cudaStream_t s, WaitCtx* w);
__device__ __forceinline__ uint32_t wait_limit(const WaitCtx& w, uint32_t dflt) {
  return w.lim ? w.lim : dflt;
}
// Records a wait that gave up (the first code on the stream is kept).
__device__ __forceinline__ void wait_gave_up(const WaitCtx& w, int code) { atomicCAS(w.st, 0, code); }

// Synchronises s and takes (reads and clears) the status word of stream s
// (stream-ordered copies; returns TIMEOUT with *code set when a wait gave up).
int device_status_on(cudaStream_t s, int32_t* code);

// Device-to-host reads after the work queued on s: every chunk and the
// stream's status word are copied in order on s into a pinned staging
// buffer of the calling thread, s is synchronised once, and the chunks are
// copied out.  Returns TIMEOUT (status word taken and cleared) when a
// bounded wait gave up on s.
struct ReadChunk {
  void* dst;
  const void* src;
  size_t bytes;
};
int read_back(cudaStream_t s, const ReadChunk* chunks, int n);

// spsvm_line_search with Eq. 4's bias in basis slot 0 (point index -1):
// b0 = &beta_0 on the device, or NULL without a bias.
int line_search_impl(const float* o, const float* u, const float* y, int64_t n, const double* d,
                     const int64_t* J, int32_t m, double lambda, double* t_host, double* t_dev,
                     void* scratch, size_t scratch_bytes, void* stream, const double* b0);

// line_search_impl without a host round trip: t (0 when no descent or when
// a grid barrier gave up) and the barrier error word go to device memory,
// in order on the stream.
int line_search_async(const float* o, const float* u, const float* y, int64_t n, const double* d,
                      const int64_t* J, int32_t m, double lambda, double* t_dev, int32_t* err_dev,
                      void* scratch, size_t scratch_bytes, void* stream, const double* b0);

// spsvm_solve_mixed right after spsvm_cholesky_mixed with its info word
// read at the first refinement check (SPSVM_ERR_NOT_PD when it is nonzero).
int solve_mixed_after_factor(const double* H, int64_t m, int64_t ldh, double shift,
                             const double* b, double* x, int32_t max_iter, double tol,
                             void* work, size_t work_bytes, const int32_t* factor_info,
                             void* stream);

// spsvm_compact_active whose K_SJ copy is written only when *kc_cond (read
// on the device) is nonzero; kc_cond NULL: always.
int compact_active_impl(const spsvm_kmat* K, const uint8_t* active, const float* w1,
                        const float* w2, double* w1out, double* w2out, spsvm_kmat* Kc,
                        const unsigned long long* kc_cond, int64_t* n_active, int32_t* pos,
                        void* scratch, size_t scratch_bytes, void* stream);

}  // namespace spsvm
