// Error reporting, device facts and point preparation (row norms, BF16
// split planes).
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "internal.h"

namespace spsvm {

static thread_local char g_last_error[512] = "";

int set_error(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
  va_end(ap);
  return code;
}

int sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
  if (cached[dev] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0)
      v = 148;
    cached[dev] = v;
  }
  return cached[dev];
}

int check_kmat(const spsvm_kmat* K, const char* what) {
  if (!K || !K->data) return set_error(SPSVM_ERR_ARG, "%s: NULL kernel matrix", what);
  if (K->format != SPSVM_FP32 && K->format != SPSVM_BF16X3)
    return set_error(SPSVM_ERR_ARG, "%s: bad format %d", what, K->format);
  if (K->n < 0 || K->rows < 0 || K->ld < K->n || (K->ld % 8) != 0)
    return set_error(SPSVM_ERR_ARG, "%s: bad shape n=%lld rows=%lld ld=%lld", what,
                     (long long)K->n, (long long)K->rows, (long long)K->ld);
  if (K->format == SPSVM_BF16X3 && K->plane < K->rows * K->ld)
    return set_error(SPSVM_ERR_ARG, "%s: hi/lo planes overlap", what);
  if ((reinterpret_cast<uintptr_t>(K->data) & 15) != 0)
    return set_error(SPSVM_ERR_ARG, "%s: data not 16-byte aligned", what);
  return SPSVM_OK;
}

// One warp per point: ||x_i||^2 in FP64, and the BF16 split of the row.
__global__ void prepare_points_kernel(const float* __restrict__ X, int64_t n, int64_t d,
                                      int64_t ldx, float* __restrict__ norms,
                                      __nv_bfloat16* __restrict__ hi,
                                      __nv_bfloat16* __restrict__ lo, int64_t ldh) {
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= n) return;
  const float* x = X + i * ldx;
  double acc = 0.0;
  for (int64_t k = lane; k < d; k += 32) {
    float v = x[k];
    acc += (double)v * (double)v;
  }
  acc = warp_sum(acc);
  if (lane == 0) norms[i] = (float)acc;
  if (hi) {
    for (int64_t k = lane; k < ldh; k += 32) {
      __nv_bfloat16 h = __float2bfloat16_rn(0.0f), l = h;
      if (k < d) split_bf16(x[k], h, l);
      hi[i * ldh + k] = h;
      lo[i * ldh + k] = l;
    }
  }
}

}  // namespace spsvm

using namespace spsvm;

extern "C" const char* spsvm_strerror(int code) {
  switch (code) {
    case SPSVM_OK: return "ok";
    case SPSVM_ERR_ARG: return "invalid argument";
    case SPSVM_ERR_OOM: return "out of memory / workspace too small";
    case SPSVM_ERR_NOT_PD: return "Newton matrix not positive definite";
    case SPSVM_ERR_NO_CONVERGE: return "Newton iteration limit reached";
    case SPSVM_ERR_CUDA: return "CUDA error";
    case SPSVM_ERR_TIMEOUT: return "bounded device wait timed out";
    case SPSVM_ERR_BUSY: return "not admitted yet";
    default: return "unknown status";
  }
}

extern "C" const char* spsvm_last_error(void) { return g_last_error; }

extern "C" const char* spsvm_version(void) {
  return "spsvm 0.1 (sm_103a, tcgen05)";
}

extern "C" int spsvm_prepare_points(spsvm_points* p, int32_t precision, void* stream) {
  if (!p || !p->X || !p->norms) return set_error(SPSVM_ERR_ARG, "prepare_points: NULL pointer");
  if (p->n < 0 || p->d < 1 || p->ldx < p->d)
    return set_error(SPSVM_ERR_ARG, "prepare_points: bad shape n=%lld d=%lld ldx=%lld",
                     (long long)p->n, (long long)p->d, (long long)p->ldx);
  if (precision == SPSVM_BF16X3) {
    if (!p->hi || !p->lo || p->ldh < p->d || (p->ldh % 64) != 0)
      return set_error(SPSVM_ERR_ARG, "prepare_points: BF16X3 needs hi/lo planes with ldh %% 64 == 0");
  } else if (precision != SPSVM_FP32) {
    return set_error(SPSVM_ERR_ARG, "prepare_points: bad precision %d", precision);
  }
  if (p->n == 0) return SPSVM_OK;
  const int warps = 8;
  dim3 grid((unsigned)ceil_div(p->n, warps));
  prepare_points_kernel<<<grid, warps * 32, 0, as_stream(stream)>>>(
      p->X, p->n, p->d, p->ldx, p->norms,
      precision == SPSVM_BF16X3 ? reinterpret_cast<__nv_bfloat16*>(p->hi) : nullptr,
      precision == SPSVM_BF16X3 ? reinterpret_cast<__nv_bfloat16*>(p->lo) : nullptr, p->ldh);
  SPSVM_LAUNCH_CHECK();
  return SPSVM_OK;
}
