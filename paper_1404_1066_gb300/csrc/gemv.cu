// HBM-bound passes over the stored kernel matrix K_nJ (basis-major):
//   * o = K_nJ beta with the active set, loss and error count of Eq. 4;
//   * u = K_nJ v (line-search direction);
//   * active-set compaction K_SJ with the masked transposed products
//     K_SJ^T w (gradient and Newton right-hand side of Eq. 4).
// Products are FP32; every 32 terms the running sum is promoted to FP64.
#include "internal.h"

namespace spsvm {

namespace {

constexpr int GV_T = 256;          // threads per block
constexpr int GV_P = 2;            // consecutive points per thread
constexpr int GV_PTS = GV_T * GV_P;
constexpr int GV_CHUNK = 32;       // terms summed in FP32 before promotion (all in flight)
constexpr int GV_BETA = 2048;      // beta entries staged in shared memory per pass

__device__ __forceinline__ float bf_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }

// Loads the thread's 2 consecutive kernel values of row j from point i
// (i even, i + 1 < n) as FP32: one 8-byte load (FP32), or one 4-byte load
// per BF16 plane.  A warp's load instruction covers 256 contiguous bytes of
// a row; with a whole chunk of 32 rows in flight per thread this layout
// streams at the HBM read rate (fewer, wider loads per thread kept fewer
// bytes in flight).
template <int FMT>
__device__ __forceinline__ void load2(const KView& K, int64_t j, int64_t i, float k[2]) {
  if (FMT == SPSVM_FP32) {
    const float2 a = *reinterpret_cast<const float2*>(static_cast<const float*>(K.data) + j * K.ld + i);
    k[0] = a.x;
    k[1] = a.y;
  } else {
    const uint16_t* base = static_cast<const uint16_t*>(K.data);
    const uint32_t h = *reinterpret_cast<const uint32_t*>(base + j * K.ld + i);
    const uint32_t l = *reinterpret_cast<const uint32_t*>(base + K.plane + j * K.ld + i);
    k[0] = bf_lo(h) + bf_lo(l);
    k[1] = bf_hi(h) + bf_hi(l);
  }
}

// acc[p] = sum_j K[j][i + p] v_j for the thread's points.
template <int FMT>
__device__ __forceinline__ void row_products(const KView& K, int64_t rows, int64_t n,
                                             const double* __restrict__ v, int64_t i,
                                             float* vs, double acc[GV_P]) {
#pragma unroll
  for (int p = 0; p < GV_P; ++p) acc[p] = 0.0;
  const bool full = (i + GV_P <= n);
  for (int64_t j0 = 0; j0 < rows; j0 += GV_BETA) {
    const int cnt = (int)min64(GV_BETA, rows - j0);
    __syncthreads();
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) vs[t] = (float)v[j0 + t];
    __syncthreads();
    if (i >= n) continue;
    for (int c0 = 0; c0 < cnt; c0 += GV_CHUNK) {
      float f[GV_P];
#pragma unroll
      for (int p = 0; p < GV_P; ++p) f[p] = 0.f;
      if (full && c0 + GV_CHUNK <= cnt) {
#pragma unroll
        for (int c = c0; c < c0 + GV_CHUNK; ++c) {
          float k[GV_P];
          load2<FMT>(K, j0 + c, i, k);
          const float b = vs[c];
#pragma unroll
          for (int p = 0; p < GV_P; ++p) f[p] = fmaf(k[p], b, f[p]);
        }
      } else {
        const int ce = min(cnt, c0 + GV_CHUNK);
        for (int c = c0; c < ce; ++c) {
          const float b = vs[c];
          for (int p = 0; p < GV_P; ++p)
            if (i + p < n) f[p] = fmaf(K.at(j0 + c, i + p), b, f[p]);
        }
      }
#pragma unroll
      for (int p = 0; p < GV_P; ++p) acc[p] += (double)f[p];
    }
  }
}

// o = K beta (or given), active flags, per-block loss / errors / |S|.
template <int FMT>
__global__ void __launch_bounds__(GV_T) outputs_kernel(
    KView K, int64_t rows, int64_t n, const double* __restrict__ beta,
    const float* __restrict__ y, float* __restrict__ o, uint8_t* __restrict__ active,
    double* __restrict__ part, int accumulate) {
  __shared__ float vs[GV_BETA];
  __shared__ double sh[32];
  const int64_t i = ((int64_t)blockIdx.x * GV_T + threadIdx.x) * GV_P;
  double acc[GV_P];
  if (beta) row_products<FMT>(K, rows, n, beta, i, vs, acc);
  double loss = 0.0, err = 0.0, act = 0.0;
  {
#pragma unroll
    for (int p = 0; p < GV_P; ++p) {
      const int64_t ii = i + p;
      if (ii >= n) break;
      float oi;
      if (beta) {
        oi = accumulate ? (float)((double)o[ii] + acc[p]) : (float)acc[p];
        o[ii] = oi;
      } else {
        oi = o[ii];
      }
      const float yi = y[ii];
      const float margin = yi * oi;
      const bool s = margin < 1.0f;
      if (active) active[ii] = s ? 1 : 0;
      if (s) {
        const double xi = 1.0 - (double)margin;
        loss += xi * xi;
        act += 1.0;
      }
      if (margin <= 0.0f) err += 1.0;
    }
  }
  if (part) {
    loss = block_sum(loss, sh);
    __syncthreads();
    err = block_sum(err, sh);
    __syncthreads();
    act = block_sum(act, sh);
    if (threadIdx.x == 0) {
      part[3 * blockIdx.x + 0] = 0.5 * loss;
      part[3 * blockIdx.x + 1] = err;
      part[3 * blockIdx.x + 2] = act;
    }
  }
}

template <int FMT>
__global__ void __launch_bounds__(GV_T) gemv_kernel(KView K, int64_t rows, int64_t n,
                                                    const double* __restrict__ v,
                                                    float* __restrict__ u, int accumulate) {
  __shared__ float vs[GV_BETA];
  const int64_t i = ((int64_t)blockIdx.x * GV_T + threadIdx.x) * GV_P;
  double acc[GV_P];
  row_products<FMT>(K, rows, n, v, i, vs, acc);
#pragma unroll
  for (int p = 0; p < GV_P; ++p) {
    const int64_t ii = i + p;
    if (ii < n) u[ii] = accumulate ? (float)((double)u[ii] + acc[p]) : (float)acc[p];
  }
}

// Fixed-order sum of per-block triples.
__global__ void sum_triples(const double* __restrict__ part, int64_t blocks, double* out) {
  __shared__ double sh[32];
  for (int c = 0; c < 3; ++c) {
    double s = 0.0;
    for (int64_t b = threadIdx.x; b < blocks; b += blockDim.x) s += part[3 * b + c];
    s = block_sum(s, sh);
    __syncthreads();
    if (threadIdx.x == 0) out[c] = s;
  }
}

// ---- active-set scan -----------------------------------------------------
constexpr int SC_T = 256;
constexpr int SC_PTS = SC_T * 4;

// The scanned flag of point i: active[i], or with ref, active[i] != ref[i].
__device__ __forceinline__ int scan_flag(const uint8_t* __restrict__ active,
                                         const uint8_t* __restrict__ ref, int64_t i) {
  return ref ? (active[i] != ref[i]) : active[i];
}

__global__ void scan_count(const uint8_t* __restrict__ active, const uint8_t* __restrict__ ref,
                           int64_t n, int32_t* __restrict__ counts) {
  __shared__ int sh[32];
  const int64_t base = (int64_t)blockIdx.x * SC_PTS;
  int c = 0;
  for (int p = 0; p < 4; ++p) {
    const int64_t i = base + threadIdx.x + (int64_t)SC_T * p;
    if (i < n) c += scan_flag(active, ref, i);
  }
  c = block_sum(c, sh);
  if (threadIdx.x == 0) counts[blockIdx.x] = c;
}

// Exclusive scan of block counts in one block; writes the total to *total.
__global__ void scan_blocks(int32_t* __restrict__ counts, int64_t nb, int64_t* __restrict__ total) {
  __shared__ int32_t sh[1024];
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t b0 = 0; b0 < nb; b0 += blockDim.x) {
    const int64_t b = b0 + threadIdx.x;
    const int32_t v = (b < nb) ? counts[b] : 0;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
      int32_t add = (threadIdx.x >= (unsigned)off) ? sh[threadIdx.x - off] : 0;
      __syncthreads();
      sh[threadIdx.x] += add;
      __syncthreads();
    }
    const int32_t incl = sh[threadIdx.x];
    if (b < nb) counts[b] = (int32_t)(carry + incl - v);
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry += incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void scan_write(const uint8_t* __restrict__ active, const uint8_t* __restrict__ ref,
                           int64_t n, const int32_t* __restrict__ offsets, int32_t* __restrict__ pos,
                           int32_t* __restrict__ list) {
  __shared__ int32_t sh[SC_PTS];
  const int64_t base = (int64_t)blockIdx.x * SC_PTS;
  for (int p = 0; p < 4; ++p) {
    const int64_t i = base + threadIdx.x * 4 + p;
    sh[threadIdx.x * 4 + p] = (i < n) ? scan_flag(active, ref, i) : 0;
  }
  __syncthreads();
  // sequential scan per thread over its 4, then block scan of thread sums
  int32_t local[4], run = 0;
  for (int p = 0; p < 4; ++p) { local[p] = run; run += sh[threadIdx.x * 4 + p]; }
  __shared__ int32_t ts[SC_T];
  ts[threadIdx.x] = run;
  __syncthreads();
  for (int off = 1; off < SC_T; off <<= 1) {
    int32_t add = (threadIdx.x >= (unsigned)off) ? ts[threadIdx.x - off] : 0;
    __syncthreads();
    ts[threadIdx.x] += add;
    __syncthreads();
  }
  const int32_t excl = ts[threadIdx.x] - run + offsets[blockIdx.x];
  for (int p = 0; p < 4; ++p) {
    const int64_t i = base + threadIdx.x * 4 + p;
    if (i < n) {
      if (pos) pos[i] = excl + local[p];
      if (sh[threadIdx.x * 4 + p]) list[excl + local[p]] = (int32_t)i;   // flagged indices, in order
    }
  }
}

// ---- compaction + masked transposed products ---------------------------
constexpr int CP_T = 256;
constexpr int CP_ROWS = 8;      // basis rows per block

// Writes kernel value v (read from K as `h` + `l` in the planes format) to
// column q of row j of the compact matrix: FP32, or hi / lo planes (copied
// from K's planes, or split from an FP32 value).
__device__ __forceinline__ void kc_put(void* kc_data, int32_t kc_format, int64_t kc_ld,
                                       int64_t kc_plane, int32_t k_format, int64_t j, int64_t q,
                                       float v, __nv_bfloat16 h, __nv_bfloat16 l) {
  if (kc_format == SPSVM_FP32) {
    static_cast<float*>(kc_data)[j * kc_ld + q] = v;
    return;
  }
  if (k_format == SPSVM_FP32) split_bf16(v, h, l);
  __nv_bfloat16* dst = static_cast<__nv_bfloat16*>(kc_data);
  dst[j * kc_ld + q] = h;
  dst[kc_plane + j * kc_ld + q] = l;
}

__global__ void __launch_bounds__(CP_T) compact_kernel(
    KView K, int64_t rows, int64_t n, const uint8_t* __restrict__ active,
    const int32_t* __restrict__ pos, const float* __restrict__ w1, const float* __restrict__ w2,
    void* kc_data, int32_t kc_format, int64_t kc_ld, int64_t kc_plane, int64_t chunks_per_block,
    double2* __restrict__ part, const int64_t* __restrict__ ns_dev, int64_t gather_max,
    const unsigned long long* __restrict__ kc_cond) {
  __shared__ double sh[32];
  if (*ns_dev <= gather_max) return;   // few active points: compact_gather does this
  if (kc_cond && *kc_cond == 0) kc_data = nullptr;   // the caller keeps the copy it has
  const int64_t j0 = (int64_t)blockIdx.x * CP_ROWS;
  const int64_t c_begin = (int64_t)blockIdx.y * chunks_per_block;
  const int64_t nchunks = ceil_div(n, (int64_t)CP_T);
  const int64_t c_end = min(nchunks, c_begin + chunks_per_block);
  double s1[CP_ROWS], s2[CP_ROWS];
  float f1[CP_ROWS], f2[CP_ROWS];
#pragma unroll
  for (int r = 0; r < CP_ROWS; ++r) { s1[r] = 0.0; s2[r] = 0.0; f1[r] = 0.f; f2[r] = 0.f; }
  int since = 0;
  for (int64_t c = c_begin; c < c_end; ++c) {
    const int64_t i = c * CP_T + threadIdx.x;
    if (i >= n) continue;
    if (!active[i]) continue;
    const int32_t q = pos[i];
    const float a = w1 ? w1[i] : 0.f, b = w2 ? w2[i] : 0.f;
#pragma unroll
    for (int r = 0; r < CP_ROWS; ++r) {
      const int64_t j = j0 + r;
      if (j >= rows) break;
      float v;
      __nv_bfloat16 h = __float2bfloat16_rn(0.f), l = h;
      if (K.format == SPSVM_FP32) {
        v = static_cast<const float*>(K.data)[j * K.ld + i];
      } else {
        const __nv_bfloat16* src = static_cast<const __nv_bfloat16*>(K.data);
        h = src[j * K.ld + i];
        l = src[K.plane + j * K.ld + i];
        v = __bfloat162float(h) + __bfloat162float(l);
      }
      if (kc_data) kc_put(kc_data, kc_format, kc_ld, kc_plane, K.format, j, q, v, h, l);
      f1[r] = fmaf(a, v, f1[r]);
      f2[r] = fmaf(b, v, f2[r]);
    }
    if (++since == 32) {
#pragma unroll
      for (int r = 0; r < CP_ROWS; ++r) {
        s1[r] += (double)f1[r]; s2[r] += (double)f2[r]; f1[r] = 0.f; f2[r] = 0.f;
      }
      since = 0;
    }
  }
#pragma unroll
  for (int r = 0; r < CP_ROWS; ++r) { s1[r] += (double)f1[r]; s2[r] += (double)f2[r]; }
  for (int r = 0; r < CP_ROWS; ++r) {
    const double a = block_sum(s1[r], sh);
    __syncthreads();
    const double b = block_sum(s2[r], sh);
    __syncthreads();
    const int64_t j = j0 + r;
    if (threadIdx.x == 0 && j < rows) part[(int64_t)blockIdx.y * rows + j] = make_double2(a, b);
  }
}

// Few active points (at most gather_max): one block per CP_ROWS basis rows
// walks the list of active indices, reads their kernel values (scattered,
// one sector each), writes them compacted and reduces the two weighted sums
// into partial slice 0 (same chunked FP32 -> FP64 promotion as the scan).
__global__ void __launch_bounds__(CP_T) compact_gather(
    KView K, int64_t rows, const int32_t* __restrict__ list, const int64_t* __restrict__ ns_dev,
    int64_t gather_max, const float* __restrict__ w1, const float* __restrict__ w2, void* kc_data,
    int32_t kc_format, int64_t kc_ld, int64_t kc_plane, double2* __restrict__ part,
    const unsigned long long* __restrict__ kc_cond) {
  __shared__ double sh[32];
  const int64_t ns = *ns_dev;
  if (ns > gather_max) return;
  if (kc_cond && *kc_cond == 0) kc_data = nullptr;
  const int64_t j0 = (int64_t)blockIdx.x * CP_ROWS;
  double s1[CP_ROWS], s2[CP_ROWS];
  float f1[CP_ROWS], f2[CP_ROWS];
#pragma unroll
  for (int r = 0; r < CP_ROWS; ++r) { s1[r] = 0.0; s2[r] = 0.0; f1[r] = 0.f; f2[r] = 0.f; }
  int since = 0;
  for (int64_t q = threadIdx.x; q < ns; q += CP_T) {
    const int64_t i = list[q];
    const float a = w1 ? w1[i] : 0.f, b = w2 ? w2[i] : 0.f;
#pragma unroll
    for (int r = 0; r < CP_ROWS; ++r) {
      const int64_t j = j0 + r;
      if (j >= rows) break;
      float v;
      __nv_bfloat16 h = __float2bfloat16_rn(0.f), l = h;
      if (K.format == SPSVM_FP32) {
        v = static_cast<const float*>(K.data)[j * K.ld + i];
      } else {
        const __nv_bfloat16* src = static_cast<const __nv_bfloat16*>(K.data);
        h = src[j * K.ld + i];
        l = src[K.plane + j * K.ld + i];
        v = __bfloat162float(h) + __bfloat162float(l);
      }
      if (kc_data) kc_put(kc_data, kc_format, kc_ld, kc_plane, K.format, j, q, v, h, l);
      f1[r] = fmaf(a, v, f1[r]);
      f2[r] = fmaf(b, v, f2[r]);
    }
    if (++since == 32) {
#pragma unroll
      for (int r = 0; r < CP_ROWS; ++r) {
        s1[r] += (double)f1[r]; s2[r] += (double)f2[r]; f1[r] = 0.f; f2[r] = 0.f;
      }
      since = 0;
    }
  }
#pragma unroll
  for (int r = 0; r < CP_ROWS; ++r) { s1[r] += (double)f1[r]; s2[r] += (double)f2[r]; }
  for (int r = 0; r < CP_ROWS; ++r) {
    const double a = block_sum(s1[r], sh);
    __syncthreads();
    const double b = block_sum(s2[r], sh);
    __syncthreads();
    const int64_t j = j0 + r;
    if (threadIdx.x == 0 && j < rows) part[j] = make_double2(a, b);
  }
}

// Sums the partial slices of the path that ran (one slice for the gather).
__global__ void compact_finish(const double2* __restrict__ part, int64_t ysplit, int64_t rows,
                               double* w1out, double* w2out, const int64_t* __restrict__ ns_dev,
                               int64_t gather_max) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= rows) return;
  if (*ns_dev <= gather_max) ysplit = 1;
  double a = 0.0, b = 0.0;
  for (int64_t s = 0; s < ysplit; ++s) {
    const double2 p = part[s * rows + j];
    a += p.x;
    b += p.y;
  }
  if (w1out) w1out[j] = a;
  if (w2out) w2out[j] = b;
}

// Zero columns [ns, kc_n) of every row of the compact matrix.
__global__ void zero_tail(void* kc_data, int32_t format, int64_t rows, int64_t kc_ld,
                          int64_t kc_plane, int64_t kc_n, const int64_t* __restrict__ ns_dev,
                          const unsigned long long* __restrict__ kc_cond) {
  if (kc_cond && *kc_cond == 0) return;
  const int64_t ns = *ns_dev;
  const int64_t end = min(kc_n, round_up(ns, (int64_t)128));
  const int64_t width = end - ns;
  if (width <= 0) return;
  const int64_t total = rows * width;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / width, c = ns + e % width;
    if (format == SPSVM_FP32) {
      static_cast<float*>(kc_data)[j * kc_ld + c] = 0.f;
    } else {
      __nv_bfloat16* p = static_cast<__nv_bfloat16*>(kc_data);
      p[j * kc_ld + c] = __float2bfloat16_rn(0.f);
      p[kc_plane + j * kc_ld + c] = __float2bfloat16_rn(0.f);
    }
  }
}

// Wt[j][r] = K[j][list[r]] for the k = *k_dev listed points (nothing when
// k > kmax); sign[r] = +1 when list[r] is active, else -1.  Blocks stride
// over the basis rows, threads over the points.
__global__ void diff_gather(KView K, int64_t rows, const int32_t* __restrict__ list,
                            const int32_t* __restrict__ k_dev, int32_t kmax,
                            const uint8_t* __restrict__ active, float* __restrict__ Wt,
                            int64_t ldw, float* __restrict__ sign) {
  const int32_t k = *k_dev;
  if (k > kmax) return;
  if (blockIdx.x == 0)
    for (int r = threadIdx.x; r < k; r += blockDim.x) sign[r] = active[list[r]] ? 1.0f : -1.0f;
  for (int64_t j = blockIdx.x; j < rows; j += gridDim.x)
    for (int r = threadIdx.x; r < k; r += blockDim.x) Wt[j * ldw + r] = K.at(j, list[r]);
}

// *k_dev = (int32) *total
__global__ void store_count(const int64_t* __restrict__ total, int32_t* __restrict__ k_dev) {
  *k_dev = (int32_t)*total;
}

}  // namespace
}  // namespace spsvm

using namespace spsvm;

extern "C" size_t spsvm_reduce_scratch_bytes(int64_t n) {
  if (n < 0) return 0;
  return (size_t)(ceil_div(n, GV_PTS) * 3 * sizeof(double) + 64);
}

extern "C" int spsvm_outputs(const spsvm_kmat* K, const double* beta, const float* y, float* o,
                             uint8_t* active, double* stats, void* scratch, size_t scratch_bytes,
                             void* stream) {
  SPSVM_TRY(check_kmat(K, "outputs"));
  if (!y || !o) return set_error(SPSVM_ERR_ARG, "outputs: NULL y/o");
  if (K->n == 0) return SPSVM_OK;
  if (stats && (!scratch || scratch_bytes < spsvm_reduce_scratch_bytes(K->n)))
    return set_error(SPSVM_ERR_OOM, "outputs: scratch too small");
  cudaStream_t s = as_stream(stream);
  ProfScope prof(PROF_OUTPUTS, s, beta ? 4.0 * (double)K->rows * K->n : 9.0 * K->n);
  const int64_t blocks = ceil_div(K->n, GV_PTS);
  double* part = stats ? static_cast<double*>(scratch) : nullptr;
  if (K->format == SPSVM_FP32)
    outputs_kernel<SPSVM_FP32><<<(unsigned)blocks, GV_T, 0, s>>>(view(K), K->rows, K->n, beta, y,
                                                                  o, active, part, 0);
  else
    outputs_kernel<SPSVM_BF16SPLIT><<<(unsigned)blocks, GV_T, 0, s>>>(view(K), K->rows, K->n, beta,
                                                                    y, o, active, part, 0);
  SPSVM_LAUNCH_CHECK();
  if (stats) {
    sum_triples<<<1, 256, 0, s>>>(part, blocks, stats);
    SPSVM_LAUNCH_CHECK();
  }
  return SPSVM_OK;
}

extern "C" int spsvm_gemv(const spsvm_kmat* K, const double* v, float* u, int32_t accumulate,
                          void* stream) {
  SPSVM_TRY(check_kmat(K, "gemv"));
  if (!v || !u) return set_error(SPSVM_ERR_ARG, "gemv: NULL pointer");
  if (K->n == 0) return SPSVM_OK;
  const int64_t blocks = ceil_div(K->n, GV_PTS);
  ProfScope prof(PROF_GEMV, as_stream(stream), 4.0 * (double)K->rows * K->n);
  if (K->format == SPSVM_FP32)
    gemv_kernel<SPSVM_FP32><<<(unsigned)blocks, GV_T, 0, as_stream(stream)>>>(
        view(K), K->rows, K->n, v, u, accumulate);
  else
    gemv_kernel<SPSVM_BF16SPLIT><<<(unsigned)blocks, GV_T, 0, as_stream(stream)>>>(
        view(K), K->rows, K->n, v, u, accumulate);
  SPSVM_LAUNCH_CHECK();
  return SPSVM_OK;
}

namespace {
int64_t compact_ysplit(int64_t n, int64_t rows) {
  const int64_t rowblocks = ceil_div(rows, CP_ROWS);
  const int64_t nchunks = ceil_div(n, CP_T);
  int64_t want = ceil_div(4 * (int64_t)sm_count(), rowblocks);
  if (want < 1) want = 1;
  if (want > nchunks) want = nchunks;
  return want;
}
}  // namespace

extern "C" size_t spsvm_compact_scratch_bytes(int64_t n, int64_t rows) {
  if (n < 0 || rows < 0) return 0;
  const int64_t scan_blocks_n = ceil_div(n, SC_PTS);
  // partials for the largest split the launcher may pick (bounded by chunks)
  const int64_t ysplit = ceil_div(n, CP_T) < 1024 ? ceil_div(n, CP_T) : 1024;
  return (size_t)(round_up(scan_blocks_n * 4, 256) +
                  round_up((ysplit > 0 ? ysplit : 1) * (rows > 0 ? rows : 1) * 16, 256) +
                  round_up((n > 0 ? n : 1) * 4, 256));   // list of active indices
}

extern "C" int spsvm_compact_active(const spsvm_kmat* K, const uint8_t* active, const float* w1,
                                    const float* w2, double* w1out, double* w2out,
                                    spsvm_kmat* Kc, int64_t* n_active, int32_t* pos,
                                    void* scratch, size_t scratch_bytes, void* stream) {
  return compact_active_impl(K, active, w1, w2, w1out, w2out, Kc, nullptr, n_active, pos, scratch,
                             scratch_bytes, stream);
}

// With kc_cond, K_SJ is written only when *kc_cond (read on the device) is
// nonzero: the fit passes the count of points whose active flag changed, so
// an unchanged active set keeps the copy in hand without a host round trip.
int spsvm::compact_active_impl(const spsvm_kmat* K, const uint8_t* active, const float* w1,
                               const float* w2, double* w1out, double* w2out, spsvm_kmat* Kc,
                               const unsigned long long* kc_cond, int64_t* n_active,
                               int32_t* pos, void* scratch, size_t scratch_bytes, void* stream) {
  SPSVM_TRY(check_kmat(K, "compact"));
  if (!active || !n_active || !pos) return set_error(SPSVM_ERR_ARG, "compact: NULL pointer");
  if (Kc) {
    SPSVM_TRY(check_kmat(Kc, "compact(out)"));
    // the compact copy keeps K's format, or splits FP32 values into hi / lo planes
    const bool fmt_ok = Kc->format == K->format || (K->format == SPSVM_FP32 && Kc->format == SPSVM_BF16SPLIT);
    if (!fmt_ok || Kc->rows < K->rows || Kc->n < round_up(K->n, 128))
      return set_error(SPSVM_ERR_ARG, "compact: output matrix too small or wrong format");
  }
  if ((w1out && !w1) || (w2out && !w2)) return set_error(SPSVM_ERR_ARG, "compact: missing weights");
  if (!scratch || scratch_bytes < spsvm_compact_scratch_bytes(K->n, K->rows))
    return set_error(SPSVM_ERR_OOM, "compact: scratch too small");
  cudaStream_t s = as_stream(stream);
  ProfScope prof(PROF_COMPACT, s, 4.0 * (double)K->rows * K->n);
  const int64_t n = K->n;
  const int64_t sb = ceil_div(n, SC_PTS);
  int32_t* counts = static_cast<int32_t*>(scratch);
  double2* part = reinterpret_cast<double2*>(static_cast<char*>(scratch) + round_up(sb * 4, 256));
  const int64_t ysplit_max = ceil_div(n, CP_T) < 1024 ? ceil_div(n, CP_T) : 1024;
  int32_t* list = reinterpret_cast<int32_t*>(
      static_cast<char*>(scratch) + round_up(sb * 4, 256) +
      round_up((ysplit_max > 0 ? ysplit_max : 1) * (K->rows > 0 ? K->rows : 1) * 16, 256));
  // below this many active points the scattered gather beats the full scan
  const int64_t gather_max = n / 64;
  if (n == 0) {
    SPSVM_CUDA_TRY(cudaMemsetAsync(n_active, 0, sizeof(int64_t), s));
  } else {
    scan_count<<<(unsigned)sb, SC_T, 0, s>>>(active, nullptr, n, counts);
    SPSVM_LAUNCH_CHECK();
    scan_blocks<<<1, 1024, 0, s>>>(counts, sb, n_active);
    SPSVM_LAUNCH_CHECK();
    scan_write<<<(unsigned)sb, SC_T, 0, s>>>(active, nullptr, n, counts, pos, list);
    SPSVM_LAUNCH_CHECK();
  }
  if (K->rows > 0 && n > 0) {
    int64_t ysplit = compact_ysplit(n, K->rows);
    if (ysplit > 1024) ysplit = 1024;
    const int64_t nchunks = ceil_div(n, CP_T);
    const int64_t per = ceil_div(nchunks, ysplit);
    ysplit = ceil_div(nchunks, per);
    dim3 grid((unsigned)ceil_div(K->rows, CP_ROWS), (unsigned)ysplit);
    compact_kernel<<<grid, CP_T, 0, s>>>(view(K), K->rows, n, active, pos, w1, w2,
                                         Kc ? Kc->data : nullptr, Kc ? Kc->format : 0,
                                         Kc ? Kc->ld : 0, Kc ? Kc->plane : 0, per, part, n_active,
                                         gather_max, kc_cond);
    SPSVM_LAUNCH_CHECK();
    compact_gather<<<(unsigned)ceil_div(K->rows, CP_ROWS), CP_T, 0, s>>>(
        view(K), K->rows, list, n_active, gather_max, w1, w2, Kc ? Kc->data : nullptr,
        Kc ? Kc->format : 0, Kc ? Kc->ld : 0, Kc ? Kc->plane : 0, part, kc_cond);
    SPSVM_LAUNCH_CHECK();
    if (w1out || w2out) {
      compact_finish<<<(unsigned)ceil_div(K->rows, 256), 256, 0, s>>>(part, ysplit, K->rows,
                                                                       w1out, w2out, n_active,
                                                                       gather_max);
      SPSVM_LAUNCH_CHECK();
    }
  } else if (K->rows > 0) {
    if (w1out) SPSVM_CUDA_TRY(cudaMemsetAsync(w1out, 0, K->rows * sizeof(double), s));
    if (w2out) SPSVM_CUDA_TRY(cudaMemsetAsync(w2out, 0, K->rows * sizeof(double), s));
  }
  if (Kc && K->rows > 0) {
    const int64_t kc_n = round_up(n, 128) <= Kc->n ? round_up(n, 128) : Kc->n;
    zero_tail<<<4 * sm_count(), 256, 0, s>>>(Kc->data, Kc->format, K->rows, Kc->ld, Kc->plane,
                                             kc_n, n_active, kc_cond);
    SPSVM_LAUNCH_CHECK();
  }
  return SPSVM_OK;
}

extern "C" int spsvm_active_diff(const spsvm_kmat* K, const uint8_t* active, const uint8_t* ref,
                                 int32_t kmax, float* Wt, int64_t ldw, float* sign, int32_t* k_dev,
                                 void* scratch, size_t scratch_bytes, void* stream) {
  SPSVM_TRY(check_kmat(K, "active_diff"));
  if (!active || !ref || !k_dev || kmax < 0 || (kmax > 0 && (!Wt || !sign || ldw < kmax)))
    return set_error(SPSVM_ERR_ARG, "active_diff: bad arguments");
  if (!scratch || scratch_bytes < spsvm_compact_scratch_bytes(K->n, 0))
    return set_error(SPSVM_ERR_OOM, "active_diff: scratch too small");
  cudaStream_t s = as_stream(stream);
  const int64_t n = K->n;
  if (n == 0) {
    SPSVM_CUDA_TRY(cudaMemsetAsync(k_dev, 0, sizeof(int32_t), s));
    return SPSVM_OK;
  }
  const int64_t sb = ceil_div(n, SC_PTS);
  int32_t* counts = static_cast<int32_t*>(scratch);
  // the compaction's scratch: counts, partial sums (one slot for no rows), list
  int64_t* total = reinterpret_cast<int64_t*>(static_cast<char*>(scratch) + round_up(sb * 4, 256));
  const int64_t ysplit_max = ceil_div(n, CP_T) < 1024 ? ceil_div(n, CP_T) : 1024;
  int32_t* list = reinterpret_cast<int32_t*>(
      static_cast<char*>(scratch) + round_up(sb * 4, 256) + round_up(ysplit_max * 16, 256));
  scan_count<<<(unsigned)sb, SC_T, 0, s>>>(active, ref, n, counts);
  SPSVM_LAUNCH_CHECK();
  scan_blocks<<<1, 1024, 0, s>>>(counts, sb, total);
  SPSVM_LAUNCH_CHECK();
  scan_write<<<(unsigned)sb, SC_T, 0, s>>>(active, ref, n, counts, nullptr, list);
  SPSVM_LAUNCH_CHECK();
  store_count<<<1, 1, 0, s>>>(total, k_dev);
  SPSVM_LAUNCH_CHECK();
  if (kmax > 0 && K->rows > 0) {
    diff_gather<<<(unsigned)min64(K->rows, 4 * (int64_t)sm_count()), 128, 0, s>>>(
        view(K), K->rows, list, k_dev, kmax, active, Wt, ldw, sign);
    SPSVM_LAUNCH_CHECK();
  }
  return SPSVM_OK;
}
