// FP64 Cholesky trailing update on the tensor cores (an Ozaki-type split):
//   A22 -= L21 L21^T,  L21 = rows >= k0 + 64 of the 64-column panel [k0, k0+64).
// Each panel row r is scaled by 2^-e_r (e_r from the row's largest |value|),
// so its 64 values v lie in (-1, 1), and is cut into OZ_SLICES integer slices
// of 7 bits: v = sum_s a_s 2^-7s + (residual < 2^-56), |a_s| <= 127, each a_s
// exact in BF16.  For a pair of rows, sum_k v_rk v_ck = sum_{s,t} 2^-7(s+t)
// P_st with P_st = sum_k a_s a_t an exact integer; pairs are grouped by level
// u = s + t (u <= OZ_SLICES + 1) into one FP32 TMEM accumulator per level,
// each holding at most 8 x 64 x 127^2 < 2^24 (exact).  The epilogue combines
// the levels in FP64 with exact power-of-two scales and subtracts
// 2^(e_r + e_c) times the result from A22: the update matches an FP64 dot
// product of the 64 terms to within a few units of FP64 rounding.
#include <cudaTypedefs.h>

#include "internal.h"
#include "tc_ptx.h"

namespace spsvm {

namespace {

using namespace tc;

constexpr int OZ_PB = 64;        // panel width
constexpr int OZ_SLICES = 8;     // 7-bit slices: 56 bits
constexpr int OZ_LEVELS = OZ_SLICES;   // u = 2 .. OZ_SLICES + 1
constexpr int OZ_TM = 128;       // rows per tile (MMA M)
constexpr int OZ_TN = 64;        // columns per tile (MMA N)
constexpr int OZ_A_SLICE = OZ_TM * 128;   // 16 KB
constexpr int OZ_B_SLICE = OZ_TN * 128;   // 8 KB
constexpr int OZ_B_OFF = OZ_SLICES * OZ_A_SLICE;
constexpr int OZ_BAR_OFF = OZ_B_OFF + OZ_SLICES * OZ_B_SLICE;
constexpr int OZ_EXP_OFF = OZ_BAR_OFF + 64;
constexpr int OZ_SMEM = OZ_EXP_OFF + OZ_TN * 4 + 1024;


__device__ __forceinline__ uint8_t* align1024(uint8_t* p) {
  const uint32_t a = smem_u32(p);
  return p + ((1024u - (a & 1023u)) & 1023u);
}

// 2^k for integer k (exact power of two).
__device__ __forceinline__ double pow2(int k) {
  if (k >= -1022 && k <= 1023) return __longlong_as_double((long long)(k + 1023) << 52);
  return ldexp(1.0, k);
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// One warp per panel row r >= r0: exponent e_r and the OZ_SLICES slices of
// the row's 64 values (2 per lane), stored as BF16 planes [s][r][64].
__global__ void oz_slice(const double* __restrict__ H, int64_t ldh, int64_t m, int64_t k0,
                         int64_t r0, uint16_t* __restrict__ sl, int32_t* __restrict__ ex,
                         const int32_t* __restrict__ info) {
  if (*info != 0) return;
  const int lane = threadIdx.x & 31;
  const int64_t r = r0 + (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= m) return;
  const double v0 = H[r * ldh + k0 + 2 * lane], v1 = H[r * ldh + k0 + 2 * lane + 1];
  double mx = fmax(fabs(v0), fabs(v1));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  int e = 0;
  if (mx > 0.0) frexp(mx, &e);   // mx = f 2^e, f in [0.5, 1)
  double a = ldexp(v0, -e), b = ldexp(v1, -e);   // exact, |a|, |b| < 1
  const int64_t plane = m * OZ_PB;
#pragma unroll
  for (int s = 0; s < OZ_SLICES; ++s) {
    a *= 128.0;
    b *= 128.0;
    const double ta = trunc(a), tb = trunc(b);
    a -= ta;   // exact
    b -= tb;
    const __nv_bfloat162 pr = __floats2bfloat162_rn((float)ta, (float)tb);   // exact integers
    *reinterpret_cast<__nv_bfloat162*>(sl + s * plane + r * OZ_PB + 2 * lane) = pr;
  }
  if (lane == 0) ex[r] = e;
}

// Lower tile (ti, tj) of the trailing update restricted to columns
// [cbase, cend): rows cbase + 128 ti .., columns cbase + 64 tj ...  (rows
// below the diagonal only; the slices cover every row >= cbase).
__global__ void __launch_bounds__(128, 1) oz_trailing(const __grid_constant__ CUtensorMap map_a,
                                                      const __grid_constant__ CUtensorMap map_b,
                                                      double* __restrict__ H, int64_t ldh,
                                                      int64_t m, int64_t cbase, int64_t cend,
                                                      const int32_t* __restrict__ ex,
                                                      const int32_t* __restrict__ info,
                                                      WaitCtx wc) {
  extern __shared__ uint8_t smem_raw[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t ti = blockIdx.y, tj = blockIdx.x;
  const int64_t r0 = cbase + ti * OZ_TM, c0 = cbase + tj * OZ_TN;
  // only tiles touching the lower triangle
  if (c0 > r0 + OZ_TM - 1) return;
  if (__syncthreads_or(tid == 0 && (*(volatile int*)wc.st != 0 || *info != 0))) return;
  uint8_t* smem = align1024(smem_raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + OZ_BAR_OFF);
  uint64_t* done = full + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(full + 2);
  int32_t* ec = reinterpret_cast<int32_t*>(smem + OZ_EXP_OFF);
  if (tid == 0) {
    mbar_init(full, 1);
    mbar_init(done, 1);
    fence_barrier_init();
  }
  if (warp == 0) tmem_alloc(tmem_slot, 512);
  if (tid < OZ_TN) ec[tid] = (c0 + tid < cend) ? ex[c0 + tid] : 0;
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  bool ok = true;
  if (tid == 0) {
    mbar_expect_tx(full, OZ_SLICES * (OZ_A_SLICE + OZ_B_SLICE));
    for (int s = 0; s < OZ_SLICES; ++s) {
      tma_load_3d(smem + s * OZ_A_SLICE, &map_a, 0, (int)r0, s, full);
      tma_load_3d(smem + OZ_B_OFF + s * OZ_B_SLICE, &map_b, 0, (int)c0, s, full);
    }
    ok = mbar_wait(full, 0, wc.st, 101, wc.lim);
    if (ok) {
      fence_after_sync();
      constexpr uint32_t IDESC = idesc_bf16_f32(OZ_TM, OZ_TN);
      for (int lv = 0; lv < OZ_LEVELS; ++lv) {        // level u = lv + 2
        const uint32_t d = tmem + lv * OZ_TN;
        bool first = true;
        for (int s = 0; s < OZ_SLICES; ++s) {         // slice index s + 1
          const int t = lv - s;                          // slice index t + 1, (s+1)+(t+1) = lv+2
          if (t < 0 || t >= OZ_SLICES) continue;
          const uint32_t a = smem_u32(smem + s * OZ_A_SLICE);
          const uint32_t b = smem_u32(smem + OZ_B_OFF + t * OZ_B_SLICE);
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            mma_bf16(d, desc_sw128(a + k * 32), desc_sw128(b + k * 32), IDESC, first ? 0u : 1u);
            first = false;
          }
        }
      }
    }
    mma_commit(done);
  }
  ok = __syncthreads_and(ok);
  const bool got = __syncthreads_and(mbar_wait(done, 0, wc.st, 102, wc.lim)) && ok;
  fence_after_sync();
  if (got) {
    const int64_t r = r0 + 32 * warp + lane;
    const bool rin = r < m;
    const int er = rin ? ex[r] : 0;
    const uint32_t tb = tmem + ((uint32_t)(32 * warp) << 16);
    for (int cc = 0; cc < OZ_TN / 32; ++cc) {
      // each level sum is an exact integer below 2^24; levels 0-3 and 4-7
      // combine exactly into two 64-bit integers (below 2^46 each)
      long long hi[32], lo[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        hi[j] = 0;
        lo[j] = 0;
      }
#pragma unroll
      for (int lv = 0; lv < OZ_LEVELS; ++lv) {
        float v[32];
        tmem_ld32(tb + lv * OZ_TN + cc * 32, v);
        const int sh = 7 * (3 - (lv & 3));
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const long long q = (long long)__float2int_rn(v[j]) * (1LL << sh);
          if (lv < 4) hi[j] += q;
          else lo[j] += q;
        }
      }
      if (rin) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int64_t c = c0 + cc * 32 + j;
          if (c <= r && c < cend) {
            // value = hi 2^-35 + lo 2^-63, times 2^(e_r + e_c)
            const int e = er + ec[cc * 32 + j];
            const double val = fma((double)lo[j], pow2(e - 63), (double)hi[j] * pow2(e - 35));
            double* p = H + r * ldh + c;
            *p -= val;
          }
        }
      }
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    fence_after_sync();
    tmem_dealloc(tmem, 512);
  }
}

// Rank-32 update of the block column [k0 + 32, k0 + 64) (rows >= k0 + 32)
// with the first half of the panel, plain FP64.
__global__ void __launch_bounds__(256) oz_panel_update(double* __restrict__ H, int64_t ldh,
                                                       int64_t m, int64_t k0,
                                                       const int32_t* __restrict__ info) {
  __shared__ double Lc[32][33];   // L[k0+32+c][k0+l]
  if (*info != 0) return;
  const int64_t cbase = k0 + 32;
  for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
    const int c = e / 32, l = e % 32;
    Lc[c][l] = (cbase + c < m) ? H[(cbase + c) * ldh + k0 + l] : 0.0;
  }
  __syncthreads();
  const int c = threadIdx.x & 31;
  const int64_t r = cbase + (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (r >= m || cbase + c > r || cbase + c >= m) return;
  const double* Lr = H + r * ldh + k0;
  double s0 = 0.0, s1 = 0.0;
#pragma unroll
  for (int l = 0; l < 32; l += 2) {
    s0 = fma(Lr[l], Lc[c][l], s0);
    s1 = fma(Lr[l + 1], Lc[c][l + 1], s1);
  }
  H[r * ldh + cbase + c] -= (s0 + s1);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  // thread-safe one-time lookup of the driver's tensor-map encoder
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    cudaGetLastError();
    return (PFN_cuTensorMapEncodeTiled_v12000) nullptr;
  }();
  return fn;
}

// 3-D map over the slice planes [OZ_SLICES][m][64] BF16, boxes of 64 x rows x 1.
int make_slice_map(CUtensorMap* map, const uint16_t* base, int64_t m, uint32_t rows) {
  auto fn = encode_fn();
  if (!fn) return set_error(SPSVM_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
  cuuint64_t dims[3] = {(cuuint64_t)OZ_PB, (cuuint64_t)m, (cuuint64_t)OZ_SLICES};
  cuuint64_t strides[2] = {(cuuint64_t)OZ_PB * 2, (cuuint64_t)(m * OZ_PB * 2)};
  cuuint32_t box[3] = {OZ_PB, rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<uint16_t*>(base), dims,
                  strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(SPSVM_ERR_CUDA, "slice map encode failed (%d)", (int)r);
  return SPSVM_OK;
}

}  // namespace

// Slice planes and exponents of one panel.
static size_t slice_buf_bytes(int64_t m) {
  return (size_t)round_up(OZ_SLICES * m * OZ_PB * 2, 256) + (size_t)round_up(m * 4, 256);
}

// Two slice buffers, so that the update of one panel can still read its
// slices while the next panel is being sliced.
size_t chol_tc_work_bytes(int64_t m) { return 2 * slice_buf_bytes(m); }

// Rank-32 update of the second half of the panel at k0 with its first half.
int chol_tc_panel_update(double* H, int64_t ldh, int64_t m, int64_t k0, const int32_t* info,
                         cudaStream_t s) {
  const int64_t rows = m - (k0 + 32);
  if (rows <= 0) return SPSVM_OK;
  oz_panel_update<<<(unsigned)ceil_div(rows, (int64_t)8), 256, 0, s>>>(H, ldh, m, k0, info);
  SPSVM_LAUNCH_CHECK();
  return SPSVM_OK;
}

// The panel-side kernels of this file take the largest shared-memory
// carveout, like the update, so that they can share SMs with it.
int chol_tc_carveout() {
  SPSVM_CUDA_TRY(cudaFuncSetAttribute(oz_panel_update, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      (int)cudaSharedmemCarveoutMaxShared));
  SPSVM_CUDA_TRY(cudaFuncSetAttribute(oz_slice, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      (int)cudaSharedmemCarveoutMaxShared));
  return SPSVM_OK;
}

// Slices of the rows >= k0 + 64 of the factored panel [k0, k0 + 64) into
// buffer `buf` (0 or 1) of the work area.
int chol_tc_slice(const double* H, int64_t ldh, int64_t m, int64_t k0, const int32_t* info,
                  void* work, int buf, cudaStream_t s) {
  const int64_t base = k0 + OZ_PB;
  const int64_t R = m - base;
  if (R <= 0) return SPSVM_OK;
  char* w = static_cast<char*>(work) + buf * slice_buf_bytes(m);
  uint16_t* sl = reinterpret_cast<uint16_t*>(w);
  int32_t* ex = reinterpret_cast<int32_t*>(w + round_up(OZ_SLICES * m * OZ_PB * 2, 256));
  oz_slice<<<(unsigned)ceil_div(R, (int64_t)8), 256, 0, s>>>(H, ldh, m, k0, base, sl, ex, info);
  SPSVM_LAUNCH_CHECK();
  return SPSVM_OK;
}

// Trailing update A[r][c] -= sum_l L[r][k0+l] L[c][k0+l] for the columns
// cbase <= c < cend (cbase >= k0 + 64) and rows r >= c, from the slices in
// buffer `buf`.
int chol_tc_update(double* H, int64_t ldh, int64_t m, int64_t cbase, int64_t cend,
                   const int32_t* info, void* work, int buf, cudaStream_t s) {
  const int64_t R = m - cbase;
  if (R <= 0 || cend <= cbase) return SPSVM_OK;
  char* w = static_cast<char*>(work) + buf * slice_buf_bytes(m);
  const uint16_t* sl = reinterpret_cast<const uint16_t*>(w);
  const int32_t* ex = reinterpret_cast<const int32_t*>(w + round_up(OZ_SLICES * m * OZ_PB * 2, 256));
  CUtensorMap ma, mb;
  SPSVM_TRY(make_slice_map(&ma, sl, m, OZ_TM));
  SPSVM_TRY(make_slice_map(&mb, sl, m, OZ_TN));
  SPSVM_CUDA_TRY(cudaFuncSetAttribute(oz_trailing, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      OZ_SMEM));
  dim3 grid((unsigned)ceil_div(cend - cbase, (int64_t)OZ_TN), (unsigned)ceil_div(R, (int64_t)OZ_TM));
  WaitCtx wc;
  SPSVM_TRY(wait_ctx(s, &wc));
  oz_trailing<<<grid, 128, OZ_SMEM, s>>>(ma, mb, H, ldh, m, cbase, cend, ex, info, wc);
  SPSVM_LAUNCH_CHECK();
  return SPSVM_OK;
}


}  // namespace spsvm
