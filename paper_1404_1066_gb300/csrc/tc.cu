// tcgen05 (sm_103a) tensor-core kernels of the SPSVM_BF16X3 form.  Every
// FP32 operand x is split as hi + lo (both BF16) and a product x*z is formed
// as hi*hi + hi*lo + lo*hi (three BF16 MMAs accumulating in FP32 in TMEM);
// the dropped lo*lo term is below 2^-16 of |x z|.
//
//   * kernel block / candidate scores (RBF kernel of Section 2 through the
//     distance expansion; the basis-vector score of Section 4): points X
//     (TMA, 128 rows per tile) times gathered basis / candidate rows, fused
//     epilogue exp(-gamma max(0, |x|^2 + |z|^2 - 2 x.z)) that either stores
//     the kernel values or reduces the score sums without storing them;
//   * masked Gram matrix K_SJ^T K_SJ (the Hessian term of Eq. 4 on the
//     active set): warp-specialised TMA producer / MMA issuer / epilogue over
//     128 x 128 upper-triangular tiles with two TMEM accumulators, FP32
//     partial sums per 8192 points promoted to FP64.
#include <cudaTypedefs.h>

#include "gram.h"
#include "internal.h"
#include "tc_ptx.h"

namespace spsvm {

namespace {

using namespace tc;

__device__ int g_tc_status = 0;

__device__ __forceinline__ uint8_t* align1024(uint8_t* p) {
  const uint32_t a = smem_u32(p);
  return p + ((1024u - (a & 1023u)) & 1023u);
}

// ---------------------------------------------------------------------------
// Kernel block / scores: D[c][i] = z_c . x_i over one tile of 128 basis (or
// candidate) rows c (the MMA M dimension, gathered by index into shared
// memory) and 256 points i (the N dimension, loaded by TMA).  TMEM lane c
// holds row c, so each thread writes or reduces a contiguous run of points.
// ---------------------------------------------------------------------------
constexpr int KB_THREADS = 128;
constexpr int KB_M = 128;                  // basis rows per tile
constexpr int KB_N = 256;                  // points per tile
constexpr int KB_A_BYTES = KB_M * 128;     // one plane: 128 rows x 64 BF16
constexpr int KB_B_BYTES = KB_N * 128;     // one plane: 256 rows x 64 BF16
constexpr int KB_STAGE = 2 * KB_A_BYTES + 2 * KB_B_BYTES;
constexpr int KB_BAR_OFF = 2 * KB_STAGE;   // 5 mbarriers + TMEM slot
constexpr int KB_ZROW_OFF = KB_BAR_OFF + 64;
constexpr int KB_XN_OFF = KB_ZROW_OFF + KB_M * 8;
constexpr int KB_RES_OFF = KB_XN_OFF + KB_N * 4;
constexpr int KB_ACT_OFF = KB_RES_OFF + KB_N * 4;
constexpr int KB_SMEM = KB_ACT_OFF + KB_N * 4 + 1024;   // + alignment slack

template <bool SCORE>
__global__ void __launch_bounds__(KB_THREADS, 1) kblock_tc_kernel(
    const __grid_constant__ CUtensorMap map_hi, const __grid_constant__ CUtensorMap map_lo,
    const uint16_t* __restrict__ Xhi, const uint16_t* __restrict__ Xlo, int64_t ldh, int64_t n,
    const float* __restrict__ norms, const int64_t* __restrict__ idx, int32_t m, float gamma,
    uint16_t* __restrict__ out, int64_t ld, int64_t plane, int64_t row0,
    const float* __restrict__ y, const float* __restrict__ o, double2* __restrict__ part,
    int32_t kappa) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = align1024(smem_raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + KB_BAR_OFF);
  uint64_t* empty = full + 2;
  uint64_t* done = full + 4;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(full + 5);
  int64_t* zrow = reinterpret_cast<int64_t*>(smem + KB_ZROW_OFF);
  float* xn_s = reinterpret_cast<float*>(smem + KB_XN_OFF);
  float* res_s = reinterpret_cast<float*>(smem + KB_RES_OFF);
  float* act_s = reinterpret_cast<float*>(smem + KB_ACT_OFF);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int c0 = blockIdx.x * KB_M;
  const int64_t i0 = (int64_t)blockIdx.y * KB_N;
  const int m_here = min(KB_M, m - c0);
  constexpr uint32_t IDESC = idesc_bf16_f32(KB_M, KB_N);
  // once any block has given up a wait, the remaining blocks exit at once
  if (__syncthreads_or(tid == 0 && *(volatile int*)&g_tc_status != 0)) return;

  if (tid == 0) {
    mbar_init(&full[0], 1);
    mbar_init(&full[1], 1);
    mbar_init(&empty[0], 1);
    mbar_init(&empty[1], 1);
    mbar_init(done, 1);
    fence_barrier_init();
    prefetch_tmap(&map_hi);
    prefetch_tmap(&map_lo);
  }
  if (warp == 0) tmem_alloc(tmem_slot, KB_N);
  {
    const int c = tid;   // KB_THREADS == KB_M
    zrow[c] = (c < m_here) ? idx[c0 + c] : -1;
  }
  for (int j = tid; j < KB_N; j += KB_THREADS) {
    const int64_t i = i0 + j;
    const bool in = i < n;
    xn_s[j] = in ? norms[i] : 0.f;
    if (SCORE) {
      float r = 0.f, a = 0.f;
      if (in) {
        const float oi = o[i], yi = y[i];
        if (yi * oi < 1.0f) {
          r = oi - yi;
          a = 1.f;
        }
      }
      res_s[j] = r;
      act_s[j] = a;
    }
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  const int nK = (int)(ldh / 64);
  bool ok = true;
  int last_kc[2] = {-1, -1};   // thread 0: last chunk loaded into each stage
  int used_kc[2] = {-1, -1};   // thread 0: last chunk whose load was waited on
  for (int kc = 0; kc < nK; ++kc) {
    const int s = kc & 1;
    uint8_t* st = smem + s * KB_STAGE;
    if (kc >= 2 && ok) ok = mbar_wait(&empty[s], ((kc - 2) >> 1) & 1, &g_tc_status, 1);
    if (!__syncthreads_and(ok)) {
      ok = false;
      break;
    }
    uint8_t* ah = st;
    uint8_t* al = st + KB_A_BYTES;
    uint8_t* bh = st + 2 * KB_A_BYTES;
    uint8_t* bl = bh + KB_B_BYTES;
    if (tid == 0) {
      mbar_expect_tx(&full[s], 2 * KB_B_BYTES);
      tma_load_2d(bh, &map_hi, kc * 64, (int)i0, &full[s]);
      tma_load_2d(bl, &map_lo, kc * 64, (int)i0, &full[s]);
      last_kc[s] = kc;
    }
    // gather the basis rows (128-byte swizzle, as TMA would lay them out)
    for (int e = tid; e < KB_M * 8; e += KB_THREADS) {
      const int r = e >> 3, ch = e & 7;
      uint4 vh = make_uint4(0, 0, 0, 0), vl = vh;
      const int64_t zr = zrow[r];
      if (zr >= 0) {
        const int64_t off = zr * ldh + (int64_t)kc * 64 + ch * 8;
        vh = *reinterpret_cast<const uint4*>(Xhi + off);
        vl = *reinterpret_cast<const uint4*>(Xlo + off);
      }
      const int so = r * 128 + ((ch ^ (r & 7)) << 4);
      *reinterpret_cast<uint4*>(ah + so) = vh;
      *reinterpret_cast<uint4*>(al + so) = vl;
    }
    fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      if (mbar_wait(&full[s], (kc >> 1) & 1, &g_tc_status, 2)) {
        used_kc[s] = kc;
        fence_after_sync();
        const uint32_t a_hi = smem_u32(ah), a_lo = smem_u32(al);
        const uint32_t b_hi = smem_u32(bh), b_lo = smem_u32(bl);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const uint32_t koff = k * 32;
          mma_bf16(tmem, desc_sw128(a_hi + koff), desc_sw128(b_hi + koff), IDESC,
                   (kc | k) != 0);
          mma_bf16(tmem, desc_sw128(a_hi + koff), desc_sw128(b_lo + koff), IDESC, 1);
          mma_bf16(tmem, desc_sw128(a_lo + koff), desc_sw128(b_hi + koff), IDESC, 1);
        }
        mma_commit(&empty[s]);
      } else {
        ok = false;
      }
    }
  }
  if (tid == 0) {
    mma_commit(done);
    // no TMA copy may still be in flight when the block exits
    for (int s = 0; s < 2; ++s)
      if (last_kc[s] >= 0 && last_kc[s] != used_kc[s])
        mbar_wait(&full[s], (uint32_t)((last_kc[s] >> 1) & 1), &g_tc_status, 4);
  }
  ok = __syncthreads_and(ok);
  bool got = mbar_wait(done, 0, &g_tc_status, 3);
  got = __syncthreads_and(got) && ok;
  fence_after_sync();

  if (got) {
    const int c = 32 * warp + lane;               // basis row of this thread
    const bool crow = c < m_here;
    const float zn = crow ? norms[zrow[c]] : 0.f;
    // K = 2^(g2 (2 dot - |x|^2 - |z|^2)), g2 = gamma log2(e)
    const float g2 = gamma * 1.4426950408889634f;
    const int64_t npts = min64(KB_N, n - i0);
    const uint32_t tbase = tmem + ((uint32_t)(32 * warp) << 16);
    float gs = 0.f, hs = 0.f;
    for (int cc = 0; cc < KB_N / 32; ++cc) {
      if (cc * 32 >= npts) break;                 // uniform across the block
      float v[32];
      tmem_ld32(tbase + cc * 32, v);
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const float d2 = fmaxf(xn_s[cc * 32 + j] + zn - 2.0f * v[j], 0.0f);
        v[j] = exp2f(-g2 * d2);
      }
      if (!SCORE) {
        if (crow) {
          uint16_t* dh = out + (row0 + c0 + c) * ld + i0 + cc * 32;
          uint16_t* dl = dh + plane;
          if (cc * 32 + 32 <= npts) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              uint32_t wh[4], wl[4];
#pragma unroll
              for (int t = 0; t < 4; ++t) {
                __nv_bfloat16 h0, l0, h1, l1;
                split_bf16(v[8 * q + 2 * t], h0, l0);
                split_bf16(v[8 * q + 2 * t + 1], h1, l1);
                wh[t] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
                wl[t] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
              }
              *reinterpret_cast<uint4*>(dh + 8 * q) = make_uint4(wh[0], wh[1], wh[2], wh[3]);
              *reinterpret_cast<uint4*>(dl + 8 * q) = make_uint4(wl[0], wl[1], wl[2], wl[3]);
            }
          } else {
            for (int j = 0; j < 32; ++j) {
              if (cc * 32 + j >= npts) break;
              __nv_bfloat16 h, l;
              split_bf16(v[j], h, l);
              dh[j] = __bfloat16_as_ushort(h);
              dl[j] = __bfloat16_as_ushort(l);
            }
          }
        }
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const float kv = v[j];
          gs = fmaf(res_s[cc * 32 + j], kv, gs);
          hs = fmaf(act_s[cc * 32 + j] * kv, kv, hs);
        }
      }
    }
    if (SCORE && crow) part[(int64_t)blockIdx.y * kappa + c0 + c] = make_double2(gs, hs);
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    fence_after_sync();
    tmem_dealloc(tmem, KB_N);
  }
}

// ---------------------------------------------------------------------------
// Masked Gram matrix: P[a][b] (+)= sum_p Kc[a][p] Kc[b][p] over 128 x 128
// upper-triangular tiles.  Warp 0: TMEM owner and TMA producer; warp 1: MMA
// issuer; warps 2-5: epilogue.
// ---------------------------------------------------------------------------
constexpr int GR_THREADS = 192;
constexpr int GR_STAGES = 3;
constexpr int GR_TILE = 128;
constexpr int GR_PLANE_BYTES = GR_TILE * 128;
constexpr int GR_STAGE = 4 * GR_PLANE_BYTES;   // A hi, A lo, B hi, B lo
constexpr int GR_BAR_OFF = GR_STAGES * GR_STAGE;
constexpr int GR_SMEM = GR_BAR_OFF + 256 + 1024;
constexpr int64_t GR_CHUNKS_PER_SLICE = GRAM_SLICE / 64;

__global__ void __launch_bounds__(GR_THREADS, 1) gram_tc_kernel(
    const __grid_constant__ CUtensorMap map_hi, const __grid_constant__ CUtensorMap map_lo,
    int64_t m, const int64_t* __restrict__ ns_dev, int64_t slices_per_split,
    double* __restrict__ part, int64_t ldp) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = align1024(smem_raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + GR_BAR_OFF);
  uint64_t* empty = full + GR_STAGES;
  uint64_t* accf = empty + GR_STAGES;
  uint64_t* acce = accf + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acce + 2);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (__syncthreads_or(tid == 0 && *(volatile int*)&g_tc_status != 0)) return;
  // upper-triangular tile (ta <= tb)
  const int64_t T = ceil_div(m, (int64_t)GR_TILE);
  int64_t rem = blockIdx.x, ta = 0;
  while (rem >= T - ta) {
    rem -= T - ta;
    ++ta;
  }
  const int64_t tb = ta + rem;
  const int64_t a0 = ta * GR_TILE, b0 = tb * GR_TILE;
  const int64_t ns = *ns_dev;
  const int64_t chunks = ceil_div(ns, (int64_t)64);
  const int64_t c_begin = min64(chunks, (int64_t)blockIdx.y * slices_per_split * GR_CHUNKS_PER_SLICE);
  const int64_t c_end = min64(chunks, c_begin + slices_per_split * GR_CHUNKS_PER_SLICE);
  const int64_t nch = c_end - c_begin;
  const int64_t nslices = ceil_div(nch, GR_CHUNKS_PER_SLICE);
  constexpr uint32_t IDESC = idesc_bf16_f32(GR_TILE, GR_TILE);
  double* P = part + (int64_t)blockIdx.y * ldp * ldp;

  if (tid == 0) {
    for (int s = 0; s < GR_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&accf[a], 1);
      mbar_init(&acce[a], 128);
    }
    fence_barrier_init();
    prefetch_tmap(&map_hi);
    prefetch_tmap(&map_lo);
  }
  if (warp == 0) tmem_alloc(tmem_slot, 256);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer
    int64_t issued = 0;
    for (int64_t q = 0; q < nch; ++q) {
      const int s = (int)(q % GR_STAGES);
      const uint32_t ph = (uint32_t)((q / GR_STAGES) & 1);
      if (!mbar_wait(&empty[s], ph ^ 1u, &g_tc_status, 11)) break;
      uint8_t* st = smem + s * GR_STAGE;
      const int x = (int)((c_begin + q) * 64);
      mbar_expect_tx(&full[s], GR_STAGE);
      tma_load_2d(st, &map_hi, x, (int)a0, &full[s]);
      tma_load_2d(st + GR_PLANE_BYTES, &map_lo, x, (int)a0, &full[s]);
      tma_load_2d(st + 2 * GR_PLANE_BYTES, &map_hi, x, (int)b0, &full[s]);
      tma_load_2d(st + 3 * GR_PLANE_BYTES, &map_lo, x, (int)b0, &full[s]);
      issued = q + 1;
    }
    // wait for the copies of the last stages so none is in flight at exit
    for (int64_t q = (issued > GR_STAGES ? issued - GR_STAGES : 0); q < issued; ++q)
      mbar_wait(&full[q % GR_STAGES], (uint32_t)((q / GR_STAGES) & 1), &g_tc_status, 12);
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer
    bool ok = true;
    for (int64_t t = 0; t < nslices && ok; ++t) {
      const int acc = (int)(t & 1);
      const uint32_t use = (uint32_t)((t >> 1) & 1);
      if (!mbar_wait(&acce[acc], use ^ 1u, &g_tc_status, 13)) break;
      fence_after_sync();
      const uint32_t d = tmem + acc * GR_TILE;
      const int64_t q0 = t * GR_CHUNKS_PER_SLICE;
      const int64_t q1 = min64(nch, q0 + GR_CHUNKS_PER_SLICE);
      for (int64_t q = q0; q < q1; ++q) {
        const int s = (int)(q % GR_STAGES);
        const uint32_t ph = (uint32_t)((q / GR_STAGES) & 1);
        if (!mbar_wait(&full[s], ph, &g_tc_status, 14)) {
          ok = false;
          break;
        }
        fence_after_sync();
        const uint32_t base = smem_u32(smem + s * GR_STAGE);
        const uint32_t a_hi = base, a_lo = base + GR_PLANE_BYTES;
        const uint32_t b_hi = base + 2 * GR_PLANE_BYTES, b_lo = base + 3 * GR_PLANE_BYTES;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const uint32_t koff = k * 32;
          mma_bf16(d, desc_sw128(a_hi + koff), desc_sw128(b_hi + koff), IDESC,
                   (q != q0 || k != 0) ? 1u : 0u);
          mma_bf16(d, desc_sw128(a_hi + koff), desc_sw128(b_lo + koff), IDESC, 1u);
          mma_bf16(d, desc_sw128(a_lo + koff), desc_sw128(b_hi + koff), IDESC, 1u);
        }
        mma_commit(&empty[s]);
      }
      mma_commit(&accf[acc]);
    }
  } else if (warp >= 2) {
    // ---- epilogue: TMEM lanes 32 * (warp % 4) .. + 31
    const int quarter = warp & 3;
    const int64_t a = a0 + 32 * quarter + lane;
    if (nslices == 0) {
      if (a < m)
        for (int64_t b = b0; b < min64(m, b0 + GR_TILE); ++b) P[a * ldp + b] = 0.0;
    }
    for (int64_t t = 0; t < nslices; ++t) {
      const int acc = (int)(t & 1);
      const uint32_t use = (uint32_t)((t >> 1) & 1);
      if (!mbar_wait(&accf[acc], use, &g_tc_status, 15)) break;
      fence_after_sync();
      const uint32_t tbase = tmem + acc * GR_TILE + ((uint32_t)(32 * quarter) << 16);
      for (int cc = 0; cc < GR_TILE / 32; ++cc) {
        float v[32];
        tmem_ld32(tbase + cc * 32, v);
        if (a < m) {
          double* row = P + a * ldp + b0 + cc * 32;
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            if (b0 + cc * 32 + j < m) row[j] = (t == 0) ? (double)v[j] : row[j] + (double)v[j];
          }
        }
      }
      fence_before_sync();
      mbar_arrive(&acce[acc]);
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    fence_after_sync();
    tmem_dealloc(tmem, 256);
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

// 2-D BF16 map over rows x inner (row pitch `pitch_elems`), 64 x box_rows boxes,
// 128-byte swizzle, zero fill outside the tensor.
int make_map(CUtensorMap* map, const void* base, int64_t inner, int64_t rows, int64_t pitch_elems,
             uint32_t box_rows) {
  auto fn = encode_fn();
  if (!fn) return set_error(SPSVM_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
  if ((reinterpret_cast<uintptr_t>(base) & 15) || (pitch_elems * 2) % 16)
    return set_error(SPSVM_ERR_ARG, "tensor map: base or pitch not 16-byte aligned");
  cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)(rows > 0 ? rows : 1)};
  cuuint64_t strides[1] = {(cuuint64_t)(pitch_elems * 2)};
  cuuint32_t box[2] = {64, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides,
                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(SPSVM_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return SPSVM_OK;
}

template <bool SCORE>
int launch_kb(const spsvm_points* p, const int64_t* idx, int32_t m, float gamma, uint16_t* out,
              int64_t ld, int64_t plane, int64_t row0, const float* y, const float* o,
              double2* part, int32_t kappa, cudaStream_t s) {
  if (ceil_div(p->n, (int64_t)KB_N) > 65535)
    return set_error(SPSVM_ERR_ARG, "BF16X3 kernel block: n > 16,776,960 points");
  CUtensorMap mh, ml;
  SPSVM_TRY(make_map(&mh, p->hi, p->ldh, p->n, p->ldh, KB_N));
  SPSVM_TRY(make_map(&ml, p->lo, p->ldh, p->n, p->ldh, KB_N));
  auto kern = kblock_tc_kernel<SCORE>;
  static bool attr = false;
  if (!attr) {
    SPSVM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, KB_SMEM));
    attr = true;
  }
  dim3 grid((unsigned)ceil_div(m, KB_M), (unsigned)ceil_div(p->n, (int64_t)KB_N));
  kern<<<grid, KB_THREADS, KB_SMEM, s>>>(mh, ml, p->hi, p->lo, p->ldh, p->n, p->norms, idx, m,
                                         gamma, out, ld, plane, row0, y, o, part, kappa);
  SPSVM_LAUNCH_CHECK();
  return SPSVM_OK;
}

}  // namespace

bool tc_available() { return encode_fn() != nullptr; }

int launch_kernel_block_tc(const spsvm_points* p, const int64_t* idx, int32_t m, float gamma,
                           spsvm_kmat* out, int64_t row0, cudaStream_t s) {
  if (m == 0 || p->n == 0) return SPSVM_OK;
  if (out->format != SPSVM_BF16X3 || (out->ld % 8) != 0 || (out->plane % 8) != 0)
    return set_error(SPSVM_ERR_ARG,
                     "BF16X3 kernel block: needs BF16X3 storage with ld %% 8 == 0, plane %% 8 == 0");
  return launch_kb<false>(p, idx, m, gamma, static_cast<uint16_t*>(out->data), out->ld, out->plane,
                          row0, nullptr, nullptr, nullptr, 0, s);
}

int64_t score_tc_tiles(int64_t n) { return ceil_div(n, (int64_t)KB_N); }

int launch_score_tc(const spsvm_points* p, const float* y, const float* o, const int64_t* idx,
                    int32_t kappa, float gamma, double2* part, int64_t tiles, cudaStream_t s) {
  (void)tiles;
  return launch_kb<true>(p, idx, kappa, gamma, nullptr, 0, 0, 0, y, o, part, kappa, s);
}

int64_t gram_tc_splits(int64_t m, int64_t ns_max) {
  const int64_t T = ceil_div(m, (int64_t)GR_TILE);
  const int64_t tiles = T * (T + 1) / 2;
  const int64_t slices = ceil_div(ns_max > 0 ? ns_max : 1, GRAM_SLICE);
  int64_t want = ceil_div(2 * (int64_t)sm_count(), tiles > 0 ? tiles : 1);
  if (want < 1) want = 1;
  if (want > slices) want = slices;
  return want;
}

int launch_gram_tc(const spsvm_kmat* Kc, const int64_t* ns_dev, int64_t ns_max, int64_t m,
                   double* part, int64_t ldp, int64_t splits, cudaStream_t s) {
  const uint16_t* hi = static_cast<const uint16_t*>(Kc->data);
  const uint16_t* lo = hi + Kc->plane;
  CUtensorMap mh, ml;
  SPSVM_TRY(make_map(&mh, hi, Kc->ld, m, Kc->ld, GR_TILE));
  SPSVM_TRY(make_map(&ml, lo, Kc->ld, m, Kc->ld, GR_TILE));
  static bool attr = false;
  if (!attr) {
    SPSVM_CUDA_TRY(cudaFuncSetAttribute(gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        GR_SMEM));
    attr = true;
  }
  const int64_t T = ceil_div(m, (int64_t)GR_TILE);
  const int64_t tiles = T * (T + 1) / 2;
  const int64_t slices = ceil_div(ns_max > 0 ? ns_max : 1, GRAM_SLICE);
  const int64_t per = ceil_div(slices, splits);
  dim3 grid((unsigned)tiles, (unsigned)splits);
  gram_tc_kernel<<<grid, GR_THREADS, GR_SMEM, s>>>(mh, ml, m, ns_dev, per, part, ldp);
  SPSVM_LAUNCH_CHECK();
  return SPSVM_OK;
}

int tc_take_status() {
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_tc_status, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  if (v != 0) {
    const int zero = 0;
    cudaMemcpyToSymbol(g_tc_status, &zero, sizeof(int));
  }
  return v;
}

}  // namespace spsvm

extern "C" int spsvm_device_status(int32_t* code) {
  const int v = spsvm::tc_take_status();
  if (code) *code = v;
  if (v < 0) return spsvm::set_error(SPSVM_ERR_CUDA, "device status unreadable");
  if (v > 0) return spsvm::set_error(SPSVM_ERR_TIMEOUT, "a bounded device wait gave up (site %d)", v);
  return SPSVM_OK;
}
