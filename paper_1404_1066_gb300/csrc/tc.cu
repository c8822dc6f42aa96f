// tcgen05 (sm_103a) tensor-core kernels of the SPSVM_BF16SPLIT form.
//
//   * kernel block / candidate scores / decision values (RBF kernel of
//     Section 2 through the distance expansion; the basis-vector score of
//     Section 4; the classifier h(x) = w^T phi(x) on the basis): points X
//     (TMA, 128 rows per tile) times gathered basis / candidate rows, each
//     FP32 value split into three BF16 terms hi + mid + lo (exact) and
//     multiplied as six products, with a fused epilogue
//     exp(-gamma max(0, |x|^2 + |z|^2 - 2 x.z)) that stores the kernel
//     values (FP32), or reduces the score sums or the beta-weighted decision
//     sums without storing them;
//   * masked Gram matrix K_SJ^T K_SJ (the Hessian term of Eq. 4 on the
//     active set): the compact copy split as hi + lo (lo = bf16(x - hi)) and
//     all four plane products, warp-specialised TMA producer / MMA issuer /
//     epilogue over 128 x 128 upper-triangular tiles with two TMEM
//     accumulators, FP32 partial sums per 8192 points promoted to FP64.
#include <cudaTypedefs.h>

#include <mutex>

#include "gram.h"
#include "internal.h"
#include "tc_ptx.h"

namespace spsvm {

namespace {

using namespace tc;

__device__ __forceinline__ uint8_t* align1024(uint8_t* p) {
  const uint32_t a = smem_u32(p);
  return p + ((1024u - (a & 1023u)) & 1023u);
}

// ---------------------------------------------------------------------------
// Kernel block / scores, persistent and warp-specialised.  D[c][i] = z_c . x_i
// over tiles of 128 basis (or candidate) rows c (MMA M; the rows gathered
// beforehand into contiguous BF16 planes Z) by 128 points i (MMA N), both
// operands streamed by TMA through a 3-stage shared-memory ring (32-element
// K slices, 64-byte swizzle) holding the three planes of each (x = hi + mid
// + lo, exact for FP32) and multiplied as the six products hi hi, hi mid,
// mid hi, mid mid, hi lo, lo hi (the three dropped ones are below 2^-24 of
// |x z|), hi hi into one TMEM accumulator and the rest into a second (the
// FP32 accumulation's rounding grows with the MMAs a sum takes, and only the
// few large-term ones then count).  Warp 0 issues the TMA loads, warp 1 the
// MMAs into one of two tile buffers, warps 2-9 drain the other (TMEM lane c =
// row c; warps w and w + 4 share a lane quarter and split the 128 columns),
// so the epilogue of one tile overlaps the MMAs of the next.  Tiles are ordered point-tile major so the CTAs in flight share their
// X tiles through L2.
// ---------------------------------------------------------------------------
constexpr int PK_M = 128;
constexpr int PK_N = 128;
constexpr int PK_KC = 32;                                  // K elements per stage (64-byte rows)
constexpr int PK_WP = PK_N / 2;                            // points per epilogue warp
constexpr int PK_ACC_COLS = 2 * PK_N;                      // TMEM per tile: large + small terms
constexpr int PK_STAGES = 3;
constexpr int PK_PLANE_A = PK_M * PK_KC * 2;               // 8 KB: 128 rows x 32 BF16
constexpr int PK_PLANE_B = PK_N * PK_KC * 2;               // 8 KB
constexpr int PK_STAGE = 3 * PK_PLANE_A + 3 * PK_PLANE_B;  // 48 KB
constexpr int PK_EPI_WARPS = 8;
constexpr int PK_THREADS = 32 * (2 + PK_EPI_WARPS);
constexpr int PK_OUT_BOX = 32 * 128;                       // 32 rows x 32 FP32
constexpr int PK_OUT_OFF = PK_STAGES * PK_STAGE;           // per epilogue warp: two boxes
constexpr int PK_BAR_OFF = PK_OUT_OFF + PK_EPI_WARPS * 2 * PK_OUT_BOX;
constexpr int PK_RED_OFF = PK_BAR_OFF + 256;
constexpr int PK_STAGE_OFF = PK_RED_OFF + 4 * 32 * 8;      // per epilogue warp: 3 x 64 floats
constexpr int PK_SMEM = PK_STAGE_OFF + PK_EPI_WARPS * 3 * PK_WP * 4 + 1024;   // + alignment slack
static_assert(PK_SMEM <= 227 * 1024, "kernel block shared memory");
static_assert(2 * PK_ACC_COLS <= 512, "two tiles of two accumulators fit TMEM");

__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, int x, int y, const void* src) {
  asm volatile(
      "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
          reinterpret_cast<uint64_t>(map)),
      "r"(x), "r"(y), "r"(smem_u32(src))
      : "memory");
}
__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// Waits until the shared-memory sources of every committed bulk store have been read.
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// Tile order: groups of PK_GROUP consecutive point tiles, each group swept
// over all basis blocks with the point tile varying fastest.  The CTAs in
// flight then share a few X tiles through L2 while each basis row receives
// PK_GROUP x 256 contiguous bytes, so the kernel-matrix writes reach DRAM in
// long runs.
constexpr int64_t PK_GROUP = 32;
__device__ __forceinline__ void tile_coords(int64_t t, int64_t nCB, int64_t nPT, int& cb,
                                            int64_t& pt) {
  const int64_t per = nCB * PK_GROUP;
  const int64_t g = t / per, r = t % per;
  const int64_t g0 = g * PK_GROUP;
  const int64_t gw = min64(PK_GROUP, nPT - g0);   // the last group may be narrower
  cb = (int)(r / gw);
  pt = g0 + r % gw;
}

// Epilogue modes: store the FP32 kernel values, reduce the candidate-score
// sums without storing them, or reduce the decision values
// f(x_i) = sum_c beta_c k(z_c, x_i) (Z the basis rows, X the queries) over
// each warp's 32 basis rows, also without storing the kernel values.
enum KbMode { KB_STORE_F32 = 0, KB_SCORE = 2, KB_DECIDE = 3 };


template <int MODE>
__global__ void __launch_bounds__(PK_THREADS, 1) kblock_tc_kernel(
    const __grid_constant__ CUtensorMap map_zhi, const __grid_constant__ CUtensorMap map_zmid,
    const __grid_constant__ CUtensorMap map_zlo, const __grid_constant__ CUtensorMap map_xhi,
    const __grid_constant__ CUtensorMap map_xmid, const __grid_constant__ CUtensorMap map_xlo,
    const __grid_constant__ CUtensorMap map_out, int64_t ldh, int64_t n, int32_t m,
    const float* __restrict__ norms, const int64_t* __restrict__ idx, float gamma, int64_t row0,
    const float* __restrict__ y, const float* __restrict__ o, double2* __restrict__ part,
    int32_t kappa, const float* __restrict__ znorm, const double* __restrict__ beta,
    float* __restrict__ dpart, int64_t ldp, WaitCtx wc) {
  constexpr bool SCORE = MODE == KB_SCORE;
  constexpr bool STORE = MODE == KB_STORE_F32;
  constexpr bool DECIDE = MODE == KB_DECIDE;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = align1024(smem_raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + PK_BAR_OFF);
  uint64_t* empty = full + PK_STAGES;
  uint64_t* tfull = empty + PK_STAGES;
  uint64_t* tempty = tfull + 2;
  uint64_t* redf = tempty + 2;   // per lane quarter: half-tile sums written
  uint64_t* rede = redf + 4;     // per lane quarter: half-tile sums consumed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(rede + 4);
  float2* red = reinterpret_cast<float2*>(smem + PK_RED_OFF);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (__syncthreads_or(tid == 0 && *(volatile int*)wc.st != 0)) return;
  const int64_t nCB = ceil_div((int64_t)m, (int64_t)PK_M);
  const int64_t nPT = ceil_div(n, (int64_t)PK_N);
  const int64_t T = nCB * nPT;
  const int nK = (int)(ldh / PK_KC);
  constexpr uint32_t IDESC = idesc_bf16_f32(PK_M, PK_N);

  if (tid == 0) {
    for (int s = 0; s < PK_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&tfull[a], 1);
      mbar_init(&tempty[a], 32 * PK_EPI_WARPS);
    }
    for (int qd = 0; qd < 4; ++qd) {
      mbar_init(&redf[qd], 32);
      mbar_init(&rede[qd], 32);
    }
    fence_barrier_init();
    prefetch_tmap(&map_zhi);
    prefetch_tmap(&map_zmid);
    prefetch_tmap(&map_zlo);
    prefetch_tmap(&map_xhi);
    prefetch_tmap(&map_xmid);
    prefetch_tmap(&map_xlo);
    if (STORE) prefetch_tmap(&map_out);
  }
  if (warp == 0) tmem_alloc(tmem_slot, 2 * PK_ACC_COLS);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---- TMA producer
      int64_t q = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < T && ok; t += gridDim.x) {
        int cb;
        int64_t pt;
        tile_coords(t, nCB, nPT, cb, pt);
        for (int kc = 0; kc < nK; ++kc, ++q) {
          const int s = (int)(q % PK_STAGES);
          const uint32_t ph = (uint32_t)((q / PK_STAGES) & 1);
          if (!mbar_wait(&empty[s], ph ^ 1u, wc.st, 21, wc.lim)) {
            ok = false;
            break;
          }
          uint8_t* st = smem + s * PK_STAGE;
          uint8_t* sb = st + 3 * PK_PLANE_A;
          mbar_expect_tx(&full[s], PK_STAGE);
          tma_load_2d(st, &map_zhi, kc * PK_KC, cb * PK_M, &full[s]);
          tma_load_2d(st + PK_PLANE_A, &map_zmid, kc * PK_KC, cb * PK_M, &full[s]);
          tma_load_2d(st + 2 * PK_PLANE_A, &map_zlo, kc * PK_KC, cb * PK_M, &full[s]);
          tma_load_2d(sb, &map_xhi, kc * PK_KC, (int)(pt * PK_N), &full[s]);
          tma_load_2d(sb + PK_PLANE_B, &map_xmid, kc * PK_KC, (int)(pt * PK_N), &full[s]);
          tma_load_2d(sb + 2 * PK_PLANE_B, &map_xlo, kc * PK_KC, (int)(pt * PK_N), &full[s]);
        }
      }
      // no copy may be in flight when the block exits
      for (int64_t r = (q > PK_STAGES ? q - PK_STAGES : 0); r < q; ++r)
        mbar_wait(&full[r % PK_STAGES], (uint32_t)((r / PK_STAGES) & 1), wc.st, 22, wc.lim);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer
      int64_t q = 0, j = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < T && ok; t += gridDim.x, ++j) {
        const int acc = (int)(j & 1);
        if (!mbar_wait(&tempty[acc], (uint32_t)(((j >> 1) & 1) ^ 1), wc.st, 23, wc.lim)) break;
        fence_after_sync();
        // hi hi products in one accumulator, the five smaller ones (2^-8 and
        // below) in another: the FP32 accumulation's rounding then grows with
        // the few large-term MMAs only
        const uint32_t d_big = tmem + acc * PK_ACC_COLS;
        const uint32_t d_small = d_big + PK_N;
        for (int kc = 0; kc < nK; ++kc, ++q) {
          const int s = (int)(q % PK_STAGES);
          const uint32_t ph = (uint32_t)((q / PK_STAGES) & 1);
          if (!mbar_wait(&full[s], ph, wc.st, 24, wc.lim)) {
            ok = false;
            break;
          }
          fence_after_sync();
          const uint32_t base = smem_u32(smem + s * PK_STAGE);
          const uint32_t a_hi = base, a_mid = base + PK_PLANE_A, a_lo = base + 2 * PK_PLANE_A;
          const uint32_t b_hi = base + 3 * PK_PLANE_A, b_mid = b_hi + PK_PLANE_B,
                         b_lo = b_hi + 2 * PK_PLANE_B;
#pragma unroll
          for (int k = 0; k < PK_KC / 16; ++k) {
            const uint32_t koff = k * 32;
            const uint32_t first = (kc | k) != 0 ? 1u : 0u;
            mma_bf16(d_small, desc_sw64(a_lo + koff), desc_sw64(b_hi + koff), IDESC, first);
            mma_bf16(d_small, desc_sw64(a_hi + koff), desc_sw64(b_lo + koff), IDESC, 1u);
            mma_bf16(d_small, desc_sw64(a_mid + koff), desc_sw64(b_mid + koff), IDESC, 1u);
            mma_bf16(d_small, desc_sw64(a_mid + koff), desc_sw64(b_hi + koff), IDESC, 1u);
            mma_bf16(d_small, desc_sw64(a_hi + koff), desc_sw64(b_mid + koff), IDESC, 1u);
            mma_bf16(d_big, desc_sw64(a_hi + koff), desc_sw64(b_hi + koff), IDESC, first);
          }
          mma_commit(&empty[s]);
        }
        mma_commit(&tfull[acc]);
      }
    }
  } else {
    // ---- epilogue: warp w drains lane quarter w % 4, points half * 64 ..
    const int quarter = warp & 3;
    const int half = (warp - 2) >> 2;
    const int c_in = 32 * quarter + lane;
    const float g2 = gamma * 1.4426950408889634f;   // K = 2^(-g2 |x - z|^2)
    float* stage = reinterpret_cast<float*>(smem + PK_STAGE_OFF) + (warp - 2) * 3 * PK_WP;
    uint8_t* obox = smem + PK_OUT_OFF + (warp - 2) * 2 * PK_OUT_BOX;
    int64_t j = 0;
    for (int64_t t = blockIdx.x; t < T; t += gridDim.x, ++j) {
      int cb;
      int64_t pt;
      tile_coords(t, nCB, nPT, cb, pt);
      const int64_t c = (int64_t)cb * PK_M + c_in;
      const bool crow = c < m;
      const float zn = crow ? (DECIDE ? znorm[c] : norms[idx[c]]) : 0.f;
      const float bc = DECIDE && crow ? (float)beta[c] : 0.f;
      const int64_t ib = pt * PK_N + half * PK_WP;
      const int64_t npts = min64(PK_WP, n - ib);
      // this warp's 64 points: norms (and for scores the active residual / flag)
      for (int h2 = 0; h2 < PK_WP / 32; ++h2) {
        const int jj = h2 * 32 + lane;
        const int64_t i = ib + jj;
        const bool in = jj < npts;
        stage[jj] = in ? norms[i] : 0.f;
        if (SCORE) {
          float r = 0.f, a = 0.f;
          if (in) {
            const float oi = o[i], yi = y[i];
            if (yi * oi < 1.0f) {
              r = oi - yi;
              a = 1.f;
            }
          }
          stage[PK_WP + jj] = r;
          stage[2 * PK_WP + jj] = a;
        }
      }
      __syncwarp();
      const int acc = (int)(j & 1);
      if (!mbar_wait(&tfull[acc], (uint32_t)((j >> 1) & 1), wc.st, 25, wc.lim)) break;
      fence_after_sync();
      float gs = 0.f, hs = 0.f;
      const uint32_t tb = tmem + acc * PK_ACC_COLS + half * PK_WP + ((uint32_t)(32 * quarter) << 16);
      if (STORE) {
        // the previous tile's boxes must have been read out before they are rewritten
        if (lane == 0) bulk_wait_read();
        __syncwarp();
      }
      const float zz = -g2 * zn;
      for (int cc = 0; cc < PK_WP / 32; ++cc) {
        if (cc * 32 >= npts) break;   // uniform per warp
        float v[32], w[32];
        tmem_ld32(tb + cc * 32, v);
        tmem_ld32(tb + PK_N + cc * 32, w);
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) v[jj] += w[jj];   // x.z = large terms + small terms
        // arg = -g2 * max(|x|^2 + |z|^2 - 2 x.z, 0); points past n carry zero
        // norms here and are clipped by the store or weighted by zero flags
#pragma unroll
        for (int jj = 0; jj < 32; jj += 4) {
          const float4 x4 = *reinterpret_cast<const float4*>(stage + cc * 32 + jj);
          v[jj + 0] = ex2_approx(fminf(fmaf(-g2, x4.x, fmaf(2.0f * g2, v[jj + 0], zz)), 0.0f));
          v[jj + 1] = ex2_approx(fminf(fmaf(-g2, x4.y, fmaf(2.0f * g2, v[jj + 1], zz)), 0.0f));
          v[jj + 2] = ex2_approx(fminf(fmaf(-g2, x4.z, fmaf(2.0f * g2, v[jj + 2], zz)), 0.0f));
          v[jj + 3] = ex2_approx(fminf(fmaf(-g2, x4.w, fmaf(2.0f * g2, v[jj + 3], zz)), 0.0f));
        }
        if (STORE) {
          // 32 FP32 values into box cc of this warp (row = lane, 128-byte
          // swizzle: 16-byte chunk ch of row r at chunk ch ^ (r & 7))
          uint8_t* bx = obox + cc * PK_OUT_BOX;
#pragma unroll
          for (int ch = 0; ch < 8; ++ch) {
            const int so = lane * 128 + ((ch ^ (lane & 7)) << 4);
            *reinterpret_cast<float4*>(bx + so) =
                make_float4(v[4 * ch], v[4 * ch + 1], v[4 * ch + 2], v[4 * ch + 3]);
          }
        } else if (SCORE) {
#pragma unroll
          for (int jj = 0; jj < 32; ++jj) {
            const float kv = v[jj];
            gs = fmaf(stage[PK_WP + cc * 32 + jj], kv, gs);
            hs = fmaf(stage[2 * PK_WP + cc * 32 + jj] * kv, kv, hs);
          }
        } else {
          // beta_c k(z_c, x_i) summed over this warp's 32 basis rows (rows
          // past m carry beta 0); one partial per (basis block, lane
          // quarter) and query, summed in a fixed order by the finish
#pragma unroll
          for (int jj = 0; jj < 32; ++jj) v[jj] *= bc;
          const float f = warp_column_sums(v, lane);
          if (cc * 32 + lane < npts)
            dpart[((int64_t)cb * 4 + quarter) * ldp + ib + cc * 32 + lane] = f;
        }
      }
      fence_before_sync();
      mbar_arrive(&tempty[acc]);
      if (STORE && npts > 0) {
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) {
          const int x = (int)ib, yrow = (int)(row0 + (int64_t)cb * PK_M + 32 * quarter);
          // boxes of 32 points; the second starts past n only when npts <= 32
          tma_store_2d(&map_out, x, yrow, obox);
          if (npts > 32) tma_store_2d(&map_out, x + 32, yrow, obox + PK_OUT_BOX);
          bulk_commit();
        }
      }
      if (SCORE) {
        // the two warps of a lane quarter combine their halves of the tile
        const uint32_t par = (uint32_t)(j & 1);
        if (half == 1) {
          if (!mbar_wait(&rede[quarter], par ^ 1u, wc.st, 26, wc.lim)) break;
          red[quarter * 32 + lane] = make_float2(gs, hs);
          mbar_arrive(&redf[quarter]);
        } else {
          if (!mbar_wait(&redf[quarter], par, wc.st, 27, wc.lim)) break;
          const float2 r2 = red[quarter * 32 + lane];
          mbar_arrive(&rede[quarter]);
          if (crow)
            part[pt * kappa + c] = make_double2((double)gs + (double)r2.x, (double)hs + (double)r2.y);
        }
      }
      __syncwarp();
    }
    if (STORE && lane == 0) bulk_wait_all();
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    fence_after_sync();
    tmem_dealloc(tmem, 2 * PK_ACC_COLS);
  }
}

// Z planes: rows idx[0..m) of the three split X planes, zero rows up to m_pad.
__global__ void gather_rows_bf16(const uint16_t* __restrict__ Xhi, const uint16_t* __restrict__ Xmid,
                                 const uint16_t* __restrict__ Xlo, int64_t ldh,
                                 const int64_t* __restrict__ idx, int32_t m, int64_t m_pad,
                                 uint16_t* __restrict__ Zhi, uint16_t* __restrict__ Zmid,
                                 uint16_t* __restrict__ Zlo) {
  const int64_t chunks = ldh / 8;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m_pad * chunks) return;
  const int64_t r = e / chunks, ch = e % chunks;
  uint4 vh = make_uint4(0, 0, 0, 0), vm = vh, vl = vh;
  if (r < m) {
    const int64_t src = idx[r] * ldh + ch * 8;
    vh = *reinterpret_cast<const uint4*>(Xhi + src);
    vm = *reinterpret_cast<const uint4*>(Xmid + src);
    vl = *reinterpret_cast<const uint4*>(Xlo + src);
  }
  *reinterpret_cast<uint4*>(Zhi + r * ldh + ch * 8) = vh;
  *reinterpret_cast<uint4*>(Zmid + r * ldh + ch * 8) = vm;
  *reinterpret_cast<uint4*>(Zlo + r * ldh + ch * 8) = vl;
}

// ---------------------------------------------------------------------------
// Masked Gram matrix: P[a][b] (+)= sum_p Kc[a][p] Kc[b][p] over 128 x 128
// upper-triangular tiles, Kc = hi + lo with all four plane products, so P
// is the Gram matrix of the stored values up to FP32 accumulation rounding
// (positive semidefinite to that level).  Warp 0: TMEM owner and TMA producer; warp 1: MMA
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
    double* __restrict__ part, int64_t ldp, WaitCtx wc) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = align1024(smem_raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + GR_BAR_OFF);
  uint64_t* empty = full + GR_STAGES;
  uint64_t* accf = empty + GR_STAGES;
  uint64_t* acce = accf + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acce + 2);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (__syncthreads_or(tid == 0 && *(volatile int*)wc.st != 0)) return;
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
      if (!mbar_wait(&empty[s], ph ^ 1u, wc.st, 11, wc.lim)) break;
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
      mbar_wait(&full[q % GR_STAGES], (uint32_t)((q / GR_STAGES) & 1), wc.st, 12, wc.lim);
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer
    bool ok = true;
    for (int64_t t = 0; t < nslices && ok; ++t) {
      const int acc = (int)(t & 1);
      const uint32_t use = (uint32_t)((t >> 1) & 1);
      if (!mbar_wait(&acce[acc], use ^ 1u, wc.st, 13, wc.lim)) break;
      fence_after_sync();
      const uint32_t d = tmem + acc * GR_TILE;
      const int64_t q0 = t * GR_CHUNKS_PER_SLICE;
      const int64_t q1 = min64(nch, q0 + GR_CHUNKS_PER_SLICE);
      for (int64_t q = q0; q < q1; ++q) {
        const int s = (int)(q % GR_STAGES);
        const uint32_t ph = (uint32_t)((q / GR_STAGES) & 1);
        if (!mbar_wait(&full[s], ph, wc.st, 14, wc.lim)) {
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
          // lo x lo too: without it the sum is (hi + lo)^T (hi + lo) - lo^T lo,
          // indefinite in the null space of a short K_SJ
          mma_bf16(d, desc_sw128(a_lo + koff), desc_sw128(b_lo + koff), IDESC, 1u);
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
      if (!mbar_wait(&accf[acc], use, wc.st, 15, wc.lim)) break;
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

// 2-D map over rows x inner (row pitch `pitch_elems`) of BF16 (or FP32 with
// f32), box_inner x box_rows boxes of 128 bytes per row, 128-byte swizzle,
// zero fill outside the tensor.
int make_map(CUtensorMap* map, const void* base, int64_t inner, int64_t rows, int64_t pitch_elems,
             uint32_t box_rows, uint32_t box_inner, bool f32 = false) {
  auto fn = encode_fn();
  if (!fn) return set_error(SPSVM_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
  const int64_t esz = f32 ? 4 : 2;
  const int64_t row_bytes = box_inner * esz;   // 128-byte rows swizzled by 128, 64-byte rows by 64
  if ((reinterpret_cast<uintptr_t>(base) & 15) || (pitch_elems * esz) % 16 ||
      (row_bytes != 128 && row_bytes != 64))
    return set_error(SPSVM_ERR_ARG, "tensor map: base or pitch not 16-byte aligned, or box row not 64/128 bytes");
  cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)(rows > 0 ? rows : 1)};
  cuuint64_t strides[1] = {(cuuint64_t)(pitch_elems * esz)};
  cuuint32_t box[2] = {box_inner, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                  const_cast<void*>(base), dims, strides,
                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  row_bytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(SPSVM_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return SPSVM_OK;
}

// Extra arguments of the decision mode: basis norms, beta, the partial sums
// and their row pitch.
struct DecideArgs {
  const float* znorm = nullptr;
  const double* beta = nullptr;
  float* dpart = nullptr;
  int64_t ldp = 0;
};

// STORE / SCORE: the m rows idx of the points' planes are gathered into zbuf
// first (zero rows up to a multiple of 128).  DECIDE: zbuf already holds the
// basis planes (m rows of pitch ldh; the tensor maps zero-fill past m).
template <int MODE>
int launch_kb(const spsvm_points* p, const int64_t* idx, int32_t m, float gamma, void* out,
              int64_t ld, int64_t row0, const float* y, const float* o, double2* part,
              int32_t kappa, void* zbuf, size_t zbytes, cudaStream_t s,
              const DecideArgs& da = DecideArgs()) {
  const int64_t m_pad = round_up(m, (int64_t)PK_M);
  const int64_t zrows = MODE == KB_DECIDE ? (int64_t)m : m_pad;
  if (!zbuf || zbytes < (size_t)(zrows * p->ldh * 6))
    return set_error(SPSVM_ERR_OOM, "BF16SPLIT kernel block: scratch too small for the basis planes");
  uint16_t* zhi = static_cast<uint16_t*>(zbuf);
  uint16_t* zmid = zhi + zrows * p->ldh;
  uint16_t* zlo = zmid + zrows * p->ldh;
  if (MODE != KB_DECIDE) {
    const int64_t work = m_pad * (p->ldh / 8);
    gather_rows_bf16<<<(unsigned)ceil_div(work, (int64_t)256), 256, 0, s>>>(
        p->hi, p->mid, p->lo, p->ldh, idx, m, m_pad, zhi, zmid, zlo);
    SPSVM_LAUNCH_CHECK();
  }
  CUtensorMap mzh, mzm, mzl, mxh, mxm, mxl, mo;
  SPSVM_TRY(make_map(&mzh, zhi, p->ldh, zrows, p->ldh, PK_M, PK_KC));
  SPSVM_TRY(make_map(&mzm, zmid, p->ldh, zrows, p->ldh, PK_M, PK_KC));
  SPSVM_TRY(make_map(&mzl, zlo, p->ldh, zrows, p->ldh, PK_M, PK_KC));
  SPSVM_TRY(make_map(&mxh, p->hi, p->ldh, p->n, p->ldh, PK_N, PK_KC));
  SPSVM_TRY(make_map(&mxm, p->mid, p->ldh, p->n, p->ldh, PK_N, PK_KC));
  SPSVM_TRY(make_map(&mxl, p->lo, p->ldh, p->n, p->ldh, PK_N, PK_KC));
  // output rows [0, row0 + m): rows past the basis block are clipped, never written
  if (MODE == KB_STORE_F32) SPSVM_TRY(make_map(&mo, out, p->n, row0 + m, ld, 32, 32, true));
  else mo = mxh;
  auto kern = kblock_tc_kernel<MODE>;
  SPSVM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, PK_SMEM));
  const int64_t tiles = ceil_div((int64_t)m, (int64_t)PK_M) * ceil_div(p->n, (int64_t)PK_N);
  const int grid = (int)min64(tiles, (int64_t)sm_count());
  WaitCtx wc;
  SPSVM_TRY(wait_ctx(s, &wc));
  kern<<<grid, PK_THREADS, PK_SMEM, s>>>(mzh, mzm, mzl, mxh, mxm, mxl, mo, p->ldh, p->n, m,
                                         p->norms, idx, gamma, row0, y, o, part, kappa, da.znorm,
                                         da.beta, da.dpart, da.ldp, wc);
  SPSVM_LAUNCH_CHECK();
  return SPSVM_OK;
}

}  // namespace

bool tc_available() { return encode_fn() != nullptr; }

size_t kernel_block_tc_scratch(int64_t m, int64_t ldh) {
  return (size_t)(round_up(m, (int64_t)PK_M) * ldh * 6);   // three BF16 planes of the rows
}

int launch_kernel_block_tc(const spsvm_points* p, const int64_t* idx, int32_t m, float gamma,
                           spsvm_kmat* out, int64_t row0, void* scratch, size_t scratch_bytes,
                           cudaStream_t s) {
  if (m == 0 || p->n == 0) return SPSVM_OK;
  if (out->format != SPSVM_FP32 || (out->ld % 8) != 0)
    return set_error(SPSVM_ERR_ARG, "BF16SPLIT kernel block: stores FP32 (ld %% 8 == 0)");
  return launch_kb<KB_STORE_F32>(p, idx, m, gamma, out->data, out->ld, row0, nullptr, nullptr,
                                 nullptr, 0, scratch, scratch_bytes, s);
}

int64_t score_tc_tiles(int64_t n) { return ceil_div(n, (int64_t)PK_N); }

int launch_score_tc(const spsvm_points* p, const float* y, const float* o, const int64_t* idx,
                    int32_t kappa, float gamma, double2* part, int64_t tiles, void* zbuf,
                    size_t zbytes, cudaStream_t s) {
  (void)tiles;
  return launch_kb<KB_SCORE>(p, idx, kappa, gamma, nullptr, 0, 0, y, o, part, kappa, zbuf, zbytes, s);
}

int64_t decision_tc_parts(int64_t m) { return 4 * ceil_div(m, (int64_t)PK_M); }

int launch_decision_tc(const spsvm_points* q, const void* zplanes, size_t zbytes, int64_t m,
                       const float* znorm, const double* beta, float gamma, float* dpart,
                       int64_t ldp, cudaStream_t s) {
  if (m == 0 || q->n == 0) return SPSVM_OK;
  DecideArgs da;
  da.znorm = znorm;
  da.beta = beta;
  da.dpart = dpart;
  da.ldp = ldp;
  return launch_kb<KB_DECIDE>(q, nullptr, (int32_t)m, gamma, nullptr, 0, 0, nullptr, nullptr,
                              nullptr, 0, const_cast<void*>(zplanes), zbytes, s, da);
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
  SPSVM_TRY(make_map(&mh, hi, Kc->ld, m, Kc->ld, GR_TILE, 64));
  SPSVM_TRY(make_map(&ml, lo, Kc->ld, m, Kc->ld, GR_TILE, 64));
  SPSVM_CUDA_TRY(cudaFuncSetAttribute(gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      GR_SMEM));
  const int64_t T = ceil_div(m, (int64_t)GR_TILE);
  const int64_t tiles = T * (T + 1) / 2;
  const int64_t slices = ceil_div(ns_max > 0 ? ns_max : 1, GRAM_SLICE);
  const int64_t per = ceil_div(slices, splits);
  dim3 grid((unsigned)tiles, (unsigned)splits);
  WaitCtx wc;
  SPSVM_TRY(wait_ctx(s, &wc));
  gram_tc_kernel<<<grid, GR_THREADS, GR_SMEM, s>>>(mh, ml, m, ns_dev, per, part, ldp, wc);
  SPSVM_LAUNCH_CHECK();
  return SPSVM_OK;
}

}  // namespace spsvm

