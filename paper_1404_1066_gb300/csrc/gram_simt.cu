// Masked Gram matrix H = lambda K_JJ + K_SJ^T K_SJ (the generalised Hessian
// of Eq. 4 on the active set S) in FP32 SIMT arithmetic, with FP32 sums per
// slice of 8192 points promoted to FP64.  Also the FP64 finishing pass
// shared by both arithmetic forms.
#include "internal.h"
#include "gram.h"

namespace spsvm {

namespace {

constexpr int GT = 64;      // output tile
constexpr int GK = 32;      // points per smem stage
constexpr int GNT = 256;    // 16 x 16 threads, 4 x 4 outputs each

// Maps a linear index to the (ta <= tb) upper-triangular tile pair.
__device__ __forceinline__ void tri_index(int64_t t, int64_t T, int& ta, int& tb) {
  // rows of the upper triangle: row a has T - a tiles
  int a = 0;
  int64_t rem = t;
  while (rem >= T - a) { rem -= T - a; ++a; }
  ta = a;
  tb = a + (int)rem;
}

__global__ void __launch_bounds__(GNT) gram_simt_kernel(
    KView Kc, int64_t m, const int64_t* __restrict__ ns_dev, int64_t slices_per_split,
    double* __restrict__ part, int64_t ldp) {
  __shared__ float As[GK][GT + 1];
  __shared__ float Bs[GK][GT + 1];
  const int64_t T = ceil_div(m, (int64_t)GT);
  int ta, tb;
  tri_index(blockIdx.x, T, ta, tb);
  const int64_t a0 = (int64_t)ta * GT, b0 = (int64_t)tb * GT;
  const int64_t ns = *ns_dev;
  const int64_t p_begin = (int64_t)blockIdx.y * slices_per_split * GRAM_SLICE;
  const int64_t p_end = min(ns, p_begin + slices_per_split * GRAM_SLICE);
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  double accd[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) accd[r][c] = 0.0;
  for (int64_t s0 = p_begin; s0 < p_end; s0 += GRAM_SLICE) {
    const int64_t s1 = min(p_end, s0 + GRAM_SLICE);
    float acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[r][c] = 0.f;
    for (int64_t p0 = s0; p0 < s1; p0 += GK) {
#pragma unroll
      for (int r = 0; r < (GT * GK) / GNT; ++r) {
        const int e = t + GNT * r;
        const int row = e / GK, col = e % GK;
        const int64_t p = p0 + col;
        const bool okp = p < s1;
        As[col][row] = (okp && a0 + row < m) ? Kc.at(a0 + row, p) : 0.f;
        Bs[col][row] = (okp && b0 + row < m) ? Kc.at(b0 + row, p) : 0.f;
      }
      __syncthreads();
#pragma unroll 8
      for (int kk = 0; kk < GK; ++kk) {
        float av[4], bv[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) av[r] = As[kk][ty + 16 * r];
#pragma unroll
        for (int c = 0; c < 4; ++c) bv[c] = Bs[kk][tx + 16 * c];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(av[r], bv[c], acc[r][c]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) accd[r][c] += (double)acc[r][c];
  }
  double* P = part + (int64_t)blockIdx.y * ldp * ldp;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int64_t a = a0 + ty + 16 * r;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int64_t b = b0 + tx + 16 * c;
      if (a < m && b < m) P[a * ldp + b] = accd[r][c];
    }
  }
}

}  // namespace

int64_t gram_simt_splits(int64_t m, int64_t ns_max) {
  const int64_t T = ceil_div(m, (int64_t)GT);
  const int64_t tiles = T * (T + 1) / 2;
  const int64_t slices = ceil_div(ns_max > 0 ? ns_max : 1, GRAM_SLICE);
  int64_t want = ceil_div(2 * (int64_t)sm_count(), tiles > 0 ? tiles : 1);
  if (want < 1) want = 1;
  if (want > slices) want = slices;
  return want;
}

int launch_gram_simt(const spsvm_kmat* Kc, const int64_t* ns_dev, int64_t ns_max, int64_t m,
                     double* part, int64_t ldp, int64_t splits, cudaStream_t s) {
  const int64_t T = ceil_div(m, (int64_t)GT);
  const int64_t tiles = T * (T + 1) / 2;
  const int64_t slices = ceil_div(ns_max > 0 ? ns_max : 1, GRAM_SLICE);
  const int64_t per = ceil_div(slices, splits);
  dim3 grid((unsigned)tiles, (unsigned)splits);
  gram_simt_kernel<<<grid, GNT, 0, s>>>(view(Kc), m, ns_dev, per, part, ldp);
  SPSVM_LAUNCH_CHECK();
  return SPSVM_OK;
}

// K_JJ[a][b] = (K[b][J[a]] + K[a][J[b]]) / 2 (the stored values made
// symmetric; exact in FP64) for the rows and columns from row0 on: thread
// (r, c), r >= row0, writes (r, c) and (c, r).  A fit keeps K_JJ in its
// workspace and extends it once per round, so the Gram finish reads it
// coalesced instead of gathering two scattered kernel values per entry.
__global__ void kjj_fill_kernel(KView K, const int64_t* __restrict__ J, int64_t m, int64_t row0,
                                double* __restrict__ kjj, int64_t ldk) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t rows = m - row0;
  if (e >= rows * m) return;
  const int64_t r = row0 + e / m, c = e % m;
  // the bias slot (point index -1) has no regulariser row or column
  const double v = (J[r] < 0 || J[c] < 0) ? 0.0 : 0.5 * ((double)K.at(c, J[r]) + (double)K.at(r, J[c]));
  kjj[r * ldk + c] = v;
  kjj[c * ldk + r] = v;
}

// H[a][b] = H[b][a] = lambda K_JJ[a][b] + sum_s part[s][min(a,b)][max(a,b)]
// over 32 x 32 upper tiles: the partials, K_JJ and both halves of H move
// through shared memory so that every global access is coalesced.
constexpr int FT = 32;
__global__ void __launch_bounds__(FT * 8) gram_finish_kernel(const double* __restrict__ part,
                                                             int64_t splits, int64_t ldp,
                                                             const double* __restrict__ kjj,
                                                             int64_t ldk, int64_t m, double lambda,
                                                             double* __restrict__ H, int64_t ldh) {
  __shared__ double P[FT][FT + 1];
  __shared__ double Kt[FT][FT + 1];
  const int64_t T = ceil_div(m, (int64_t)FT);
  int64_t rem = blockIdx.x, ta = 0;
  while (rem >= T - ta) {
    rem -= T - ta;
    ++ta;
  }
  const int64_t tb = ta + rem;
  const int64_t a0 = ta * FT, b0 = tb * FT;
  const int c = threadIdx.x;
  const int64_t b = b0 + c;
  for (int r = threadIdx.y; r < FT; r += 8) {
    const int64_t a = a0 + r;
    double sum = 0.0, kv = 0.0;
    if (a < m && b < m) {
      for (int64_t k = 0; k < splits; ++k) sum += part[k * ldp * ldp + a * ldp + b];
      kv = kjj[a * ldk + b];
    }
    P[r][c] = sum;
    Kt[r][c] = kv;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < FT; r += 8) {
    const int64_t a = a0 + r;
    if (a < m && b < m) {
      // the partial of the upper triangle for both orientations
      const double pv = (ta == tb && r > c) ? P[c][r] : P[r][c];
      H[a * ldh + b] = lambda * Kt[r][c] + pv;
    }
  }
  if (ta != tb) {   // mirror tile: H[b0 + r][a0 + c] from the transposed values
    const int64_t a = a0 + c;
    for (int r = threadIdx.y; r < FT; r += 8) {
      const int64_t bb = b0 + r;
      if (a < m && bb < m) H[bb * ldh + a] = lambda * Kt[c][r] + P[c][r];
    }
  }
}

int launch_gram_finish(const double* part, int64_t splits, int64_t ldp, const double* kjj,
                       int64_t ldk, int64_t m, double lambda, double* H, int64_t ldh,
                       cudaStream_t s) {
  const int64_t T = ceil_div(m, (int64_t)FT);
  gram_finish_kernel<<<(unsigned)(T * (T + 1) / 2), dim3(FT, 8), 0, s>>>(part, splits, ldp, kjj,
                                                                         ldk, m, lambda, H, ldh);
  SPSVM_LAUNCH_CHECK();
  return SPSVM_OK;
}

size_t gram_part_bytes(int64_t m, int64_t ns) {
  if (m < 0 || ns < 0) return 0;
  const int64_t ldp = round_up(m > 0 ? m : 1, 64);
  int64_t splits = gram_simt_splits(m, ns);
  const int64_t tc = gram_tc_splits(m, ns);
  if (tc > splits) splits = tc;
  return (size_t)(splits * ldp * ldp * (int64_t)sizeof(double));
}

int kjj_fill(const spsvm_kmat* K, const int64_t* J, int64_t m, int64_t row0, double* kjj,
             int64_t ldk, cudaStream_t s) {
  if (m <= row0) return SPSVM_OK;
  const int64_t total = (m - row0) * m;
  kjj_fill_kernel<<<(unsigned)ceil_div(total, 256), 256, 0, s>>>(view(K), J, m, row0, kjj, ldk);
  SPSVM_LAUNCH_CHECK();
  return SPSVM_OK;
}

}  // namespace spsvm

using namespace spsvm;

extern "C" size_t spsvm_gram_scratch_bytes(int64_t m, int64_t ns) {
  if (m < 0 || ns < 0) return 0;
  const int64_t ldp = round_up(m > 0 ? m : 1, 64);
  // the partial sums, then K_JJ gathered from K (a fit keeps its own)
  return gram_part_bytes(m, ns) + (size_t)(ldp * ldp * (int64_t)sizeof(double));
}

namespace spsvm {
int gram_impl(const spsvm_kmat* Kc, const int64_t* ns_dev, int64_t ns_max, const spsvm_kmat* K,
              const int64_t* J, double lambda, int32_t precision, double* H, int64_t ldh,
              void* scratch, size_t scratch_bytes, cudaStream_t s, double ns_work,
              const double* kjj, int64_t ldk) {
  SPSVM_TRY(check_kmat(Kc, "gram(Kc)"));
  SPSVM_TRY(check_kmat(K, "gram(K)"));
  if (!ns_dev || !J || !H) return set_error(SPSVM_ERR_ARG, "gram: NULL pointer");
  const int64_t m = K->rows;
  if (Kc->rows < m || ldh < m || ns_max < 0 || ns_max > Kc->n || !(lambda > 0.0))
    return set_error(SPSVM_ERR_ARG, "gram: bad shapes m=%lld Kc.rows=%lld ldh=%lld ns_max=%lld",
                     (long long)m, (long long)Kc->rows, (long long)ldh, (long long)ns_max);
  if (m == 0) return SPSVM_OK;
  const size_t need = kjj ? gram_part_bytes(m, ns_max) : spsvm_gram_scratch_bytes(m, ns_max);
  if (!scratch || scratch_bytes < need) return set_error(SPSVM_ERR_OOM, "gram: scratch too small");
  // algorithmic work: one multiply-add per active point per unique entry,
  // times the four plane products of the BF16SPLIT form
  ProfScope prof(PROF_GRAM, s,
                 (precision == SPSVM_BF16SPLIT ? 4.0 : 1.0) * ns_work * (double)m * (double)(m + 1));
  const int64_t ldp = round_up(m, 64);
  double* part = static_cast<double*>(scratch);
  if (!kjj) {   // gather K_JJ into the scratch behind the partial sums
    double* kj = reinterpret_cast<double*>(static_cast<char*>(scratch) + gram_part_bytes(m, ns_max));
    SPSVM_TRY(kjj_fill(K, J, m, 0, kj, ldp, s));
    kjj = kj;
    ldk = ldp;
  }
  int64_t splits;
  if (precision == SPSVM_BF16SPLIT) {
    if (Kc->format != SPSVM_BF16SPLIT) return set_error(SPSVM_ERR_ARG, "gram: BF16SPLIT needs split planes");
    splits = gram_tc_splits(m, ns_max);
    SPSVM_TRY(launch_gram_tc(Kc, ns_dev, ns_max, m, part, ldp, splits, s));
  } else if (precision == SPSVM_FP32) {
    splits = gram_simt_splits(m, ns_max);
    SPSVM_TRY(launch_gram_simt(Kc, ns_dev, ns_max, m, part, ldp, splits, s));
  } else {
    return set_error(SPSVM_ERR_ARG, "gram: bad precision");
  }
  return launch_gram_finish(part, splits, ldp, kjj, ldk, m, lambda, H, ldh, s);
}
}  // namespace spsvm

extern "C" int spsvm_gram(const spsvm_kmat* Kc, const int64_t* ns_dev, int64_t ns_max,
                          const spsvm_kmat* K, const int64_t* J, double lambda, int32_t precision,
                          double* H, int64_t ldh, void* scratch, size_t scratch_bytes,
                          void* stream) {
  return gram_impl(Kc, ns_dev, ns_max, K, J, lambda, precision, H, ldh, scratch, scratch_bytes,
                   as_stream(stream), (double)ns_max, nullptr, 0);
}
