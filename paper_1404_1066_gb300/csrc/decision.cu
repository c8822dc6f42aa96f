// Decision values f(q) = sum_j beta_j k(q, b_j) (Section 4: the classifier
// h(x) = w^T phi(x) with w restricted to the basis J), tile by tile, never
// storing the query-by-basis kernel block.  SPSVM_FP32: plain FP32 SIMT dot
// products, FP64 accumulation of beta_j k(q, b_j) per tile of 64 basis
// vectors.  SPSVM_BF16SPLIT: the tensor-core kernel block engine with the
// basis rows and the queries split into three BF16 planes each, FP32 sums of
// beta_j k over 32 basis rows per partial, the partials summed in FP64 in a
// fixed order.
#include "internal.h"

namespace spsvm {

int64_t decision_tc_parts(int64_t m);
int launch_decision_tc(const spsvm_points* q, const void* zplanes, size_t zbytes, int64_t m,
                       const float* znorm, const double* beta, float gamma, float* dpart,
                       int64_t ldp, cudaStream_t s);

namespace {

constexpr int QM = 128;   // queries per block
constexpr int QN = 64;    // basis vectors per tile
constexpr int QK = 16;
constexpr int QT = 256;

__global__ void row_norms_kernel(const float* __restrict__ A, int64_t m, int64_t d, int64_t lda,
                                 float* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= m) return;
  double acc = 0.0;
  for (int64_t k = lane; k < d; k += 32) {
    const float v = A[i * lda + k];
    acc += (double)v * (double)v;
  }
  acc = warp_sum(acc);
  if (lane == 0) out[i] = (float)acc;
}

__global__ void __launch_bounds__(QT) decision_simt(
    const float* __restrict__ B, int64_t m, int64_t ldb, const float* __restrict__ bnorm,
    const double* __restrict__ beta, const float* __restrict__ Q, int64_t nq, int64_t ldq,
    int64_t d, float gamma, float* __restrict__ out) {
  __shared__ float Qs[QK][QM + 4];
  __shared__ float Bs[QK][QN + 4];
  __shared__ float qn[QM];
  __shared__ float bn[QN];
  __shared__ double bs[QN];
  __shared__ double red[8][QM];
  const int t = threadIdx.x, tx = t & 31, ty = t >> 5;
  const int64_t q0 = (int64_t)blockIdx.x * QM;
  // query norms (FP64 accumulation), one warp per query
  for (int r = ty; r < QM; r += 8) {
    const int64_t q = q0 + r;
    double acc = 0.0;
    if (q < nq)
      for (int64_t k = tx; k < d; k += 32) {
        const float v = Q[q * ldq + k];
        acc += (double)v * (double)v;
      }
    acc = warp_sum(acc);
    if (tx == 0) qn[r] = (float)acc;
  }
  double accd[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t b0 = 0; b0 < m; b0 += QN) {
    __syncthreads();
    if (t < QN) {
      const int64_t b = b0 + t;
      bn[t] = (b < m) ? bnorm[b] : 0.f;
      bs[t] = (b < m) ? beta[b] : 0.0;
    }
    float acc[4][8];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 8; ++c) acc[a][c] = 0.f;
    for (int64_t k0 = 0; k0 < d; k0 += QK) {
#pragma unroll
      for (int r = 0; r < (QM * QK) / QT; ++r) {
        const int e = t + QT * r;
        const int row = e / QK, col = e % QK;
        const int64_t q = q0 + row, k = k0 + col;
        Qs[col][row] = (q < nq && k < d) ? Q[q * ldq + k] : 0.f;
      }
#pragma unroll
      for (int r = 0; r < (QN * QK) / QT; ++r) {
        const int e = t + QT * r;
        const int row = e / QK, col = e % QK;
        const int64_t b = b0 + row, k = k0 + col;
        Bs[col][row] = (b < m && k < d) ? B[b * ldb + k] : 0.f;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < QK; ++kk) {
        float av[4], bv[8];
#pragma unroll
        for (int a = 0; a < 4; ++a) av[a] = Qs[kk][tx + 32 * a];
#pragma unroll
        for (int c = 0; c < 8; ++c) bv[c] = Bs[kk][ty + 8 * c];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int c = 0; c < 8; ++c) acc[a][c] = fmaf(av[a], bv[c], acc[a][c]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const float xn = qn[tx + 32 * a];
      double s = 0.0;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int cc = ty + 8 * c;
        if (b0 + cc < m) s += bs[cc] * (double)rbf_from_dot(xn, bn[cc], acc[a][c], gamma);
      }
      accd[a] += s;
    }
  }
  __syncthreads();
#pragma unroll
  for (int a = 0; a < 4; ++a) red[ty][tx + 32 * a] = accd[a];
  __syncthreads();
  if (t < QM) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w][t];
    const int64_t q = q0 + t;
    if (q < nq) out[q] = (float)s;
  }
}

// out[i] = sum over the P partials of column i, in FP64, in order.
__global__ void decision_finish(const float* __restrict__ part, int64_t P, int64_t ldp,
                                int64_t nq, float* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nq) return;
  double s = 0.0;
  for (int64_t p = 0; p < P; ++p) s += (double)part[p * ldp + i];
  out[i] = (float)s;
}

// Queries per pass of the tensor-core form (bounds the scratch).
constexpr int64_t kDecideChunk = 32768;

struct DecideLayout {
  int64_t ldh, qc, parts;
  size_t off_zn, off_z, z_bytes, off_qn, off_q, q_plane, off_part, total;
};

DecideLayout decide_layout(int64_t nq, int64_t m, int64_t d) {
  DecideLayout L;
  auto al = [](size_t b) { return (size_t)round_up((int64_t)b, 256); };
  L.ldh = round_up(d, 64);
  L.qc = round_up(min64(max64(nq, 1), kDecideChunk), 128);
  L.parts = decision_tc_parts(m);
  size_t o = 0;
  L.off_zn = o;
  o += al((size_t)m * 4);
  L.off_z = o;
  L.z_bytes = (size_t)m * L.ldh * 6;
  o += al(L.z_bytes);
  L.off_qn = o;
  o += al((size_t)L.qc * 4);
  L.off_q = o;
  L.q_plane = (size_t)L.qc * L.ldh * 2;
  o += al(3 * L.q_plane);
  L.off_part = o;
  o += al((size_t)L.parts * L.qc * 4);
  L.total = o;
  return L;
}

}  // namespace
}  // namespace spsvm

using namespace spsvm;

extern "C" size_t spsvm_decision_scratch_bytes(int64_t nq, int64_t m, int64_t d, int32_t precision) {
  if (m < 0 || d < 1) return 0;
  if (precision == SPSVM_BF16SPLIT) return decide_layout(nq, m, d).total;
  return (size_t)round_up(m * 4 + 16, 256);
}

extern "C" int spsvm_decision(const float* B, int64_t m, int64_t ldb, const double* beta,
                              const float* Q, int64_t nq, int64_t ldq, int64_t d, float gamma,
                              int32_t precision, float* out, void* scratch, size_t scratch_bytes,
                              void* stream) {
  if (!B || !beta || !Q || !out || m < 0 || nq < 0 || d < 1 || ldb < d || ldq < d || !(gamma > 0.f))
    return set_error(SPSVM_ERR_ARG, "decision: bad arguments");
  if (precision != SPSVM_FP32 && precision != SPSVM_BF16SPLIT)
    return set_error(SPSVM_ERR_ARG, "decision: bad precision");
  if (nq == 0) return SPSVM_OK;
  if (!scratch || scratch_bytes < spsvm_decision_scratch_bytes(nq, m, d, precision))
    return set_error(SPSVM_ERR_OOM, "decision: scratch too small");
  cudaStream_t s = as_stream(stream);
  if (precision == SPSVM_BF16SPLIT) {
    // algorithmic work: 2 nq m d multiply-adds, times the six plane products
    ProfScope prof(PROF_DECISION, s, 12.0 * (double)nq * m * (double)d);
    if (m == 0) {
      SPSVM_CUDA_TRY(cudaMemsetAsync(out, 0, (size_t)nq * 4, s));
      return SPSVM_OK;
    }
    const DecideLayout L = decide_layout(nq, m, d);
    char* w = static_cast<char*>(scratch);
    // the basis rows' norms and planes (rows past m read as zeros)
    uint16_t* zp = reinterpret_cast<uint16_t*>(w + L.off_z);
    spsvm_points zb{B, m, d, ldb, reinterpret_cast<float*>(w + L.off_zn), zp, zp + 2 * m * L.ldh,
                    L.ldh, zp + m * L.ldh};
    SPSVM_TRY(spsvm_prepare_points(&zb, SPSVM_BF16SPLIT, stream));
    uint16_t* qp = reinterpret_cast<uint16_t*>(w + L.off_q);
    float* part = reinterpret_cast<float*>(w + L.off_part);
    for (int64_t q0 = 0; q0 < nq; q0 += L.qc) {
      const int64_t cnt = min64(L.qc, nq - q0);
      spsvm_points qb{Q + q0 * ldq, cnt, d, ldq, reinterpret_cast<float*>(w + L.off_qn), qp,
                      qp + 2 * L.qc * L.ldh, L.ldh, qp + L.qc * L.ldh};
      SPSVM_TRY(spsvm_prepare_points(&qb, SPSVM_BF16SPLIT, stream));
      SPSVM_TRY(launch_decision_tc(&qb, zp, L.z_bytes, m, zb.norms, beta, gamma, part, L.qc, s));
      decision_finish<<<(unsigned)ceil_div(cnt, (int64_t)256), 256, 0, s>>>(part, L.parts, L.qc,
                                                                           cnt, out + q0);
      SPSVM_LAUNCH_CHECK();
    }
    return SPSVM_OK;
  }
  ProfScope prof(PROF_DECISION, s, 2.0 * (double)nq * m * (double)d);
  float* bnorm = static_cast<float*>(scratch);
  if (m > 0) {
    row_norms_kernel<<<(unsigned)ceil_div(m, 8), 256, 0, s>>>(B, m, d, ldb, bnorm);
    SPSVM_LAUNCH_CHECK();
  }
  decision_simt<<<(unsigned)ceil_div(nq, QM), QT, 0, s>>>(B, m, ldb, bnorm, beta, Q, nq, ldq, d,
                                                          gamma, out);
  SPSVM_LAUNCH_CHECK();
  return SPSVM_OK;
}
