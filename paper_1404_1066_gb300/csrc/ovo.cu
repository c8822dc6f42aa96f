// One-vs-one multiclass SP-SVM (Section 5 trains its multiclass sets one
// against one): the C(C-1)/2 binary problems of the class pairs fitted as
// one batch on the shared X, and prediction by voting over the pair models.
#include <vector>

#include "internal.h"

namespace spsvm {
namespace {

constexpr int OV_T = 256;
constexpr int OV_MAX_CLASSES = 64;

// Pair p = (a, b) (order (0,1), (0,2), ..., (1,2), ...) votes a where its
// decision value is >= 0, else b; the class with the most votes wins, ties
// to the smaller class.
__global__ void __launch_bounds__(OV_T) ovo_vote_kernel(const float* __restrict__ dec, int64_t nq,
                                                        int32_t classes,
                                                        int32_t* __restrict__ labels,
                                                        int32_t* __restrict__ votes) {
  const int64_t i = (int64_t)blockIdx.x * OV_T + threadIdx.x;
  if (i >= nq) return;
  int32_t v[OV_MAX_CLASSES];
  for (int c = 0; c < classes; ++c) v[c] = 0;
  int64_t p = 0;
  for (int a = 0; a < classes; ++a)
    for (int b = a + 1; b < classes; ++b, ++p) {
      if (dec[p * nq + i] >= 0.0f) ++v[a];
      else ++v[b];
    }
  int best = 0;
  for (int c = 1; c < classes; ++c)
    if (v[c] > v[best]) best = c;
  labels[i] = best;
  if (votes)
    for (int c = 0; c < classes; ++c) votes[i * classes + c] = v[c];
}

int64_t ovo_count(int32_t classes) { return (int64_t)classes * (classes - 1) / 2; }

}  // namespace
}  // namespace spsvm

using namespace spsvm;

extern "C" int spsvm_fit_ovo(const float* X, int64_t n, int64_t d, int64_t ldx,
                             const int32_t* labels, int32_t classes, float gamma, double lambda,
                             int32_t basis_budget, double tol, const spsvm_options* opt,
                             int32_t workers, spsvm_model** outs, int32_t* status) {
  if (!X || !labels || !outs || !status || n < 1 || d < 1 || ldx < d)
    return set_error(SPSVM_ERR_ARG, "fit_ovo: bad arguments");
  if (classes < 2 || classes > OV_MAX_CLASSES)
    return set_error(SPSVM_ERR_ARG, "fit_ovo: classes must be in [2, %d]", OV_MAX_CLASSES);
  if (basis_budget < 1) return set_error(SPSVM_ERR_ARG, "fit_ovo: basis budget < 1");
  std::vector<std::vector<int64_t>> members(classes);
  for (int64_t i = 0; i < n; ++i) {
    if (labels[i] < 0 || labels[i] >= classes)
      return set_error(SPSVM_ERR_ARG, "fit_ovo: label %d of row %lld out of range", (int)labels[i],
                       (long long)i);
    members[labels[i]].push_back(i);
  }
  for (int c = 0; c < classes; ++c)
    if (members[c].empty()) return set_error(SPSVM_ERR_ARG, "fit_ovo: class %d has no rows", c);
  const int64_t P = ovo_count(classes);
  std::vector<std::vector<int64_t>> rows(P);
  std::vector<std::vector<float>> ys(P);
  std::vector<spsvm_problem> probs(P);
  int64_t p = 0;
  for (int a = 0; a < classes; ++a)
    for (int b = a + 1; b < classes; ++b, ++p) {
      // the pair's rows in X order, y = +1 for class a
      auto& r = rows[p];
      auto& y = ys[p];
      r.reserve(members[a].size() + members[b].size());
      for (int64_t i = 0; i < n; ++i)
        if (labels[i] == a || labels[i] == b) {
          r.push_back(i);
          y.push_back(labels[i] == a ? 1.0f : -1.0f);
        }
      spsvm_problem q{};
      q.rows = r.data();
      q.n_rows = (int64_t)r.size();
      q.y = y.data();
      q.gamma = gamma;
      q.lambda = lambda;
      q.basis_budget = (int32_t)min64(basis_budget, q.n_rows);
      q.tol = tol;
      q.seed = 0;
      probs[p] = q;
    }
  return spsvm_fit_batched(X, n, d, ldx, probs.data(), (int32_t)P, opt, workers, outs, status);
}

extern "C" size_t spsvm_predict_ovo_work_bytes(int32_t classes, int64_t nq) {
  if (classes < 2 || nq < 0) return 0;
  return (size_t)round_up(ovo_count(classes) * (nq > 0 ? nq : 1) * 4, (int64_t)256);
}

extern "C" int spsvm_predict_ovo(const spsvm_model* const* models, int32_t classes,
                                 const float* Xq, int64_t nq, int64_t ldq, int32_t* labels,
                                 int32_t* votes, void* work, size_t work_bytes, void* stream) {
  if (!models || !labels || nq < 0 || (nq > 0 && !Xq))
    return set_error(SPSVM_ERR_ARG, "predict_ovo: bad arguments");
  if (classes < 2 || classes > OV_MAX_CLASSES)
    return set_error(SPSVM_ERR_ARG, "predict_ovo: classes must be in [2, %d]", OV_MAX_CLASSES);
  const int64_t P = ovo_count(classes);
  for (int64_t p = 0; p < P; ++p)
    if (!models[p]) return set_error(SPSVM_ERR_ARG, "predict_ovo: model %lld missing", (long long)p);
  if (nq == 0) return SPSVM_OK;
  if (!work || work_bytes < spsvm_predict_ovo_work_bytes(classes, nq))
    return set_error(SPSVM_ERR_OOM, "predict_ovo: work too small");
  float* dec = static_cast<float*>(work);
  for (int64_t p = 0; p < P; ++p) SPSVM_TRY(spsvm_predict(models[p], Xq, nq, ldq, dec + p * nq, stream));
  ovo_vote_kernel<<<(unsigned)ceil_div(nq, (int64_t)OV_T), OV_T, 0, as_stream(stream)>>>(
      dec, nq, classes, labels, votes);
  SPSVM_LAUNCH_CHECK();
  return SPSVM_OK;
}
