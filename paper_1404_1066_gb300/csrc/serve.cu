// Batched fits and the serving loop.  Neither has a counterpart in the
// paper beyond its multiclass wrapper (Section 5 trains one binary SP-SVM per
// class pair); both run many independent SP-SVM fits (Section 4) at once.
//
//  * spsvm_fit_batched: problems on rows of one shared device X, spread over
//    worker threads, each with its own CUDA stream and workspace, largest
//    problem first.  A problem's result does not depend on which worker ran
//    it or what ran beside it (each fit's reductions have a fixed order).
//  * spsvm_server: requests (fit, predict) admitted first-come against an
//    HBM budget that counts what the server holds (its workers' buffers, kept
//    and grown across requests, and the resident models); a request that does
//    not fit waits while later ones that do fit run (continuous batching),
//    and a request that has waited longer than two seconds blocks later ones
//    until it is admitted (idle workers then give their buffers back).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace spsvm {
namespace {

__global__ void gather_rows_f32(const float* __restrict__ X, int64_t ldx, int64_t d,
                                const int64_t* __restrict__ rows, int64_t nr,
                                float* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nr * d) return;
  const int64_t r = e / d, k = e % d;
  out[e] = X[rows[r] * ldx + k];
}

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct DeviceBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DeviceBuf() = default;
  DeviceBuf(const DeviceBuf&) = delete;
  DeviceBuf& operator=(const DeviceBuf&) = delete;
  void reset() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  int ensure(size_t want) {
    if (want <= bytes) return SPSVM_OK;
    reset();
    if (want == 0) return SPSVM_OK;
    if (cudaMalloc(&p, want) != cudaSuccess) {
      cudaGetLastError();
      return set_error(SPSVM_ERR_OOM, "cannot allocate %zu device bytes", want);
    }
    bytes = want;
    return SPSVM_OK;
  }
  ~DeviceBuf() {
    if (p) cudaFree(p);
  }
};

}  // namespace
}  // namespace spsvm

using namespace spsvm;

// ---------------------------------------------------------------------------
// Batched fits
// ---------------------------------------------------------------------------
extern "C" int spsvm_fit_batched(const float* X, int64_t n, int64_t d, int64_t ldx,
                                 const spsvm_problem* probs, int32_t count,
                                 const spsvm_options* opt, int32_t workers, spsvm_model** outs,
                                 int32_t* status) {
  if (!X || n < 1 || d < 1 || ldx < d || count < 0 || (count > 0 && (!probs || !outs || !status)))
    return set_error(SPSVM_ERR_ARG, "fit_batched: bad arguments");
  for (int32_t p = 0; p < count; ++p) {
    outs[p] = nullptr;
    status[p] = SPSVM_ERR_ARG;
    const spsvm_problem& q = probs[p];
    if (!q.y || q.n_rows < 1 || (q.rows == nullptr && q.n_rows != n))
      return set_error(SPSVM_ERR_ARG, "fit_batched: problem %d has no rows or labels", p);
    if (q.rows)
      for (int64_t i = 0; i < q.n_rows; ++i)
        if (q.rows[i] < 0 || q.rows[i] >= n)
          return set_error(SPSVM_ERR_ARG, "fit_batched: problem %d row %lld out of range", p,
                           (long long)q.rows[i]);
  }
  if (count == 0) return SPSVM_OK;
  if (workers < 1) workers = 1;
  if (workers > count) workers = count;
  int dev = 0;
  SPSVM_CUDA_TRY(cudaGetDevice(&dev));
  // largest problems first
  std::vector<int32_t> order(count);
  for (int32_t p = 0; p < count; ++p) order[p] = p;
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
    return probs[a].n_rows * (int64_t)probs[a].basis_budget >
           probs[b].n_rows * (int64_t)probs[b].basis_budget;
  });
  std::atomic<int32_t> next{0};
  std::atomic<int> first_error{SPSVM_OK};
  auto work = [&]() {
    if (cudaSetDevice(dev) != cudaSuccess) {
      first_error.store(SPSVM_ERR_CUDA);
      return;
    }
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      first_error.store(SPSVM_ERR_CUDA);
      return;
    }
    DeviceBuf xs, ys, rows, ws;
    for (;;) {
      const int32_t k = next.fetch_add(1);
      if (k >= count) break;
      const int32_t p = order[k];
      const spsvm_problem& q = probs[p];
      spsvm_options o{};
      if (opt) o = *opt;
      o.stream = s;
      if (q.seed) o.seed = q.seed;
      const int64_t nr = q.n_rows;
      const size_t wsb = spsvm_fit_workspace_bytes(nr, d, q.basis_budget, &o);
      int rc = xs.ensure((size_t)nr * d * 4);
      if (rc == SPSVM_OK) rc = ys.ensure((size_t)nr * 4);
      if (rc == SPSVM_OK && q.rows) rc = rows.ensure((size_t)nr * 8);
      if (rc == SPSVM_OK) rc = ws.ensure(wsb);
      const float* Xp = X;
      int64_t ldp = ldx;
      if (rc == SPSVM_OK && q.rows) {
        if (cudaMemcpyAsync(rows.p, q.rows, nr * 8, cudaMemcpyHostToDevice, s) != cudaSuccess) {
          rc = SPSVM_ERR_CUDA;
        } else {
          gather_rows_f32<<<(unsigned)ceil_div(nr * d, 256), 256, 0, s>>>(
              X, ldx, d, static_cast<const int64_t*>(rows.p), nr, static_cast<float*>(xs.p));
          count_launch();
          if (cudaGetLastError() != cudaSuccess) rc = SPSVM_ERR_CUDA;
          Xp = static_cast<const float*>(xs.p);
          ldp = d;
        }
      }
      if (rc == SPSVM_OK &&
          cudaMemcpyAsync(ys.p, q.y, nr * 4, cudaMemcpyHostToDevice, s) != cudaSuccess)
        rc = SPSVM_ERR_CUDA;
      if (rc == SPSVM_OK)
        rc = spsvm_fit(Xp, nr, d, ldp, static_cast<const float*>(ys.p), q.gamma, q.lambda,
                       q.basis_budget, q.tol, &o, ws.p, ws.bytes, &outs[p]);
      status[p] = rc;
      if (rc != SPSVM_OK && rc != SPSVM_ERR_NO_CONVERGE) {
        int expected = SPSVM_OK;
        first_error.compare_exchange_strong(expected, rc);
      }
    }
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  };
  std::vector<std::thread> pool;
  for (int32_t w = 0; w < workers; ++w) pool.emplace_back(work);
  for (auto& t : pool) t.join();
  const int e = first_error.load();
  return e == SPSVM_OK ? SPSVM_OK
                       : set_error(e, "fit_batched: at least one problem failed (see status[])");
}

// ---------------------------------------------------------------------------
// Serving loop
// ---------------------------------------------------------------------------
struct SpsvmRequest {
  int64_t id = 0;
  int kind = 0;   // 0 fit, 1 predict
  // fit
  std::vector<float> X, y;
  int64_t n = 0, d = 0;
  float gamma = 0.f;
  double lambda = 0.0, tol = 0.0;
  int32_t budget = 0;
  spsvm_options opt{};
  std::vector<int64_t> init_basis;
  spsvm_model* model = nullptr;
  // predict
  int64_t fit_id = -1;
  std::vector<float> Xq, out;
  int64_t nq = 0;
  // bookkeeping
  size_t footprint = 0;     // device bytes the request needs (checked against the budget)
  size_t model_bytes = 0;   // device bytes of the fitted model while resident
  size_t work_bytes = 0;    // a predict's decision work (at most, for the fit's budget)
  double t_submit = 0, t_start = 0, t_end = 0;
  int state = 0;   // 0 queued, 1 running, 2 done
  int32_t status = SPSVM_OK;
};

struct spsvm_server {
  // in_use: device bytes the server holds -- every worker's buffers (kept
  // across requests, grown on demand) and every resident model (until
  // spsvm_server_release or destroy), plus the model reserve of a fit that
  // is running
  size_t budget = 0, in_use = 0, peak = 0;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<int64_t> queue;
  std::unordered_map<int64_t, std::shared_ptr<SpsvmRequest>> reqs;
  int64_t next_id = 1;
  int64_t done = 0;
  bool stop = false;
  std::vector<std::thread> workers;
};

namespace {

// A worker's device buffers, kept across requests (grown, never shrunk
// while requests keep fitting the budget).
struct WorkerBufs {
  DeviceBuf X, y, ws, Q, out, pw;
  size_t held() const { return X.bytes + y.bytes + ws.bytes + Q.bytes + out.bytes + pw.bytes; }
  void release() {
    X.reset();
    y.reset();
    ws.reset();
    Q.reset();
    out.reset();
    pw.reset();
  }
};

// Device bytes a fit's model holds at most (basis rows, beta, decision scratch).
size_t model_reserve(const SpsvmRequest& r) {
  return (size_t)r.budget * r.d * 4 + (size_t)r.budget * 8 +
         spsvm_decision_scratch_bytes(0, r.budget, r.d, SPSVM_FP32);
}

size_t grow_of(const DeviceBuf& b, size_t want) { return want > b.bytes ? want - b.bytes : 0; }

// Device bytes the worker must add to run r (its buffers grown to r's needs,
// plus the model reserve of a fit).
size_t extra_for(const SpsvmRequest& r, const WorkerBufs& W) {
  if (r.kind == 0)
    return grow_of(W.X, r.X.size() * 4) + grow_of(W.y, r.y.size() * 4) +
           grow_of(W.ws, spsvm_fit_workspace_bytes(r.n, r.d, r.budget, &r.opt)) + model_reserve(r);
  return grow_of(W.Q, r.Xq.size() * 4) + grow_of(W.out, (size_t)r.nq * 4) +
         grow_of(W.pw, r.work_bytes);
}

// First admissible request in FIFO order for this worker (lock held): its
// extra bytes fit the budget; the bytes are reserved.  A request waiting
// longer than two seconds blocks later ones; *aged is set when that head
// does not fit, and the caller then gives its own buffers back.
std::shared_ptr<SpsvmRequest> take_admissible(spsvm_server* S, const WorkerBufs& W, bool* aged) {
  const double t = now_ms();
  *aged = false;
  for (auto it = S->queue.begin(); it != S->queue.end(); ++it) {
    auto r = S->reqs[*it];
    bool ready = true;
    if (r->kind == 1) {
      auto f = S->reqs.find(r->fit_id);
      ready = (f != S->reqs.end() && f->second->state == 2);
    }
    const size_t extra = ready ? extra_for(*r, W) : 0;
    if (ready && S->in_use + extra <= S->budget) {
      S->queue.erase(it);
      S->in_use += extra;
      S->peak = std::max(S->peak, S->in_use);
      r->state = 1;
      r->t_start = t;
      return r;
    }
    if (ready && t - r->t_submit > 2000.0) {   // aged head blocks the rest
      *aged = true;
      return nullptr;
    }
  }
  return nullptr;
}

int run_fit(SpsvmRequest& r, WorkerBufs& W, cudaStream_t s) {
  SPSVM_TRY(W.X.ensure(r.X.size() * 4));
  SPSVM_TRY(W.y.ensure(r.y.size() * 4));
  spsvm_options o = r.opt;
  o.stream = s;
  if (!r.init_basis.empty()) {
    o.initial_basis = r.init_basis.data();
    o.n_initial = (int32_t)r.init_basis.size();
  }
  SPSVM_TRY(W.ws.ensure(spsvm_fit_workspace_bytes(r.n, r.d, r.budget, &o)));
  SPSVM_CUDA_TRY(cudaMemcpyAsync(W.X.p, r.X.data(), r.X.size() * 4, cudaMemcpyHostToDevice, s));
  SPSVM_CUDA_TRY(cudaMemcpyAsync(W.y.p, r.y.data(), r.y.size() * 4, cudaMemcpyHostToDevice, s));
  const int rc = spsvm_fit(static_cast<float*>(W.X.p), r.n, r.d, r.d, static_cast<float*>(W.y.p),
                           r.gamma, r.lambda, r.budget, r.tol, &o, W.ws.p, W.ws.bytes, &r.model);
  cudaStreamSynchronize(s);
  return rc;
}

int run_predict(SpsvmRequest& r, spsvm_model* m, WorkerBufs& W, cudaStream_t s) {
  SPSVM_TRY(W.Q.ensure(r.Xq.size() * 4));
  SPSVM_TRY(W.out.ensure((size_t)r.nq * 4));
  SPSVM_TRY(W.pw.ensure(r.work_bytes));
  SPSVM_CUDA_TRY(cudaMemcpyAsync(W.Q.p, r.Xq.data(), r.Xq.size() * 4, cudaMemcpyHostToDevice, s));
  SPSVM_TRY(spsvm_predict_ws(m, static_cast<float*>(W.Q.p), r.nq, r.d, static_cast<float*>(W.out.p),
                             W.pw.p, W.pw.bytes, s));
  r.out.resize(r.nq);
  SPSVM_CUDA_TRY(cudaMemcpyAsync(r.out.data(), W.out.p, r.nq * 4, cudaMemcpyDeviceToHost, s));
  SPSVM_CUDA_TRY(cudaStreamSynchronize(s));
  return SPSVM_OK;
}

void worker_loop(spsvm_server* S) {
  cudaSetDevice(S->device);
  cudaStream_t s = nullptr;
  cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  WorkerBufs W;
  for (;;) {
    std::shared_ptr<SpsvmRequest> r;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      for (;;) {
        if (S->stop) {
          S->in_use -= W.held();
          lk.unlock();
          W.release();
          cudaStreamDestroy(s);
          return;
        }
        bool aged = false;
        r = take_admissible(S, W, &aged);
        if (r) break;
        if (aged && W.held() > 0) {
          // an aged request does not fit: give this worker's buffers back
          // (a device-synchronising free, on this rare path only)
          S->in_use -= W.held();
          lk.unlock();
          W.release();
          lk.lock();
          continue;
        }
        S->cv.wait_for(lk, std::chrono::milliseconds(50));
      }
    }
    int rc;
    spsvm_model* fm = nullptr;
    if (r->kind == 0) {
      rc = run_fit(*r, W, s);
    } else {
      {
        std::lock_guard<std::mutex> lk(S->mu);
        fm = S->reqs[r->fit_id]->model;
      }
      rc = fm ? run_predict(*r, fm, W, s) : set_error(SPSVM_ERR_ARG, "predict: fit produced no model");
    }
    {
      std::lock_guard<std::mutex> lk(S->mu);
      r->status = rc;
      r->t_end = now_ms();
      r->state = 2;
      r->X.clear();
      r->X.shrink_to_fit();
      r->Xq.clear();
      r->Xq.shrink_to_fit();
      // a fit's model reserve becomes the model's actual bytes (resident
      // until released); a failed fit returns its reserve
      if (r->kind == 0) {
        S->in_use -= model_reserve(*r);
        r->model_bytes = spsvm_model_device_bytes(r->model);
        S->in_use += r->model_bytes;
      }
      ++S->done;
    }
    S->cv.notify_all();
  }
}

int enqueue(spsvm_server* S, std::shared_ptr<SpsvmRequest> r, int64_t* id) {
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (r->footprint > S->budget)
      return set_error(SPSVM_ERR_OOM, "request needs %zu bytes, budget is %zu", r->footprint,
                       S->budget);
    r->id = S->next_id++;
    r->t_submit = now_ms();
    S->reqs[r->id] = r;
    S->queue.push_back(r->id);
    *id = r->id;
  }
  S->cv.notify_all();
  return SPSVM_OK;
}

}  // namespace

extern "C" int spsvm_server_create(size_t hbm_budget_bytes, int32_t workers, spsvm_server** out) {
  if (!out || hbm_budget_bytes == 0 || workers < 1)
    return set_error(SPSVM_ERR_ARG, "server_create: bad arguments");
  auto* S = new spsvm_server();
  S->budget = hbm_budget_bytes;
  if (cudaGetDevice(&S->device) != cudaSuccess) {
    cudaGetLastError();
    delete S;
    return set_error(SPSVM_ERR_CUDA, "server_create: no device");
  }
  for (int32_t w = 0; w < workers; ++w) S->workers.emplace_back(worker_loop, S);
  *out = S;
  return SPSVM_OK;
}

extern "C" int spsvm_server_submit_fit(spsvm_server* S, const float* X, int64_t n, int64_t d,
                                       const float* y, float gamma, double lambda,
                                       int32_t basis_budget, double tol, const spsvm_options* opt,
                                       int64_t* request_id) {
  if (!S || !X || !y || !request_id || n < 1 || d < 1 || !(gamma > 0.f) || !(lambda > 0.0) ||
      basis_budget < 1 || basis_budget > n)
    return set_error(SPSVM_ERR_ARG, "server_submit_fit: bad arguments");
  auto r = std::make_shared<SpsvmRequest>();
  r->kind = 0;
  r->X.assign(X, X + n * d);
  r->y.assign(y, y + n);
  r->n = n;
  r->d = d;
  r->gamma = gamma;
  r->lambda = lambda;
  r->tol = tol;
  r->budget = basis_budget;
  if (opt) {
    r->opt = *opt;
    if (opt->initial_basis && opt->n_initial > 0)
      r->init_basis.assign(opt->initial_basis, opt->initial_basis + opt->n_initial);
  }
  r->opt.initial_basis = nullptr;
  r->opt.n_initial = 0;
  r->footprint = (size_t)n * d * 4 + (size_t)n * 4 +
                 spsvm_fit_workspace_bytes(n, d, basis_budget, &r->opt) + model_reserve(*r);
  return enqueue(S, r, request_id);
}

extern "C" int spsvm_server_submit_predict(spsvm_server* S, int64_t fit_id, const float* Xq,
                                           int64_t nq, int64_t* request_id) {
  if (!S || !Xq || nq < 1 || !request_id)
    return set_error(SPSVM_ERR_ARG, "server_submit_predict: bad arguments");
  int64_t d = 0;
  size_t work = 0;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    auto f = S->reqs.find(fit_id);
    if (f == S->reqs.end() || f->second->kind != 0)
      return set_error(SPSVM_ERR_ARG, "server_submit_predict: unknown fit request %lld",
                       (long long)fit_id);
    if (f->second->state == 2 && !f->second->model)
      return set_error(SPSVM_ERR_ARG, "server_submit_predict: fit request %lld has no model "
                       "(failed or released)", (long long)fit_id);
    d = f->second->d;
    // the decision work of the split form, for the fit's basis budget
    if (f->second->opt.precision == SPSVM_BF16SPLIT)
      work = spsvm_decision_scratch_bytes(nq, f->second->budget, d, SPSVM_BF16SPLIT);
  }
  auto r = std::make_shared<SpsvmRequest>();
  r->kind = 1;
  r->fit_id = fit_id;
  r->d = d;
  r->nq = nq;
  r->Xq.assign(Xq, Xq + nq * d);
  r->work_bytes = work;
  r->footprint = (size_t)nq * d * 4 + (size_t)nq * 4 + work;
  return enqueue(S, r, request_id);
}

extern "C" int spsvm_server_wait(spsvm_server* S, int64_t request_id, double timeout_s,
                                 int32_t* status, double* latency_ms) {
  if (!S) return set_error(SPSVM_ERR_ARG, "server_wait: NULL server");
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(request_id);
  if (it == S->reqs.end()) return set_error(SPSVM_ERR_ARG, "server_wait: unknown request");
  auto r = it->second;
  const auto deadline = std::chrono::steady_clock::now() +
                        std::chrono::microseconds((int64_t)(timeout_s * 1e6));
  while (r->state != 2) {
    if (timeout_s >= 0 && std::chrono::steady_clock::now() >= deadline)
      return set_error(SPSVM_ERR_TIMEOUT, "server_wait: request %lld not finished",
                       (long long)request_id);
    S->cv.wait_for(lk, std::chrono::milliseconds(20));
  }
  if (status) *status = r->status;
  if (latency_ms) *latency_ms = r->t_end - r->t_submit;
  return SPSVM_OK;
}

extern "C" int spsvm_server_result(spsvm_server* S, int64_t request_id, float* decision,
                                   int64_t cap, spsvm_model** model) {
  if (!S) return set_error(SPSVM_ERR_ARG, "server_result: NULL server");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(request_id);
  if (it == S->reqs.end() || it->second->state != 2)
    return set_error(SPSVM_ERR_ARG, "server_result: request unknown or not finished");
  auto& r = *it->second;
  if (model) *model = (r.kind == 0) ? r.model : nullptr;
  if (decision && r.kind == 1) {
    if (cap < r.nq) return set_error(SPSVM_ERR_ARG, "server_result: output too small");
    std::copy(r.out.begin(), r.out.end(), decision);
  }
  return SPSVM_OK;
}

extern "C" int spsvm_server_release(spsvm_server* S, int64_t fit_request_id) {
  if (!S) return set_error(SPSVM_ERR_ARG, "server_release: NULL server");
  spsvm_model* m = nullptr;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(fit_request_id);
    if (it == S->reqs.end() || it->second->kind != 0 || it->second->state != 2)
      return set_error(SPSVM_ERR_ARG, "server_release: %lld is not a finished fit",
                       (long long)fit_request_id);
    for (auto& kv : S->reqs)   // predicts of this model still queued or running
      if (kv.second->kind == 1 && kv.second->fit_id == fit_request_id && kv.second->state != 2)
        return set_error(SPSVM_ERR_BUSY, "server_release: predicts of %lld pending",
                         (long long)fit_request_id);
    m = it->second->model;
    it->second->model = nullptr;
    S->in_use -= it->second->model_bytes;
    it->second->model_bytes = 0;
  }
  spsvm_free(m);
  S->cv.notify_all();
  return SPSVM_OK;
}

extern "C" int spsvm_server_stats(spsvm_server* S, int64_t* done, int64_t* queued,
                                  size_t* hbm_in_use, size_t* hbm_peak) {
  if (!S) return set_error(SPSVM_ERR_ARG, "server_stats: NULL server");
  std::lock_guard<std::mutex> lk(S->mu);
  if (done) *done = S->done;
  if (queued) *queued = (int64_t)S->queue.size();
  if (hbm_in_use) *hbm_in_use = S->in_use;
  if (hbm_peak) *hbm_peak = S->peak;
  return SPSVM_OK;
}

extern "C" void spsvm_server_destroy(spsvm_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv.notify_all();
  for (auto& t : S->workers) t.join();
  for (auto& kv : S->reqs)
    if (kv.second->model) spsvm_free(kv.second->model);
  delete S;
}
