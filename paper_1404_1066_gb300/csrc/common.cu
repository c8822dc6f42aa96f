// Error reporting, device facts and point preparation (row norms, BF16
// split planes).
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <mutex>
#include <unordered_map>
#include <vector>

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
  if (K->format != SPSVM_FP32 && K->format != SPSVM_BF16SPLIT)
    return set_error(SPSVM_ERR_ARG, "%s: bad format %d", what, K->format);
  if (K->n < 0 || K->rows < 0 || K->ld < K->n || (K->ld % 8) != 0)
    return set_error(SPSVM_ERR_ARG, "%s: bad shape n=%lld rows=%lld ld=%lld", what,
                     (long long)K->n, (long long)K->rows, (long long)K->ld);
  if (K->format == SPSVM_BF16SPLIT && K->plane < K->rows * K->ld)
    return set_error(SPSVM_ERR_ARG, "%s: hi/lo planes overlap", what);
  if ((reinterpret_cast<uintptr_t>(K->data) & 15) != 0)
    return set_error(SPSVM_ERR_ARG, "%s: data not 16-byte aligned", what);
  return SPSVM_OK;
}

// One warp per point: ||x_i||^2 in FP64, and the three-term BF16 split of
// the row (hi = bf16(x), mid = bf16(x - hi), lo = bf16(x - hi - mid); the
// differences are exact in FP32).
__global__ void prepare_points_kernel(const float* __restrict__ X, int64_t n, int64_t d,
                                      int64_t ldx, float* __restrict__ norms,
                                      __nv_bfloat16* __restrict__ hi,
                                      __nv_bfloat16* __restrict__ mid,
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
      __nv_bfloat16 h = __float2bfloat16_rn(0.0f), md = h, l = h;
      if (k < d) {
        const float v = x[k];
        split_bf16(v, h, md);                                  // h, md = bf16(v - h)
        l = __float2bfloat16_rn((v - __bfloat162float(h)) - __bfloat162float(md));
      }
      hi[i * ldh + k] = h;
      mid[i * ldh + k] = md;
      lo[i * ldh + k] = l;
    }
  }
}

static std::atomic<unsigned long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// ---- status words of the bounded device waits, one per stream --------------
namespace {
constexpr int kStatusSlots = 1024;
__device__ int g_wait_status[kStatusSlots];
std::atomic<uint32_t> g_wait_limit{0};
std::mutex g_slot_mu;
struct SlotUse {
  int slot;
  uint64_t last;
};
std::unordered_map<cudaStream_t, SlotUse> g_slot_of;
uint64_t g_slot_clock = 0;
}  // namespace

// The stream's slot is assigned on its first use (zeroed in order on the
// stream) and kept; with every slot taken, the least recently used stream's
// slot is handed over.  The table's device address is looked up on each call
// (no cached address survives a context reset).
int wait_ctx(cudaStream_t s, WaitCtx* w) {
  void* base = nullptr;
  SPSVM_CUDA_TRY(cudaGetSymbolAddress(&base, g_wait_status));
  int slot = -1;
  bool fresh = false;
  {
    std::lock_guard<std::mutex> lk(g_slot_mu);
    ++g_slot_clock;
    auto it = g_slot_of.find(s);
    if (it != g_slot_of.end()) {
      it->second.last = g_slot_clock;
      slot = it->second.slot;
    } else {
      if ((int)g_slot_of.size() < kStatusSlots) {
        slot = (int)g_slot_of.size();
      } else {
        auto lru = g_slot_of.begin();
        for (auto jt = g_slot_of.begin(); jt != g_slot_of.end(); ++jt)
          if (jt->second.last < lru->second.last) lru = jt;
        slot = lru->second.slot;
        g_slot_of.erase(lru);
      }
      g_slot_of[s] = SlotUse{slot, g_slot_clock};
      fresh = true;
    }
  }
  w->st = static_cast<int*>(base) + slot;
  w->lim = g_wait_limit.load(std::memory_order_relaxed);
  if (fresh) SPSVM_CUDA_TRY(cudaMemsetAsync(w->st, 0, sizeof(int), s));
  return SPSVM_OK;
}

namespace {
// Pinned staging memory of one host thread for read_back (grown on demand,
// released at thread exit).
struct PinnedStage {
  void* p = nullptr;
  size_t bytes = 0;
  ~PinnedStage() {
    if (p) cudaFreeHost(p);
  }
};
thread_local PinnedStage t_stage;

int read_back_code(cudaStream_t s, const ReadChunk* c, int n, int32_t* code) {
  size_t total = 16;
  for (int k = 0; k < n; ++k) total += (size_t)round_up((int64_t)c[k].bytes, 16);
  if (t_stage.bytes < total) {
    if (t_stage.p) cudaFreeHost(t_stage.p);
    t_stage.p = nullptr;
    t_stage.bytes = 0;
    const size_t want = total < 4096 ? 4096 : total;
    SPSVM_CUDA_TRY(cudaMallocHost(&t_stage.p, want));
    t_stage.bytes = want;
  }
  WaitCtx w;
  SPSVM_TRY(wait_ctx(s, &w));
  char* h = static_cast<char*>(t_stage.p);
  size_t off = 16;
  for (int k = 0; k < n; ++k) {
    if (c[k].bytes)
      SPSVM_CUDA_TRY(cudaMemcpyAsync(h + off, c[k].src, c[k].bytes, cudaMemcpyDeviceToHost, s));
    off += (size_t)round_up((int64_t)c[k].bytes, 16);
  }
  SPSVM_CUDA_TRY(cudaMemcpyAsync(h, w.st, sizeof(int), cudaMemcpyDeviceToHost, s));
  SPSVM_CUDA_TRY(cudaStreamSynchronize(s));
  off = 16;
  for (int k = 0; k < n; ++k) {
    if (c[k].bytes) memcpy(c[k].dst, h + off, c[k].bytes);
    off += (size_t)round_up((int64_t)c[k].bytes, 16);
  }
  int v = 0;
  memcpy(&v, h, sizeof(int));
  if (code) *code = v;
  if (v != 0) {
    SPSVM_CUDA_TRY(cudaMemsetAsync(w.st, 0, sizeof(int), s));
    SPSVM_CUDA_TRY(cudaStreamSynchronize(s));
    return set_error(SPSVM_ERR_TIMEOUT, "a bounded device wait gave up (site %d)", v);
  }
  return SPSVM_OK;
}
}  // namespace

int read_back(cudaStream_t s, const ReadChunk* chunks, int n) {
  return read_back_code(s, chunks, n, nullptr);
}

int device_status_on(cudaStream_t s, int32_t* code) { return read_back_code(s, nullptr, 0, code); }

// ---- kernel timing -----------------------------------------------------
namespace {
const char* kSlotNames[PROF_SLOTS] = {"kernel_block", "score", "outputs", "gemv", "compact",
                                      "gram", "cholesky", "solve", "line_search", "decision",
                                      "fit", "lowrank"};
struct Pending {
  int slot;
  cudaEvent_t e0, e1;
  double work;
};
struct Totals {
  long long launches = 0;
  double ms = 0.0, work = 0.0;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_free_events;
Totals g_totals[PROF_SLOTS];

cudaEvent_t take_event() {
  if (!g_free_events.empty()) {
    cudaEvent_t e = g_free_events.back();
    g_free_events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

void resolve_locked() {
  for (auto& p : g_pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(p.e1) == cudaSuccess &&
        cudaEventElapsedTime(&ms, p.e0, p.e1) == cudaSuccess) {
      g_totals[p.slot].launches += 1;
      g_totals[p.slot].ms += ms;
      g_totals[p.slot].work += p.work;
    } else {
      cudaGetLastError();
    }
    g_free_events.push_back(p.e0);
    g_free_events.push_back(p.e1);
  }
  g_pending.clear();
}
}  // namespace

ProfScope::ProfScope(int slot_, cudaStream_t s_, double work_)
    : slot(slot_), s(s_), work(work_), e0(nullptr) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (!g_prof_on) return;
  cudaEvent_t e = take_event();
  if (e && cudaEventRecord(e, s) == cudaSuccess) e0 = e;
}

ProfScope::~ProfScope() {
  if (!e0) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  cudaEvent_t e1 = take_event();
  if (!e1 || cudaEventRecord(e1, s) != cudaSuccess) {
    g_free_events.push_back(static_cast<cudaEvent_t>(e0));
    return;
  }
  g_pending.push_back(Pending{slot, static_cast<cudaEvent_t>(e0), e1, work});
  if (g_pending.size() > 4096) resolve_locked();
}

}  // namespace spsvm

using namespace spsvm;

extern "C" uint64_t spsvm_launch_count(void) { return g_launches.load(); }

extern "C" int spsvm_profile_enable(int32_t on) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  resolve_locked();
  for (auto& t : g_totals) t = Totals{};
  g_prof_on = on != 0;
  return SPSVM_OK;
}

extern "C" int spsvm_profile_read(int32_t slot, const char** name, int64_t* launches,
                                  double* ms, double* work) {
  if (slot < 0 || slot >= PROF_SLOTS) return set_error(SPSVM_ERR_ARG, "profile_read: bad slot");
  std::lock_guard<std::mutex> lk(g_prof_mu);
  resolve_locked();
  if (name) *name = kSlotNames[slot];
  if (launches) *launches = g_totals[slot].launches;
  if (ms) *ms = g_totals[slot].ms;
  if (work) *work = g_totals[slot].work;
  return SPSVM_OK;
}

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
  if (precision == SPSVM_BF16SPLIT) {
    if (!p->hi || !p->mid || !p->lo || p->ldh < p->d || (p->ldh % 64) != 0)
      return set_error(SPSVM_ERR_ARG,
                       "prepare_points: BF16SPLIT needs hi / mid / lo planes with ldh %% 64 == 0");
  } else if (precision != SPSVM_FP32) {
    return set_error(SPSVM_ERR_ARG, "prepare_points: bad precision %d", precision);
  }
  if (p->n == 0) return SPSVM_OK;
  const int warps = 8;
  dim3 grid((unsigned)ceil_div(p->n, warps));
  prepare_points_kernel<<<grid, warps * 32, 0, as_stream(stream)>>>(
      p->X, p->n, p->d, p->ldx, p->norms,
      precision == SPSVM_BF16SPLIT ? reinterpret_cast<__nv_bfloat16*>(p->hi) : nullptr,
      precision == SPSVM_BF16SPLIT ? reinterpret_cast<__nv_bfloat16*>(p->mid) : nullptr,
      precision == SPSVM_BF16SPLIT ? reinterpret_cast<__nv_bfloat16*>(p->lo) : nullptr, p->ldh);
  SPSVM_LAUNCH_CHECK();
  return SPSVM_OK;
}

extern "C" int spsvm_stream_status(void* stream, int32_t* code) {
  if (code) *code = 0;
  const int rc = spsvm::device_status_on(as_stream(stream), code);
  if (rc == SPSVM_ERR_CUDA && code) *code = -1;
  return rc;
}

extern "C" int spsvm_device_status(int32_t* code) { return spsvm_stream_status(nullptr, code); }

extern "C" void spsvm_set_wait_limit(uint32_t polls) {
  spsvm::g_wait_limit.store(polls, std::memory_order_relaxed);
}
