// Optional per-kernel timing: when enabled, every kernel launch of the library is
// bracketed by two CUDA events on the launching stream and tagged with a category name
// and the algorithmic flops and bytes of that launch.  hps_timing_get reduces the events
// into per-category totals.  Disabled (the default), a scope costs one atomic load.
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "hps_internal.h"

namespace hps {

namespace {

struct Rec {
  int cat;
  cudaEvent_t e0, e1;
  double flops, bytes;
  int launches;
};

struct Cat {
  std::string name;
  long long launches = 0;
  double ms = 0.0, flops = 0.0, bytes = 0.0;
};

std::atomic<bool> g_on{false};
std::mutex g_mu;
std::vector<Rec> g_pending;
std::vector<cudaEvent_t> g_pool;
std::vector<Cat> g_cats;
std::map<std::string, int> g_ids;

cudaEvent_t take_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

int drain() {
  std::lock_guard<std::mutex> lk(g_mu);
  int rc = 0;
  for (Rec& r : g_pending) {
    float ms = 0.0f;
    if (cudaEventSynchronize(r.e1) != cudaSuccess || cudaEventElapsedTime(&ms, r.e0, r.e1) != cudaSuccess) {
      cudaGetLastError();
      rc = 1;
    }
    Cat& c = g_cats[r.cat];
    c.launches += r.launches;
    c.ms += ms;
    c.flops += r.flops;
    c.bytes += r.bytes;
    g_pool.push_back(r.e0);
    g_pool.push_back(r.e1);
  }
  g_pending.clear();
  return rc;
}

}  // namespace

thread_local int g_suspended = 0;

bool timing_enabled() { return g_on.load(std::memory_order_relaxed) && !g_suspended; }
void timing_suspend(bool on) { g_suspended += on ? 1 : -1; }

TimingScope::TimingScope(const char* name, cudaStream_t s, double flops, double bytes, int launches)
    : stream_(s), flops_(flops), bytes_(bytes), launches_(launches) {
  if (!timing_enabled()) return;
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_ids.find(name);
  if (it == g_ids.end()) {
    cat_ = (int)g_cats.size();
    g_ids[name] = cat_;
    g_cats.push_back(Cat());
    g_cats.back().name = name;
  } else {
    cat_ = it->second;
  }
  e0_ = take_event();
  e1_ = take_event();
  if (!e0_ || !e1_) {
    cat_ = -1;
    return;
  }
  cudaEventRecord((cudaEvent_t)e0_, s);
}

TimingScope::~TimingScope() {
  if (cat_ < 0) return;
  cudaEventRecord((cudaEvent_t)e1_, stream_);
  std::lock_guard<std::mutex> lk(g_mu);
  g_pending.push_back({cat_, (cudaEvent_t)e0_, (cudaEvent_t)e1_, flops_, bytes_, launches_});
}

}  // namespace hps

using namespace hps;

extern "C" {

int hps_timing_enable(int on) {
  g_on.store(on != 0);
  return HPS_OK;
}

int hps_timing_reset(void) {
  drain();
  std::lock_guard<std::mutex> lk(g_mu);
  for (Cat& c : g_cats) {
    c.launches = 0;
    c.ms = c.flops = c.bytes = 0.0;
  }
  return HPS_OK;
}

int hps_timing_count(int* n) {
  if (!n) return HPS_ERR_INVALID_ARG;
  const int rc = drain();
  std::lock_guard<std::mutex> lk(g_mu);
  *n = (int)g_cats.size();
  return rc ? HPS_ERR_CUDA : HPS_OK;
}

int hps_timing_get(int i, char* name, int name_len, int64_t* launches, double* ms, double* flops, double* bytes) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (i < 0 || i >= (int)g_cats.size()) return HPS_ERR_INVALID_ARG;
  const Cat& c = g_cats[i];
  if (name && name_len > 0) {
    std::strncpy(name, c.name.c_str(), (size_t)name_len - 1);
    name[name_len - 1] = '\0';
  }
  if (launches) *launches = c.launches;
  if (ms) *ms = c.ms;
  if (flops) *flops = c.flops;
  if (bytes) *bytes = c.bytes;
  return HPS_OK;
}

}  // extern "C"
